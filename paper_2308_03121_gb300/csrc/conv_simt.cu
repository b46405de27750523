// FP32 SIMT convolution and modulated deformable convolution (the "plain" path).
//
// The networks NNVISR hosts are stacks of 3x3 convolutions (Section 3.1) plus
// the DCN v2 operator the paper ships (Section 3.1, torchvision semantics).
// This file computes both on the FP32 CUDA-core lanes, as implicit GEMM:
//   M = output pixels (a 128-pixel row segment per block),
//   N = output channels (NB per block),
//   K = taps x input channels, walked in slices of 8 input channels.
// Per slice a block stages the input halo (conv: 8 ch x KS rows x 130 px) or
// the bilinear-sampled, mask-weighted im2col tile (DCN: 8 ch x 9 taps x 128
// px) in shared memory, plus the weights [8][KS*KS][NB]; each thread
// accumulates 8 pixels x 4 output channels in registers.  The epilogue fuses
// bias, LeakyReLU(0.1), the residual add, and -- for a network's last layer
// -- PixelShuffle(2) plus the skip (nearest / bilinear upsample of the input
// frame) into a planar float32 image.
//
// Tensors use the blocked layout [C/4][H][W][4] (16-byte channel chunks).
#include "common.cuh"
#include "epilogue.cuh"

namespace nvisr {

namespace {

constexpr int TW = 128;  // output pixels per block (one row segment)

// Bilinear sample with zero contribution from out-of-image corners, 4 channels.
__device__ __forceinline__ float4 bilinear4(const float4 *plane, int H, int W, float sy, float sx) {
    float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
    const float fy = floorf(sy), fx = floorf(sx);
    const int y0 = (int)fy, x0 = (int)fx;
    const float ly = sy - fy, lx = sx - fx;
#pragma unroll
    for (int dy = 0; dy < 2; ++dy) {
        const int yy = y0 + dy;
        if (yy < 0 || yy >= H) continue;
        const float wy = dy ? ly : 1.f - ly;
#pragma unroll
        for (int dx = 0; dx < 2; ++dx) {
            const int xx = x0 + dx;
            if (xx < 0 || xx >= W) continue;
            const float wgt = wy * (dx ? lx : 1.f - lx);
            const float4 t = plane[(int64_t)yy * W + xx];
            v.x += wgt * t.x; v.y += wgt * t.y; v.z += wgt * t.z; v.w += wgt * t.w;
        }
    }
    return v;
}

// MODE 0: convolution (halo staging); MODE 1: DCN (sampled im2col staging).
template <int NB, int KS, int MODE>
__global__ void __launch_bounds__(16 * NB / 4) conv_simt_kernel(ConvArgs a, DcnArgs d) {
    constexpr int NT = 16 * NB / 4;
    constexpr int KK = KS * KS;
    constexpr int PAD = (KS - 1) / 2;
    constexpr int APX = (MODE == 0) ? (KS == 3 ? 132 : 128) : 128;  // row pitch of the staged tile
    constexpr int AROWS = (MODE == 0) ? KS : KK;                   // halo rows or taps
    extern __shared__ __align__(16) float smem_f[];
    float(*As)[AROWS][APX] = reinterpret_cast<float(*)[AROWS][APX]>(smem_f);
    float(*Bs)[KK][NB] = reinterpret_cast<float(*)[KK][NB]>(smem_f + 8 * AROWS * APX);

    const int H = MODE == 0 ? a.H : d.H;
    const int W = MODE == 0 ? a.W : d.W;
    const int cin_pad = MODE == 0 ? a.cin_pad : d.cin_pad;
    const int cout_pad = MODE == 0 ? a.cout_pad : d.cout_pad;
    const float *wts = (const float *)(MODE == 0 ? a.w : d.w);
    const float4 *xin = (const float4 *)(MODE == 0 ? a.x : d.x);

    const int tiles_x = (W + TW - 1) / TW;
    const int tile = blockIdx.x;
    const int img = tile / (tiles_x * H);
    const int rem = tile - img * tiles_x * H;
    const int y = rem / tiles_x;
    const int x0 = (rem - y * tiles_x) * TW;
    const int ot = blockIdx.y;
    const int tid = threadIdx.x;
    const int pg = tid % 16, og = tid / 16;
    const int64_t HW = (int64_t)H * W;
    const float4 *ximg = xin + (int64_t)img * (cin_pad / 4) * HW;

    float acc[8][4];
#pragma unroll
    for (int p = 0; p < 8; ++p)
#pragma unroll
        for (int n = 0; n < 4; ++n) acc[p][n] = 0.f;

    for (int s = 0; s < cin_pad / 8; ++s) {
        // ---- stage A
        if (MODE == 0) {
            constexpr int PXN = TW + KS - 1;
            for (int i = tid; i < 2 * KS * PXN; i += NT) {
                const int cl = i / (KS * PXN);
                const int r = (i / PXN) % KS;
                const int p = i % PXN;
                const int iy = y + r - PAD, ix = x0 + p - PAD;
                float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
                if (iy >= 0 && iy < H && ix >= 0 && ix < W)
                    v = ximg[(int64_t)(s * 2 + cl) * HW + (int64_t)iy * W + ix];
                As[cl * 4 + 0][r][p] = v.x;
                As[cl * 4 + 1][r][p] = v.y;
                As[cl * 4 + 2][r][p] = v.z;
                As[cl * 4 + 3][r][p] = v.w;
            }
        } else {
            const int cpg = d.cin_pad / d.groups;
            for (int i = tid; i < 2 * KK * TW; i += NT) {
                const int cl = i / (KK * TW);
                const int k = (i / TW) % KK;
                const int p = i % TW;
                const int xx = x0 + p;
                float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
                if (xx < W) {
                    const int c = (s * 2 + cl) * 4;
                    const int g = c / cpg;
                    const int64_t pix = (int64_t)y * W + xx;
                    auto omv = [&](int ch) { return d.om[((int64_t)(ch >> 2) * HW + pix) * 4 + (ch & 3)]; };
                    const int cd = dcn_off_channel(g, k, d.groups, d.om_tap_major != 0);
                    const float dy = omv(cd);
                    const float dx = omv(cd + 1);
                    float m = omv(dcn_mask_channel(g, k, d.groups, d.om_tap_major != 0));
                    if (d.mask_logits) m = 1.f / (1.f + expf(-m));
                    const float sy = (float)(y + k / 3 - 1) + dy;
                    const float sx = (float)(xx + k % 3 - 1) + dx;
                    v = bilinear4(ximg + (int64_t)(s * 2 + cl) * HW, H, W, sy, sx);
                    v.x *= m; v.y *= m; v.z *= m; v.w *= m;
                }
                As[cl * 4 + 0][k][p] = v.x;
                As[cl * 4 + 1][k][p] = v.y;
                As[cl * 4 + 2][k][p] = v.z;
                As[cl * 4 + 3][k][p] = v.w;
            }
        }
        // ---- stage B: weights [cin_pad][KK][cout_pad] -> Bs[8][KK][NB]
        for (int i = tid; i < 8 * KK * NB / 4; i += NT) {
            const int c = i / (KK * NB / 4);
            const int t = (i / (NB / 4)) % KK;
            const int n4 = i % (NB / 4);
            const float4 v = *reinterpret_cast<const float4 *>(
                wts + ((int64_t)(s * 8 + c) * KK + t) * cout_pad + ot * NB + n4 * 4);
            *reinterpret_cast<float4 *>(&Bs[c][t][n4 * 4]) = v;
        }
        __syncthreads();
        // ---- multiply
#pragma unroll 2
        for (int c = 0; c < 8; ++c) {
            if (MODE == 0) {
#pragma unroll
                for (int ky = 0; ky < KS; ++ky) {
                    float av[8 + KS - 1];
                    const float *ar = &As[c][ky][pg * 8];
                    const float4 a0 = *reinterpret_cast<const float4 *>(ar);
                    const float4 a1 = *reinterpret_cast<const float4 *>(ar + 4);
                    av[0] = a0.x; av[1] = a0.y; av[2] = a0.z; av[3] = a0.w;
                    av[4] = a1.x; av[5] = a1.y; av[6] = a1.z; av[7] = a1.w;
                    if (KS == 3) {
                        const float2 a2 = *reinterpret_cast<const float2 *>(ar + 8);
                        av[8 % (8 + KS - 1)] = a2.x;
                        av[9 % (8 + KS - 1)] = a2.y;
                    }
#pragma unroll
                    for (int kx = 0; kx < KS; ++kx) {
                        const float4 b = *reinterpret_cast<const float4 *>(&Bs[c][ky * KS + kx][og * 4]);
#pragma unroll
                        for (int p = 0; p < 8; ++p) {
                            const float v = av[p + kx];
                            acc[p][0] += v * b.x; acc[p][1] += v * b.y;
                            acc[p][2] += v * b.z; acc[p][3] += v * b.w;
                        }
                    }
                }
            } else {
#pragma unroll
                for (int k = 0; k < KK; ++k) {
                    const float *ar = &As[c][k][pg * 8];
                    const float4 a0 = *reinterpret_cast<const float4 *>(ar);
                    const float4 a1 = *reinterpret_cast<const float4 *>(ar + 4);
                    const float av[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
                    const float4 b = *reinterpret_cast<const float4 *>(&Bs[c][k][og * 4]);
#pragma unroll
                    for (int p = 0; p < 8; ++p) {
                        acc[p][0] += av[p] * b.x; acc[p][1] += av[p] * b.y;
                        acc[p][2] += av[p] * b.z; acc[p][3] += av[p] * b.w;
                    }
                }
            }
        }
        __syncthreads();
    }

    // ---- epilogue
    const int oc0 = ot * NB + og * 4;
    const float *bias = MODE == 0 ? a.bias : d.bias;
    const float accs = MODE == 0 ? a.acc_scale : d.acc_scale;
    const float4 bv = *reinterpret_cast<const float4 *>(bias + oc0);
    const int act = MODE == 0 ? a.act : 0;
    float4 *yout = (float4 *)(MODE == 0 ? a.y : d.y);
    for (int p = 0; p < 8; ++p) {
        const int xx = x0 + pg * 8 + p;
        if (xx >= W) break;
        float v[4] = {acc[p][0] * accs + bv.x, acc[p][1] * accs + bv.y,
                      acc[p][2] * accs + bv.z, acc[p][3] * accs + bv.w};
        if (act == 1) {
#pragma unroll
            for (int n = 0; n < 4; ++n) v[n] = lrelu(v[n]);
        }
        if (MODE == 0 && a.ps > 0) {
            // PixelShuffle(2): channels oc0..oc0+3 are output channel oc0/4 at
            // sub-positions (i, j) = (0,0), (0,1), (1,0), (1,1).
            const int c = oc0 / 4;
            if (oc0 + 3 >= a.cout) continue;
            if (a.ps_out) {
                for (int ij = 0; ij < 4; ++ij) {
                    const int Y = 2 * y + (ij >> 1), X = 2 * xx + (ij & 1);
                    float o = v[ij] + skip_value(a, c, Y, X, a.skip_scale, a.skip_h, a.skip_w);
                    a.ps_out[(int64_t)c * a.ps_pitch * (2 * H) + (int64_t)Y * a.ps_pitch + X] = o;
                }
            } else {
                float *yo = (float *)a.y + (int64_t)img * (a.cout / 4) * 4 * HW;
                for (int ij = 0; ij < 4; ++ij) {
                    const int Y = 2 * y + (ij >> 1), X = 2 * xx + (ij & 1);
                    float o = v[ij];
                    if (a.ps_act == 1) o = lrelu(o);
                    yo[(((int64_t)(c / 4) * (2 * H) + Y) * (2 * W) + X) * 4 + (c % 4)] = o;
                }
            }
            continue;
        }
        const int64_t off = (int64_t)img * (cout_pad / 4) * HW + (int64_t)(oc0 / 4) * HW +
                            (int64_t)y * W + xx;
        if (MODE == 0 && a.res) {
            const float4 r = reinterpret_cast<const float4 *>(a.res)[off];
            v[0] += r.x; v[1] += r.y; v[2] += r.z; v[3] += r.w;
        }
        yout[off] = make_float4(v[0], v[1], v[2], v[3]);
    }
}

template <int NB, int KS, int MODE>
cudaError_t launch_nb(const ConvArgs &a, const DcnArgs &d, int H, int W, int nimg, int cout_pad,
                      cudaStream_t st) {
    constexpr int KK = KS * KS;
    constexpr int APX = (MODE == 0) ? (KS == 3 ? 132 : 128) : 128;
    constexpr int AROWS = (MODE == 0) ? KS : KK;
    constexpr size_t smem = sizeof(float) * (8 * AROWS * APX + 8 * KK * NB);
    static bool configured = false;
    if (!configured) {
        cudaError_t e = cudaFuncSetAttribute(conv_simt_kernel<NB, KS, MODE>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        configured = true;
    }
    dim3 grid(((W + TW - 1) / TW) * H * nimg, cout_pad / NB);
    conv_simt_kernel<NB, KS, MODE><<<grid, 16 * NB / 4, smem, st>>>(a, d);
    return cudaGetLastError();
}

}  // namespace

size_t simt_weight_bytes(int cin_pad, int cout_pad, int k) {
    return (size_t)cin_pad * k * k * cout_pad * sizeof(float);
}

void prepare_weights_simt(const float *w, int cout, int cin, int k, int cin_pad, int cout_pad, float *dst) {
    const int kk = k * k;
    for (size_t i = 0; i < (size_t)cin_pad * kk * cout_pad; ++i) dst[i] = 0.f;
    for (int o = 0; o < cout; ++o)
        for (int c = 0; c < cin; ++c)
            for (int t = 0; t < kk; ++t)
                dst[((size_t)c * kk + t) * cout_pad + o] = w[((size_t)o * cin + c) * kk + t];
}

cudaError_t launch_conv_simt(const ConvArgs &a, cudaStream_t st) {
    if (a.rq.on) return cudaErrorNotSupported;  // requantise is fused into tensor-core tails only
    DcnArgs d{};
    if (a.cin_pad % 8 || a.cout_pad % 16) return cudaErrorInvalidValue;
    const int nb = a.cout_pad % 64 == 0 ? 64 : (a.cout_pad % 32 == 0 ? 32 : 16);
    const int use_nb = a.ps > 0 ? 16 : nb;  // PixelShuffle epilogue groups 4 channels per thread
    if (a.k == 3) {
        if (use_nb == 64) return launch_nb<64, 3, 0>(a, d, a.H, a.W, a.nimg, a.cout_pad, st);
        if (use_nb == 32) return launch_nb<32, 3, 0>(a, d, a.H, a.W, a.nimg, a.cout_pad, st);
        return launch_nb<16, 3, 0>(a, d, a.H, a.W, a.nimg, a.cout_pad, st);
    }
    if (a.k == 1) {
        if (use_nb == 64) return launch_nb<64, 1, 0>(a, d, a.H, a.W, a.nimg, a.cout_pad, st);
        if (use_nb == 32) return launch_nb<32, 1, 0>(a, d, a.H, a.W, a.nimg, a.cout_pad, st);
        return launch_nb<16, 1, 0>(a, d, a.H, a.W, a.nimg, a.cout_pad, st);
    }
    return cudaErrorInvalidValue;
}

cudaError_t launch_dcn_simt(const DcnArgs &d, cudaStream_t st) {
    ConvArgs a{};
    if (d.cin_pad % 8 || d.cout_pad % 16 || (d.cin_pad / d.groups) % 4) return cudaErrorInvalidValue;
    const int nb = d.cout_pad % 64 == 0 ? 64 : (d.cout_pad % 32 == 0 ? 32 : 16);
    if (nb == 64) return launch_nb<64, 3, 1>(a, d, d.H, d.W, 1, d.cout_pad, st);
    if (nb == 32) return launch_nb<32, 3, 1>(a, d, d.H, d.W, 1, d.cout_pad, st);
    return launch_nb<16, 3, 1>(a, d, d.H, d.W, 1, d.cout_pad, st);
}

}  // namespace nvisr
