// Ingest, requantise and layout kernels: the format side of the hot path.
//
// Ingest turns the integer Y'CbCr planes NNVISR receives from the host
// framework into the float R'G'B' frame an RGB network consumes, and
// requantise turns the network's float output back into integer planes
// (Section 3.1: RGB and YUV pixel formats, YUV420 halving two of the three
// channels, colour-space-aware processing).  Conventions (ITU-T H.273 /
// BT.709, read into the paper, which fixes no numbers):
//   limited: Y' = (Y - 16m)/(219m), C' = (C - 128m)/(224m), m = 2^(b-8)
//   full:    Y' = Y/(2^b - 1),       C' = (C - 2^(b-1))/(2^b - 1)
//   R = Y' + 2(1-Kr)Cr', B = Y' + 2(1-Kb)Cb', G = (Y' - Kr R - Kb B)/Kg
//   Kr = 0.2126, Kb = 0.0722 (BT.709); no clamping in float.
//   4:2:0 siting: LEFT = co-sited columns / centred rows, CENTER = centred
//   both ways, POINT = replicate; downsampling: LEFT = [1 2 1]/4 on columns
//   and row-pair mean, CENTER/POINT = 2x2 mean.  Edges clamp.
//   Quantisation: round half to even, clamp to [0, 2^b - 1].
// Both kernels are HBM-bound streaming passes: each thread handles four
// consecutive pixels (ingest) or a 2x8 luma block (requantise 4:2:0) with
// vector loads/stores along rows.
#include "common.cuh"
#include "rq_math.cuh"
#include "sm100_ptx.cuh"

namespace nvisr {

namespace {


struct RangeConst {
    float y_off, y_den, c_off, c_den;  // normalise: (v - off) / den
    float y_mul, y_add, c_mul, c_add;  // scale back: v * mul + add
    float vmax;
    float y_rden, c_rden;              // 1 / den (the streaming kernels multiply)
    // colour matrix (BT.709 or BT.2020 non-constant luminance): luma weights and
    // the derived factors 2(1 - Kr), 2(1 - Kb), 1 / Kg, 1 / (2(1 - Kb)), 1 / (2(1 - Kr))
    float kr, kb, kg, cr_r, cb_b, rkg, cb_s, cr_s;
    int yuv;  // the network sees Y'Cb'Cr' planes: no matrix either way
    int transfer;  // nvisr_transfer: the network sees linear light (PQ / HLG)
};

RangeConst range_const(int bits, int range, int matrix, int yuv, int transfer) {
    RangeConst r;
    r.yuv = yuv;
    r.transfer = transfer;
    r.kr = matrix == NVISR_MATRIX_BT2020 ? 0.2627f : 0.2126f;
    r.kb = matrix == NVISR_MATRIX_BT2020 ? 0.0593f : 0.0722f;
    r.kg = 1.0f - r.kr - r.kb;
    r.cr_r = 2.0f * (1.0f - r.kr);
    r.cb_b = 2.0f * (1.0f - r.kb);
    r.rkg = 1.0f / r.kg;
    r.cb_s = 1.0f / (2.0f * (1.0f - r.kb));
    r.cr_s = 1.0f / (2.0f * (1.0f - r.kr));
    if (range == NVISR_RANGE_LIMITED) {
        float m = (float)(1 << (bits - 8));
        r.y_off = 16.f * m; r.y_den = 219.f * m; r.c_off = 128.f * m; r.c_den = 224.f * m;
        r.y_mul = 219.f * m; r.y_add = 16.f * m; r.c_mul = 224.f * m; r.c_add = 128.f * m;
    } else {
        float top = (float)((1 << bits) - 1);
        r.y_off = 0.f; r.y_den = top; r.c_off = (float)(1 << (bits - 1)); r.c_den = top;
        r.y_mul = top; r.y_add = 0.f; r.c_mul = top; r.c_add = (float)(1 << (bits - 1));
    }
    if (matrix == NVISR_MATRIX_RGB) {
        // R'G'B' planes: every channel takes the luma range equations, no matrix
        r.c_off = r.y_off; r.c_den = r.y_den; r.c_mul = r.y_mul; r.c_add = r.y_add;
        r.yuv = 1;
    }
    r.vmax = (float)((1 << bits) - 1);
    r.y_rden = 1.0f / r.y_den;
    r.c_rden = 1.0f / r.c_den;
    return r;
}

// HDR transfer (SMPTE ST 2084 PQ, BT.2100 HLG), float32.  to_linear: coded R'G'B' value,
// clamped to [0, 1] (where the functions are defined; the PQ EOTF has a pole above 1) ->
// linear light; from_linear: linear light, clamped to [0, 1] -> coded value.  Not inlined:
// each kernel calls them at many sites, and only HDR formats take that branch, so one
// out-of-line copy keeps the common (SDR) code of the format kernels small.
constexpr float PQ_M1 = 2610.f / 16384.f, PQ_M2 = 2523.f / 4096.f * 128.f;
constexpr float PQ_C1 = 3424.f / 4096.f, PQ_C2 = 2413.f / 4096.f * 32.f, PQ_C3 = 2392.f / 4096.f * 32.f;
constexpr float HLG_A = 0.17883277f, HLG_B = 1.f - 4.f * HLG_A, HLG_C = 0.55991073f;

__device__ __noinline__ float to_linear(int tf, float e) {
    if (tf == NVISR_TRANSFER_NONE) return e;
    e = fminf(fmaxf(e, 0.f), 1.f);
    if (tf == NVISR_TRANSFER_PQ) {
        const float ep = powf(e, 1.f / PQ_M2);
        return powf(fmaxf(ep - PQ_C1, 0.f) / (PQ_C2 - PQ_C3 * ep), 1.f / PQ_M1);
    }
    if (tf == NVISR_TRANSFER_HLG) return e <= 0.5f ? e * e / 3.f : (expf((e - HLG_C) / HLG_A) + HLG_B) / 12.f;
    return e;
}

__device__ __noinline__ float from_linear(int tf, float l) {
    if (tf == NVISR_TRANSFER_PQ) {
        const float ym = powf(fminf(fmaxf(l, 0.f), 1.f), PQ_M1);
        return powf((PQ_C1 + PQ_C2 * ym) / (1.f + PQ_C3 * ym), PQ_M2);
    }
    if (tf == NVISR_TRANSFER_HLG) {
        const float e = fminf(fmaxf(l, 0.f), 1.f);
        return e <= 1.f / 12.f ? sqrtf(3.f * e) : HLG_A * logf(12.f * e - HLG_B) + HLG_C;
    }
    return l;
}

template <typename S>
__device__ __forceinline__ float ld_sample(const S *row, int i) { return (float)row[i]; }

__device__ __forceinline__ int clampi(int v, int lo, int hi) { return v < lo ? lo : (v > hi ? hi : v); }

// Normalised chroma at chroma (row j, col i) (clamped indices).
template <typename S>
__device__ __forceinline__ float chroma_at(const uint8_t *base, int64_t pitch, int Hc, int Wc,
                                           int j, int i, float off, float den) {
    j = clampi(j, 0, Hc - 1);
    i = clampi(i, 0, Wc - 1);
    const S *row = reinterpret_cast<const S *>(base + (int64_t)j * pitch);
    return (ld_sample(row, i) - off) / den;
}

// Vertically interpolated chroma column i for luma row y (4:2:0).
template <typename S>
__device__ __forceinline__ float chroma_v(const uint8_t *base, int64_t pitch, int Hc, int Wc,
                                          int y, int i, int loc, float off, float den) {
    const int j = y >> 1;
    const float c0 = chroma_at<S>(base, pitch, Hc, Wc, j, i, off, den);
    if (loc == NVISR_CHROMA_POINT) return c0;
    const int jn = (y & 1) ? j + 1 : j - 1;
    const float c1 = chroma_at<S>(base, pitch, Hc, Wc, jn, i, off, den);
    return 0.75f * c0 + 0.25f * c1;
}

// Full-resolution chroma at luma (y, x) for 4:2:0, given the format siting.
template <typename S>
__device__ __forceinline__ float chroma_up(const uint8_t *base, int64_t pitch, int Hc, int Wc,
                                           int y, int x, int loc, float off, float den) {
    const int i = x >> 1;
    const float v0 = chroma_v<S>(base, pitch, Hc, Wc, y, i, loc, off, den);
    if (loc == NVISR_CHROMA_POINT) return v0;
    if (loc == NVISR_CHROMA_LEFT) {
        if ((x & 1) == 0) return v0;
        const float v1 = chroma_v<S>(base, pitch, Hc, Wc, y, i + 1, loc, off, den);
        return 0.5f * (v0 + v1);
    }
    const int in = (x & 1) ? i + 1 : i - 1;  // CENTER
    const float v1 = chroma_v<S>(base, pitch, Hc, Wc, y, in, loc, off, den);
    return 0.75f * v0 + 0.25f * v1;
}

template <typename S>
__global__ void __launch_bounds__(256) ingest_kernel(
    const uint8_t *__restrict__ yp, int64_t py, const uint8_t *__restrict__ up, int64_t pu,
    const uint8_t *__restrict__ vp, int64_t pv, int H, int W, int sub420, int loc, RangeConst rc,
    float *__restrict__ out, int64_t pitch) {
    const int qx = blockIdx.x * blockDim.x + threadIdx.x;  // quad of 4 pixels
    const int y = blockIdx.y;
    const int x0 = qx * 4;
    if (x0 >= W) return;
    const int Hc = sub420 ? H / 2 : H, Wc = sub420 ? W / 2 : W;
    const S *yrow = reinterpret_cast<const S *>(yp + (int64_t)y * py);
    float r[4], g[4], b[4];
#pragma unroll
    for (int e = 0; e < 4; ++e) {
        const int x = min(x0 + e, W - 1);
        const float Y = (ld_sample(yrow, x) - rc.y_off) / rc.y_den;
        float cb, cr;
        if (sub420) {
            cb = chroma_up<S>(up, pu, Hc, Wc, y, x, loc, rc.c_off, rc.c_den);
            cr = chroma_up<S>(vp, pv, Hc, Wc, y, x, loc, rc.c_off, rc.c_den);
        } else {
            cb = chroma_at<S>(up, pu, Hc, Wc, y, x, rc.c_off, rc.c_den);
            cr = chroma_at<S>(vp, pv, Hc, Wc, y, x, rc.c_off, rc.c_den);
        }
        if (rc.yuv) {
            r[e] = Y;
            g[e] = cb;
            b[e] = cr;
        } else {
            r[e] = Y + rc.cr_r * cr;
            b[e] = Y + rc.cb_b * cb;
            g[e] = (Y - rc.kr * r[e] - rc.kb * b[e]) / rc.kg;
        }
        if (rc.transfer) {
            r[e] = to_linear(rc.transfer, r[e]);
            g[e] = to_linear(rc.transfer, g[e]);
            b[e] = to_linear(rc.transfer, b[e]);
        }
    }
    const int64_t plane = pitch * H;
    float *o = out + (int64_t)y * pitch + x0;
    const bool vec = (x0 + 4 <= W) && ((reinterpret_cast<uintptr_t>(o) & 15) == 0) && (pitch % 4 == 0);
    if (vec) {
        *reinterpret_cast<float4 *>(o) = make_float4(r[0], r[1], r[2], r[3]);
        *reinterpret_cast<float4 *>(o + plane) = make_float4(g[0], g[1], g[2], g[3]);
        *reinterpret_cast<float4 *>(o + 2 * plane) = make_float4(b[0], b[1], b[2], b[3]);
    } else {
        for (int e = 0; e < 4 && x0 + e < W; ++e) {
            o[e] = r[e];
            o[plane + e] = g[e];
            o[2 * plane + e] = b[e];
        }
    }
}

// 4:2:0 ingest, one thread per luma row 2j + blockIdx.z and 8 columns (4 chroma
// columns): the chroma rows j-1 .. j+1 and columns 4q-1 .. 4q+4 it needs are
// read into registers (normalised), then every luma sample's chroma is
// interpolated from them in the same order as the scalar form (vertical, then
// horizontal), and the three planes are written with 16-byte stores.
// Divisions are replaced by multiplications with the reciprocal.  (One row
// per thread rather than the chroma row's two doubles the threads of this
// short, latency-bound pass; the repeated chroma reads hit L2.)
template <typename S>
__global__ void __launch_bounds__(128) ingest420_kernel(
    const uint8_t *__restrict__ yp, int64_t py, const uint8_t *__restrict__ up, int64_t pu,
    const uint8_t *__restrict__ vp, int64_t pv, int H, int W, int loc, RangeConst rc,
    float *__restrict__ out, int64_t pitch) {
    // launched as a dependent: the ring slot may still be read by the stream's previous kernel
    griddep_wait();
    griddep_launch_dependents();
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y;
    const int x0 = q * 8;
    if (x0 >= W) return;
    const int Hc = H / 2, Wc = W / 2;
    float cu[3][6], cv[3][6];
    // chroma columns 4q .. 4q+3 as one 4-sample load when inside the row and aligned
    const bool cvec = 4 * q + 3 <= Wc - 1 && ((pu | pv) % (4 * (int64_t)sizeof(S))) == 0 &&
                      ((reinterpret_cast<uintptr_t>(up) | reinterpret_cast<uintptr_t>(vp)) % (4 * sizeof(S))) == 0;
    auto load4 = [&](const S *r, float *dst) {
        float t[4];
        if (sizeof(S) == 2) {
            const uint2 w = __ldg(reinterpret_cast<const uint2 *>(r));
            t[0] = (float)(w.x & 0xffffu); t[1] = (float)(w.x >> 16); t[2] = (float)(w.y & 0xffffu); t[3] = (float)(w.y >> 16);
        } else {
            const uint32_t w = __ldg(reinterpret_cast<const uint32_t *>(r));
            t[0] = (float)(w & 0xffu); t[1] = (float)((w >> 8) & 0xffu); t[2] = (float)((w >> 16) & 0xffu); t[3] = (float)(w >> 24);
        }
#pragma unroll
        for (int k = 0; k < 4; ++k) dst[k] = (t[k] - rc.c_off) * rc.c_rden;
    };
#pragma unroll
    for (int rr = 0; rr < 3; ++rr) {
        const int row = clampi(j - 1 + rr, 0, Hc - 1);
        const S *ur = reinterpret_cast<const S *>(up + (int64_t)row * pu);
        const S *vr = reinterpret_cast<const S *>(vp + (int64_t)row * pv);
        if (cvec) {
            load4(ur + 4 * q, &cu[rr][1]);
            load4(vr + 4 * q, &cv[rr][1]);
#pragma unroll
            for (int cc = 0; cc < 6; cc += 5) {
                const int col = clampi(4 * q - 1 + cc, 0, Wc - 1);
                cu[rr][cc] = ((float)__ldg(ur + col) - rc.c_off) * rc.c_rden;
                cv[rr][cc] = ((float)__ldg(vr + col) - rc.c_off) * rc.c_rden;
            }
        } else {
#pragma unroll
            for (int cc = 0; cc < 6; ++cc) {
                const int col = clampi(4 * q - 1 + cc, 0, Wc - 1);
                cu[rr][cc] = ((float)__ldg(ur + col) - rc.c_off) * rc.c_rden;
                cv[rr][cc] = ((float)__ldg(vr + col) - rc.c_off) * rc.c_rden;
            }
        }
    }
    const int64_t plane = pitch * H;
    const bool vec = x0 + 8 <= W && (pitch & 3) == 0 && (reinterpret_cast<uintptr_t>(out) & 15) == 0;
    {
        const int a = blockIdx.z;
        const int y = 2 * j + a;
        if (y >= H) return;
        // vertical interpolation: luma row 2j uses chroma rows (j, j-1), row 2j+1 uses (j, j+1)
        float vu[6], vvv[6];
#pragma unroll
        for (int cc = 0; cc < 6; ++cc) {
            if (loc == NVISR_CHROMA_POINT) {
                vu[cc] = cu[1][cc];
                vvv[cc] = cv[1][cc];
            } else {
                vu[cc] = 0.75f * cu[1][cc] + 0.25f * cu[a ? 2 : 0][cc];
                vvv[cc] = 0.75f * cv[1][cc] + 0.25f * cv[a ? 2 : 0][cc];
            }
        }
        const S *yr = reinterpret_cast<const S *>(yp + (int64_t)y * py);
        float ys[8];
        if (x0 + 8 <= W && (reinterpret_cast<uintptr_t>(yr + x0) & (8 * sizeof(S) - 1)) == 0) {
            if (sizeof(S) == 2) {
                const uint4 w = __ldg(reinterpret_cast<const uint4 *>(yr + x0));
                const uint32_t ww[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    ys[2 * k] = (float)(ww[k] & 0xffffu);
                    ys[2 * k + 1] = (float)(ww[k] >> 16);
                }
            } else {
                const uint2 w = __ldg(reinterpret_cast<const uint2 *>(yr + x0));
                const uint32_t ww[2] = {w.x, w.y};
#pragma unroll
                for (int k = 0; k < 8; ++k) ys[k] = (float)((ww[k >> 2] >> (8 * (k & 3))) & 0xffu);
            }
        } else {
#pragma unroll
            for (int e = 0; e < 8; ++e) ys[e] = (float)__ldg(yr + min(x0 + e, W - 1));
        }
        float r[8], g[8], b[8];
#pragma unroll
        for (int e = 0; e < 8; ++e) {
            const int li = (e >> 1) + 1;  // local index of chroma column x >> 1
            float cb, cr;
            if (loc == NVISR_CHROMA_LEFT) {
                cb = (e & 1) ? 0.5f * (vu[li] + vu[li + 1]) : vu[li];
                cr = (e & 1) ? 0.5f * (vvv[li] + vvv[li + 1]) : vvv[li];
            } else if (loc == NVISR_CHROMA_CENTER) {
                cb = (e & 1) ? 0.75f * vu[li] + 0.25f * vu[li + 1] : 0.75f * vu[li] + 0.25f * vu[li - 1];
                cr = (e & 1) ? 0.75f * vvv[li] + 0.25f * vvv[li + 1] : 0.75f * vvv[li] + 0.25f * vvv[li - 1];
            } else {
                cb = vu[li];
                cr = vvv[li];
            }
            const float Y = (ys[e] - rc.y_off) * rc.y_rden;
            if (rc.yuv) {
                r[e] = Y;
                g[e] = cb;
                b[e] = cr;
            } else {
                r[e] = Y + rc.cr_r * cr;
                b[e] = Y + rc.cb_b * cb;
                g[e] = (Y - rc.kr * r[e] - rc.kb * b[e]) * rc.rkg;
            }
            if (rc.transfer) {
                r[e] = to_linear(rc.transfer, r[e]);
                g[e] = to_linear(rc.transfer, g[e]);
                b[e] = to_linear(rc.transfer, b[e]);
            }
        }
        float *o = out + (int64_t)y * pitch + x0;
        if (vec) {
            *reinterpret_cast<float4 *>(o) = make_float4(r[0], r[1], r[2], r[3]);
            *reinterpret_cast<float4 *>(o + 4) = make_float4(r[4], r[5], r[6], r[7]);
            *reinterpret_cast<float4 *>(o + plane) = make_float4(g[0], g[1], g[2], g[3]);
            *reinterpret_cast<float4 *>(o + plane + 4) = make_float4(g[4], g[5], g[6], g[7]);
            *reinterpret_cast<float4 *>(o + 2 * plane) = make_float4(b[0], b[1], b[2], b[3]);
            *reinterpret_cast<float4 *>(o + 2 * plane + 4) = make_float4(b[4], b[5], b[6], b[7]);
        } else {
#pragma unroll
            for (int e = 0; e < 8; ++e) {
                if (x0 + e >= W) break;
                o[e] = r[e];
                o[plane + e] = g[e];
                o[2 * plane + e] = b[e];
            }
        }
    }
}

template <typename S>
__device__ __forceinline__ void st_sample(uint8_t *base, int64_t pitch, int y, int x, float v) {
    reinterpret_cast<S *>(base + (int64_t)y * pitch)[x] = (S)(int)v;
}

// Bilinear blend of the corners (row 0: a00, a01; row 1: a10, a11) at fractions (lx, ly).
__device__ __forceinline__ float bilerp(float a00, float a01, float a10, float a11, float lx, float ly) {
    return rq_bilerp(a00, a01, a10, a11, lx, ly);
}

// Skip value (mean of the skip frames, upsampled) at output (c, Y, X).
__device__ __forceinline__ float skip_at(const SkipArgs &k, int c, int Y, int X) {
    float acc = 0.f;
    for (int f = 0; f < k.n; ++f) {
        const float *p = k.src[f] + (int64_t)c * k.plane;
        float v;
        const int sv = k.scale_y > 0 ? k.scale_y : k.scale;  // vertical scale
        if (k.mode == 1) {
            v = p[(int64_t)(Y / sv) * k.pitch + X / k.scale];
        } else {
            const float inv = 1.0f / (float)k.scale, inv_y = 1.0f / (float)sv;
            const float sy = fmaxf(((float)Y + 0.5f) * inv_y - 0.5f, 0.f);
            const float sx = fmaxf(((float)X + 0.5f) * inv - 0.5f, 0.f);
            const int y0 = min((int)sy, k.h - 1), x0 = min((int)sx, k.w - 1);
            const int y1 = min(y0 + 1, k.h - 1), x1 = min(x0 + 1, k.w - 1);
            const float ly = sy - (float)y0, lx = sx - (float)x0;
            const float *r0 = p + (int64_t)y0 * k.pitch;
            const float *r1 = p + (int64_t)y1 * k.pitch;
            v = bilerp(r0[x0], r0[x1], r1[x0], r1[x1], lx, ly);
        }
        acc = __fadd_rn(acc, v);
    }
    return k.n == 2 ? acc * 0.5f : acc;
}

// Network output sample (residual + skip) of channel c at (Y, X).
__device__ __forceinline__ float out_at(const float *in, int64_t pitch, int64_t plane, const SkipArgs &k, int c,
                                        int Y, int X) {
    const float v = in[(int64_t)c * plane + (int64_t)Y * pitch + X];
    return k.n ? __fadd_rn(v, skip_at(k, c, Y, X)) : v;
}

__device__ __forceinline__ void rgb2ycc(const RangeConst &rc, float r, float g, float b, float &y, float &cb,
                                        float &cr) {
    if (rc.transfer) {
        r = from_linear(rc.transfer, r);
        g = from_linear(rc.transfer, g);
        b = from_linear(rc.transfer, b);
    }
    if (rc.yuv) {  // channels are Y'Cb'Cr' (or R'G'B' planes) already
        y = r;
        cb = g;
        cr = b;
        return;
    }
    rq_ycc(r, g, b, rc.kr, rc.kg, rc.kb, rc.cb_s, rc.cr_s, y, cb, cr);
}

// 4:4:4: one thread per 4 pixels of a row.
template <typename S>
__global__ void __launch_bounds__(256) requant444_kernel(const float *__restrict__ in, int64_t pitch,
                                                         int H, int W, RangeConst rc, uint8_t *yp,
                                                         int64_t py, uint8_t *up, int64_t pu,
                                                         uint8_t *vp, int64_t pv, const __grid_constant__ SkipArgs sk) {
    const int x0 = (blockIdx.x * blockDim.x + threadIdx.x) * 4;
    const int y = blockIdx.y;
    if (x0 >= W) return;
    const int64_t plane = pitch * H;
    for (int e = 0; e < 4 && x0 + e < W; ++e) {
        float Y, cb, cr;
        rgb2ycc(rc, out_at(in, pitch, plane, sk, 0, y, x0 + e), out_at(in, pitch, plane, sk, 1, y, x0 + e),
                out_at(in, pitch, plane, sk, 2, y, x0 + e), Y, cb, cr);
        st_sample<S>(yp, py, y, x0 + e, rq_code(Y, rc.y_mul, rc.y_add, rc.vmax));
        st_sample<S>(up, pu, y, x0 + e, rq_code(cb, rc.c_mul, rc.c_add, rc.vmax));
        st_sample<S>(vp, pv, y, x0 + e, rq_code(cr, rc.c_mul, rc.c_add, rc.vmax));
    }
}

// 4:2:0: one thread per (chroma row j, 4 chroma columns): luma rows 2j, 2j+1,
// columns 8q .. 8q+7; chroma needs columns 8q-1 .. 8q+7 for LEFT siting.  The
// network output of those 2 x 9 pixels is loaded once (two 16-byte loads and
// one scalar per row and channel when the rows are 16-byte aligned), luma is
// written with one 8- or 16-byte store per row and chroma with one per plane.
// SKS = 2: the skip is one frame upsampled 2x bilinearly (align_corners = false,
// edge clamp).  Output rows 2j, 2j+1 and columns 8q-1 .. 8q+7 then read
// low-resolution rows j-1 .. j+1 and columns 4q-1 .. 4q+4 (clamped), loaded
// once into registers; every output sample blends two rows and two columns
// with the fixed weights 1/4, 3/4 in the same order as the general formula.
// SKS = 4: the mean of NF frames upsampled 4x bilinearly.  Both output rows
// blend the same two low-resolution rows, and columns 8q-1 .. 8q+7 blend
// columns 2q-1 .. 2q+2 with the fractions 3/8, 5/8, 7/8, 1/8, ... that the
// general formula gives exactly; those 2 x 4 values per channel and frame are
// loaded once, at columns clamped to the image.  At the right edge this is the
// general formula's arithmetic; at the left edge, where the formula clamps the
// position to column 0, it blends two copies of column 0 (within one FP32 ulp
// of it).  Columns past W - 1 are computed but never stored.
template <typename S, int SKS, int NF>
__global__ void __launch_bounds__(128) requant420_kernel(const float *__restrict__ in, int64_t pitch,
                                                         int H, int W, int loc, RangeConst rc,
                                                         uint8_t *yp, int64_t py, uint8_t *up,
                                                         int64_t pu, uint8_t *vp, int64_t pv, const __grid_constant__ SkipArgs sk) {
    // launched as a dependent: the network output comes from the stream's previous kernel
    griddep_wait();
    griddep_launch_dependents();
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y;
    const int xb = q * 8;
    if (xb >= W) return;
    const int64_t plane = pitch * H;
    const int Wc = W / 2;
    // px[ch][a][c9]: network output of channel ch, row 2j + a, column xb - 1 + c9 (clamped)
    float px[3][2][9];
    const bool vin = xb + 8 <= W && (pitch & 3) == 0 && (reinterpret_cast<uintptr_t>(in) & 15) == 0;
#pragma unroll
    for (int ch = 0; ch < 3; ++ch)
#pragma unroll
        for (int a = 0; a < 2; ++a) {
            const float *row = in + (int64_t)ch * plane + (int64_t)(2 * j + a) * pitch;
            px[ch][a][0] = __ldg(row + clampi(xb - 1, 0, W - 1));
            if (vin) {
                const float4 v0 = __ldg(reinterpret_cast<const float4 *>(row + xb));
                const float4 v1 = __ldg(reinterpret_cast<const float4 *>(row + xb + 4));
                px[ch][a][1] = v0.x; px[ch][a][2] = v0.y; px[ch][a][3] = v0.z; px[ch][a][4] = v0.w;
                px[ch][a][5] = v1.x; px[ch][a][6] = v1.y; px[ch][a][7] = v1.z; px[ch][a][8] = v1.w;
            } else {
#pragma unroll
                for (int c = 1; c < 9; ++c) px[ch][a][c] = __ldg(row + clampi(xb - 1 + c, 0, W - 1));
            }
        }
    constexpr bool SKIP2 = SKS == 2;
    float lr[SKIP2 ? 3 : 1][3][6];
    float l4[SKS == 4 ? NF : 1][3][2][4];
    float ly4[2] = {0.f, 0.f};
    if (SKS == 4) {
        int r0 = 0, r1 = 0;
#pragma unroll
        for (int a = 0; a < 2; ++a) {
            // the general formula; rows 2j and 2j + 1 give the same (y0, y1)
            const float sy = fmaxf(((float)(2 * j + a) + 0.5f) * 0.25f - 0.5f, 0.f);
            const int y0 = min((int)sy, sk.h - 1);
            ly4[a] = sy - (float)y0;
            if (a == 0) {
                r0 = y0;
                r1 = min(y0 + 1, sk.h - 1);
            }
        }
        int lc[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) lc[i] = clampi(2 * q - 1 + i, 0, sk.w - 1);
#pragma unroll
        for (int f = 0; f < NF; ++f)
#pragma unroll
            for (int c = 0; c < 3; ++c)
#pragma unroll
                for (int rr = 0; rr < 2; ++rr) {
                    const float *row = sk.src[f] + (int64_t)c * sk.plane + (int64_t)(rr ? r1 : r0) * sk.pitch;
#pragma unroll
                    for (int i = 0; i < 4; ++i) l4[f][c][rr][i] = __ldg(row + lc[i]);
                }
    }
    if (SKIP2) {
        const bool svec = 4 * q + 3 <= sk.w - 1 && (sk.pitch & 3) == 0 && (sk.plane & 3) == 0 &&
                          (reinterpret_cast<uintptr_t>(sk.src[0]) & 15) == 0;
#pragma unroll
        for (int c = 0; c < 3; ++c)
#pragma unroll
            for (int rr = 0; rr < 3; ++rr) {
                const float *row = sk.src[0] + (int64_t)c * sk.plane + (int64_t)clampi(j - 1 + rr, 0, sk.h - 1) * sk.pitch;
                if (svec) {
                    const float4 m = __ldg(reinterpret_cast<const float4 *>(row + 4 * q));
                    lr[c][rr][0] = __ldg(row + max(4 * q - 1, 0));
                    lr[c][rr][1] = m.x; lr[c][rr][2] = m.y; lr[c][rr][3] = m.z; lr[c][rr][4] = m.w;
                    lr[c][rr][5] = __ldg(row + min(4 * q + 4, sk.w - 1));
                } else {
#pragma unroll
                    for (int cc = 0; cc < 6; ++cc) lr[c][rr][cc] = __ldg(row + clampi(4 * q - 1 + cc, 0, sk.w - 1));
                }
            }
    }
    // output (row 2j + a, column xb - 1 + c9) of channel ch: residual + skip
    auto sample = [&](int ch, int a, int c9, int x) -> float {
        const float v = px[ch][a][c9];
        if (SKS == 4) {
            const int i0 = (c9 + 1) / 4;                     // column 2q - 1 + i0
            const float lx = (float)((c9 + 1) % 4) * 0.25f + 0.125f;
            float acc = 0.f;
#pragma unroll
            for (int f = 0; f < NF; ++f)
                acc = __fadd_rn(acc, bilerp(l4[f][ch][0][i0], l4[f][ch][0][i0 + 1], l4[f][ch][1][i0],
                                            l4[f][ch][1][i0 + 1], lx, ly4[a]));
            return __fadd_rn(v, NF == 2 ? acc * 0.5f : acc);
        }
        if (!SKIP2) return sk.n ? __fadd_rn(v, skip_at(sk, ch, 2 * j + a, x)) : v;
        // horizontal: even c9 -> odd column 2i+1 (3/4 col i, 1/4 col i+1), odd c9 -> even 2i (1/4 col i-1, 3/4 col i)
        const int c0 = (c9 & 1) ? (c9 - 1) / 2 : c9 / 2;
        const float wl = (c9 & 1) ? 0.25f : 0.75f, wr = (c9 & 1) ? 0.75f : 0.25f;
        const int r0 = a;  // a = 0: rows (j-1, j) with (1/4, 3/4); a = 1: rows (j, j+1) with (3/4, 1/4)
        const float wt = a ? 0.75f : 0.25f, wb = a ? 0.25f : 0.75f;
        const float top = rq_blend(lr[ch][r0][c0], wl, lr[ch][r0][c0 + 1], wr);
        const float bot = rq_blend(lr[ch][r0 + 1][c0], wl, lr[ch][r0 + 1][c0 + 1], wr);
        return __fadd_rn(v, rq_blend(top, wt, bot, wb));
    };
    // columns xb-1 .. xb+7 (9 columns), clamped; two rows.
    float cbv[9], crv[9];  // row-pair mean of full-resolution chroma
    float yq[2][8];
#pragma unroll
    for (int c = 0; c < 9; ++c) {
        const int x = clampi(xb - 1 + c, 0, W - 1);
        float cb2[2], cr2[2];
#pragma unroll
        for (int rr = 0; rr < 2; ++rr) {
            float Y, cb, cr;
            rgb2ycc(rc, sample(0, rr, c, x), sample(1, rr, c, x), sample(2, rr, c, x), Y, cb, cr);
            cb2[rr] = cb;
            cr2[rr] = cr;
            if (c >= 1) yq[rr][c - 1] = rq_code(Y, rc.y_mul, rc.y_add, rc.vmax);
        }
        cbv[c] = rq_mean2(cb2[0], cb2[1]);
        crv[c] = rq_mean2(cr2[0], cr2[1]);
    }
#pragma unroll
    for (int rr = 0; rr < 2; ++rr) {
        S *yrow = reinterpret_cast<S *>(yp + (int64_t)(2 * j + rr) * py) + xb;
        if (xb + 8 <= W && (reinterpret_cast<uintptr_t>(yrow) & (8 * sizeof(S) - 1)) == 0) {
            uint32_t w[4];
            if (sizeof(S) == 2) {
#pragma unroll
                for (int k = 0; k < 4; ++k) w[k] = (uint32_t)(int)yq[rr][2 * k] | ((uint32_t)(int)yq[rr][2 * k + 1] << 16);
                *reinterpret_cast<uint4 *>(yrow) = make_uint4(w[0], w[1], w[2], w[3]);
            } else {
#pragma unroll
                for (int k = 0; k < 2; ++k)
                    w[k] = (uint32_t)(int)yq[rr][4 * k] | ((uint32_t)(int)yq[rr][4 * k + 1] << 8) |
                           ((uint32_t)(int)yq[rr][4 * k + 2] << 16) | ((uint32_t)(int)yq[rr][4 * k + 3] << 24);
                *reinterpret_cast<uint2 *>(yrow) = make_uint2(w[0], w[1]);
            }
        } else {
#pragma unroll
            for (int e = 0; e < 8; ++e)
                if (xb + e < W) yrow[e] = (S)(int)yq[rr][e];
        }
    }
    float cq[2][4];
#pragma unroll
    for (int e = 0; e < 4; ++e) {
        const int c = 1 + 2 * e;  // index of column 2i
        float cb, cr;
        if (loc == NVISR_CHROMA_LEFT) {
            cb = rq_121(cbv[c - 1], cbv[c], cbv[c + 1]);
            cr = rq_121(crv[c - 1], crv[c], crv[c + 1]);
        } else {
            cb = rq_mean2(cbv[c], cbv[c + 1]);
            cr = rq_mean2(crv[c], crv[c + 1]);
        }
        cq[0][e] = rq_code(cb, rc.c_mul, rc.c_add, rc.vmax);
        cq[1][e] = rq_code(cr, rc.c_mul, rc.c_add, rc.vmax);
    }
    const int i0 = q * 4;
#pragma unroll
    for (int pl = 0; pl < 2; ++pl) {
        S *crow = reinterpret_cast<S *>((pl ? vp : up) + (int64_t)j * (pl ? pv : pu)) + i0;
        if (i0 + 4 <= Wc && (reinterpret_cast<uintptr_t>(crow) & (4 * sizeof(S) - 1)) == 0) {
            if (sizeof(S) == 2)
                *reinterpret_cast<uint2 *>(crow) =
                    make_uint2((uint32_t)(int)cq[pl][0] | ((uint32_t)(int)cq[pl][1] << 16),
                               (uint32_t)(int)cq[pl][2] | ((uint32_t)(int)cq[pl][3] << 16));
            else
                *reinterpret_cast<uint32_t *>(crow) = (uint32_t)(int)cq[pl][0] | ((uint32_t)(int)cq[pl][1] << 8) |
                                                      ((uint32_t)(int)cq[pl][2] << 16) | ((uint32_t)(int)cq[pl][3] << 24);
        } else {
#pragma unroll
            for (int e = 0; e < 4; ++e)
                if (i0 + e < Wc) crow[e] = (S)(int)cq[pl][e];
        }
    }
}

template <typename T>
__device__ __forceinline__ T cvt_out(float v);
template <>
__device__ __forceinline__ float cvt_out<float>(float v) { return v; }
template <>
__device__ __forceinline__ __nv_bfloat16 cvt_out<__nv_bfloat16>(float v) { return __float2bfloat16_rn(v); }
template <>
__device__ __forceinline__ __half cvt_out<__half>(float v) { return __float2half_rn(v); }
template <>
__device__ __forceinline__ __nv_fp8_e4m3 cvt_out<__nv_fp8_e4m3>(float v) { return __nv_fp8_e4m3(v); }

template <typename T>
__device__ __forceinline__ float cvt_in(T v) { return (float)v; }
template <>
__device__ __forceinline__ float cvt_in<__nv_bfloat16>(__nv_bfloat16 v) { return __bfloat162float(v); }
template <>
__device__ __forceinline__ float cvt_in<__half>(__half v) { return __half2float(v); }

// One thread per 16-byte unit of the destination, in memory order: unit idx
// is (chunk c, pixel p, unit v of the chunk) with idx = (c*HW + p)*upch + v.
template <typename T>
__global__ void __launch_bounds__(256) pack_kernel(PackArgs a) {
    constexpr int UPC = 16 / sizeof(T);  // channels per unit
    const int64_t HW = (int64_t)a.H * a.W;
    const int upch = a.cpc / UPC;         // units per chunk
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= HW * (a.cpad / UPC)) return;
    const int64_t cp = idx / upch;
    const int v = (int)(idx - cp * upch);
    const int c = (int)(cp / HW);
    const int64_t p = cp - (int64_t)c * HW;
    const int y = (int)(p / a.W), x = (int)(p - (int64_t)y * a.W);
    const int creal = a.nsrc * a.ch_per_src;
    alignas(16) T vals[UPC];
    float amax = 0.f;
#pragma unroll
    for (int e = 0; e < UPC; ++e) {
        const int ch = c * a.cpc + v * UPC + e;
        float val = 0.f;
        if (ch < creal) {
            const int s = ch / a.ch_per_src, cc = ch - s * a.ch_per_src;
            val = a.src[s][cc * a.src_plane + (int64_t)y * a.src_pitch + x];
        }
        amax = fmaxf(amax, fabsf(val));
        vals[e] = cvt_out<T>(val * a.scale);
    }
    *reinterpret_cast<uint4 *>(reinterpret_cast<uint8_t *>(a.dst) + idx * 16) =
        *reinterpret_cast<const uint4 *>(vals);
    if (a.amax) atomicMax(a.amax, __float_as_uint(amax));
}

// 16 bytes of UPC consecutive channels, converted from float.
template <typename T>
__device__ __forceinline__ uint4 pack_unit(const float *v);
template <>
__device__ __forceinline__ uint4 pack_unit<float>(const float *v) {
    return make_uint4(__float_as_uint(v[0]), __float_as_uint(v[1]), __float_as_uint(v[2]), __float_as_uint(v[3]));
}
template <>
__device__ __forceinline__ uint4 pack_unit<__nv_bfloat16>(const float *v) {
    uint32_t w[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const __nv_bfloat162 h = __floats2bfloat162_rn(v[2 * k], v[2 * k + 1]);
        w[k] = *reinterpret_cast<const uint32_t *>(&h);
    }
    return make_uint4(w[0], w[1], w[2], w[3]);
}
template <>
__device__ __forceinline__ uint4 pack_unit<__half>(const float *v) {
    uint32_t w[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const __half2 h = __floats2half2_rn(v[2 * k], v[2 * k + 1]);
        w[k] = *reinterpret_cast<const uint32_t *>(&h);
    }
    return make_uint4(w[0], w[1], w[2], w[3]);
}
template <>
__device__ __forceinline__ uint4 pack_unit<__nv_fp8_e4m3>(const float *v) {
    uint32_t w[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        uint32_t b = 0;
#pragma unroll
        for (int e = 0; e < 4; ++e) b |= (uint32_t)__nv_fp8_e4m3(v[4 * k + e]).__x << (8 * e);
        w[k] = b;
    }
    return make_uint4(w[0], w[1], w[2], w[3]);
}

// Row-tiled pack: one thread per 4 consecutive pixels of a row and all padded
// channels.  Each source channel row segment is one 16-byte load; each
// destination unit of the 4 pixels is one 16-byte store, contiguous across the
// 4 pixels (and across the warp) for every unit index.  Needs 16-byte aligned
// source rows whose pitch covers W rounded up to 4 (the last group of a row
// reads into that padding and stores only pixels < W); otherwise the per-unit
// kernel above runs.
template <typename T>
__device__ __forceinline__ void pack_rows(const PackArgs &a) {
    constexpr int UPC = 16 / sizeof(T);
    const int x0 = (blockIdx.x * blockDim.x + threadIdx.x) * 4;
    const int y = blockIdx.y;
    if (x0 >= a.W || y >= a.H) return;
    const int64_t HW = (int64_t)a.H * a.W;
    const int upch = a.cpc / UPC;
    const int creal = a.nsrc * a.ch_per_src;
    const int64_t p0 = (int64_t)y * a.W + x0;
    float amax = 0.f;
    for (int u = 0; u < a.cpad / UPC; ++u) {  // unit index over all channels
        float v[4][UPC];
#pragma unroll
        for (int e = 0; e < UPC; ++e) {
            const int ch = u * UPC + e;
            float4 f = make_float4(0.f, 0.f, 0.f, 0.f);
            if (ch < creal) {
                const int s = ch / a.ch_per_src, cc = ch - s * a.ch_per_src;
                f = __ldg(reinterpret_cast<const float4 *>(a.src[s] + cc * a.src_plane + (int64_t)y * a.src_pitch + x0));
            }
            amax = fmaxf(amax, fmaxf(fmaxf(fabsf(f.x), fabsf(f.y)), fmaxf(fabsf(f.z), fabsf(f.w))));
            v[0][e] = f.x * a.scale;
            v[1][e] = f.y * a.scale;
            v[2][e] = f.z * a.scale;
            v[3][e] = f.w * a.scale;
        }
        const int c = u / upch, vv = u - c * upch;
        uint8_t *d = reinterpret_cast<uint8_t *>(a.dst) + (((int64_t)c * HW + p0) * upch + vv) * 16;
#pragma unroll
        for (int k = 0; k < 4; ++k)
            if (x0 + k < a.W) *reinterpret_cast<uint4 *>(d + (int64_t)k * upch * 16) = pack_unit<T>(v[k]);
    }
    if (a.amax) {
        const unsigned m = __reduce_max_sync(__activemask(), __float_as_uint(amax));
        if ((threadIdx.x & 31) == (__ffs(__activemask()) - 1)) atomicMax(a.amax, m);
    }
}

template <typename T>
__global__ void __launch_bounds__(128) pack_rows_kernel(const __grid_constant__ PackArgs a) {
    pack_rows<T>(a);
}

// Batched form: blockIdx.z selects one of several packs (e.g. the tuples of
// several streams) whose arguments are read from a device table.
template <typename T>
__global__ void __launch_bounds__(128) pack_rows_table_kernel(const PackArgs *__restrict__ tab) {
    pack_rows<T>(tab[blockIdx.z]);
}

template <typename T>
__global__ void __launch_bounds__(256) unpack_kernel(const uint8_t *__restrict__ src, int cpad, int cpc, int C,
                                                     int H, int W, float scale, float *dst, int64_t pitch) {
    constexpr int UPC = 16 / sizeof(T);
    const int64_t HW = (int64_t)H * W;
    const int upch = cpc / UPC;
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= HW * (cpad / UPC)) return;
    const int64_t cp = idx / upch;
    const int v = (int)(idx - cp * upch);
    const int c = (int)(cp / HW);
    const int64_t p = cp - (int64_t)c * HW;
    const int y = (int)(p / W), x = (int)(p - (int64_t)y * W);
    alignas(16) T vals[UPC];
    *reinterpret_cast<uint4 *>(vals) = *reinterpret_cast<const uint4 *>(src + idx * 16);
#pragma unroll
    for (int e = 0; e < UPC; ++e) {
        const int ch = c * cpc + v * UPC + e;
        if (ch < C) dst[(int64_t)ch * pitch * H + (int64_t)y * pitch + x] = cvt_in<T>(vals[e]) * scale;
    }
}

}  // namespace

namespace {

// One thread per low-resolution pixel: its 3 * ry * rx channels (float32, 4 per 16-byte
// unit) scattered to the ry x rx block of each of the 3 planar output channels.
__global__ void __launch_bounds__(256) shuffle_planar_kernel(const float *__restrict__ src, int H, int W, int ry,
                                                             int rx, float *__restrict__ dst, int64_t dst_pitch) {
    griddep_wait();  // launched as a dependent of the layer that produced src
    griddep_launch_dependents();
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y;
    if (x >= W || y >= H) return;
    const int64_t HW = (int64_t)H * W;
    const int64_t plane = dst_pitch * H * ry;
    for (int c = 0; c < 3; ++c)
        for (int i = 0; i < ry; ++i)
            for (int j = 0; j < rx; ++j) {
                const int ch = (c * ry + i) * rx + j;
                const float v = src[((int64_t)(ch >> 2) * HW + (int64_t)y * W + x) * 4 + (ch & 3)];
                dst[c * plane + (int64_t)(ry * y + i) * dst_pitch + rx * x + j] = v;
            }
}

}  // namespace

cudaError_t launch_shuffle_planar(const float *src, int H, int W, int ry, int rx, float *dst, int64_t dst_pitch,
                                  cudaStream_t st) {
    if (H < 1 || W < 1 || ry < 1 || ry > 2 || rx < 1 || rx > 2 || dst_pitch < (int64_t)W * rx)
        return cudaErrorInvalidValue;
    return launch_dependent(shuffle_planar_kernel, dim3((unsigned)((W + 255) / 256), (unsigned)H), dim3(256), 0, st,
                            src, H, W, ry, rx, dst, dst_pitch);
}

cudaError_t launch_ingest(const nvisr_format &f, const void *y, int64_t py, const void *u, int64_t pu,
                          const void *v, int64_t pv, float *out, int64_t out_pitch, cudaStream_t st, int yuv) {
    const RangeConst rc = range_const(f.bit_depth, f.range, f.matrix, yuv, f.transfer);
    if (f.subsampling == NVISR_SUB_420) {
        dim3 blk(128);
        dim3 grd((f.width + 8 * 128 - 1) / (8 * 128), (f.height + 1) / 2, 2);
        if (f.bit_depth <= 8)
            return launch_dependent(ingest420_kernel<uint8_t>, grd, blk, 0, st, (const uint8_t *)y, py,
                                    (const uint8_t *)u, pu, (const uint8_t *)v, pv, f.height, f.width, f.chroma_loc,
                                    rc, out, out_pitch);
        return launch_dependent(ingest420_kernel<uint16_t>, grd, blk, 0, st, (const uint8_t *)y, py,
                                (const uint8_t *)u, pu, (const uint8_t *)v, pv, f.height, f.width, f.chroma_loc, rc,
                                out, out_pitch);
    }
    dim3 block(64);
    dim3 grid((f.width / 4 + 1 + block.x - 1) / block.x, f.height);
    const int sub = f.subsampling == NVISR_SUB_420;
    if (f.bit_depth <= 8)
        ingest_kernel<uint8_t><<<grid, block, 0, st>>>((const uint8_t *)y, py, (const uint8_t *)u, pu,
                                                       (const uint8_t *)v, pv, f.height, f.width, sub,
                                                       f.chroma_loc, rc, out, out_pitch);
    else
        ingest_kernel<uint16_t><<<grid, block, 0, st>>>((const uint8_t *)y, py, (const uint8_t *)u, pu,
                                                        (const uint8_t *)v, pv, f.height, f.width, sub,
                                                        f.chroma_loc, rc, out, out_pitch);
    return cudaGetLastError();
}

cudaError_t launch_requant(const nvisr_format &f, const float *in, int64_t in_pitch, void *y, int64_t py,
                           void *u, int64_t pu, void *v, int64_t pv, cudaStream_t st, const SkipArgs *skip,
                           int yuv) {
    const RangeConst rc = range_const(f.bit_depth, f.range, f.matrix, yuv, f.transfer);
    SkipArgs sk{};
    if (skip) sk = *skip;
    dim3 block(64);
    if (f.subsampling == NVISR_SUB_420) {
        cudaError_t e = cudaSuccess;
        block = dim3(128);
        dim3 grid((f.width + 8 * 128 - 1) / (8 * 128), f.height / 2);
        const bool iso = sk.scale_y == 0 || sk.scale_y == sk.scale;
        const bool skip2 = iso && sk.n == 1 && sk.mode == 2 && sk.scale == 2 && sk.h * 2 == f.height &&
                           sk.w * 2 == f.width;
        const bool skip4 = iso && (sk.n == 1 || sk.n == 2) && sk.mode == 2 && sk.scale == 4 && sk.h * 4 == f.height &&
                           sk.w * 4 == f.width;
#define NVISR_RQ(S_, K_, N_)                                                                                 \
    e = launch_dependent(requant420_kernel<S_, K_, N_>, grid, block, 0, st, in, in_pitch, f.height, f.width, \
                         f.chroma_loc, rc, (uint8_t *)y, py, (uint8_t *)u, pu, (uint8_t *)v, pv, sk)
#define NVISR_RQ_ALL(S_)                  \
    if (skip2) NVISR_RQ(S_, 2, 1);        \
    else if (skip4 && sk.n == 1) NVISR_RQ(S_, 4, 1); \
    else if (skip4) NVISR_RQ(S_, 4, 2);   \
    else NVISR_RQ(S_, 0, 1)
        if (f.bit_depth <= 8) {
            NVISR_RQ_ALL(uint8_t);
        } else {
            NVISR_RQ_ALL(uint16_t);
        }
#undef NVISR_RQ_ALL
#undef NVISR_RQ
        return e;
    } else {
        dim3 grid((f.width / 4 + 1 + block.x - 1) / block.x, f.height);
        if (f.bit_depth <= 8)
            requant444_kernel<uint8_t><<<grid, block, 0, st>>>(in, in_pitch, f.height, f.width, rc,
                                                               (uint8_t *)y, py, (uint8_t *)u, pu,
                                                               (uint8_t *)v, pv, sk);
        else
            requant444_kernel<uint16_t><<<grid, block, 0, st>>>(in, in_pitch, f.height, f.width, rc,
                                                                (uint8_t *)y, py, (uint8_t *)u, pu,
                                                                (uint8_t *)v, pv, sk);
    }
    return cudaGetLastError();
}

cudaError_t launch_pack(const PackArgs &a0, cudaStream_t st) {
    PackArgs a = a0;
    const int upc = chunk_channels(a.dt);
    if (a.cpc == 0) a.cpc = upc;
    if (a.cpc % upc || a.cpad % a.cpc) return cudaErrorInvalidValue;
    if (pack_rows_fits(a)) {
        dim3 blk(128), grd((a.W / 4 + 127) / 128, a.H);
        switch (a.dt) {
            case DT_F32: pack_rows_kernel<float><<<grd, blk, 0, st>>>(a); break;
            case DT_BF16: pack_rows_kernel<__nv_bfloat16><<<grd, blk, 0, st>>>(a); break;
            case DT_F16: pack_rows_kernel<__half><<<grd, blk, 0, st>>>(a); break;
            default: pack_rows_kernel<__nv_fp8_e4m3><<<grd, blk, 0, st>>>(a); break;
        }
        return cudaGetLastError();
    }
    const int64_t n = (int64_t)a.H * a.W * (a.cpad / upc);
    const int block = 256;
    const int64_t grid = (n + block - 1) / block;
    switch (a.dt) {
        case DT_F32: pack_kernel<float><<<(unsigned)grid, block, 0, st>>>(a); break;
        case DT_BF16: pack_kernel<__nv_bfloat16><<<(unsigned)grid, block, 0, st>>>(a); break;
        case DT_F16: pack_kernel<__half><<<(unsigned)grid, block, 0, st>>>(a); break;
        default: pack_kernel<__nv_fp8_e4m3><<<(unsigned)grid, block, 0, st>>>(a); break;
    }
    return cudaGetLastError();
}

bool pack_rows_fits(const PackArgs &a) {
    const int upc = chunk_channels(a.dt);
    const int cpc = a.cpc ? a.cpc : upc;
    bool ok = a.src_pitch % 4 == 0 && a.src_pitch >= (a.W + 3) / 4 * 4 && a.src_plane % 4 == 0 && cpc % upc == 0 &&
              a.cpad % cpc == 0;
    for (int s = 0; s < a.nsrc; ++s) ok = ok && (reinterpret_cast<uintptr_t>(a.src[s]) & 15) == 0;
    return ok;
}

cudaError_t launch_pack_table(const PackArgs *host_tab, const PackArgs *dev_tab, int n, cudaStream_t st) {
    if (n < 1) return cudaSuccess;
    int maxw = 0, maxh = 0;
    for (int i = 0; i < n; ++i) {
        const PackArgs &a = host_tab[i];
        if (!pack_rows_fits(a) || a.dt != host_tab[0].dt || a.cpc == 0) return cudaErrorInvalidValue;
        maxw = std::max(maxw, a.W);
        maxh = std::max(maxh, a.H);
    }
    dim3 blk(128), grd((maxw / 4 + 127) / 128, maxh, n);
    switch (host_tab[0].dt) {
        case DT_F32: pack_rows_table_kernel<float><<<grd, blk, 0, st>>>(dev_tab); break;
        case DT_BF16: pack_rows_table_kernel<__nv_bfloat16><<<grd, blk, 0, st>>>(dev_tab); break;
        case DT_F16: pack_rows_table_kernel<__half><<<grd, blk, 0, st>>>(dev_tab); break;
        default: pack_rows_table_kernel<__nv_fp8_e4m3><<<grd, blk, 0, st>>>(dev_tab); break;
    }
    return cudaGetLastError();
}

cudaError_t launch_unpack(const void *src, int dt, int cpad, int cpc, int C, int H, int W, float scale, float *dst,
                          int64_t dst_pitch, cudaStream_t st) {
    const int upc = chunk_channels(dt);
    if (cpc == 0) cpc = upc;
    if (cpc % upc || cpad % cpc) return cudaErrorInvalidValue;
    const int64_t n = (int64_t)H * W * (cpad / upc);
    const int block = 256;
    const unsigned grid = (unsigned)((n + block - 1) / block);
    const uint8_t *s = (const uint8_t *)src;
    switch (dt) {
        case DT_F32: unpack_kernel<float><<<grid, block, 0, st>>>(s, cpad, cpc, C, H, W, scale, dst, dst_pitch); break;
        case DT_BF16: unpack_kernel<__nv_bfloat16><<<grid, block, 0, st>>>(s, cpad, cpc, C, H, W, scale, dst, dst_pitch); break;
        case DT_F16: unpack_kernel<__half><<<grid, block, 0, st>>>(s, cpad, cpc, C, H, W, scale, dst, dst_pitch); break;
        default: unpack_kernel<__nv_fp8_e4m3><<<grid, block, 0, st>>>(s, cpad, cpc, C, H, W, scale, dst, dst_pitch); break;
    }
    return cudaGetLastError();
}

// ---------------------------------------------------------------- fused requantise helpers

bool fused_rq_format(const nvisr_format &f, int yuv, FusedRq *rq) {
    if (yuv || f.transfer != NVISR_TRANSFER_NONE || f.matrix == NVISR_MATRIX_RGB) return false;
    const RangeConst rc = range_const(f.bit_depth, f.range, f.matrix, yuv, f.transfer);
    rq->on = 1;
    rq->wide = f.bit_depth > 8;
    rq->sub420 = f.subsampling == NVISR_SUB_420;
    rq->loc = f.chroma_loc;
    rq->y_mul = rc.y_mul;
    rq->y_add = rc.y_add;
    rq->c_mul = rc.c_mul;
    rq->c_add = rc.c_add;
    rq->vmax = rc.vmax;
    rq->kr = rc.kr;
    rq->kg = rc.kg;
    rq->kb = rc.kb;
    rq->cb_s = rc.cb_s;
    rq->cr_s = rc.cr_s;
    return true;
}

namespace {

// One thread per (low-resolution row, 128-pixel tile after the first): the LEFT-sited
// chroma sample at the tile's first column, from the columns the two tiles' CTAs left
// in rq.edge: [k * 6 + 0..3] = this tile's first pixel (Cb' even, Cb' odd, Cr' even,
// Cr' odd column, each the mean of its two rows), [k * 6 + 4..5] = the previous tile's
// last pixel's odd column (Cb', Cr').  The arithmetic is requant420_kernel's.
template <typename S>
__global__ void rq_edge_fixup_kernel(FusedRq rq, int H, int W, int tiles) {
    griddep_wait();  // launched as a dependent of the output layer
    griddep_launch_dependents();
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int n = H * (tiles - 1);
    if (i >= n) return;
    const int o = i / (tiles - 1), t = 1 + i % (tiles - 1);
    const float *e = rq.edge + ((int64_t)o * tiles + t) * 6;
    const float cb = rq_121(e[4], e[0], e[1]);
    const float cr = rq_121(e[5], e[2], e[3]);
    const int x = t * 128;
    reinterpret_cast<S *>(rq.up + (int64_t)o * rq.pu)[x] = (S)(int)rq_code(cb, rq.c_mul, rq.c_add, rq.vmax);
    reinterpret_cast<S *>(rq.vp + (int64_t)o * rq.pv)[x] = (S)(int)rq_code(cr, rq.c_mul, rq.c_add, rq.vmax);
}

}  // namespace

bool rq_edge_fixup_runs(const FusedRq &rq, int W) {
    return rq.on && rq.sub420 && rq.loc == NVISR_CHROMA_LEFT && (W + 127) / 128 >= 2;
}

cudaError_t launch_rq_edge_fixup(const FusedRq &rq, int H, int W, cudaStream_t st) {
    const int tiles = (W + 127) / 128;
    if (!rq_edge_fixup_runs(rq, W)) return cudaSuccess;
    const int n = H * (tiles - 1);
    const dim3 grid((n + 127) / 128), block(128);
    return rq.wide ? launch_dependent(rq_edge_fixup_kernel<uint16_t>, grid, block, 0, st, rq, H, W, tiles)
                   : launch_dependent(rq_edge_fixup_kernel<uint8_t>, grid, block, 0, st, rq, H, W, tiles);
}

}  // namespace nvisr
