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

namespace nvisr {

namespace {

constexpr float KR = 0.2126f;
constexpr float KB = 0.0722f;
constexpr float KG = 1.0f - 0.2126f - 0.0722f;

struct RangeConst {
    float y_off, y_den, c_off, c_den;  // normalise: (v - off) / den
    float y_mul, y_add, c_mul, c_add;  // scale back: v * mul + add
    float vmax;
};

RangeConst range_const(int bits, int range) {
    RangeConst r;
    if (range == NVISR_RANGE_LIMITED) {
        float m = (float)(1 << (bits - 8));
        r.y_off = 16.f * m; r.y_den = 219.f * m; r.c_off = 128.f * m; r.c_den = 224.f * m;
        r.y_mul = 219.f * m; r.y_add = 16.f * m; r.c_mul = 224.f * m; r.c_add = 128.f * m;
    } else {
        float top = (float)((1 << bits) - 1);
        r.y_off = 0.f; r.y_den = top; r.c_off = (float)(1 << (bits - 1)); r.c_den = top;
        r.y_mul = top; r.y_add = 0.f; r.c_mul = top; r.c_add = (float)(1 << (bits - 1));
    }
    r.vmax = (float)((1 << bits) - 1);
    return r;
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
        r[e] = Y + (2.0f * (1.0f - KR)) * cr;
        b[e] = Y + (2.0f * (1.0f - KB)) * cb;
        g[e] = (Y - KR * r[e] - KB * b[e]) / KG;
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

__device__ __forceinline__ float quant(float v, float vmax) {
    v = rintf(v);  // round half to even
    return fminf(fmaxf(v, 0.0f), vmax);
}

template <typename S>
__device__ __forceinline__ void st_sample(uint8_t *base, int64_t pitch, int y, int x, float v) {
    reinterpret_cast<S *>(base + (int64_t)y * pitch)[x] = (S)(int)v;
}

__device__ __forceinline__ void rgb2ycc(float r, float g, float b, float &y, float &cb, float &cr) {
    y = KR * r + KG * g + KB * b;
    cb = (b - y) / (2.0f * (1.0f - KB));
    cr = (r - y) / (2.0f * (1.0f - KR));
}

// 4:4:4: one thread per 4 pixels of a row.
template <typename S>
__global__ void __launch_bounds__(256) requant444_kernel(const float *__restrict__ in, int64_t pitch,
                                                         int H, int W, RangeConst rc, uint8_t *yp,
                                                         int64_t py, uint8_t *up, int64_t pu,
                                                         uint8_t *vp, int64_t pv) {
    const int x0 = (blockIdx.x * blockDim.x + threadIdx.x) * 4;
    const int y = blockIdx.y;
    if (x0 >= W) return;
    const int64_t plane = pitch * H;
    const float *row = in + (int64_t)y * pitch;
    for (int e = 0; e < 4 && x0 + e < W; ++e) {
        float Y, cb, cr;
        rgb2ycc(row[x0 + e], row[plane + x0 + e], row[2 * plane + x0 + e], Y, cb, cr);
        st_sample<S>(yp, py, y, x0 + e, quant(Y * rc.y_mul + rc.y_add, rc.vmax));
        st_sample<S>(up, pu, y, x0 + e, quant(cb * rc.c_mul + rc.c_add, rc.vmax));
        st_sample<S>(vp, pv, y, x0 + e, quant(cr * rc.c_mul + rc.c_add, rc.vmax));
    }
}

// 4:2:0: one thread per (chroma row j, 4 chroma columns): luma rows 2j, 2j+1,
// columns 8q .. 8q+7; chroma needs columns 8q-1 .. 8q+7 for LEFT siting.
template <typename S>
__global__ void __launch_bounds__(256) requant420_kernel(const float *__restrict__ in, int64_t pitch,
                                                         int H, int W, int loc, RangeConst rc,
                                                         uint8_t *yp, int64_t py, uint8_t *up,
                                                         int64_t pu, uint8_t *vp, int64_t pv) {
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y;
    const int xb = q * 8;
    if (xb >= W) return;
    const int64_t plane = pitch * H;
    const int Wc = W / 2;
    // columns xb-1 .. xb+7 (9 columns), clamped; two rows.
    float cbv[9], crv[9];  // row-pair mean of full-resolution chroma
#pragma unroll
    for (int c = 0; c < 9; ++c) {
        const int x = clampi(xb - 1 + c, 0, W - 1);
        float cb2[2], cr2[2];
#pragma unroll
        for (int rr = 0; rr < 2; ++rr) {
            const int y = 2 * j + rr;
            const float *row = in + (int64_t)y * pitch;
            float Y, cb, cr;
            rgb2ycc(row[x], row[plane + x], row[2 * plane + x], Y, cb, cr);
            cb2[rr] = cb;
            cr2[rr] = cr;
            if (c >= 1 && c <= 8 && xb - 1 + c < W)
                st_sample<S>(yp, py, y, x, quant(Y * rc.y_mul + rc.y_add, rc.vmax));
        }
        cbv[c] = 0.5f * (cb2[0] + cb2[1]);
        crv[c] = 0.5f * (cr2[0] + cr2[1]);
    }
#pragma unroll
    for (int e = 0; e < 4; ++e) {
        const int i = q * 4 + e;
        if (i >= Wc) break;
        const int c = 1 + 2 * e;  // index of column 2i
        float cb, cr;
        if (loc == NVISR_CHROMA_LEFT) {
            cb = 0.25f * (cbv[c - 1] + 2.0f * cbv[c] + cbv[c + 1]);
            cr = 0.25f * (crv[c - 1] + 2.0f * crv[c] + crv[c + 1]);
        } else {
            cb = 0.5f * (cbv[c] + cbv[c + 1]);
            cr = 0.5f * (crv[c] + crv[c + 1]);
        }
        st_sample<S>(up, pu, j, i, quant(cb * rc.c_mul + rc.c_add, rc.vmax));
        st_sample<S>(vp, pv, j, i, quant(cr * rc.c_mul + rc.c_add, rc.vmax));
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

// One thread per (pixel, 16-byte chunk).
template <typename T>
__global__ void __launch_bounds__(256) pack_kernel(PackArgs a) {
    constexpr int CPC = 16 / sizeof(T);
    const int64_t HW = (int64_t)a.H * a.W;
    const int nchunks = a.cpad / CPC;
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= HW * nchunks) return;
    const int cc = (int)(idx / HW);
    const int64_t p = idx - (int64_t)cc * HW;
    const int y = (int)(p / a.W), x = (int)(p - (int64_t)y * a.W);
    const int creal = a.nsrc * a.ch_per_src;
    alignas(16) T vals[CPC];
    float amax = 0.f;
#pragma unroll
    for (int e = 0; e < CPC; ++e) {
        const int ch = cc * CPC + e;
        float v = 0.f;
        if (ch < creal) {
            const int s = ch / a.ch_per_src, c = ch - s * a.ch_per_src;
            v = a.src[s][c * a.src_plane + (int64_t)y * a.src_pitch + x];
        }
        amax = fmaxf(amax, fabsf(v));
        vals[e] = cvt_out<T>(v * a.scale);
    }
    *reinterpret_cast<uint4 *>(reinterpret_cast<uint8_t *>(a.dst) + idx * 16) =
        *reinterpret_cast<const uint4 *>(vals);
    if (a.amax) atomicMax(a.amax, __float_as_uint(amax));
}

template <typename T>
__global__ void __launch_bounds__(256) unpack_kernel(const uint8_t *__restrict__ src, int cpad, int C,
                                                     int H, int W, float scale, float *dst,
                                                     int64_t pitch) {
    constexpr int CPC = 16 / sizeof(T);
    const int64_t HW = (int64_t)H * W;
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= HW * (cpad / CPC)) return;
    const int cc = (int)(idx / HW);
    const int64_t p = idx - (int64_t)cc * HW;
    const int y = (int)(p / W), x = (int)(p - (int64_t)y * W);
    alignas(16) T vals[CPC];
    *reinterpret_cast<uint4 *>(vals) = *reinterpret_cast<const uint4 *>(src + idx * 16);
#pragma unroll
    for (int e = 0; e < CPC; ++e) {
        const int ch = cc * CPC + e;
        if (ch < C) dst[(int64_t)ch * pitch * H + (int64_t)y * pitch + x] = cvt_in<T>(vals[e]) * scale;
    }
}

}  // namespace

cudaError_t launch_ingest(const nvisr_format &f, const void *y, int64_t py, const void *u, int64_t pu,
                          const void *v, int64_t pv, float *out, int64_t out_pitch, cudaStream_t st) {
    const RangeConst rc = range_const(f.bit_depth, f.range);
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
                           void *u, int64_t pu, void *v, int64_t pv, cudaStream_t st) {
    const RangeConst rc = range_const(f.bit_depth, f.range);
    dim3 block(64);
    if (f.subsampling == NVISR_SUB_420) {
        dim3 grid((f.width / 8 + 1 + block.x - 1) / block.x, f.height / 2);
        if (f.bit_depth <= 8)
            requant420_kernel<uint8_t><<<grid, block, 0, st>>>(in, in_pitch, f.height, f.width, f.chroma_loc,
                                                               rc, (uint8_t *)y, py, (uint8_t *)u, pu,
                                                               (uint8_t *)v, pv);
        else
            requant420_kernel<uint16_t><<<grid, block, 0, st>>>(in, in_pitch, f.height, f.width, f.chroma_loc,
                                                                rc, (uint8_t *)y, py, (uint8_t *)u, pu,
                                                                (uint8_t *)v, pv);
    } else {
        dim3 grid((f.width / 4 + 1 + block.x - 1) / block.x, f.height);
        if (f.bit_depth <= 8)
            requant444_kernel<uint8_t><<<grid, block, 0, st>>>(in, in_pitch, f.height, f.width, rc,
                                                               (uint8_t *)y, py, (uint8_t *)u, pu,
                                                               (uint8_t *)v, pv);
        else
            requant444_kernel<uint16_t><<<grid, block, 0, st>>>(in, in_pitch, f.height, f.width, rc,
                                                                (uint8_t *)y, py, (uint8_t *)u, pu,
                                                                (uint8_t *)v, pv);
    }
    return cudaGetLastError();
}

cudaError_t launch_pack(const PackArgs &a, cudaStream_t st) {
    const int cpc = chunk_channels(a.dt);
    const int64_t n = (int64_t)a.H * a.W * (a.cpad / cpc);
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

cudaError_t launch_unpack(const void *src, int dt, int cpad, int C, int H, int W, float scale, float *dst,
                          int64_t dst_pitch, cudaStream_t st) {
    const int cpc = chunk_channels(dt);
    const int64_t n = (int64_t)H * W * (cpad / cpc);
    const int block = 256;
    const unsigned grid = (unsigned)((n + block - 1) / block);
    const uint8_t *s = (const uint8_t *)src;
    switch (dt) {
        case DT_F32: unpack_kernel<float><<<grid, block, 0, st>>>(s, cpad, C, H, W, scale, dst, dst_pitch); break;
        case DT_BF16: unpack_kernel<__nv_bfloat16><<<grid, block, 0, st>>>(s, cpad, C, H, W, scale, dst, dst_pitch); break;
        case DT_F16: unpack_kernel<__half><<<grid, block, 0, st>>>(s, cpad, C, H, W, scale, dst, dst_pitch); break;
        default: unpack_kernel<__nv_fp8_e4m3><<<grid, block, 0, st>>>(s, cpad, C, H, W, scale, dst, dst_pitch); break;
    }
    return cudaGetLastError();
}

}  // namespace nvisr
