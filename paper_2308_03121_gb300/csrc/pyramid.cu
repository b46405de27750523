// Resampling of the extract stage's feature pyramid (Section 3.1: the extract
// stage produces "a pyramid of features in different spatial dimensions"):
//   pool: the 2x2 mean, out[c, y, x] = (in[2y, 2x] + in[2y, 2x+1] + in[2y+1, 2x] + in[2y+1, 2x+1]) / 4;
//   up:   bilinear x2 with align_corners = False and edge clamp, source row
//         max((Y + 1/2) / 2 - 1/2, 0) between rows floor and floor + 1 (clamped), likewise columns.
// Both work on the blocked activation layout [C/cpc][H][W][cpc] (BF16, FP16 or
// float32), one thread per output pixel and 16-byte unit of channels, FP32
// arithmetic, one rounding to the stored type.  They stream their tensors once
// (HBM-bound: read 4 and write 1 value per pooled value; up reads each input
// value about 4 times through L1/L2 and writes 4).
#include <algorithm>

#include "common.cuh"

namespace nvisr {

namespace {

template <typename T>
struct Unit;  // 16 bytes of channels <-> floats
template <>
struct Unit<float> {
    static constexpr int N = 4;
    __device__ static void load(const uint8_t *p, float (&v)[N]) {
        const float4 q = *reinterpret_cast<const float4 *>(p);
        v[0] = q.x; v[1] = q.y; v[2] = q.z; v[3] = q.w;
    }
    __device__ static void store(uint8_t *p, const float (&v)[N]) {
        *reinterpret_cast<float4 *>(p) = make_float4(v[0], v[1], v[2], v[3]);
    }
};
template <>
struct Unit<__nv_bfloat16> {
    static constexpr int N = 8;
    __device__ static void load(const uint8_t *p, float (&v)[N]) {
        const uint4 q = *reinterpret_cast<const uint4 *>(p);
        const __nv_bfloat162 *h = reinterpret_cast<const __nv_bfloat162 *>(&q);
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const float2 f = __bfloat1622float2(h[i]);
            v[2 * i] = f.x;
            v[2 * i + 1] = f.y;
        }
    }
    __device__ static void store(uint8_t *p, const float (&v)[N]) {
        uint4 q;
        __nv_bfloat162 *h = reinterpret_cast<__nv_bfloat162 *>(&q);
#pragma unroll
        for (int i = 0; i < 4; ++i) h[i] = __floats2bfloat162_rn(v[2 * i], v[2 * i + 1]);
        *reinterpret_cast<uint4 *>(p) = q;
    }
};
template <>
struct Unit<__half> {
    static constexpr int N = 8;
    __device__ static void load(const uint8_t *p, float (&v)[N]) {
        const uint4 q = *reinterpret_cast<const uint4 *>(p);
        const __half2 *h = reinterpret_cast<const __half2 *>(&q);
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const float2 f = __half22float2(h[i]);
            v[2 * i] = f.x;
            v[2 * i + 1] = f.y;
        }
    }
    __device__ static void store(uint8_t *p, const float (&v)[N]) {
        uint4 q;
        __half2 *h = reinterpret_cast<__half2 *>(&q);
#pragma unroll
        for (int i = 0; i < 4; ++i) h[i] = __floats2half2_rn(v[2 * i], v[2 * i + 1]);
        *reinterpret_cast<uint4 *>(p) = q;
    }
};

// Byte address of the 16-byte unit holding channels [c, c + N) of pixel pix.
__device__ __forceinline__ int64_t unit_off(int c, int64_t pix, int64_t hw, int cpc, int esz) {
    return ((int64_t)(c / cpc) * hw + pix) * cpc * esz + (int64_t)(c % cpc) * esz;
}

template <typename T>
__global__ void pool2_kernel(const uint8_t *__restrict__ x, int xcpc, uint8_t *__restrict__ y, int ycpc, int C,
                             int H, int W) {
    using U = Unit<T>;
    constexpr int esz = (int)sizeof(T);
    const int Ho = H / 2, Wo = W / 2;
    const int units = C / U::N;
    const int64_t n = (int64_t)Ho * Wo * units;
    const int64_t hwi = (int64_t)H * W, hwo = (int64_t)Ho * Wo;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int u = (int)(i % units);  // consecutive threads: consecutive units of one pixel
        const int64_t po = i / units;
        const int yo = (int)(po / Wo), xo = (int)(po % Wo);
        const int c = u * U::N;
        float a[U::N], b[U::N], d[U::N], e[U::N], o[U::N];
        const int64_t p00 = (int64_t)(2 * yo) * W + 2 * xo;
        U::load(x + unit_off(c, p00, hwi, xcpc, esz), a);
        U::load(x + unit_off(c, p00 + 1, hwi, xcpc, esz), b);
        U::load(x + unit_off(c, p00 + W, hwi, xcpc, esz), d);
        U::load(x + unit_off(c, p00 + W + 1, hwi, xcpc, esz), e);
#pragma unroll
        for (int k = 0; k < U::N; ++k) o[k] = ((a[k] + b[k]) + (d[k] + e[k])) * 0.25f;
        U::store(y + unit_off(c, po, hwo, ycpc, esz), o);
    }
}

template <typename T>
__global__ void up2_kernel(const uint8_t *__restrict__ x, int xcpc, uint8_t *__restrict__ y, int ycpc, int C, int H,
                           int W) {
    using U = Unit<T>;
    constexpr int esz = (int)sizeof(T);
    const int Ho = 2 * H, Wo = 2 * W;
    const int units = C / U::N;
    const int64_t n = (int64_t)Ho * Wo * units;
    const int64_t hwi = (int64_t)H * W, hwo = (int64_t)Ho * Wo;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int u = (int)(i % units);
        const int64_t po = i / units;
        const int yo = (int)(po / Wo), xo = (int)(po % Wo);
        const int c = u * U::N;
        // source position of the output pixel centre, clamped at the top / left edge
        const float sy = fmaxf((yo + 0.5f) * 0.5f - 0.5f, 0.f), sx = fmaxf((xo + 0.5f) * 0.5f - 0.5f, 0.f);
        const int y0 = (int)sy, x0 = (int)sx;  // sy, sx >= 0: truncation is floor
        const int y1 = min(y0 + 1, H - 1), x1 = min(x0 + 1, W - 1);
        const float fy = sy - (float)y0, fx = sx - (float)x0;
        float a[U::N], b[U::N], d[U::N], e[U::N], o[U::N];
        U::load(x + unit_off(c, (int64_t)y0 * W + x0, hwi, xcpc, esz), a);
        U::load(x + unit_off(c, (int64_t)y0 * W + x1, hwi, xcpc, esz), b);
        U::load(x + unit_off(c, (int64_t)y1 * W + x0, hwi, xcpc, esz), d);
        U::load(x + unit_off(c, (int64_t)y1 * W + x1, hwi, xcpc, esz), e);
#pragma unroll
        for (int k = 0; k < U::N; ++k) {
            const float top = a[k] * (1.f - fx) + b[k] * fx;
            const float bot = d[k] * (1.f - fx) + e[k] * fx;
            o[k] = top * (1.f - fy) + bot * fy;
        }
        U::store(y + unit_off(c, po, hwo, ycpc, esz), o);
    }
}

template <typename T>
cudaError_t run_resample(bool up, const void *x, int xcpc, void *y, int ycpc, int C, int H, int W, cudaStream_t st) {
    const int64_t px = up ? (int64_t)4 * H * W : (int64_t)(H / 2) * (W / 2);
    const int64_t n = px * (C / Unit<T>::N);
    const int threads = 256;
    const int64_t blocks = std::min<int64_t>((n + threads - 1) / threads, (int64_t)device_sm_count() * 16);
    if (blocks < 1) return cudaSuccess;
    if (up)
        up2_kernel<T><<<(int)blocks, threads, 0, st>>>(static_cast<const uint8_t *>(x), xcpc,
                                                        static_cast<uint8_t *>(y), ycpc, C, H, W);
    else
        pool2_kernel<T><<<(int)blocks, threads, 0, st>>>(static_cast<const uint8_t *>(x), xcpc,
                                                          static_cast<uint8_t *>(y), ycpc, C, H, W);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_resample2(bool up, int dt, const void *x, int xcpc, void *y, int ycpc, int C, int H, int W,
                             cudaStream_t st) {
    const int n = chunk_channels(dt);
    // whole 16-byte units inside each chunk; pooling needs even sizes
    if (C % n || xcpc % n || ycpc % n || H < 1 || W < 1 || (!up && (H % 2 || W % 2))) return cudaErrorInvalidValue;
    if (dt == DT_F32) return run_resample<float>(up, x, xcpc, y, ycpc, C, H, W, st);
    if (dt == DT_BF16) return run_resample<__nv_bfloat16>(up, x, xcpc, y, ycpc, C, H, W, st);
    if (dt == DT_F16) return run_resample<__half>(up, x, xcpc, y, ycpc, C, H, W, st);
    return cudaErrorNotSupported;
}

}  // namespace nvisr
