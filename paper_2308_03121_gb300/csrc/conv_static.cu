// nvisr_conv2d_static: the one-layer convolution of nvisr_conv2d with every
// working buffer carved out of one fixed device array of this module instead
// of memory allocated per call.
//
// Who needs it: callers that must not allocate while they run.  cudaMalloc can
// fail once a process has handed its device memory to other work, and cudaFree
// synchronises the whole device, stalling every other stream of the process;
// a real-time caller, or one whose memory is fully reserved in advance, can
// afford neither.  This entry point makes no allocation of its own: the
// 32 MiB area below is set aside when the module is loaded, and the layout of
// the weights and bias runs in device kernels reading the caller's buffers
// (nothing is staged on the host).
//
// Limits: one area per device, shared by every call on that device, so calls
// that overlap in time on one device (from several host threads, or on several
// streams) race on it and must be serialised by the caller.  A problem whose
// buffers exceed the area is rejected with NVISR_OVER_BUDGET before any device
// work.  The first call on each device looks up the area's address; make that
// first call before any stream capture begins.  FP8 (which measures a
// per-tensor scale on the host side) is not offered here.
#include <mutex>
#include <string>
#include <vector>

#include "common.cuh"

// The working area (weights image, bias, blocked x / y / residual, error word).
static __device__ __align__(256) uint8_t conv_static_scratch[NVISR_CONV2D_STATIC_SCRATCH_BYTES];

namespace nvisr {

void set_error(const std::string &msg);
nvisr_status cuda_status(cudaError_t e, const char *where);

namespace {

// The area's address per (device, context): a context created anew for a device
// (after cudaDeviceReset, say) loads the module again, at a new address.
struct AreaRec {
    int dev;
    void *ctx;
    uint8_t *ptr;
};
std::mutex g_area_mu;
std::vector<AreaRec> g_area;

// SIMT image [cin_pad][k*k][cout_pad] float32, written whole (padding = 0).
__global__ void simt_weights_kernel(const float *__restrict__ w, int cout, int cin, int kk, int cin_pad,
                                    int cout_pad, float *__restrict__ dst) {
    const int64_t n = (int64_t)cin_pad * kk * cout_pad;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int o = (int)(i % cout_pad);
        const int64_t ct = i / cout_pad;
        const int t = (int)(ct % kk), c = (int)(ct / kk);
        dst[i] = (o < cout && c < cin) ? w[((int64_t)o * cin + c) * kk + t] : 0.f;
    }
}

template <typename T>
__device__ __forceinline__ T to_elem(float v);
template <>
__device__ __forceinline__ __nv_bfloat16 to_elem<__nv_bfloat16>(float v) { return __float2bfloat16_rn(v); }
template <>
__device__ __forceinline__ __half to_elem<__half>(float v) { return __float2half_rn(v); }

// Tensor-core image per output slice of ns channels: [slice][tap][K chunk][n][chunk bytes],
// with the 16-byte units of row n rotated by n & 7 in the 128-byte-swizzled form.
// One thread per weight element; the destination was zeroed beforehand.
template <typename T>
__global__ void tc_weights_kernel(const float *__restrict__ w, int cout, int cin, int kk, int cin_pad, int ns,
                                  int cpc, int sw128, uint8_t *__restrict__ dst) {
    constexpr int esz = (int)sizeof(T);
    const int cb = cpc * esz, chunks = cin_pad / cpc;
    const int64_t n_el = (int64_t)cout * cin * kk;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n_el;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int t = (int)(i % kk);
        const int c = (int)((i / kk) % cin);
        const int o = (int)(i / ((int64_t)kk * cin));
        const int sl = o / ns, n = o % ns, kc = c / cpc, e = c % cpc;
        int64_t off = (int64_t)sl * kk * chunks * ns * cb + (((int64_t)t * chunks + kc) * ns + n) * cb;
        off += sw128 ? (int64_t)((((e * esz) >> 4) ^ (n & 7)) << 4) + (e * esz) % 16 : (int64_t)e * esz;
        *reinterpret_cast<T *>(dst + off) = to_elem<T>(w[i]);
    }
}

// Row-streaming 64 -> 64 image [kx][2 - ky][64 out][128 B swizzled 64 in]; one
// thread per weight element, every destination byte written.
template <typename T>
__global__ void rows_weights_kernel(const float *__restrict__ w, uint8_t *__restrict__ dst) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= 64 * 64 * 9) return;
    const int kx = i % 3, ky = (i / 3) % 3, c = (i / 9) % 64, n = i / 576;
    const int64_t row = (int64_t)(2 - ky) * 64 + n;
    const int64_t off = (int64_t)kx * 3 * 64 * 128 + row * 128 + (((c >> 3) ^ (n & 7)) << 4) + (c & 7) * 2;
    *reinterpret_cast<T *>(dst + off) = to_elem<T>(w[i]);
}

// Bump allocator over the fixed area: 256-byte aligned slices, sizes checked
// in 64-bit arithmetic before any device work.
struct Carve {
    uint64_t used = 0;
    bool ok = true;
    uint64_t take(uint64_t bytes) {
        const uint64_t at = used;
        const uint64_t sz = (bytes + 255) / 256 * 256;
        if (sz > NVISR_CONV2D_STATIC_SCRATCH_BYTES || at > NVISR_CONV2D_STATIC_SCRATCH_BYTES - sz) ok = false;
        else used = at + sz;
        return at;
    }
};

nvisr_status fail(nvisr_status s, const std::string &msg) {
    set_error(msg);
    return s;
}

#define CS_TRY(x)                                                       \
    do {                                                                \
        cudaError_t e_ = (x);                                           \
        if (e_ != cudaSuccess) return cuda_status(e_, "conv2d_static"); \
    } while (0)

// The current context (the driver's cuCtxGetCurrent, reached through the runtime).
void *current_context() {
    typedef int (*CtxGetCurrent)(void **);
    static CtxGetCurrent fn = [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            return (CtxGetCurrent)p;
        return (CtxGetCurrent) nullptr;
    }();
    void *ctx = nullptr;
    if (fn) fn(&ctx);
    return ctx;
}

// Set-up: looks up the address of the area, once per device and context, with
// that device current.
nvisr_status area_for_current_device(uint8_t **out) {
    int dev = -1;
    CS_TRY(cudaGetDevice(&dev));
    std::lock_guard<std::mutex> lock(g_area_mu);
    if (void *ctx = current_context())
        for (const AreaRec &r : g_area)
            if (r.dev == dev && r.ctx == ctx) {
                *out = r.ptr;
                return NVISR_OK;
            }
    // no context yet, or a new one: the lookup also initialises the device's context
    void *p = nullptr;
    CS_TRY(cudaGetSymbolAddress(&p, conv_static_scratch));
    g_area.push_back({dev, current_context(), static_cast<uint8_t *>(p)});
    *out = static_cast<uint8_t *>(p);
    return NVISR_OK;
}

int grid_for(int64_t n, int threads) {
    const int64_t blocks = (n + threads - 1) / threads;
    return (int)std::min<int64_t>(std::max<int64_t>(blocks, 1), (int64_t)device_sm_count() * 16);
}

}  // namespace
}  // namespace nvisr

using namespace nvisr;

extern "C" nvisr_status nvisr_conv2d_static(int32_t precision, const float *x, int32_t cin, int32_t h, int32_t w,
                                            const float *weight, const float *bias, int32_t cout, int32_t k,
                                            int32_t act, const float *res, float *y, void *stream) {
    if (!x || !weight || !y || cin < 1 || cout < 1 || h < 1 || w < 1 || (k != 1 && k != 3) || act < 0 || act > 1)
        return fail(NVISR_INVALID_ARG, "conv2d_static: bad arguments");
    if (precision < NVISR_PREC_FP32 || precision > NVISR_PREC_FP8)
        return fail(NVISR_INVALID_ARG, "conv2d_static: unknown precision");
    if (precision == NVISR_PREC_FP8)
        return fail(NVISR_UNSUPPORTED_FORMAT, "conv2d_static: precision must be FP32, BF16 or FP16");
    const uint64_t cap = NVISR_CONV2D_STATIC_SCRATCH_BYTES;
    if ((uint64_t)cin > cap || (uint64_t)cout > cap || (uint64_t)h * (uint64_t)w > cap)
        return fail(NVISR_OVER_BUDGET, "conv2d_static: problem exceeds the static scratch area");
    const bool tc = precision != NVISR_PREC_FP32;
    const int dt = precision == NVISR_PREC_FP32 ? DT_F32 : (precision == NVISR_PREC_FP16 ? DT_F16 : DT_BF16);
    const int esz = dtype_size(dt);
    const int cin_pad = tc ? round_up(cin, 16) : round_up(cin, 8);
    const int cout_pad = round_up(cout, 16);
    const bool rows = tc && k == 3 && cin == 64 && cout == 64;
    const uint64_t px = (uint64_t)h * (uint64_t)w;
    const uint64_t wbytes = tc ? (uint64_t)tc_weight_bytes(cin_pad, cout_pad, k, dt)
                               : (uint64_t)simt_weight_bytes(cin_pad, cout_pad, k);
    Carve cv;
    const uint64_t o_err = cv.take(sizeof(int));
    const uint64_t o_bias = cv.take((uint64_t)cout_pad * 4);
    const uint64_t o_w = cv.take(wbytes);
    const uint64_t o_rows = rows ? cv.take(tc_rows_weight_bytes()) : 0;
    const uint64_t o_x = cv.take((uint64_t)cin_pad * px * esz);
    const uint64_t o_y = cv.take((uint64_t)cout_pad * px * esz);
    const uint64_t o_r = res ? cv.take((uint64_t)cout_pad * px * esz) : 0;
    if (!cv.ok)
        return fail(NVISR_OVER_BUDGET, "conv2d_static: problem needs more than the " +
                                           std::to_string(NVISR_CONV2D_STATIC_SCRATCH_BYTES) +
                                           "-byte static scratch area");
    uint8_t *area = nullptr;
    nvisr_status s = area_for_current_device(&area);
    if (s != NVISR_OK) return s;
    cudaStream_t st = (cudaStream_t)stream;
    int *err = reinterpret_cast<int *>(area + o_err);
    float *db = reinterpret_cast<float *>(area + o_bias);
    uint8_t *dw = area + o_w, *dwr = rows ? area + o_rows : nullptr;
    void *dx = area + o_x, *dy = area + o_y, *dr = res ? (void *)(area + o_r) : nullptr;

    // what must start at zero: the error word, the bias padding, the weight image padding
    CS_TRY(cudaMemsetAsync(err, 0, sizeof(int), st));
    CS_TRY(cudaMemsetAsync(db, 0, (size_t)cout_pad * 4, st));
    if (bias) CS_TRY(cudaMemcpyAsync(db, bias, (size_t)cout * 4, cudaMemcpyDeviceToDevice, st));
    const int kk = k * k;
    if (tc) {
        CS_TRY(cudaMemsetAsync(dw, 0, wbytes, st));
        const int ns = cout_pad / tc_nslice(cin_pad, cout_pad, k, dt);
        const int sw128 = layout_cpc(dt, cin_pad) == 64;
        const int cpc = sw128 ? 64 : 16 / esz;
        const int64_t n_el = (int64_t)cout * cin * kk;
        if (dt == DT_BF16)
            tc_weights_kernel<__nv_bfloat16><<<grid_for(n_el, 256), 256, 0, st>>>(weight, cout, cin, kk, cin_pad, ns,
                                                                                  cpc, sw128, dw);
        else
            tc_weights_kernel<__half><<<grid_for(n_el, 256), 256, 0, st>>>(weight, cout, cin, kk, cin_pad, ns, cpc,
                                                                           sw128, dw);
        CS_TRY(cudaGetLastError());
        if (rows) {
            CS_TRY(cudaMemsetAsync(dwr, 0, tc_rows_weight_bytes(), st));
            if (dt == DT_BF16) rows_weights_kernel<__nv_bfloat16><<<(64 * 64 * 9 + 255) / 256, 256, 0, st>>>(weight, dwr);
            else rows_weights_kernel<__half><<<(64 * 64 * 9 + 255) / 256, 256, 0, st>>>(weight, dwr);
            CS_TRY(cudaGetLastError());
        }
    } else {
        const int64_t n = (int64_t)cin_pad * kk * cout_pad;
        simt_weights_kernel<<<grid_for(n, 256), 256, 0, st>>>(weight, cout, cin, kk, cin_pad, cout_pad,
                                                             reinterpret_cast<float *>(dw));
        CS_TRY(cudaGetLastError());
    }

    const int in_cpc = layout_cpc(dt, cin_pad), out_cpc = layout_cpc(dt, cout_pad);
    PackArgs pa{};
    pa.src[0] = x;
    pa.nsrc = 1;
    pa.ch_per_src = cin;
    pa.src_pitch = w;
    pa.src_plane = (int64_t)w * h;
    pa.H = h;
    pa.W = w;
    pa.dst = dx;
    pa.cpad = cin_pad;
    pa.dt = dt;
    pa.cpc = in_cpc;
    pa.scale = 1.f;
    CS_TRY(launch_pack(pa, st));
    if (res) {
        PackArgs pr = pa;
        pr.src[0] = res;
        pr.ch_per_src = cout;
        pr.dst = dr;
        pr.cpad = cout_pad;
        pr.cpc = out_cpc;
        CS_TRY(launch_pack(pr, st));
    }
    ConvArgs a{};
    a.x = dx; a.cin_pad = cin_pad; a.H = h; a.W = w; a.nimg = 1; a.w = dw; a.w_rows = dwr; a.bias = db;
    a.cout = cout; a.cout_pad = cout_pad; a.k = k; a.act = act; a.res = dr; a.y = dy;
    a.in_dt = dt; a.out_dt = dt; a.acc_scale = 1.f; a.out_scale = 1.f; a.y2_scale = 1.f; a.err = err;
    a.in_cpc = in_cpc; a.out_cpc = out_cpc;
    CS_TRY(tc ? launch_conv_tc(a, st) : launch_conv_simt(a, st));
    CS_TRY(launch_unpack(dy, dt, cout_pad, out_cpc, cout, h, w, 1.f, y, w, st));
    int herr = 0;
    CS_TRY(cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, st));
    CS_TRY(cudaStreamSynchronize(st));
    if (herr) return fail(NVISR_DEVICE_TIMEOUT, "conv2d_static: a device-side wait exceeded its bound");
    return NVISR_OK;
}
