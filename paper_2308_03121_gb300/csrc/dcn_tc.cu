// Modulated deformable convolution (DCN v2) on the tensor cores, sm_103a.
//
// The paper ships a DCN v2 operator compatible with torchvision's
// deform_conv2d because video enhancement networks align neighbouring frames
// with it (Section 3.1).  For output pixel p, tap k and input channel c of
// offset group g:
//     y[o,p] = b[o] + sum_{c,k} w[o,c,k] * m[g,k](p) * bilinear(x_c, p + p_k + d[g,k](p))
// with out-of-image bilinear corners contributing zero.
//
// Kernel: one CTA per SM walks 128-pixel row tiles.  For each tile and tap,
// sixteen producer warps (four threads per pixel, each taking a quarter of
// the 8-channel groups) read the tap's offsets and mask, issue the four bilinear
// corner loads of all their channel groups before using any (so many gathers
// are in flight at once), blend them in FP32, scale by the mask and store
// 16-byte rows of the canonical no-swizzle K-major A tile in shared memory
// (the sampled im2col tile of that tap).  A single thread issues the tap's
// tcgen05.mma's against the resident weights into a double-buffered TMEM
// accumulator; four epilogue warps add the bias and store the blocked
// output.  Every wait is bounded in time.
#include "common.cuh"
#include "sm100_ptx.cuh"

namespace nvisr {

namespace {

constexpr int TM = 128;
constexpr int NGATHER = 512;            // gather threads (four per pixel)
constexpr int MMA_WARP = NGATHER / 32;  // then the MMA / TMEM / weights warp, then 4 epilogue warps
constexpr int NT = NGATHER + 32 + 128;
constexpr uint64_t WAIT_NS = 2000000000ull;
constexpr int SMEM_LIMIT = 232448;

template <typename T>
struct Cv;
template <>
struct Cv<__nv_bfloat16> {
    static __device__ __forceinline__ float in(__nv_bfloat16 v) { return __bfloat162float(v); }
    static __device__ __forceinline__ __nv_bfloat16 out(float v) { return __float2bfloat16_rn(v); }
};
template <>
struct Cv<__half> {
    static __device__ __forceinline__ float in(__half v) { return __half2float(v); }
    static __device__ __forceinline__ __half out(float v) { return __float2half_rn(v); }
};

// T: 16-bit element type of x / y; NS: output channels (one slice); C: input channels.
template <typename T, int NS, int C>
__global__ void __launch_bounds__(NT, 1) dcn_tc_kernel(const DcnArgs a, int stages) {
    constexpr int CPC = 8;                 // channels per 16-byte chunk
    constexpr int NCH = C / CPC;           // chunks per tap (= K / 8)
    constexpr uint32_t LBO = TM * 16;      // chunk stride inside a stage
    constexpr uint32_t STAGE = NCH * LBO;  // one tap's A tile
    constexpr int AFMT = std::is_same<T, __nv_bfloat16>::value ? 1 : 0;
    constexpr uint32_t IDESC = instr_desc(TM, NS, AFMT, AFMT);
    constexpr uint32_t NCOLS = 2 * NS <= 32 ? 32 : (2 * NS <= 64 ? 64 : (2 * NS <= 128 ? 128 : 256));
    static_assert(NCH % 2 == 0, "two chunks per MMA");

    extern __shared__ uint8_t smem_raw[];
    uint8_t *smem = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    uint64_t *full = reinterpret_cast<uint64_t *>(smem);
    uint64_t *empty = full + 8;
    uint64_t *tfull = empty + 8;
    uint64_t *tempty = tfull + 2;
    uint64_t *wbar = tempty + 2;
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(wbar + 1);
    volatile int *abort = reinterpret_cast<volatile int *>(tmem_slot + 1);
    const uint32_t wbytes = 9 * NCH * NS * 16;
    uint8_t *wsm = smem + 1024;
    uint8_t *stage0 = wsm + ((wbytes + 1023) & ~1023u);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int H = a.H, W = a.W;
    // blocked layouts [C/cpc][H][W][cpc]: byte address of the 8-channel unit starting at channel c
    const int xcpc = a.x_cpc, ycpc = a.y_cpc;
    const int64_t HW = (int64_t)H * W;
    const int tiles_x = (W + TM - 1) / TM;
    const int ntiles = tiles_x * H;
    const int S = stages;

    if (threadIdx.x == 0) {
        for (int s = 0; s < S; ++s) {
            mbar_init(&full[s], NGATHER);
            mbar_init(&empty[s], 1);
        }
        for (int i = 0; i < 2; ++i) {
            mbar_init(&tfull[i], 1);
            mbar_init(&tempty[i], 128);
        }
        mbar_init(wbar, 1);
        *abort = 0;
        fence_mbarrier_init();
    }
    if (warp == MMA_WARP) {
        tmem_alloc(tmem_slot, NCOLS);
        tmem_relinquish();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem_base = *tmem_slot;

    if (warp < NGATHER / 32) {
        // ------------------------------------------------ gather producers
        // thread = (8-channel group cc, pixel): the 8 threads of a pixel read the
        // pixel's 128-byte channel line of a corner together (full-line loads)
        constexpr int PPP = NGATHER / NCH;           // pixels per pass
        constexpr int NPASS = TM / PPP;              // passes over the tile's pixels
        static_assert(NGATHER % NCH == 0 && TM % PPP == 0, "gather mapping");
        const int cc = threadIdx.x % NCH;            // channel group (16-byte chunk)
        const int mp = threadIdx.x / NCH;            // pixel within a pass
        const uint8_t *x = static_cast<const uint8_t *>(a.x);
        const int cpg = a.cin_pad / a.groups;
        const int G = a.groups;
        const int g = (cc * CPC) / cpg;
        const uint8_t *plane = x + (int64_t)((cc * CPC) / xcpc) * HW * xcpc * 2 + ((cc * CPC) % xcpc) * 2;
        int s = 0;
        uint32_t ph = 0;
        bool ok = true;
        // offsets (dy, dx adjacent in one 4-channel unit) and mask of every pass's pixel
        // for tap k; the next tap's are loaded while this tap's corners are in flight
        auto load_om = [&](int y, int xb, int k, float2 (&d)[NPASS], float (&mk)[NPASS]) {
            const int cd = 2 * (g * 9 + k), cm = 18 * G + g * 9 + k;
#pragma unroll
            for (int h = 0; h < NPASS; ++h) {
                const int64_t pix = (int64_t)y * W + min(xb + mp + h * PPP, W - 1);
                d[h] = __ldg(reinterpret_cast<const float2 *>(a.om + ((int64_t)(cd >> 2) * HW + pix) * 4 + (cd & 3)));
                mk[h] = __ldg(a.om + ((int64_t)(cm >> 2) * HW + pix) * 4 + (cm & 3));
            }
        };
        for (int t = blockIdx.x; t < ntiles && ok; t += gridDim.x) {
            const int y = t / tiles_x;
            const int xb = (t - y * tiles_x) * TM;
            float2 dn[NPASS];
            float mn[NPASS];
            load_om(y, xb, 0, dn, mn);
            for (int k = 0; k < 9; ++k) {
                float dy[NPASS], dx[NPASS], msk[NPASS];
#pragma unroll
                for (int h = 0; h < NPASS; ++h) {
                    dy[h] = dn[h].x;
                    dx[h] = dn[h].y;
                    msk[h] = mn[h];
                }
                if (!mbar_wait_bounded(&empty[s], ph ^ 1, abort, WAIT_NS)) {
                    *abort = 1;
                    if (a.err) atomicExch(a.err, DEVERR_TIMEOUT);
                    ok = false;
                    break;
                }
                uint8_t *stg = stage0 + (size_t)s * STAGE + (size_t)cc * LBO;
                // every corner load of every pass first, then the blends
                uint4 v[NPASS][4];
                float wq[NPASS][4];
#pragma unroll
                for (int h = 0; h < NPASS; ++h) {
                    const int xx = xb + mp + h * PPP;
                    const float sy = (float)(y + k / 3 - 1) + dy[h];
                    const float sx = (float)(xx + k % 3 - 1) + dx[h];
                    const float fy = floorf(sy), fx = floorf(sx);
                    const int y0 = (int)fy, x0 = (int)fx;
                    const float ly = sy - fy, lx = sx - fx;
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        const int yy = y0 + (q >> 1), xq = x0 + (q & 1);
                        const bool in = xx < W && yy >= 0 && yy < H && xq >= 0 && xq < W;
                        wq[h][q] = in ? ((q >> 1) ? ly : 1.f - ly) * ((q & 1) ? lx : 1.f - lx) : 0.f;
                        v[h][q] = in ? __ldg(reinterpret_cast<const uint4 *>(plane + ((int64_t)yy * W + xq) * xcpc * 2))
                                     : make_uint4(0u, 0u, 0u, 0u);
                    }
                }
                if (k < 8) load_om(y, xb, k + 1, dn, mn);
#pragma unroll
                for (int h = 0; h < NPASS; ++h) {
                    float acc[CPC];
#pragma unroll
                    for (int e = 0; e < CPC; ++e) acc[e] = 0.f;
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        const T *vv = reinterpret_cast<const T *>(&v[h][q]);
#pragma unroll
                        for (int e = 0; e < CPC; ++e) acc[e] += wq[h][q] * Cv<T>::in(vv[e]);
                    }
                    float mm = msk[h];
                    if (a.mask_logits) mm = 1.f / (1.f + expf(-mm));
                    alignas(16) T o[CPC];
#pragma unroll
                    for (int e = 0; e < CPC; ++e) o[e] = Cv<T>::out(acc[e] * mm);
                    *reinterpret_cast<uint4 *>(stg + (size_t)(mp + h * PPP) * 16) = *reinterpret_cast<const uint4 *>(o);
                }
                fence_proxy_async();  // generic smem writes -> visible to the tensor core
                mbar_arrive(&full[s]);
                if (++s == S) { s = 0; ph ^= 1; }
            }
        }
    } else if (warp == MMA_WARP) {
        if (lane == 0) {
            // ------------------------------------------------ weights + MMA issue
            mbar_arrive_expect_tx(wbar, wbytes);
            for (uint32_t off = 0; off < wbytes; off += 32768u)
                bulk_load(wsm + off, static_cast<const uint8_t *>(a.w) + off, min(32768u, wbytes - off), wbar);
            bool ok = mbar_wait_bounded(wbar, 0, abort, WAIT_NS);
            if (!ok) {
                *abort = 1;
                if (a.err) atomicExch(a.err, DEVERR_TIMEOUT);
            }
            const uint32_t wbase = smem_u32(wsm);
            int s = 0, it = 0, last_a = -1;
            uint32_t ph = 0, last_par = 0;
            for (int t = blockIdx.x; t < ntiles && ok; t += gridDim.x, ++it) {
                const int ab = it & 1;
                const uint32_t u = (uint32_t)(it >> 1);
                if (!mbar_wait_bounded(&tempty[ab], (u & 1) ^ 1, abort, WAIT_NS)) {
                    *abort = 1;
                    if (a.err) atomicExch(a.err, DEVERR_TIMEOUT);
                    break;
                }
                tc_fence_after();
                const uint32_t d_tmem = tmem_base + (uint32_t)(ab * NS);
                for (int k = 0; k < 9; ++k) {
                    if (!mbar_wait_bounded(&full[s], ph, abort, WAIT_NS)) {
                        *abort = 1;
                        if (a.err) atomicExch(a.err, DEVERR_TIMEOUT);
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    const uint32_t sb = smem_u32(stage0 + (size_t)s * STAGE);
#pragma unroll
                    for (int j = 0; j < NCH / 2; ++j) {
                        const uint64_t ad = smem_desc(sb + 2 * j * LBO, LBO, 128);
                        const uint64_t bd = smem_desc(wbase + (uint32_t)((k * NCH + 2 * j) * NS * 16), NS * 16, 128);
                        umma<0>(d_tmem, ad, bd, IDESC, (k | j) != 0 ? 1u : 0u);
                    }
                    umma_commit(&empty[s]);
                    if (++s == S) { s = 0; ph ^= 1; }
                }
                if (!ok) break;
                umma_commit(&tfull[ab]);
                last_a = ab;
                last_par = u & 1;
            }
            if (last_a >= 0) mbar_wait_bounded(&tfull[last_a], last_par, nullptr, WAIT_NS);
            mbar_wait_bounded(wbar, 0, nullptr, WAIT_NS);
        }
    } else {
        // ------------------------------------------------ epilogue (the last 4 warps, one per lane quadrant)
        const int q = warp & 3;
        const int m = q * 32 + lane;
        uint8_t *yb = static_cast<uint8_t *>(a.y);
        int it = 0;
        for (int t = blockIdx.x; t < ntiles; t += gridDim.x, ++it) {
            const int ab = it & 1;
            const uint32_t u = (uint32_t)(it >> 1);
            bool ok = mbar_wait_bounded(&tfull[ab], u & 1, abort, WAIT_NS);
            ok = __all_sync(0xffffffffu, ok);
            if (!ok) {
                if (lane == 0) {
                    *abort = 1;
                    if (a.err) atomicExch(a.err, DEVERR_TIMEOUT);
                }
                break;
            }
            tc_fence_after();
            const int y = t / tiles_x;
            const int xx = (t - y * tiles_x) * TM + m;
            const int64_t pix = (int64_t)y * W + xx;
            const uint32_t taddr = tmem_base + ((uint32_t)(q * 32) << 16) + (uint32_t)(ab * NS);
#pragma unroll
            for (int j = 0; j < NS / 16; ++j) {
                float v[16];
                tmem_ld16(taddr + (uint32_t)(j * 16), v);
                if (xx >= W) continue;
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    alignas(16) T o[CPC];
#pragma unroll
                    for (int e = 0; e < CPC; ++e) {
                        const int n = j * 16 + h * 8 + e;
                        o[e] = Cv<T>::out(v[h * 8 + e] * a.acc_scale + a.bias[n]);
                    }
                    const int n = j * 16 + h * 8;
                    *reinterpret_cast<uint4 *>(yb + ((int64_t)(n / ycpc) * HW + pix) * ycpc * 2 + (n % ycpc) * 2) =
                        *reinterpret_cast<const uint4 *>(o);
                }
            }
            tc_fence_before();
            mbar_arrive(&tempty[ab]);
        }
    }
    __syncthreads();
    if (warp == MMA_WARP) {
        __syncwarp();
        tc_fence_after();
        tmem_dealloc(tmem_base, NCOLS);
    }
}

template <typename T, int NS, int C>
cudaError_t run(const DcnArgs &a, cudaStream_t st) {
    constexpr uint32_t STAGE = (C / 8) * TM * 16;
    constexpr uint32_t wbytes = 9 * (C / 8) * NS * 16;
    const uint32_t wround = (wbytes + 1023) & ~1023u;
    int stages = (SMEM_LIMIT - 2048 - (int)wround) / (int)STAGE;
    if (stages > 8) stages = 8;
    if (stages < 2) return cudaErrorInvalidConfiguration;
    int smem = 2048 + (int)wround + stages * (int)STAGE;
    if (smem < 118 * 1024) smem = 118 * 1024;
    auto kern = dcn_tc_kernel<T, NS, C>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    const int tiles = ((a.W + TM - 1) / TM) * a.H;
    int grid = device_sm_count();
    if (grid > tiles) grid = tiles;
    kern<<<grid, NT, smem, st>>>(a, stages);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_dcn_tc(const DcnArgs &a0, cudaStream_t st) {
    DcnArgs a = a0;
    if (a.x_cpc == 0) a.x_cpc = 8;
    if (a.y_cpc == 0) a.y_cpc = 8;
    if (a.cin_pad != 64 || a.cout_pad != 64 || (a.cin_pad / a.groups) % 8) return cudaErrorNotSupported;
    if ((a.x_cpc != 8 && a.x_cpc != 64) || (a.y_cpc != 8 && a.y_cpc != 64)) return cudaErrorNotSupported;
    if (a.in_dt == DT_BF16 && a.out_dt == DT_BF16) return run<__nv_bfloat16, 64, 64>(a, st);
    if (a.in_dt == DT_F16 && a.out_dt == DT_F16) return run<__half, 64, 64>(a, st);
    return cudaErrorNotSupported;
}

}  // namespace nvisr
