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
// sixteen producer warps (a warp per 8-channel chunk and half tile, a lane pair
// per pixel) read the tap's offsets and mask, issue the bilinear corner loads
// of all their pixels before using any (so many gathers are in flight at
// once), blend them in FP32 with the mask folded into the row weights, and store 8-byte halves of the
// 16-byte rows of the canonical no-swizzle K-major A tile in shared memory (the
// sampled im2col tile of that tap).  A single thread issues the tap's
// tcgen05.mma's against the resident weights into a double-buffered TMEM
// accumulator; four epilogue warps add the bias and store the blocked output.
// Every wait is bounded in time.  x is best given in 8-channel planes
// (launch_dcn_relayout8), where the two columns of a bilinear corner pair share
// a cache line; any supported layout gives the same result.
#include "common.cuh"
#include "sm100_ptx.cuh"

namespace nvisr {

namespace {

constexpr int TM = 128;
constexpr int NGATHER = 512;            // gather threads (a lane pair per pixel and chunk)
constexpr int MMA_WARP = NGATHER / 32;  // then 4 epilogue warps, the first also loads the weights and issues the MMAs
constexpr int NT = NGATHER + 128;       // 20 warps: 5 per SM sub-partition leaves 96 registers a thread
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

// Two 16-bit elements of a 32-bit word (element 0 in the low half) <-> two floats.
template <typename T>
__device__ __forceinline__ float2 unpack_pair(uint32_t w);
template <>
__device__ __forceinline__ float2 unpack_pair<__nv_bfloat16>(uint32_t w) {
    return make_float2(__uint_as_float(w << 16), __uint_as_float(w & 0xffff0000u));
}
template <>
__device__ __forceinline__ float2 unpack_pair<__half>(uint32_t w) {
    return __half22float2(*reinterpret_cast<const __half2 *>(&w));
}
template <typename T>
__device__ __forceinline__ uint32_t pack_pair(float lo, float hi);
template <>
__device__ __forceinline__ uint32_t pack_pair<__nv_bfloat16>(float lo, float hi) {
    const __nv_bfloat162 h = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<const uint32_t *>(&h);
}
template <>
__device__ __forceinline__ uint32_t pack_pair<__half>(float lo, float hi) {
    const __half2 h = __floats2half2_rn(lo, hi);
    return *reinterpret_cast<const uint32_t *>(&h);
}

// acc += s * v on two lanes: one packed FP32 FMA (each lane an IEEE fma, as the scalar form).
__device__ __forceinline__ void ffma2(float2 &acc, float s, float2 v) {
    uint64_t d, x, w;
    asm("mov.b64 %0, {%1, %2};" : "=l"(d) : "f"(acc.x), "f"(acc.y));
    asm("mov.b64 %0, {%1, %2};" : "=l"(x) : "f"(v.x), "f"(v.y));
    asm("mov.b64 %0, {%1, %1};" : "=l"(w) : "f"(s));
    asm("fma.rn.f32x2 %0, %1, %2, %0;" : "+l"(d) : "l"(w), "l"(x));
    asm("mov.b64 {%0, %1}, %2;" : "=f"(acc.x), "=f"(acc.y) : "l"(d));
}

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
    // the next kernel may be scheduled once every CTA got here (after the TMEM allocation);
    // the features and offsets are read only after the previous kernels completed
    griddep_launch_dependents();
    griddep_wait();

    if (warp < NGATHER / 32) {
        // ------------------------------------------------ gather producers
        // A lane pair holds one sample row of one (pixel, 8-channel chunk): lane c
        // loads column x0 + c.  With x in 8-channel planes both columns sit in one
        // 128-byte line (unless x0 ends a line), so a warp's load of 16 pixels of
        // one chunk touches about 18 lines instead of 32 (the L1 data stage takes
        // a wavefront per line).  The pair then swaps halves: lane 0 blends
        // channels 0-3 and lane 1 channels 4-7, each from all four corners.
        constexpr int NGW = NGATHER / 32;  // gather warps
        constexpr int WPC = NGW / NCH;     // warps per chunk
        constexpr int PPW = TM / WPC;      // pixels per warp
        constexpr int NPASS = PPW / 16;    // 16 pixels (32 lanes) per pass
        static_assert(NGW % NCH == 0 && PPW % 16 == 0, "gather mapping");
        const int cc = warp % NCH;         // channel chunk of this warp
        const int c = lane & 1;            // column x0 + c of the corner pair
        const int pb = (warp / NCH) * PPW + (lane >> 1);
        const uint8_t *x = static_cast<const uint8_t *>(a.x);
        const int G = a.groups;
        const int g = (cc * CPC) / (a.cin_pad / G);
        const bool tapm = a.om_tap_major != 0;
        const uint8_t *plane = x + (int64_t)((cc * CPC) / xcpc) * HW * xcpc * 2 + ((cc * CPC) % xcpc) * 2;
        const uint32_t pstride = (uint32_t)xcpc * 2;  // bytes per pixel in the plane (the plane is < 2 GiB)
        const uint32_t rowb = (uint32_t)W * pstride;  // bytes per row of the plane
        static_assert(NPASS % 2 == 0, "passes shared by a lane pair");
        constexpr int NP2 = NPASS / 2;
        int s = 0;
        uint32_t ph = 0;
        bool ok = true;
        // Corner values.  A corner is loaded only when its weight is nonzero, which the
        // bounds checks allow only inside the image.  A skipped corner keeps the value
        // of an earlier load (or zero), which its weight of zero cancels (x is finite).
        uint4 v[NPASS][2];
#pragma unroll
        for (int j = 0; j < NPASS; ++j) v[j][0] = v[j][1] = make_uint4(0u, 0u, 0u, 0u);
        // offsets and mask of this lane's passes h = 2i + c for tap k of tile t: loaded one
        // tap ahead of their use, so that their DRAM latency overlaps the previous tap
        auto load_om = [&](int t, int k, float2 (&d)[NP2], float (&lg)[NP2]) {
            const int y = t / tiles_x;
            const int xb = (t - y * tiles_x) * TM;
            const int cd = dcn_off_channel(g, k, G, tapm), cm = dcn_mask_channel(g, k, G, tapm);
            // float offsets in 32 bits (the tensor is < 2^31 floats)
            const uint32_t od = (uint32_t)(cd >> 2) * (uint32_t)HW * 4u + (cd & 3);
            const uint32_t oms = (uint32_t)(cm >> 2) * (uint32_t)HW * 4u + (cm & 3);
#pragma unroll
            for (int i = 0; i < NP2; ++i) {
                const int px = xb + pb + (2 * i + c) * 16;
                const uint32_t pix4 = (uint32_t)(y * W + min(px, W - 1)) * 4u;
                d[i] = __ldg(reinterpret_cast<const float2 *>(a.om + od + pix4));
                lg[i] = __ldg(a.om + oms + pix4);
            }
        };
        float2 nd[NP2];
        float nlg[NP2];
        if (blockIdx.x < ntiles && !a.starve) load_om(blockIdx.x, 0, nd, nlg);
        for (int t = blockIdx.x; t < ntiles && ok && !a.starve; t += gridDim.x) {
            const int y = t / tiles_x;
            const int xb = (t - y * tiles_x) * TM;
            for (int k = 0; k < 9; ++k) {
                // The lane pair shares its sample records: lane c computes those of the
                // passes h = 2i + c (offsets, mask, corner weights, position), and both
                // lanes then read each pass's record from the lane that computed it.
                // Record: row weights wy0, wy1 (times the mask), column weights wx0, wx1
                // (each zero outside the image), and y0 * W + x0.
                float2 cd2[NP2];
                float clg[NP2];
#pragma unroll
                for (int i = 0; i < NP2; ++i) {
                    cd2[i] = nd[i];
                    clg[i] = nlg[i];
                }
                if (k < 8) load_om(t, k + 1, nd, nlg);
                else if (t + (int)gridDim.x < ntiles) load_om(t + gridDim.x, 0, nd, nlg);
                float ewy0[NP2], ewy1[NP2], ewx0[NP2], ewx1[NP2];
                uint32_t eb[NP2];
#pragma unroll
                for (int i = 0; i < NP2; ++i) {
                    const int px = xb + pb + (2 * i + c) * 16;
                    const float2 d = cd2[i];
                    const float lg = clg[i];
                    // mask = sigmoid(logit) with the fast exponential and division: a relative
                    // error near 1e-6, far below the 16-bit rounding of the sample it scales
                    // (0 and 1 at the extremes); the exact form cost 4 % of the launch
                    const float m = a.mask_logits ? __fdividef(1.f, 1.f + __expf(-lg)) : lg;
                    const float sy = (float)(y + k / 3 - 1) + d.x;
                    const float sx = (float)(px + k % 3 - 1) + d.y;
                    const float fy = floorf(sy), fx = floorf(sx);
                    const int y0 = (int)fy, x0 = (int)fx;
                    const float ly = sy - fy, lx = sx - fx;
                    const bool in = px < W;
                    ewy0[i] = in && (unsigned)y0 < (unsigned)H ? (1.f - ly) * m : 0.f;
                    ewy1[i] = in && (unsigned)(y0 + 1) < (unsigned)H ? ly * m : 0.f;
                    ewx0[i] = (unsigned)x0 < (unsigned)W ? 1.f - lx : 0.f;
                    ewx1[i] = (unsigned)(x0 + 1) < (unsigned)W ? lx : 0.f;
                    eb[i] = (uint32_t)y0 * (uint32_t)W + (uint32_t)x0;
                }
                // each pass's record from the lane that computed it, then its corner loads
                // (every load of the tap is issued before the first blend)
                float wy0[NPASS], wy1[NPASS], wxo[NPASS], wxp[NPASS];
#pragma unroll
                for (int h = 0; h < NPASS; ++h) {
                    const int src = (lane & ~1) | (h & 1);
                    wy0[h] = __shfl_sync(0xffffffffu, ewy0[h >> 1], src);
                    wy1[h] = __shfl_sync(0xffffffffu, ewy1[h >> 1], src);
                    const float x0w = __shfl_sync(0xffffffffu, ewx0[h >> 1], src);
                    const float x1w = __shfl_sync(0xffffffffu, ewx1[h >> 1], src);
                    const uint32_t bs = __shfl_sync(0xffffffffu, eb[h >> 1], src);
                    wxo[h] = c ? x1w : x0w;  // weight of this lane's column x0 + c
                    wxp[h] = c ? x0w : x1w;  // weight of the partner's column
                    const uint32_t o0 = (bs + (uint32_t)c) * pstride;
                    if (wy0[h] != 0.f && wxo[h] != 0.f) v[h][0] = __ldg(reinterpret_cast<const uint4 *>(plane + o0));
                    if (wy1[h] != 0.f && wxo[h] != 0.f) v[h][1] = __ldg(reinterpret_cast<const uint4 *>(plane + (o0 + rowb)));
                }
                // the corner loads are in flight while the warp waits for a free stage; the
                // shuffles below need the whole warp: it leaves together
                const bool got = mbar_wait_bounded(&empty[s], ph ^ 1, abort, WAIT_NS);
                if (!__all_sync(0xffffffffu, got)) {
                    *abort = 1;
                    if (a.err) atomicExch(a.err, DEVERR_TIMEOUT);
                    ok = false;
                    break;
                }
                uint8_t *stg = stage0 + (size_t)s * STAGE + (size_t)cc * LBO + c * 8;
#pragma unroll
                for (int h = 0; h < NPASS; ++h) {
                    // lane 0 blends channels 0-3 and lane 1 channels 4-7: each keeps its half
                    // of its own column x0 + c and takes the partner's half of column x0 + 1 - c
                    float2 acc[2] = {make_float2(0.f, 0.f), make_float2(0.f, 0.f)};
#pragma unroll
                    for (int r = 0; r < 2; ++r) {
                        const uint4 q = v[h][r];
                        const uint32_t k0 = c ? q.z : q.x, k1 = c ? q.w : q.y;
                        const uint32_t g0 = __shfl_xor_sync(0xffffffffu, c ? q.x : q.z, 1);
                        const uint32_t g1 = __shfl_xor_sync(0xffffffffu, c ? q.y : q.w, 1);
                        const float wr = r ? wy1[h] : wy0[h];
                        const float wa = wr * wxo[h], wb = wr * wxp[h];
                        ffma2(acc[0], wa, unpack_pair<T>(k0));
                        ffma2(acc[1], wa, unpack_pair<T>(k1));
                        ffma2(acc[0], wb, unpack_pair<T>(g0));
                        ffma2(acc[1], wb, unpack_pair<T>(g1));
                    }
                    *reinterpret_cast<uint2 *>(stg + (size_t)(pb + h * 16) * 16) =
                        make_uint2(pack_pair<T>(acc[0].x, acc[0].y), pack_pair<T>(acc[1].x, acc[1].y));
                }
                fence_proxy_async();  // generic smem writes -> visible to the tensor core
                mbar_arrive(&full[s]);
                if (++s == S) { s = 0; ph ^= 1; }
            }
        }
    } else {
        // ------------------------------------------------ epilogue (the last 4 warps, one per lane quadrant);
        // lane 0 of the first also loads the weights and issues every tile's MMAs, and
        // that warp stores its quadrant of tile i - 1 after issuing tile i
        const bool issuer = warp == MMA_WARP;
        const int q = warp & 3;
        const int m = q * 32 + lane;
        uint8_t *yb = static_cast<uint8_t *>(a.y);
        const uint32_t wbase = smem_u32(wsm);
        bool run = true;     // this warp's epilogue still runs
        bool issue = true;   // the issuer still issues
        int s = 0, last_ab = -1;
        uint32_t ph = 0, last_par = 0;
        if (issuer) {
            if (lane == 0) {
                mbar_arrive_expect_tx(wbar, wbytes);
                for (uint32_t off = 0; off < wbytes; off += 32768u)
                    bulk_load(wsm + off, static_cast<const uint8_t *>(a.w) + off, min(32768u, wbytes - off), wbar);
                issue = mbar_wait_bounded(wbar, 0, abort, WAIT_NS);
                if (!issue) {
                    *abort = 1;
                    if (a.err) atomicExch(a.err, DEVERR_TIMEOUT);
                }
            }
            issue = __shfl_sync(0xffffffffu, issue, 0);
        }
        // issues the 9 taps of tile number it (buffer it & 1); false when a wait gave up
        auto issue_tile = [&](int it) -> bool {
            bool good = true;
            if (lane == 0) {
                const int ab = it & 1;
                const uint32_t u = (uint32_t)(it >> 1);
                good = mbar_wait_bounded(&tempty[ab], (u & 1) ^ 1, abort, WAIT_NS);
                if (good) {
                    tc_fence_after();
                    const uint32_t d_tmem = tmem_base + (uint32_t)(ab * NS);
                    for (int k = 0; k < 9 && good; ++k) {
                        good = mbar_wait_bounded(&full[s], ph, abort, WAIT_NS);
                        if (!good) {
                            if (k > 0) {  // the final wait then covers the taps already issued
                                umma_commit(&tfull[ab]);
                                last_ab = ab;
                                last_par = u & 1;
                            }
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
                    if (good) {
                        umma_commit(&tfull[ab]);
                        last_ab = ab;
                        last_par = u & 1;
                    }
                }
                if (!good) {
                    *abort = 1;
                    if (a.err) atomicExch(a.err, DEVERR_TIMEOUT);
                }
            }
            return __shfl_sync(0xffffffffu, good, 0);
        };
        // stores this warp's quadrant of tile t (number it); false when the wait gave up
        auto store_tile = [&](int t, int it) -> bool {
            const int ab = it & 1;
            const uint32_t u = (uint32_t)(it >> 1);
            const bool ok = __all_sync(0xffffffffu, mbar_wait_bounded(&tfull[ab], u & 1, abort, WAIT_NS));
            if (!ok) {
                if (lane == 0) {
                    *abort = 1;
                    if (a.err) atomicExch(a.err, DEVERR_TIMEOUT);
                }
                return false;
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
            return true;
        };
        int it = 0, prev_t = -1;
        for (int t = blockIdx.x; t < ntiles && run; t += gridDim.x, ++it) {
            if (issuer) {
                if (issue) issue = issue_tile(it);
                if (!issue) break;
                if (prev_t >= 0) run = store_tile(prev_t, it - 1);
                prev_t = t;
            } else {
                run = store_tile(t, it);
            }
        }
        if (issuer && issue && run && prev_t >= 0) store_tile(prev_t, it - 1);
        if (issuer && lane == 0) {
            // nothing of this CTA's may still be in flight when it leaves
            if (last_ab >= 0) mbar_wait_bounded(&tfull[last_ab], last_par, nullptr, WAIT_NS);
            mbar_wait_bounded(wbar, 0, nullptr, WAIT_NS);
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
    return launch_dependent(kern, grid, NT, smem, st, a, stages);
}

// One thread per (pixel, 8-channel chunk), chunk fastest: a warp reads four
// pixels' 128-byte channel lines and writes 64-byte runs of eight planes.
__global__ void relayout8_kernel(const uint4 *__restrict__ x, int64_t HW, int nch, int xcpc, uint4 *__restrict__ y) {
    const int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (u >= HW * nch) return;
    const int64_t p = u / nch;
    const int cc = (int)(u - p * nch);
    const int per = xcpc / 8;  // 16-byte chunks per pixel in the source layout
    y[(int64_t)cc * HW + p] = __ldg(x + ((int64_t)(cc / per) * HW + p) * per + cc % per);
}

}  // namespace

cudaError_t launch_dcn_relayout8(const void *x, int cpad, int H, int W, int x_cpc, void *y, cudaStream_t st) {
    if (cpad % 8 || x_cpc % 8 || cpad % x_cpc) return cudaErrorInvalidValue;
    const int64_t HW = (int64_t)H * W, units = HW * (cpad / 8);
    if (units == 0) return cudaSuccess;
    const int64_t blocks = (units + 255) / 256;
    relayout8_kernel<<<(unsigned)blocks, 256, 0, st>>>(static_cast<const uint4 *>(x), HW, cpad / 8, x_cpc,
                                                       static_cast<uint4 *>(y));
    return cudaGetLastError();
}

cudaError_t launch_dcn_tc(const DcnArgs &a0, cudaStream_t st) {
    DcnArgs a = a0;
    a.starve = test_starve();
    if (a.x_cpc == 0) a.x_cpc = 8;
    if (a.y_cpc == 0) a.y_cpc = 8;
    if (a.cin_pad != 64 || a.cout_pad != 64 || (a.cin_pad / a.groups) % 8) return cudaErrorNotSupported;
    // x in 8-channel planes (launch_dcn_relayout8); y blocked by 8 or 64 channels
    if (a.x_cpc != 8 || (a.y_cpc != 8 && a.y_cpc != 64)) return cudaErrorNotSupported;
    if (a.om_tap_major && a.groups % 2) return cudaErrorNotSupported;
    // 32-bit gather offsets into a plane of x and into om
    if ((int64_t)a.H * a.W * a.x_cpc * 2 >= (int64_t(1) << 31) || (int64_t)a.H * a.W * a.om_cpad >= (int64_t(1) << 31))
        return cudaErrorNotSupported;
    if (a.in_dt == DT_BF16 && a.out_dt == DT_BF16) return run<__nv_bfloat16, 64, 64>(a, st);
    if (a.in_dt == DT_F16 && a.out_dt == DT_F16) return run<__half, 64, 64>(a, st);
    return cudaErrorNotSupported;
}

}  // namespace nvisr
