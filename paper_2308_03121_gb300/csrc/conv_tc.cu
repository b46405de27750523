// Tensor-core implicit-GEMM convolution for sm_103a (tcgen05 + TMEM + TMA).
//
// The enhancement networks NNVISR runs are stacks of 3x3 convolutions
// (Section 3.1); here each layer is one GEMM
//     D[M = pixels][N = out channels] = sum_K A[pixel][tap, in channel] B[out][tap, in]
// computed without materialising im2col:
//
//  * Tile = 128 consecutive output pixels of one row (M = 128 = the MMA's M).
//  * A producer warp TMA-loads the tile's input halo -- KS rows x (128+KS-1)
//    pixels x NCH 16-byte channel chunks -- from the blocked activation
//    [C/cpc][H][W][cpc] into shared memory, out-of-image pixels zero-filled
//    by TMA (exact zero padding).  The halo lands in the canonical no-swizzle
//    K-major layout (8 pixels x 16 bytes per core matrix), so the A operand
//    of tap (ky, kx) is the same buffer addressed (ky*(128+KS-1) + kx)*16
//    bytes further: the 9 taps share one load.
//  * The layer's weights (or a slice of its output channels) stay resident in
//    shared memory for the whole persistent CTA, pre-arranged on the host in
//    the same core-matrix layout.
//  * One thread issues tcgen05.mma (kind::f16 for BF16/FP16, kind::f8f6f4 for
//    FP8 E4M3) into a double-buffered FP32 accumulator in TMEM; commits
//    release shared-memory stages and hand finished tiles to the epilogue.
//  * Four epilogue warps read TMEM (tcgen05.ld), apply scale, bias,
//    LeakyReLU(0.1) and the residual add, and store the blocked output; the
//    network's last layer instead applies PixelShuffle(2) and adds the skip
//    (upsampled input frame) into a planar float32 image.
//
// Every mbarrier wait is bounded in time; a CTA that gives up raises a flag
// seen by its other roles, records DEVERR_TIMEOUT in the error word, drains
// its own in-flight copies and MMAs, and frees its TMEM before returning.
#include <cudaTypedefs.h>

#include <mutex>
#include <type_traits>
#include <utility>
#include <vector>

#include "common.cuh"
#include "epilogue.cuh"
#include "rq_math.cuh"
#include "sm100_ptx.cuh"
#include "tc_util.cuh"

namespace nvisr {

namespace {

constexpr int TM = 128;
// warp 0: TMA producer, warp 1: MMA issuer + TMEM owner, warps 2-9: epilogue
// (two warps per TMEM lane quadrant, each owning half of the accumulator columns)
constexpr int NTHREADS = 320;
constexpr int ROWS_THREADS = 352;     // row kernel: + one warp that performs the MMA issuer's waits
// the 16-channel head adds a twelfth warp: with warp 0 it converts the tuple's float32 frames
constexpr int rows_threads(int cin, bool multi) { return cin == 16 && !multi ? 384 : ROWS_THREADS; }
constexpr int NEPI = 256;
constexpr uint64_t WAIT_NS = 2000000000ull;
constexpr int SMEM_LIMIT = 232448;  // 227 KB per CTA
constexpr int SMEM_HDR = 1024;      // barriers + TMEM slot + abort flag
// The tuple head's float32 staging: HEAD_NSL slots of HEAD_RPB input rows of each of up to 5
// frames (3 planes x pixels x0 - 4 .. x0 + 131).  One TMA box per frame covers a slot's rows:
// the boxes, not their bytes, set the rate at which the rows arrive (a second row per box
// cost no time), so a box carries four rows.
constexpr int HEAD_RPB = 4;
constexpr int HEAD_NSL = 4;
constexpr uint32_t HEAD_FROW32 = (HEAD_RPB * 3 * 136 * 4 + 127u) & ~127u;  // one frame of a slot, 128-byte aligned
constexpr int W_MAX = 112 * 1024;   // resident weight slice budget

struct TcParams {
    int H, W, nimg, cin_chunks;      // cin_chunks = cin_pad / cpc
    int cout, cout_pad, ns, nslice;
    const uint8_t *wts;               // nslice slices of wbytes
    uint32_t wbytes;
    int stages;
    const float *bias;
    int act;
    const uint8_t *res;
    uint8_t *y;
    float acc_scale, out_scale;
    float res_scale;                  // 1 / out_scale: residual values are stored pre-scaled
    uint8_t *y2;
    float y2_scale;
    unsigned *amax;
    // final PixelShuffle + skip
    float *ps_out;
    int64_t ps_pitch;
    ConvArgs skip;  // skip_* fields only
    int ps_act;
    int no_main;                      // row kernel: no 16-bit output, the FP8 copy (y2) is the output
    int ntup;                         // row kernel, 16-channel head: > 0 = read the tuple's ntup float32
    int tslot[8];                     //   frames from the ring (slots tslot[]) instead of a packed tensor
    int *err;
    int starve;                       // test drill: the producer loads no input, the pipeline waits run out
    FusedRq rq;                       // 2 x 2 shuffle tail: requantise in the epilogue
};

template <typename T>
__device__ __forceinline__ T to_elem(float v);
template <>
__device__ __forceinline__ __nv_bfloat16 to_elem<__nv_bfloat16>(float v) { return __float2bfloat16_rn(v); }
template <>
__device__ __forceinline__ __half to_elem<__half>(float v) { return __float2half_rn(v); }
template <>
__device__ __forceinline__ __nv_fp8_e4m3 to_elem<__nv_fp8_e4m3>(float v) { return __nv_fp8_e4m3(v); }
template <>
__device__ __forceinline__ float to_elem<float>(float v) { return v; }

template <typename T>
__device__ __forceinline__ float from_elem(T v) { return (float)v; }
template <>
__device__ __forceinline__ float from_elem<__nv_bfloat16>(__nv_bfloat16 v) { return __bfloat162float(v); }
template <>
__device__ __forceinline__ float from_elem<__half>(__half v) { return __half2float(v); }

__device__ __forceinline__ void raise_abort(volatile int *abort, int *err) {
    *abort = 1;
    if (err) atomicExch(err, DEVERR_TIMEOUT);
}

// Store 16 values as 16-bit or 8-bit elements at out (16 or 32 bytes... as
// whole 16-byte chunks of the blocked layout).
template <typename T>
__device__ __forceinline__ void store_vals(uint8_t *base, int64_t chunk_stride, int chunk0, const float *v,
                                           int n) {
    constexpr int CPC = 16 / sizeof(T);
    for (int c = 0; c < n / CPC; ++c) {
        alignas(16) T o[CPC];
#pragma unroll
        for (int e = 0; e < CPC; ++e) o[e] = to_elem<T>(v[c * CPC + e]);
        *reinterpret_cast<uint4 *>(base + (int64_t)(chunk0 + c) * chunk_stride) =
            *reinterpret_cast<const uint4 *>(o);
    }
}

// IN_DT: operand dtype; OUT_DT: dtype of y/res (16-bit, or E4M3 when the
// layer feeds only an FP8 consumer); NS: output channels per CTA slice; KS:
// kernel size; NCH: 16-byte chunks per pipeline stage (even); EPI: 0 blocked
// store, 1 PixelShuffle(2) + skip into planar float32, 2 PixelShuffle(2) +
// activation into a blocked tensor at twice the resolution.
template <int IN_DT, int OUT_DT, int NS, int KS, int NCH, int EPI, int CBI, int CBO>
__global__ void __launch_bounds__(NTHREADS, 1) conv_tc_kernel(const __grid_constant__ CUtensorMap tmap,
                                                              const TcParams p) {
    using TI = typename Elem<IN_DT>::T;
    using TO = typename Elem<OUT_DT>::T;
    constexpr int KIND = IN_DT == DT_E4M3 ? 1 : 0;
    constexpr int AFMT = IN_DT == DT_BF16 ? 1 : 0;
    constexpr uint32_t IDESC = instr_desc(TM, NS, AFMT, AFMT);
    constexpr int ROWS = KS;
    constexpr int PXS = TM + KS - 1;
    constexpr int PAD = (KS - 1) / 2;
    // CBI == 16: input chunks are 16 bytes, the stage is [chunk][row][px][16 B]
    //            (no swizzle; LBO_A = chunk stride).
    // CBI == 128: input chunks are 64 channels (128 bytes), TMA writes each as
    //            a 128-byte-swizzled [row][px][128 B] region of CREG bytes.
    constexpr uint32_t LBO_A = ROWS * PXS * 16;
    constexpr uint32_t CREG = (ROWS * PXS * 128 + 1023u) & ~1023u;
    // TMA destinations must be 128-byte aligned (1 KB for the swizzled atoms).
    constexpr uint32_t STAGE_BYTES = CBI == 16 ? ((NCH * LBO_A + 1023u) & ~1023u) : NCH * CREG;
    constexpr uint32_t TX_BYTES = CBI == 16 ? NCH * LBO_A : NCH * ROWS * PXS * 128;
    constexpr uint32_t NCOLS = (2 * NS <= 32) ? 32 : (2 * NS <= 64 ? 64 : (2 * NS <= 128 ? 128 : (2 * NS <= 256 ? 256 : 512)));
    constexpr int CPC_O = CBO / sizeof(TO);  // output channels per chunk
    constexpr int UPC_O = 16 / sizeof(TO);   // output channels per 16-byte unit
    static_assert(CBI == 128 || NCH % 2 == 0, "an MMA consumes two 16-byte K chunks");
    static_assert(CBI == 16 || KIND == 0, "swizzled inputs are 16-bit");

    extern __shared__ uint8_t smem_raw[];
    uint8_t *smem = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    const int S = p.stages;
    uint64_t *full = reinterpret_cast<uint64_t *>(smem);
    uint64_t *empty = full + 8;
    uint64_t *tfull = empty + 8;
    uint64_t *tempty = tfull + 2;
    uint64_t *wbar = tempty + 2;
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(wbar + 1);
    volatile int *abort = reinterpret_cast<volatile int *>(tmem_slot + 1);
    uint64_t *drain = reinterpret_cast<uint64_t *>(smem + 256);  // the issuer's MMAs, after an abort
    float *sbias = reinterpret_cast<float *>(smem + 512);  // this slice's NS biases
    uint8_t *wsm = smem + SMEM_HDR;
    uint8_t *stage0 = wsm + ((p.wbytes + 1023) & ~1023u);
    static_assert(NS * 4 <= 512, "bias staging fits the header");

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int slice = blockIdx.x % p.nslice;
    if (threadIdx.x >= 64 && threadIdx.x < 64 + NS) sbias[threadIdx.x - 64] = p.bias[slice * NS + threadIdx.x - 64];
    const int cta_stride = gridDim.x / p.nslice;
    const int cta0 = blockIdx.x / p.nslice;
    const int tiles_x = (p.W + TM - 1) / TM;
    const int ntiles = tiles_x * p.H * p.nimg;
    const int groups = p.cin_chunks / NCH;

    if (threadIdx.x == 0) {
        for (int s = 0; s < S; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        for (int a = 0; a < 2; ++a) {
            mbar_init(&tfull[a], 1);
            mbar_init(&tempty[a], NEPI);
        }
        mbar_init(wbar, 1);
        mbar_init(drain, 1);
        *abort = 0;
        fence_mbarrier_init();
    }
    if (warp == 1) {
        tmem_alloc(tmem_slot, NCOLS);
        tmem_relinquish();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem_base = *tmem_slot;
    griddep_launch_dependents();  // as in the row kernel: after the TMEM allocation
    griddep_wait();               // activations only after the previous kernels completed

    if (warp == 0) {
        if (lane == 0) {
            // ---------------- producer: weights once, then input halos
            mbar_arrive_expect_tx(wbar, p.wbytes);
            const uint8_t *wsrc = p.wts + (size_t)slice * p.wbytes;
            for (uint32_t off = 0; off < p.wbytes; off += 32768u) {
                const uint32_t n = min(32768u, p.wbytes - off);
                bulk_load(wsm + off, wsrc + off, n, wbar);
            }
            int s = 0;
            uint32_t ph = 0;
            int issued = 0;
            bool ok = true;
            for (int t = cta0; t < ntiles && ok && !p.starve; t += cta_stride) {
                const int img = t / (tiles_x * p.H);
                const int r = t - img * tiles_x * p.H;
                const int y = r / tiles_x;
                const int x0 = (r - y * tiles_x) * TM;
                for (int g = 0; g < groups; ++g) {
                    if (!mbar_wait_bounded(&empty[s], ph ^ 1, abort, WAIT_NS)) {
                        raise_abort(abort, p.err);
                        ok = false;
                        break;
                    }
                    mbar_arrive_expect_tx(&full[s], TX_BYTES);
                    if (CBI == 16) {
                        tma_load_4d(stage0 + (size_t)s * STAGE_BYTES, &tmap, &full[s], 0, x0 - PAD, y - PAD,
                                    img * p.cin_chunks + g * NCH);
                    } else {
#pragma unroll
                        for (int c = 0; c < NCH; ++c)
                            tma_load_4d(stage0 + (size_t)s * STAGE_BYTES + c * CREG, &tmap, &full[s], 0, x0 - PAD,
                                        y - PAD, img * p.cin_chunks + g * NCH + c);
                    }
                    ++issued;
                    if (++s == S) { s = 0; ph ^= 1; }
                }
            }
            // drain: the last load of every stage must land before the CTA exits
            for (int k = 0; k < S && k < issued; ++k) {
                const int idx = issued - 1 - k;  // load number idx went to stage idx % S, phase (idx / S) & 1
                mbar_wait_bounded(&full[idx % S], (uint32_t)((idx / S) & 1), nullptr, WAIT_NS);
            }
            mbar_wait_bounded(wbar, 0, nullptr, WAIT_NS);
        }
    } else if (warp == 1) {
        if (lane == 0) {
            // ---------------- MMA issuer
            bool ok = mbar_wait_bounded(wbar, 0, abort, WAIT_NS);
            if (!ok) raise_abort(abort, p.err);
            const uint32_t wbase = smem_u32(wsm);
            int s = 0;
            uint32_t ph = 0;
            int it = 0, last_a = -1;
            uint32_t last_par = 0;
            for (int t = cta0; t < ntiles && ok; t += cta_stride, ++it) {
                const int a = it & 1;
                const uint32_t u = (uint32_t)(it >> 1);
                if (!mbar_wait_bounded(&tempty[a], (u & 1) ^ 1, abort, WAIT_NS)) {
                    raise_abort(abort, p.err);
                    break;
                }
                tc_fence_after();
                const uint32_t d_tmem = tmem_base + (uint32_t)(a * NS);
                for (int g = 0; g < groups; ++g) {
                    if (!mbar_wait_bounded(&full[s], ph, abort, WAIT_NS)) {
                        raise_abort(abort, p.err);
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    // descriptors of tap 0 / K-step 0; others add (byte offset >> 4) to the start field
                    if (CBI == 16) {
                        const uint64_t a0 = smem_desc(smem_u32(stage0 + (size_t)s * STAGE_BYTES), LBO_A, 128);
                        const uint64_t b0 = smem_desc(wbase + (uint32_t)(g * NCH) * (uint32_t)(NS * 16), NS * 16, 128);
#pragma unroll 1
                        for (int tap = 0; tap < KS * KS; ++tap) {
                            const int ky = tap / KS, kx = tap % KS;
                            const uint64_t at = a0 + (uint64_t)((ky * PXS + kx) * 16 >> 4);
                            const uint64_t bt = b0 + (uint64_t)((uint32_t)(tap * p.cin_chunks) * (uint32_t)NS);
#pragma unroll
                            for (int j = 0; j < NCH / 2; ++j) {
                                umma<KIND>(d_tmem, at + (uint64_t)(2 * j * (LBO_A >> 4)),
                                           bt + (uint64_t)(2 * j * NS), IDESC, (g | tap | j) != 0 ? 1u : 0u);
                            }
                        }
                    } else {
                        // 128-byte swizzle: a tap's A rows start (ky*PXS + kx) rows into the region;
                        // the swizzle is a function of the address, so any row start is valid with
                        // base offset 0.  K advances 32 bytes (16 BF16/FP16) per MMA inside a row.
                        const uint64_t a0 = smem_desc_sw128(smem_u32(stage0 + (size_t)s * STAGE_BYTES), 0);
                        const uint64_t b0 = smem_desc_sw128(wbase + (uint32_t)(g * NCH) * (uint32_t)(NS * 128), 0);
#pragma unroll 1
                        for (int tap = 0; tap < KS * KS; ++tap) {
                            const int ky = tap / KS, kx = tap % KS;
                            const uint64_t at = a0 + (uint64_t)((ky * PXS + kx) * 128 >> 4);
                            const uint64_t bt = b0 + (uint64_t)((uint32_t)(tap * p.cin_chunks) * (uint32_t)(NS * 128 >> 4));
#pragma unroll
                            for (int c = 0; c < NCH; ++c)
#pragma unroll
                                for (int j = 0; j < 4; ++j)
                                    umma<KIND>(d_tmem, at + (uint64_t)((c * CREG + j * 32) >> 4),
                                               bt + (uint64_t)((c * NS * 128 + j * 32) >> 4), IDESC,
                                               (g | tap | c | j) != 0 ? 1u : 0u);
                        }
                    }
                    umma_commit(&empty[s]);
                    if (++s == S) { s = 0; ph ^= 1; }
                }
                if (!ok) break;
                umma_commit(&tfull[a]);
                last_a = a;
                last_par = u & 1;
            }
            // drain: MMAs must finish before TMEM is released
            if (last_a >= 0) mbar_wait_bounded(&tfull[last_a], last_par, nullptr, WAIT_NS);
            if (*abort) {
                // an early exit may leave MMAs of an unfinished tile, which no tile commit covers
                umma_commit(drain);
                mbar_wait_bounded(drain, 0, nullptr, WAIT_NS);
            }
        }
    } else {
        // ---------------- epilogue: warps 2..9; warp w owns TMEM lane quadrant (w % 4)
        // and accumulator columns [half * NH, (half + 1) * NH) of the slice
        const int q = warp & 3;
        const int half = (warp - 2) >> 2;
        constexpr int NH = NS / 2;
        constexpr int NRU = (EPI == 0) ? NH / UPC_O : 1;  // 16-byte output units per thread
        const int m = q * 32 + lane;
        const int col0 = half * NH;                        // first column (slice-local channel)
        const int64_t HW = (int64_t)p.H * p.W;
        auto unit_addr = [&](uint8_t *base, int ocn, int img, int n, int64_t pix, int64_t hw) -> uint8_t * {
            return base + (((int64_t)img * (ocn / CPC_O) + n / CPC_O) * hw + pix) * CBO +
                   (int64_t)(n % CPC_O) * (int64_t)sizeof(TO);
        };
        // residual prefetch one tile ahead: the next tile's loads are in flight
        // while this tile is finished
        uint4 rnext[NRU];
        auto prefetch = [&](int t2) {
            if (EPI != 0 || !p.res || t2 >= ntiles) return;
            const int img2 = t2 / (tiles_x * p.H);
            const int r2 = t2 - img2 * tiles_x * p.H;
            const int y2 = r2 / tiles_x;
            const int x2 = (r2 - y2 * tiles_x) * TM + m;
            if (x2 >= p.W) return;
            const int64_t pix2 = (int64_t)y2 * p.W + x2;
#pragma unroll
            for (int uu = 0; uu < NRU; ++uu)
                rnext[uu] = __ldg(reinterpret_cast<const uint4 *>(unit_addr(
                    const_cast<uint8_t *>(p.res), p.cout_pad, img2, slice * NS + col0 + uu * UPC_O, pix2, HW)));
        };
        prefetch(cta0);
        int it = 0;
        for (int t = cta0; t < ntiles; t += cta_stride, ++it) {
            const int a = it & 1;
            const uint32_t u = (uint32_t)(it >> 1);
            const int img = t / (tiles_x * p.H);
            const int r = t - img * tiles_x * p.H;
            const int y = r / tiles_x;
            const int x = (r - y * tiles_x) * TM + m;
            const bool valid = x < p.W;
            uint4 rres[NRU];
#pragma unroll
            for (int uu = 0; uu < NRU; ++uu) rres[uu] = rnext[uu];
            prefetch(t + cta_stride);
            bool ok = mbar_wait_bounded(&tfull[a], u & 1, abort, WAIT_NS);
            ok = __all_sync(0xffffffffu, ok);
            if (!ok) {
                if (lane == 0) raise_abort(abort, p.err);
                break;
            }
            tc_fence_after();
            const uint32_t taddr = tmem_base + ((uint32_t)(q * 32) << 16) + (uint32_t)(a * NS + col0);
            float v[NH];
            {
                if constexpr (NH == 8) {
                    uint32_t r8[8];
                    tmem_ld8_nowait(taddr, r8);
                    tmem_wait_ld();
#pragma unroll
                    for (int e = 0; e < 8; ++e) v[e] = __uint_as_float(r8[e]);
                } else {
                    uint32_t rr[NH / 16][16];
#pragma unroll
                    for (int j = 0; j < NH / 16; ++j) tmem_ld16_nowait(taddr + (uint32_t)(j * 16), rr[j]);
                    tmem_wait_ld();
#pragma unroll
                    for (int j = 0; j < NH / 16; ++j)
#pragma unroll
                        for (int e = 0; e < 16; ++e) v[j * 16 + e] = __uint_as_float(rr[j][e]);
                }
            }
            if (valid) {
#pragma unroll
                for (int e = 0; e < NH; ++e) {
                    float o = v[e] * p.acc_scale + sbias[col0 + e];
                    if (EPI != 1 && p.act == 1) o = lrelu(o);
                    v[e] = o;
                }
                if (EPI == 0) {
                    const int64_t pix = (int64_t)y * p.W + x;
                    const int n0 = slice * NS + col0;
                    if (p.res) {
#pragma unroll
                        for (int uu = 0; uu < NRU; ++uu) {
                            alignas(16) TO rv[UPC_O];
                            *reinterpret_cast<uint4 *>(rv) = rres[uu];
#pragma unroll
                            for (int e = 0; e < UPC_O; ++e) v[uu * UPC_O + e] += from_elem<TO>(rv[e]) * p.res_scale;
                        }
                    }
                    if (p.amax) {
                        float amax = 0.f;
#pragma unroll
                        for (int e = 0; e < NH; ++e) amax = fmaxf(amax, fabsf(v[e]));
                        atomicMax(p.amax, __float_as_uint(amax));
                    }
                    if (p.y2) {  // FP8 copy, 16-channel (16-byte) chunks
#pragma unroll
                        for (int c = 0; c < NH / 16; ++c) {
                            alignas(16) __nv_fp8_e4m3 o8[16];
#pragma unroll
                            for (int e = 0; e < 16; ++e) o8[e] = __nv_fp8_e4m3(v[c * 16 + e] * p.y2_scale);
                            *reinterpret_cast<uint4 *>(
                                p.y2 + (((int64_t)img * (p.cout_pad / 16) + n0 / 16 + c) * HW + pix) * 16) =
                                *reinterpret_cast<const uint4 *>(o8);
                        }
                    }
#pragma unroll
                    for (int uu = 0; uu < NRU; ++uu) {
                        alignas(16) TO o[UPC_O];
#pragma unroll
                        for (int e = 0; e < UPC_O; ++e) o[e] = to_elem<TO>(v[uu * UPC_O + e] * p.out_scale);
                        *reinterpret_cast<uint4 *>(unit_addr(p.y, p.cout_pad, img, n0 + uu * UPC_O, pix, HW)) =
                            *reinterpret_cast<const uint4 *>(o);
                    }
                } else if (EPI == 1) {
                    // PixelShuffle(2): this warp's channels col0..col0+NH-1 are shuffled channels
                    // col0/4 .. at sub-positions (i, j) = (n % 4) / 2, n % 2; planar float32 out
                    const int H2 = 2 * p.H;
#pragma unroll
                    for (int cl = 0; cl < NH / 4; ++cl) {
                        const int c = col0 / 4 + cl;
                        if (c >= p.cout / 4) break;
                        float *dst = p.ps_out + (int64_t)img * (p.cout / 4) * p.ps_pitch * H2 +
                                     (int64_t)c * p.ps_pitch * H2 + (int64_t)(2 * y) * p.ps_pitch + 2 * x;
                        *reinterpret_cast<float2 *>(dst) = make_float2(v[cl * 4 + 0], v[cl * 4 + 1]);
                        *reinterpret_cast<float2 *>(dst + p.ps_pitch) = make_float2(v[cl * 4 + 2], v[cl * 4 + 3]);
                    }
                } else {
                    // PixelShuffle(2) into a blocked tensor of cout/4 channels at twice the resolution:
                    // this warp's NH columns are shuffled channels c_base .. c_base + NH/4 - 1
                    const int cps = p.cout / 4;
                    const int64_t HW4 = 4 * HW;
                    const int c_base = (slice * NS + col0) / 4;
#pragma unroll
                    for (int ij = 0; ij < 4; ++ij) {
                        const int Y = 2 * y + (ij >> 1), X = 2 * x + (ij & 1);
                        const int64_t pix2 = (int64_t)Y * (2 * p.W) + X;
#pragma unroll
                        for (int h = 0; h < NH / 4 / UPC_O; ++h) {
                            alignas(16) TO o[UPC_O];
#pragma unroll
                            for (int e = 0; e < UPC_O; ++e) {
                                float val = v[(h * UPC_O + e) * 4 + ij];
                                if (p.ps_act == 1) val = lrelu(val);
                                o[e] = to_elem<TO>(val * p.out_scale);
                            }
                            *reinterpret_cast<uint4 *>(unit_addr(p.y, cps, img, c_base + h * UPC_O, pix2, HW4)) =
                                *reinterpret_cast<const uint4 *>(o);
                        }
                    }
                }
            }
            tc_fence_before();
            mbar_arrive(&tempty[a]);
        }
    }
    __syncthreads();
    if (warp == 1) {
        __syncwarp();
        tc_fence_after();
        tmem_dealloc(tmem_base, NCOLS);
    }
}

// ---------------------------------------------------------------- row-streaming 3x3 conv

// Row-streaming variant for 64 -> 64 channel 3x3 layers (the residual trunks).
// A CTA owns a vertical strip of one 128-pixel column and walks its input rows
// top to bottom.  Input row r feeds output rows r+1, r and r-1 through the
// vertical taps ky = 0, 1, 2, so the three taps' weights are stacked along N:
// one N = 192 MMA per (kx, 16-channel K step) reads the input row once and
// accumulates into three consecutive output-row accumulators.  Accumulators
// live in a TMEM ring of 8 output rows (64 columns each); output row o
// receives its first product (accumulate = 0) from input row o-1 at kx = 0,
// K step 0, is complete after input row o+1, and is then drained by the
// epilogue, which frees its slot.  Per output row: 13 MMAs, one 130-pixel TMA
// row load (plus 2 halo rows per strip) and a third of the operand traffic of
// the per-tap form.
// Fused requantisation (FusedRq) of one low-resolution pixel (o, x) of a 2 x 2 shuffle
// tail: the same arithmetic, in the same order, as the separate requantise kernels
// (requant420_kernel's 2x skip form for 4:2:0, the general skip for 4:4:4), so the codes
// are those of the unfused path.
// Bilinear x2 skip (align_corners = False, edge clamp) at output (2o + dy, 2x + dx), the
// general form: source position max((Y + 1/2) / 2 - 1/2, 0) per axis.
__device__ __forceinline__ float rq_skip_general(const FusedRq &rq, int c, int Y, int X, int H, int W) {
    const float *pl = rq.skip + (int64_t)c * rq.skip_plane;
    const float sy = fmaxf(((float)Y + 0.5f) * 0.5f - 0.5f, 0.f);
    const float sx = fmaxf(((float)X + 0.5f) * 0.5f - 0.5f, 0.f);
    const int y0 = min((int)sy, H - 1), x0 = min((int)sx, W - 1);
    const int y1 = min(y0 + 1, H - 1), x1 = min(x0 + 1, W - 1);
    const float ly = sy - (float)y0, lx = sx - (float)x0;
    const float *r0 = pl + (int64_t)y0 * rq.skip_pitch;
    const float *r1 = pl + (int64_t)y1 * rq.skip_pitch;
    return rq_bilerp(__ldg(r0 + x0), __ldg(r0 + x1), __ldg(r1 + x0), __ldg(r1 + x1), lx, ly);
}

// The skip frame's 3 x 3 neighbourhood of pixel (o, x) per channel (rows o - 1 .. o + 1,
// columns x - 1 .. x + 1, clamped to the frame): the samples the 4:2:0 2x form of
// rq_pixel blends.  Loaded ahead of the row's accumulator, so that their latency
// overlaps the wait for it.
__device__ __forceinline__ void rq_skip_load(const FusedRq &rq, int o, int x, int H, int W, float (&lr)[3][3][3]) {
    const int rows[3] = {max(o - 1, 0), o, min(o + 1, H - 1)};
    const int cols[3] = {max(x - 1, 0), x, min(x + 1, W - 1)};
#pragma unroll
    for (int c = 0; c < 3; ++c)
#pragma unroll
        for (int rr = 0; rr < 3; ++rr) {
            const float *row = rq.skip + (int64_t)c * rq.skip_plane + (int64_t)rows[rr] * rq.skip_pitch;
#pragma unroll
            for (int cc = 0; cc < 3; ++cc) lr[c][rr][cc] = __ldg(row + cols[cc]);
        }
}

// Output samples (residual v[4c + 2dy + dx] + skip) -> luma codes yq[dy][dx], full-resolution
// chroma cb[dy][dx], cr[dy][dx] (before downsampling and rounding).  lr: the neighbourhood
// rq_skip_load read, for a 4:2:0 skip.
__device__ __forceinline__ void rq_pixel(const FusedRq &rq, const float *v, int o, int x, int H, int W,
                                         const float (&lr)[3][3][3], float (&yq)[2][2], float (&cb)[2][2],
                                         float (&cr)[2][2]) {
    float smp[3][2][2];
    if (rq.skip && rq.sub420) {
        // requant420's 2x form: rows (o-1, o) with (1/4, 3/4) for dy = 0 and (o, o+1) with
        // (3/4, 1/4) for dy = 1; columns likewise, all clamped to the frame
#pragma unroll
        for (int c = 0; c < 3; ++c) {
#pragma unroll
            for (int dy = 0; dy < 2; ++dy)
#pragma unroll
                for (int dx = 0; dx < 2; ++dx) {
                    const int c0 = dx;
                    const float wl = dx ? 0.75f : 0.25f, wr = dx ? 0.25f : 0.75f;
                    const float wt = dy ? 0.75f : 0.25f, wb = dy ? 0.25f : 0.75f;
                    const float top = rq_blend(lr[c][dy][c0], wl, lr[c][dy][c0 + 1], wr);
                    const float bot = rq_blend(lr[c][dy + 1][c0], wl, lr[c][dy + 1][c0 + 1], wr);
                    smp[c][dy][dx] = __fadd_rn(v[4 * c + 2 * dy + dx], rq_blend(top, wt, bot, wb));
                }
        }
    } else {
#pragma unroll
        for (int c = 0; c < 3; ++c)
#pragma unroll
            for (int dy = 0; dy < 2; ++dy)
#pragma unroll
                for (int dx = 0; dx < 2; ++dx) {
                    const float r = v[4 * c + 2 * dy + dx];
                    smp[c][dy][dx] = rq.skip ? __fadd_rn(r, rq_skip_general(rq, c, 2 * o + dy, 2 * x + dx, H, W)) : r;
                }
    }
#pragma unroll
    for (int dy = 0; dy < 2; ++dy)
#pragma unroll
        for (int dx = 0; dx < 2; ++dx) {
            float y;
            rq_ycc(smp[0][dy][dx], smp[1][dy][dx], smp[2][dy][dx], rq.kr, rq.kg, rq.kb, rq.cb_s, rq.cr_s, y,
                   cb[dy][dx], cr[dy][dx]);
            yq[dy][dx] = rq_code(y, rq.y_mul, rq.y_add, rq.vmax);
        }
}

// Stores two adjacent codes of row `row` at columns 2x, 2x + 1.
__device__ __forceinline__ void rq_store2(uint8_t *plane, int64_t pitch, int row, int x, bool wide, float a, float b) {
    uint8_t *p = plane + (int64_t)row * pitch;
    if (wide) *reinterpret_cast<uint32_t *>(p + 4 * (int64_t)x) = (uint32_t)(int)a | ((uint32_t)(int)b << 16);
    else *reinterpret_cast<uint16_t *>(p + 2 * (int64_t)x) = (uint16_t)((uint32_t)(int)a | ((uint32_t)(int)b << 8));
}
__device__ __forceinline__ void rq_store1(uint8_t *plane, int64_t pitch, int row, int x, bool wide, float a) {
    uint8_t *p = plane + (int64_t)row * pitch;
    if (wide) reinterpret_cast<uint16_t *>(p)[x] = (uint16_t)(int)a;
    else p[x] = (uint8_t)(int)a;
}

struct RowPlan {
    int xtiles;   // 128-pixel columns per row
    int bands;    // row bands per column (strips = xtiles * bands * nimg)
    int rps;      // rows per band
};

template <int IN_DT, int OUT_DT, int CBO, bool MULTI, int NPR, bool PS, int CIN>
__global__ void __launch_bounds__(rows_threads(CIN, MULTI), 1) conv_rows_kernel(const __grid_constant__ CUtensorMap tmap,
                                                                const __grid_constant__ CUtensorMap ymap,
                                                                const __grid_constant__ CUtensorMap rmap,
                                                                const TcParams p, const RowPlan rp,
                                                                const RowProblem *__restrict__ probs, int nprob) {
    using TO = typename Elem<OUT_DT>::T;
    constexpr int AFMT = IN_DT == DT_BF16 ? 1 : 0;       // BF16 (kind::f16) or E4M3 / F16 (0)
    constexpr bool F8IN = IN_DT == DT_E4M3;              // FP8 rows: kind::f8f6f4, K = 32
    constexpr int KIND = F8IN ? 1 : 0;
    constexpr int PXS = TM + 2;
    // CIN: input channels of a row.  64: one 128-byte line per pixel, 128-byte swizzled;
    // 128: two such lines per pixel, one 130-pixel region per 64-channel chunk
    // (chunk 1 starts 130 lines after chunk 0: the swizzle is a function of the
    // address, so a region may start inside a 1 KB atom);
    // 16 (the tuple head): two 16-byte channel chunks per pixel, canonical no-swizzle
    // layout [chunk][pixel][16 B] (K core matrices LBO_A apart)
    // FP8 (64 channels): four 16-byte chunks per pixel in the same no-swizzle
    // [chunk][pixel][16 B] layout as the 16-channel head, two chunks per K = 32 step
    static_assert(CIN == 64 || (CIN == 128 && NPR == 64 && !PS && !MULTI) || (CIN == 16 && NPR == 64 && !PS),
                  "64- or 128-channel rows or the 16-channel head");
    static_assert(!F8IN || (CIN == 64 && NPR == 64 && !PS && !MULTI), "FP8 rows: 64 -> 64 trunk layers");
    constexpr bool SW = CIN != 16 && !F8IN;                   // 128-byte swizzled operands
    constexpr int NCHK = F8IN ? 4 : 2;                        // 16-byte chunks per pixel (no-swizzle forms)
    constexpr int KSTEPS = SW ? CIN / 16 : NCHK / 2;         // MMA K steps per kx
    constexpr uint32_t AREG = PXS * 128;                      // one 64-channel chunk of a row (swizzled forms)
    constexpr uint32_t AROW = SW ? (CIN / 64) * AREG : NCHK * PXS * 16;  // bytes of one 130-pixel input row
    constexpr uint32_t ROWB = (AROW + 1023u) & ~1023u;
    constexpr uint32_t LBO_A = PXS * 16, LBO_B = 3 * NPR * 16;
    // NPR: accumulator columns of one output row (= padded output channels: 64 for the
    // trunk, 16 for the 12-channel PixelShuffle tail); PS: PixelShuffle(2) epilogue,
    // with NPR 16 into planar float32 instead of the blocked 16-bit row store, with
    // NPR 64 (a 64 -> 256 layer) into a blocked 64-channel 16-bit tensor at twice the
    // size: slice s = 2i + j holds conv channels 4n + s, i.e. all 64 channels of
    // output pixel (2o + i, 2x + j), written as one 128-byte line per pixel
    static_assert(NPR == 64 || (NPR == 16 && PS), "64-channel trunk rows or 16-channel shuffle tail");
    constexpr bool PSB = PS && NPR == 64;
    // weights of one kx: [64-channel chunk][ky' = 2 - ky][NPR][128 B] (swizzled forms) or
    // [NCHK chunks][3 * NPR][16 B] (CIN 16, FP8)
    constexpr uint32_t WKX = SW ? (CIN / 64) * 3 * NPR * 128 : NCHK * 3 * NPR * 16;
    constexpr uint32_t TILEB = TM * 128;                      // one 128-pixel output / residual row tile
    constexpr int NSLOT = 8;                                  // output-row accumulators in TMEM
    static_assert(NSLOT == 8, "slot index and phase use & 7 and >> 3");
    constexpr uint32_t NCOLS = NPR == 64 ? 512 : 128;
    constexpr int UPC_O = 16 / sizeof(TO);
    constexpr int NU = 64 / UPC_O;                            // 16-byte units of a pixel's 64 channels
    constexpr int NGRP = 128;                                 // threads of one epilogue group
    // OUT_DT F32: float32 output in 4-channel (16-byte) units, stored straight from
    // registers (no staging tile); the layer's output channels come in 64-channel
    // slices, one per CTA group (see slice below)
    constexpr bool F32OUT = OUT_DT == DT_F32;
    static_assert((CBO == 128 && sizeof(TO) == 2) || (F32OUT && CBO == 16 && CIN == 128),
                  "64-channel 16-bit tiles, or float32 4-channel units from 128-channel rows");

    extern __shared__ uint8_t smem_raw[];
    uint8_t *smem = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    const int S = p.stages;
    uint64_t *full = reinterpret_cast<uint64_t *>(smem);
    uint64_t *empty = full + 8;
    uint64_t *rowdone = empty + 8;
    uint64_t *slotfree = rowdone + NSLOT;
    uint64_t *resfull = slotfree + NSLOT;  // one per epilogue group
    uint64_t *wbar = resfull + 2;
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(wbar + 1);
    volatile int *abort = reinterpret_cast<volatile int *>(tmem_slot + 1);
    // per-group stop flags: written between a group's two per-row named
    // barriers, read after the second, so a group's warps leave on the same row
    volatile int *grp_stop = reinterpret_cast<volatile int *>(tmem_slot + 2);
    // input rows (global count) whose input has landed and whose fresh TMEM slot is
    // drained, published by the wait warp for the MMA issuer
    int *ready = reinterpret_cast<int *>(tmem_slot + 4);
    uint64_t *drain = reinterpret_cast<uint64_t *>(smem + 448);  // the issuer's MMAs, after an abort
    float *sbias = reinterpret_cast<float *>(smem + 512);
    uint8_t *wsm = smem + SMEM_HDR;
    uint8_t *stage0 = wsm + 3 * WKX;
    uint8_t *obuf = stage0 + (size_t)S * ROWB;   // output staging tile per group
    uint8_t *rbuf = obuf + 2 * TILEB;            // residual tile per group

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    // MULTI: the strips of several images of different sizes (one per problem,
    // each with its own tensor maps in global memory) share the launch
    const int strips_per_img = rp.xtiles * rp.bands;
    const int nstrips = MULTI ? probs[nprob - 1].strip0 + probs[nprob - 1].nstrips : strips_per_img * p.nimg;
    const bool has_res = MULTI ? probs[0].has_res != 0 : p.res != nullptr;
    // output-channel slices: CTA b computes slice b % nslice of strips b / nslice, + step, ...
    const int nsl = MULTI ? 1 : p.nslice;
    const int slice = (int)blockIdx.x % nsl;
    const int cta0 = (int)blockIdx.x / nsl, cstride = (int)gridDim.x / nsl;
    // unit scales: packed bias / activation / residual arithmetic (the FP8 copy and the
    // amax read the same values either way)
    const bool plain = p.acc_scale == 1.f && p.out_scale == 1.f && p.res_scale == 1.f;
    auto strip_of = [&](int sidx, int &img, int &x0, int &ra, int &rb, int &pi) {
        if (MULTI) {
            pi = 0;
            while (pi + 1 < nprob && sidx >= probs[pi + 1].strip0) ++pi;
            const RowProblem &q = probs[pi];
            const int local = sidx - q.strip0;
            const int band = local / q.xtiles;
            img = 0;
            x0 = (local - band * q.xtiles) * TM;
            ra = band * q.rps;
            rb = min(q.H, ra + q.rps);
            return;
        }
        pi = 0;
        img = sidx / strips_per_img;
        const int rem = sidx - img * strips_per_img;
        const int band = rem / rp.xtiles;
        x0 = (rem - band * rp.xtiles) * TM;
        ra = band * rp.rps;
        rb = min(p.H, ra + rp.rps);
    };
    auto tmap_of = [&](int pi) { return MULTI ? &probs[pi].tmap : &tmap; };
    auto ymap_of = [&](int pi) { return MULTI ? &probs[pi].ymap : &ymap; };
    auto rmap_of = [&](int pi) { return MULTI ? &probs[pi].rmap : &rmap; };
    auto width_of = [&](int pi) { return MULTI ? probs[pi].W : p.W; };
    if (threadIdx.x >= 64 && threadIdx.x < 64 + NPR)
        sbias[threadIdx.x - 64] = p.bias[PSB ? 4 * (threadIdx.x - 64) + slice : slice * NPR + threadIdx.x - 64];
    // 16-channel head reading the tuple's float32 frames (ntup > 0): warps 0 and 11 convert
    // each row from the float32 staging slots (TMA from the ring) into the stage
    constexpr int RPB = HEAD_RPB;                              // input rows per staging slot
    constexpr int NST32 = HEAD_NSL;                            // staging slots
    constexpr uint32_t PLN32 = RPB * 136 * 4;                  // one plane of a frame: RPB rows of x0-4 .. x0+131
    constexpr uint32_t BOX32 = 3 * PLN32;                      // one frame's box
    constexpr uint32_t FROW32 = HEAD_FROW32;                   // its place in a slot
    constexpr uint32_t SROW32 = 5 * FROW32;                    // a slot: up to 5 frames
    constexpr bool TUPF = CIN == 16 && IN_DT != DT_E4M3;
    const bool tup = TUPF && p.ntup > 0;
    uint64_t *full32 = reinterpret_cast<uint64_t *>(smem + 320);
    uint64_t *empty32 = full32 + NST32;
    if (threadIdx.x == 0) {
        for (int s = 0; s < S; ++s) {
            mbar_init(&full[s], tup ? 64 : 1);  // TMA completion, or the two converting warps' arrivals
            mbar_init(&empty[s], 1);
        }
        for (int k = 0; k < NST32; ++k) {
            mbar_init(&full32[k], 1);
            mbar_init(&empty32[k], 64);
        }
        for (int k = 0; k < NSLOT; ++k) {
            mbar_init(&rowdone[k], 1);
            mbar_init(&slotfree[k], NGRP);
        }
        mbar_init(&resfull[0], 1);
        mbar_init(&resfull[1], 1);
        mbar_init(wbar, 1);
        mbar_init(drain, 1);
        *abort = 0;
        grp_stop[0] = 0;
        grp_stop[1] = 0;
        *ready = 0;
        fence_mbarrier_init();
        // the weights are written once at filter creation, so they load before the wait
        // below, while the previous layer may still be running
        mbar_arrive_expect_tx(wbar, 3 * WKX);
        const uint8_t *wsrc = p.wts + (size_t)slice * 3 * WKX;
        for (uint32_t off = 0; off < 3 * WKX; off += 32768u)
            bulk_load(wsm + off, wsrc + off, min(32768u, 3 * WKX - off), wbar);
    }
    if (warp == 1) {
        tmem_alloc(tmem_slot, NCOLS);
        tmem_relinquish();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem_base = *tmem_slot;
    // The next layer may now be scheduled, taking each SM as this CTA leaves it (signalled
    // after the TMEM allocation, so a CTA of the next layer never holds TMEM this one waits
    // for).  Activations (inputs, residuals and the buffers this layer overwrites) belong to
    // the previous kernels of the stream: nothing below touches them before they completed.
    griddep_launch_dependents();
    griddep_wait();

    if ((warp == 0 || warp == 11) && tup) {
        // ---------------- producer (warps 0 and 11), tuple head: warp 0 lane 0 keeps up to
        // NST32 slots of the ntup float32 frames in flight, each RPB input rows of a strip
        // (TMA boxes of 136 pixels from x0 - 4, so the innermost coordinate stays 16-byte
        // aligned; OOB reads as zero); per input row the two warps convert the row (warp 0
        // pixels 0-63, warp 11 pixels 64-129) into the stage's [2 chunks][130 px][8 channels]
        // 16-bit layout, channels frame-major (the tuple pack's layout) with round-to-nearest
        // (its rounding).
        if constexpr (TUPF) {
        const bool loader = warp == 0;
        const int px0 = loader ? 0 : 64;
        using TI = typename Elem<IN_DT>::T;
        uint8_t *st32 = obuf + 2 * TILEB;
        int t_sidx = cta0, t_r = 0, t_ra = 0, t_rb = 0, t_x0 = 0, t_img = 0, t_pi = 0;
        bool t_live = false;
        // positions the load cursor on the next slot's first input row in the converting order
        // (a strip's rows ra - 1 .. rb in slots of RPB rows; the last may hold fewer)
        auto t_next = [&]() -> bool {
            if (t_live && (t_r += RPB) <= t_rb) return true;
            if (t_live) t_sidx += cstride;
            t_live = false;
            if (t_sidx >= nstrips) return false;
            strip_of(t_sidx, t_img, t_x0, t_ra, t_rb, t_pi);
            t_r = t_ra - 1;
            t_live = true;
            return true;
        };
        int gin = 0, pin = 0, issued = 0;  // pin: slots whose rows this warp has converted
        bool ok = true;
        for (int sidx = cta0; sidx < nstrips && ok; sidx += cstride) {
            int img, x0, ra, rb, pi;
            strip_of(sidx, img, x0, ra, rb, pi);
            for (int r = ra - 1; r <= rb; ++r, ++gin) {
                const int h = (r - (ra - 1)) % RPB;  // the row's place in its slot
                if (loader && lane == 0) {
                    while (ok && !p.starve && issued < pin + NST32 && t_next()) {
                        const int k = issued % NST32;
                        // the slot's previous rows (slot issued - NST32 < pin) were converted by this
                        // warp; the wait covers warp 11's half
                        if (!mbar_wait_bounded(&empty32[k], (uint32_t)((issued / NST32) & 1) ^ 1u, abort, WAIT_NS)) {
                            ok = false;
                            break;
                        }
                        mbar_arrive_expect_tx(&full32[k], (uint32_t)p.ntup * BOX32);
                        for (int f = 0; f < p.ntup; ++f)
                            tma_load_4d(st32 + (size_t)k * SROW32 + (size_t)f * FROW32, tmap_of(t_pi), &full32[k],
                                        t_x0 - 4, t_r, 0, p.tslot[f]);
                        ++issued;
                    }
                }
                const int k = pin % NST32, s = gin % S;
                bool w = __shfl_sync(0xffffffffu, ok, 0);
                if (h == 0) w = w && mbar_wait_bounded(&full32[k], (uint32_t)((pin / NST32) & 1), abort, WAIT_NS);
                w = w && mbar_wait_bounded(&empty[s], (uint32_t)((gin / S) & 1) ^ 1u, abort, WAIT_NS);
                if (!__all_sync(0xffffffffu, w)) {
                    if (lane == 0) raise_abort(abort, p.err);
                    ok = false;
                    break;
                }
                // lane l converts stage pixels px0 + l, px0 + l + 32 (warp 11: then lanes 0, 1 pixels
                // 128, 129): all loads first (conflict-free 4-byte loads), then conversion and one
                // 16-byte store per chunk and pixel (consecutive across the warp).  Stage pixel px is
                // staged float px + 3 of each channel row; channels of frames >= ntup read stale
                // staging and are replaced by zero.
                const uint32_t src = smem_u32(st32 + (size_t)k * SROW32) + (uint32_t)h * 544u + 12u;
                const uint32_t dst = smem_u32(stage0 + (size_t)s * ROWB);
                const int nch = 3 * p.ntup;
                auto chan = [](int ch) { return (uint32_t)((ch / 3) * FROW32 + (ch % 3) * PLN32); };
                auto emit = [&](int px, const float (&u)[16]) {
                    uint4 c0, c1;
                    c0.x = pack2<TI>(u[0], u[1]);   c0.y = pack2<TI>(u[2], u[3]);
                    c0.z = pack2<TI>(u[4], u[5]);   c0.w = pack2<TI>(u[6], u[7]);
                    c1.x = pack2<TI>(u[8], u[9]);   c1.y = pack2<TI>(u[10], u[11]);
                    c1.z = pack2<TI>(u[12], u[13]); c1.w = pack2<TI>(u[14], u[15]);
                    st_shared_u4(dst + (uint32_t)px * 16, c0);
                    st_shared_u4(dst + (uint32_t)(PXS + px) * 16, c1);
                };
                {
                    float v[2][16];
#pragma unroll
                    for (int ch = 0; ch < 15; ++ch)
#pragma unroll
                        for (int q = 0; q < 2; ++q)
                            v[q][ch] = ld_shared_f32(src + chan(ch) + (uint32_t)(px0 + lane + 32 * q) * 4);
#pragma unroll
                    for (int q = 0; q < 2; ++q) {
#pragma unroll
                        for (int ch = 0; ch < 15; ++ch) v[q][ch] = ch < nch ? v[q][ch] : 0.f;
                        v[q][15] = 0.f;
                        emit(px0 + lane + 32 * q, v[q]);
                    }
                }
                static_assert(PXS == 130, "two halves of 64 pixels and a two-pixel tail");
                if (!loader && lane < 2) {
                    float v[16];
#pragma unroll
                    for (int ch = 0; ch < 15; ++ch) v[ch] = ld_shared_f32(src + chan(ch) + (uint32_t)(128 + lane) * 4);
#pragma unroll
                    for (int ch = 0; ch < 15; ++ch) v[ch] = ch < nch ? v[ch] : 0.f;
                    v[15] = 0.f;
                    emit(128 + lane, v);
                }
                fence_proxy_async();  // shared-memory writes -> the tensor core's async proxy
                mbar_arrive(&full[s]);
                if (h == RPB - 1 || r == rb) {  // the slot's last row
                    mbar_arrive(&empty32[k]);
                    ++pin;
                }
            }
        }
        if (loader && lane == 0) {
            // loads still in flight after an early exit land before the CTA ends
            for (int j = pin; j < issued; ++j)
                mbar_wait_bounded(&full32[j % NST32], (uint32_t)((j / NST32) & 1), nullptr, WAIT_NS);
            mbar_wait_bounded(wbar, 0, nullptr, WAIT_NS);
        }
        }
    } else if (warp == 0) {
        if (lane == 0) {
            // ---------------- producer: one input row per stage (the weights were issued
            // in the prologue)
            int gin = 0;
            bool ok = true;
            for (int sidx = cta0; sidx < nstrips && ok && !p.starve; sidx += cstride) {
                int img, x0, ra, rb, pi;
                strip_of(sidx, img, x0, ra, rb, pi);
                for (int r = ra - 1; r <= rb; ++r, ++gin) {
                    const int s = gin % S;
                    if (!mbar_wait_bounded(&empty[s], ((gin / S) & 1) ^ 1, abort, WAIT_NS)) {
                        raise_abort(abort, p.err);
                        ok = false;
                        break;
                    }
                    mbar_arrive_expect_tx(&full[s], AROW);
                    tma_load_4d(stage0 + (size_t)s * ROWB, tmap_of(pi), &full[s], 0, x0 - 1, r,
                                SW ? (CIN == 64 ? img : 2 * img) : NCHK * img);
                    // (CIN 128, 16 and FP8: one box of all channel chunks of the row)
                }
            }
            for (int k = 0; k < S && k < gin; ++k) {
                const int idx = gin - 1 - k;
                mbar_wait_bounded(&full[idx % S], (uint32_t)((idx / S) & 1), nullptr, WAIT_NS);
            }
            mbar_wait_bounded(wbar, 0, nullptr, WAIT_NS);
        }
    } else if (warp == 1) {
        if (lane == 0) {
            // ---------------- MMA issuer.  Per input row the output rows it touches
            // form at most two contiguous TMEM slot runs (the ring may wrap); the
            // runs' descriptors are computed once per row, then the 12 (kx, K step)
            // MMAs per run only add constant offsets.
            bool ok = mbar_wait_bounded(wbar, 0, abort, WAIT_NS);
            if (!ok) raise_abort(abort, p.err);
            const uint64_t b_base = SW ? smem_desc_sw128(smem_u32(wsm), 0) : smem_desc(smem_u32(wsm), LBO_B, 128);
            // Work between MMA issues leaves the tensor pipe idle once the few queued
            // MMAs have run, and an mbarrier test made while MMAs are queued costs
            // about a hundred pipe cycles.  So this thread makes no mbarrier waits per
            // row: the wait warp publishes how many input rows are ready (input
            // landed, fresh slot drained) and the issuer re-reads that count only
            // when it runs out of ready rows.  Stage and phase advance incrementally.
            int s = 0, gout = 0, last_slot = -1, gin = 0, nready = 0;
            uint32_t last_par = 0;
            auto await_row = [&](int row) -> bool {
                if (row < nready) return true;
                nready = ld_acquire_cta(ready);
                if (row >= nready) {
                    const uint64_t t0 = globaltimer_ns();
                    for (uint32_t it = 1; row >= (nready = ld_acquire_cta(ready)); ++it) {
                        if ((it & 63) == 0 && (*abort || globaltimer_ns() - t0 > WAIT_NS)) return false;
                    }
                }
                tc_fence_after();  // the MMAs of the newly ready rows come after the acquire
                return true;
            };
            // (kx, K step) t: A advances one pixel per kx and 32 bytes per K step
            // inside the swizzled 64-channel line (CIN 64, 128: K steps 4..7 read the
            // second chunk's region); B one kx block per kx, one ky-stacked chunk
            // block per 64 channels
            auto a_off = [&](int t) {
                const int kx = t / KSTEPS, j = t % KSTEPS;
                return (uint64_t)((SW ? kx * 128 + (j >> 2) * (int)AREG + (j & 3) * 32 : kx * 16 + j * 2 * (int)LBO_A) >> 4);
            };
            auto b_off = [&](int t) {
                const int kx = t / KSTEPS, j = t % KSTEPS;
                return (uint64_t)((kx * WKX + (SW ? (j >> 2) * 3 * NPR * 128 + (j & 3) * 32 : j * 2 * (int)LBO_B)) >> 4);
            };
            auto a_desc = [&]() {
                return SW ? smem_desc_sw128(smem_u32(stage0 + (size_t)s * ROWB), 0)
                          : smem_desc(smem_u32(stage0 + (size_t)s * ROWB), LBO_A, 128);
            };
            // Any row of a strip: runs and descriptors computed from the row's position.
            auto generic_row = [&](int r, int base, int ra, int rb) -> bool {
                    const int o_lo = max(r - 1, ra), o_hi = min(r + 1, rb - 1);
                    const bool fresh = r + 1 <= rb - 1;
                    if (!await_row(gin)) return false;
                    const int sl = (base + r - 1) & (NSLOT - 1);
                    if (r - 1 >= ra && fresh && sl <= NSLOT - 3) {
                        // interior row whose three accumulator rows do not wrap the ring (6 of 8
                        // rows): one N = 3 * NPR run, the same MMAs as below with less set-up
                        const uint64_t a_base = a_desc();
                        const uint32_t id0 = instr_desc(TM, 0, AFMT, AFMT);
                        const uint32_t nstep = (uint32_t)(NPR / 8) << 17;
                        const uint32_t md = tmem_base + (uint32_t)(sl * NPR);
                        umma<KIND>(md, a_base, b_base, id0 + nstep * 2u, 1u);
                        umma<KIND>(md + 2u * NPR, a_base, b_base + (uint64_t)((2 * NPR * (SW ? 128 : 16)) >> 4),
                                   id0 + nstep, 0u);
#pragma unroll
                        for (int t = 1; t < 3 * KSTEPS; ++t)
                            umma<KIND>(md, a_base + a_off(t), b_base + b_off(t), id0 + nstep * 3u, 1u);
                    } else if (o_lo <= o_hi) {
                        const uint64_t a_base = a_desc();
                        // Output rows [o_lo, o_hi] occupy one run of contiguous TMEM slots, or two
                        // where the ring wraps.  The first MMA of the row (kx = 0, K step 0) must not
                        // accumulate into the fresh row r+1, so it is issued per run of the old rows
                        // plus once for the fresh row (accumulate = 0); the other 11 MMAs cover all
                        // of [o_lo, o_hi] with one N = 64 * rows MMA per run.  Everything is held in
                        // scalars so the unrolled issue sequence is only descriptor adds.
                        const uint32_t id0 = instr_desc(TM, 0, AFMT, AFMT);
                        const uint32_t nstep = (uint32_t)(NPR / 8) << 17;  // N += NPR
                        auto slot_of = [&](int o) { return (base + o) & (NSLOT - 1); };
                        auto bd_of = [&](int o) {
                            return b_base + (uint64_t)(((o - r + 1) * NPR * (SW ? 128 : 16)) >> 4);
                        };
                        const int sl0 = slot_of(o_lo);
                        const int len = o_hi - o_lo + 1;
                        const int m0 = min(len, NSLOT - sl0), m1 = len - m0;
                        const uint32_t md0 = tmem_base + (uint32_t)(sl0 * NPR), md1 = tmem_base;
                        const uint32_t mi0 = id0 + nstep * (uint32_t)m0, mi1 = id0 + nstep * (uint32_t)max(m1, 1);
                        const uint64_t mb0 = bd_of(o_lo), mb1 = bd_of(o_lo + m0);
                        // first MMA: old rows [o_lo, old_hi] (split at the wrap), then the fresh row
                        {
                            const int old_hi = fresh ? min(r, o_hi) : o_hi;
                            const int olen = old_hi - o_lo + 1;
                            if (olen > 0) {
                                const int f0 = min(olen, m0), f1 = olen - f0;
                                umma<KIND>(md0, a_base, mb0, id0 + nstep * (uint32_t)f0, 1u);
                                if (f1 > 0) umma<KIND>(md1, a_base, mb1, id0 + nstep * (uint32_t)f1, 1u);
                            }
                            if (fresh)
                                umma<KIND>(tmem_base + (uint32_t)(slot_of(r + 1) * NPR), a_base, bd_of(r + 1),
                                        id0 + nstep, 0u);
                        }
                        if (m1 == 0) {
#pragma unroll
                            for (int t = 1; t < 3 * KSTEPS; ++t)
                                umma<KIND>(md0, a_base + a_off(t), mb0 + b_off(t), mi0, 1u);
                        } else {
#pragma unroll
                            for (int t = 1; t < 3 * KSTEPS; ++t) {
                                const uint64_t ad = a_base + a_off(t), boff = b_off(t);
                                umma<KIND>(md0, ad, mb0 + boff, mi0, 1u);
                                umma<KIND>(md1, ad, mb1 + boff, mi1, 1u);
                            }
                        }
                    }
                    umma_commit(&empty[s]);
                    if (r - 1 >= ra) {
                        const int i = base + r - 1;
                        umma_commit(&rowdone[i & (NSLOT - 1)]);
                        last_slot = i & (NSLOT - 1);
                        last_par = (uint32_t)((i >> 3) & 1);
                    }
                    if (++s == S) s = 0;
                    ++gin;
                    return true;
            };
            // An interior row (r-1 .. r+1 inside the strip) whose first output row sits in TMEM
            // slot SL0: every run, instruction descriptor and operand offset is a compile-time
            // constant, so issuing the row is only MMAs (rows come in aligned blocks of 8, the
            // ring period, and the done-row parity is the block's).
            auto fast_row = [&](auto slc, uint32_t par) -> bool {
                constexpr int SL0 = decltype(slc)::value;
                if (!await_row(gin)) return false;
                const uint64_t a_base = a_desc();
                constexpr int M0 = SL0 <= NSLOT - 3 ? 3 : NSLOT - SL0, M1 = 3 - M0;
                constexpr int F0 = M0 >= 2 ? 2 : M0, F1 = 2 - F0;
                constexpr uint32_t ID0 = instr_desc(TM, 0, AFMT, AFMT), NST = (uint32_t)(NPR / 8) << 17;
                constexpr uint32_t MI0 = ID0 + NST * M0, MI1 = ID0 + NST * (M1 > 0 ? M1 : 1);
                constexpr uint32_t BROW = NPR * (SW ? 128 : 16);  // B bytes of one output row's taps
                const uint32_t md0 = tmem_base + (uint32_t)(SL0 * NPR), md1 = tmem_base;
                const uint64_t mb0 = b_base, mb1 = b_base + (uint64_t)((M0 * BROW) >> 4);
                umma<KIND>(md0, a_base, mb0, ID0 + NST * F0, 1u);
                if constexpr (F1 > 0) umma<KIND>(md1, a_base, mb1, ID0 + NST * F1, 1u);
                umma<KIND>(tmem_base + (uint32_t)(((SL0 + 2) & (NSLOT - 1)) * NPR), a_base,
                        b_base + (uint64_t)((2 * BROW) >> 4), ID0 + NST, 0u);
#pragma unroll
                for (int t = 1; t < 3 * KSTEPS; ++t) {
                    const uint64_t ad = a_base + a_off(t), boff = b_off(t);
                    umma<KIND>(md0, ad, mb0 + boff, MI0, 1u);
                    if constexpr (M1 > 0) umma<KIND>(md1, ad, mb1 + boff, MI1, 1u);
                }
                umma_commit(&empty[s]);
                umma_commit(&rowdone[SL0]);
                last_slot = SL0;
                last_par = par;
                if (++s == S) s = 0;
                ++gin;
                return true;
            };
            using I0 = std::integral_constant<int, 0>;
            using I1 = std::integral_constant<int, 1>;
            using I2 = std::integral_constant<int, 2>;
            using I3 = std::integral_constant<int, 3>;
            using I4 = std::integral_constant<int, 4>;
            using I5 = std::integral_constant<int, 5>;
            using I6 = std::integral_constant<int, 6>;
            using I7 = std::integral_constant<int, 7>;
            for (int sidx = cta0; sidx < nstrips && ok; sidx += cstride) {
                int img, x0, ra, rb, pi;
                strip_of(sidx, img, x0, ra, rb, pi);
                const int base = gout - ra;  // global index of this strip's output row o is base + o
                int r = ra - 1;
                while (r <= rb && ok) {
                    // (measured: the unrolled form pays for the 16-column shuffle tail; for the
                    // 64-column rows the larger code slowed the issue, so those stay generic)
                    if (NPR == 16 && r >= ra + 1 && ((base + r - 1) & (NSLOT - 1)) == 0 && r + 7 <= rb - 2) {
                        const uint32_t par = (uint32_t)(((base + r - 1) >> 3) & 1);
                        ok = fast_row(I0{}, par) && fast_row(I1{}, par) && fast_row(I2{}, par) &&
                             fast_row(I3{}, par) && fast_row(I4{}, par) && fast_row(I5{}, par) &&
                             fast_row(I6{}, par) && fast_row(I7{}, par);
                        r += 8;
                    } else {
                        ok = generic_row(r, base, ra, rb);
                        ++r;
                    }
                }
                if (!ok) raise_abort(abort, p.err);
                gout += rb - ra;
            }
            if (last_slot >= 0) mbar_wait_bounded(&rowdone[last_slot], last_par, nullptr, WAIT_NS);
            if (*abort) {
                // an early exit may leave MMAs of a strip's first row, which no row commit covers
                umma_commit(drain);
                mbar_wait_bounded(drain, 0, nullptr, WAIT_NS);
            }
        }
    } else if (warp == 11) {
        // the 16-channel head's second converter; idle unless the head reads the tuple frames
    } else if (warp == 10) {
        if (lane == 0) {
            // ---------------- wait warp: for each input row in the issuer's order, wait
            // until the slot of its fresh output row is drained and its input row has
            // landed, then publish the count of ready rows (release).
            int s = 0, gout = 0, gin = 0;
            uint32_t ph = 0;
            bool ok = true;
            for (int sidx = cta0; sidx < nstrips && ok; sidx += cstride) {
                int img, x0, ra, rb, pi;
                strip_of(sidx, img, x0, ra, rb, pi);
                const int base = gout - ra;
                for (int r = ra - 1; r <= rb; ++r) {
                    if (r + 1 <= rb - 1) {
                        const int i = base + r + 1;
                        if (!mbar_wait_bounded(&slotfree[i & (NSLOT - 1)], (uint32_t)((i >> 3) & 1) ^ 1u, abort,
                                               WAIT_NS)) {
                            ok = false;
                            break;
                        }
                    }
                    if (!mbar_wait_bounded(&full[s], ph, abort, WAIT_NS)) {
                        ok = false;
                        break;
                    }
                    st_release_cta(ready, ++gin);
                    if (++s == S) {
                        s = 0;
                        ph ^= 1u;
                    }
                }
                gout += rb - ra;
            }
            if (!ok) raise_abort(abort, p.err);
        }
    } else {
        // ---------------- epilogue: two independent groups of 4 warps (warps 2-5
        // and 6-9) take alternate output rows; warp w reads TMEM lane quadrant
        // w % 4 (pixels) and all 64 columns.  A row is staged in shared memory
        // (128-byte swizzled, as the TMA store reads it) and written by one TMA
        // store; its residual arrives by TMA, issued two rows ahead.
        const int q = warp & 3;
        const int g = (warp - 2) >> 2;
        const int m = q * 32 + lane;
        const bool leader = warp == 2 + 4 * g && lane == 0;
        const int bar_id = 1 + g;
        const int64_t HW = (int64_t)p.H * p.W;
        uint8_t *ot = obuf + g * TILEB + m * 128;
        const uint8_t *rt = rbuf + g * TILEB + m * 128;
        int gout = 0;
        int res_loads = 0;  // leader: residual loads issued into this group's buffer
        int last_res = -1;
        bool ok = true;
        for (int sidx = cta0; sidx < nstrips && ok; sidx += cstride) {
            int img, x0, ra, rb, pi;
            strip_of(sidx, img, x0, ra, rb, pi);
            const int x = x0 + m;
            const bool valid = x < width_of(pi);
            // this group's rows of the strip: global index i = gout + (o - ra) with i % 2 == g
            int o = ra + ((g - (gout & 1)) & 1);
            if (leader && has_res && o < rb) {
                mbar_arrive_expect_tx(&resfull[g], TILEB);
                tma_load_4d(rbuf + g * TILEB, rmap_of(pi), &resfull[g], 0, x0, o, img);
                last_res = res_loads++;
            }
            for (; o < rb; o += 2) {
                const int i = gout + (o - ra);
                const int slot = i % NSLOT;
                const int k = i >> 1;  // this group's row count (phase of its residual barrier)
                if (leader) bulk_wait_group_read<0>();  // the group's previous store finished reading
                // a fused requantise's 4:2:0 skip neighbourhood, loaded before the row's wait
                float lr[3][3][3];
                if constexpr (PS && !PSB)
                    if (p.rq.on && p.rq.skip && p.rq.sub420) {
                        const int Wl = width_of(pi);
                        rq_skip_load(p.rq, o, min(x, Wl - 1), p.H, Wl, lr);
                    }
                named_barrier(bar_id, NGRP);
                bool w = mbar_wait_bounded(&rowdone[slot], (uint32_t)((i / NSLOT) & 1), abort, WAIT_NS);
                w = __all_sync(0xffffffffu, w);
                if constexpr (PS && !PSB) {
                    // 12 shuffled channels: channel 4c + 2dy + dx -> output (c, 2o + dy, 2x + dx)
                    float v[16];
                    if (w) {
                        tc_fence_after();
                        uint32_t rr[16];
                        tmem_ld16_nowait(tmem_base + ((uint32_t)(q * 32) << 16) + (uint32_t)(slot * NPR), rr);
                        tmem_wait_ld();
#pragma unroll
                        for (int e = 0; e < 16; ++e) v[e] = __uint_as_float(rr[e]);
                        tc_fence_before();
                        mbar_arrive(&slotfree[slot]);
                    } else {
#pragma unroll
                        for (int e = 0; e < 16; ++e) v[e] = 0.f;
                        if (lane == 0) {
                            raise_abort(abort, p.err);
                            grp_stop[g] = 1;
                        }
                    }
#pragma unroll
                    for (int e = 0; e < 16; ++e) {
                        float ov = v[e] * p.acc_scale + sbias[e];
                        if (p.act == 1) ov = lrelu(ov);
                        if (p.ps_act == 1) ov = lrelu(ov);
                        v[e] = ov;
                    }
                    if (p.rq.on) {
                        // requantised here: residual + skip -> integer planes (see rq_pixel)
                        const FusedRq &rq = p.rq;
                        const int Wl = width_of(pi), xc = min(x, Wl - 1);
                        float yq[2][2], cb[2][2], cr[2][2];
                        rq_pixel(rq, v, o, xc, p.H, Wl, lr, yq, cb, cr);
                        const bool st = valid && w;
                        if (st)
#pragma unroll
                            for (int dy = 0; dy < 2; ++dy)
                                rq_store2(rq.yp, rq.py, 2 * o + dy, x, rq.wide, yq[dy][0], yq[dy][1]);
                        if (!rq.sub420) {
                            if (st)
#pragma unroll
                                for (int dy = 0; dy < 2; ++dy) {
                                    const float a0 = rq_code(cb[dy][0], rq.c_mul, rq.c_add, rq.vmax);
                                    const float a1 = rq_code(cb[dy][1], rq.c_mul, rq.c_add, rq.vmax);
                                    const float b0 = rq_code(cr[dy][0], rq.c_mul, rq.c_add, rq.vmax);
                                    const float b1 = rq_code(cr[dy][1], rq.c_mul, rq.c_add, rq.vmax);
                                    rq_store2(rq.up, rq.pu, 2 * o + dy, x, rq.wide, a0, a1);
                                    rq_store2(rq.vp, rq.pv, 2 * o + dy, x, rq.wide, b0, b1);
                                }
                        } else {
                            // row-pair means of the two full-resolution columns 2x, 2x + 1
                            const float cbv0 = rq_mean2(cb[0][0], cb[1][0]), cbv1 = rq_mean2(cb[0][1], cb[1][1]);
                            const float crv0 = rq_mean2(cr[0][0], cr[1][0]), crv1 = rq_mean2(cr[0][1], cr[1][1]);
                            if (rq.loc != NVISR_CHROMA_LEFT) {
                                if (st) {
                                    rq_store1(rq.up, rq.pu, o, x, rq.wide,
                                              rq_code(rq_mean2(cbv0, cbv1), rq.c_mul, rq.c_add, rq.vmax));
                                    rq_store1(rq.vp, rq.pv, o, x, rq.wide,
                                              rq_code(rq_mean2(crv0, crv1), rq.c_mul, rq.c_add, rq.vmax));
                                }
                            } else {
                                // [1 2 1] / 4 over columns 2x - 1, 2x, 2x + 1: column 2x - 1 is the left
                                // neighbour's odd column (lane - 1; the previous warp's lane 31 through
                                // shared memory; the previous tile's through rq.edge and the fix-up)
                                float cbl = __shfl_up_sync(0xffffffffu, cbv1, 1);
                                float crl = __shfl_up_sync(0xffffffffu, crv1, 1);
                                float *esm = reinterpret_cast<float *>(smem + 640) + (g * 4 + q) * 2;
                                if (lane == 31) {
                                    esm[0] = cbv1;
                                    esm[1] = crv1;
                                }
                                const int tiles = rp.xtiles;
                                const int tile = x0 / TM;
                                if (st && m == 0 && x0 > 0) {  // this tile's first column: finished by the fix-up
                                    float *e = rq.edge + ((int64_t)o * tiles + tile) * 6;
                                    e[0] = cbv0;
                                    e[1] = cbv1;
                                    e[2] = crv0;
                                    e[3] = crv1;
                                }
                                if (st && m == TM - 1 && x0 + TM < Wl) {  // the next tile's left neighbour
                                    float *e = rq.edge + ((int64_t)o * tiles + tile + 1) * 6;
                                    e[4] = cbv1;
                                    e[5] = crv1;
                                }
                                named_barrier(bar_id, NGRP);  // the group's lane-31 columns are in shared memory
                                if (lane == 0) {
                                    const float *pe = reinterpret_cast<const float *>(smem + 640) + (g * 4 + q - 1) * 2;
                                    cbl = q > 0 ? pe[0] : cbv0;  // x = 0: the clamped column is 2x itself
                                    crl = q > 0 ? pe[1] : crv0;
                                }
                                if (st && !(m == 0 && x0 > 0)) {
                                    rq_store1(rq.up, rq.pu, o, x, rq.wide,
                                              rq_code(rq_121(cbl, cbv0, cbv1), rq.c_mul, rq.c_add, rq.vmax));
                                    rq_store1(rq.vp, rq.pv, o, x, rq.wide,
                                              rq_code(rq_121(crl, crv0, crv1), rq.c_mul, rq.c_add, rq.vmax));
                                }
                            }
                        }
                    } else if (valid && w) {
                        const int64_t plane = p.ps_pitch * 2 * p.H;
#pragma unroll
                        for (int c = 0; c < 3; ++c) {
                            if (c >= p.cout / 4) break;
#pragma unroll
                            for (int dy = 0; dy < 2; ++dy)
                                *reinterpret_cast<float2 *>(p.ps_out + c * plane + (int64_t)(2 * o + dy) * p.ps_pitch +
                                                            2 * x) = make_float2(v[4 * c + 2 * dy], v[4 * c + 2 * dy + 1]);
                        }
                    }
                    if (leader && *abort) grp_stop[g] = 1;
                    named_barrier(bar_id, NGRP);
                    if (grp_stop[g]) {
                        ok = false;
                        break;
                    }
                    continue;
                }
                float v[64];
                if (w) {
                    tc_fence_after();
                    uint32_t rr[4][16];
                    const uint32_t taddr = tmem_base + ((uint32_t)(q * 32) << 16) + (uint32_t)(slot * 64);
#pragma unroll
                    for (int jj = 0; jj < 4; ++jj) tmem_ld16_nowait(taddr + (uint32_t)(jj * 16), rr[jj]);
                    tmem_wait_ld();
#pragma unroll
                    for (int jj = 0; jj < 4; ++jj)
#pragma unroll
                        for (int e = 0; e < 16; ++e) v[jj * 16 + e] = __uint_as_float(rr[jj][e]);
                    tc_fence_before();
                    mbar_arrive(&slotfree[slot]);  // the accumulator is in registers now
                } else {
#pragma unroll
                    for (int e = 0; e < 64; ++e) v[e] = 0.f;
                    if (lane == 0) {
                        raise_abort(abort, p.err);
                        grp_stop[g] = 1;
                    }
                }
                if (plain || F8IN) {
                    // 16-bit trunk layer (unit scales, no calibration) or FP8 layer: packed
                    // f32x2 arithmetic keeps the epilogue's instruction stream short, because
                    // its warps share issue slots with the MMA-issuing warp (same results as
                    // the general path)
                    const float as = p.acc_scale;
#pragma unroll
                    for (int e = 0; e < 64; e += 4) {
                        const float4 b = *reinterpret_cast<const float4 *>(sbias + e);
                        if (F8IN) {
                            fma_f32x2(v[e], v[e + 1], as, as, b.x, b.y);
                            fma_f32x2(v[e + 2], v[e + 3], as, as, b.z, b.w);
                        } else {
                            add_f32x2(v[e], v[e + 1], b.x, b.y);
                            add_f32x2(v[e + 2], v[e + 3], b.z, b.w);
                        }
                    }
                    if (p.act == 1) {
#pragma unroll
                        for (int e = 0; e < 64; e += 2) {
                            float t0 = v[e], t1 = v[e + 1];
                            mul_f32x2(t0, t1, 0.1f, 0.1f);
                            v[e] = fmaxf(v[e], t0);
                            v[e + 1] = fmaxf(v[e + 1], t1);
                        }
                    }
                } else {
                    const float as = p.acc_scale;
#pragma unroll
                    for (int e = 0; e < 64; ++e) {
                        float ov = v[e] * as + sbias[e];
                        if (p.act == 1) ov = lrelu(ov);
                        v[e] = ov;
                    }
                }
                if constexpr (!F32OUT) if (has_res) {
                    bool rw = mbar_wait_bounded(&resfull[g], (uint32_t)(k & 1), abort, WAIT_NS);
                    rw = __all_sync(0xffffffffu, rw);
                    if (!rw && lane == 0) {
                        raise_abort(abort, p.err);
                        grp_stop[g] = 1;
                    }
                    const float rs = p.res_scale;
#pragma unroll
                    for (int uu = 0; uu < NU; ++uu) {
                        const int unit = uu ^ (m & 7);
                        const uint4 raw = *reinterpret_cast<const uint4 *>(rt + unit * 16);
                        const uint32_t wd[4] = {raw.x, raw.y, raw.z, raw.w};
#pragma unroll
                        for (int h = 0; h < 4; ++h) {
                            float r0, r1;
                            unpack2<TO>(wd[h], r0, r1);
                            if (plain || (F8IN && rs == 1.f)) {
                                add_f32x2(v[uu * 8 + 2 * h], v[uu * 8 + 2 * h + 1], r0, r1);
                            } else {
                                v[uu * 8 + 2 * h] += r0 * rs;
                                v[uu * 8 + 2 * h + 1] += r1 * rs;
                            }
                        }
                    }
                }
                if (valid && p.amax) {
                    float amax = 0.f;
#pragma unroll
                    for (int e = 0; e < 64; ++e) amax = fmaxf(amax, fabsf(v[e]));
                    atomicMax(p.amax, __float_as_uint(amax));
                }
                if (valid && p.y2) {
                    // FP8 copy: scaled in pairs, converted two values per instruction
                    const int64_t pix = (int64_t)o * p.W + x;
                    const float ys = p.y2_scale;
#pragma unroll
                    for (int c = 0; c < 4; ++c) {
                        uint32_t w8[4];
#pragma unroll
                        for (int h = 0; h < 4; ++h) {
                            float a0 = v[c * 16 + 4 * h], a1 = v[c * 16 + 4 * h + 1];
                            float a2 = v[c * 16 + 4 * h + 2], a3 = v[c * 16 + 4 * h + 3];
                            mul_f32x2(a0, a1, ys, ys);
                            mul_f32x2(a2, a3, ys, ys);
                            const __nv_fp8x2_e4m3 lo(make_float2(a0, a1)), hi(make_float2(a2, a3));
                            w8[h] = (uint32_t)lo.__x | ((uint32_t)hi.__x << 16);
                        }
                        *reinterpret_cast<uint4 *>(p.y2 + (((int64_t)img * (p.cout_pad / 16) + c) * HW + pix) * 16) =
                            make_uint4(w8[0], w8[1], w8[2], w8[3]);
                    }
                }
                if (!plain && !F8IN) {
                    const float os = p.out_scale;
#pragma unroll
                    for (int e = 0; e < 64; ++e) v[e] *= os;
                }
                if constexpr (PSB) {
                    // output pixel (2o + i, 2x + j) of the shuffled tensor (64 channels, one
                    // 128-byte line), after the post-shuffle activation: staged 128-byte
                    // swizzled, and the group's row (every other pixel of output row 2o + i)
                    // written by one TMA store with an element stride of 2
                    if (p.ps_act == 1) {
#pragma unroll
                        for (int e = 0; e < 64; ++e) v[e] = lrelu(v[e]);
                    }
#pragma unroll
                    for (int uu = 0; uu < 8; ++uu) {
                        const int unit = uu ^ (m & 7);
                        uint4 ov;
                        ov.x = pack2<TO>(v[uu * 8 + 0], v[uu * 8 + 1]);
                        ov.y = pack2<TO>(v[uu * 8 + 2], v[uu * 8 + 3]);
                        ov.z = pack2<TO>(v[uu * 8 + 4], v[uu * 8 + 5]);
                        ov.w = pack2<TO>(v[uu * 8 + 6], v[uu * 8 + 7]);
                        *reinterpret_cast<uint4 *>(ot + unit * 16) = ov;
                    }
                    fence_proxy_async();  // staging writes before the async proxy
                } else if constexpr (F32OUT) {
                    // this slice's 16 4-channel units of pixel (o, x), those inside cout_pad;
                    // a warp writes 512 contiguous bytes per unit
                    if (valid && w) {
                        const int u0 = slice * (NPR / 4), nun = p.cout_pad / 4;
                        float4 *yo = reinterpret_cast<float4 *>(p.y) + ((int64_t)img * nun + u0) * HW +
                                     (int64_t)o * p.W + x;
#pragma unroll
                        for (int uu = 0; uu < NU; ++uu)
                            if (u0 + uu < nun)
                                yo[(int64_t)uu * HW] = make_float4(v[4 * uu], v[4 * uu + 1], v[4 * uu + 2], v[4 * uu + 3]);
                    }
                } else if (!p.no_main) {
#pragma unroll
                    for (int uu = 0; uu < NU; ++uu) {
                        const int unit = uu ^ (m & 7);
                        uint4 ov;
                        ov.x = pack2<TO>(v[uu * 8 + 0], v[uu * 8 + 1]);
                        ov.y = pack2<TO>(v[uu * 8 + 2], v[uu * 8 + 3]);
                        ov.z = pack2<TO>(v[uu * 8 + 4], v[uu * 8 + 5]);
                        ov.w = pack2<TO>(v[uu * 8 + 6], v[uu * 8 + 7]);
                        *reinterpret_cast<uint4 *>(ot + unit * 16) = ov;
                    }
                    fence_proxy_async();  // staging writes (and residual reads) before the async proxy
                }
                if (leader && *abort) grp_stop[g] = 1;
                named_barrier(bar_id, NGRP);
                if (grp_stop[g]) {
                    ok = false;
                    break;
                }
                if (PSB && leader) {
                    // pixels 2 x0 + j, 2 x0 + j + 2, ... of output row 2o + i; those past the
                    // image's 2W columns are not written
                    tma_store_4d(ymap_of(pi), obuf + g * TILEB, 0, 2 * x0 + (slice & 1), 2 * o + (slice >> 1), img);
                    bulk_commit_group();
                }
                if (!F32OUT && !PSB && !p.no_main && leader) {
                    tma_store_4d(ymap_of(pi), obuf + g * TILEB, 0, x0, o, img);
                    bulk_commit_group();
                    if (has_res && o + 2 < rb) {  // this group's next row; the buffer's readers are done
                        mbar_arrive_expect_tx(&resfull[g], TILEB);
                        tma_load_4d(rbuf + g * TILEB, rmap_of(pi), &resfull[g], 0, x0, o + 2, img);
                        last_res = res_loads++;
                    }
                }
            }
            gout += rb - ra;
        }
        if (leader) {
            bulk_wait_group<0>();
            // a residual load still in flight after an early exit lands before the CTA ends
            if (last_res >= 0) mbar_wait_bounded(&resfull[g], (uint32_t)(last_res & 1), nullptr, WAIT_NS);
        }
    }
    __syncthreads();
    if (warp == 1) {
        __syncwarp();
        tc_fence_after();
        tmem_dealloc(tmem_base, NCOLS);
    }
}

// ---------------------------------------------------------------- self test

// One M=128, N=16 MMA over K = 16 (BF16) or 32 (E4M3) of small integers, read
// back through tcgen05.ld and compared with the exact product.  Offsets are
// small enough that every descriptor field interpretation stays inside the
// allocated shared memory.
template <int KIND>
__global__ void __launch_bounds__(128, 1) mma_selftest_kernel(int *mismatches) {
    constexpr int K = KIND == 0 ? 16 : 32;
    constexpr int ESZ = KIND == 0 ? 2 : 1;
    constexpr int CPC = 16 / ESZ;
    extern __shared__ uint8_t smem_raw[];
    uint8_t *smem = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    uint64_t *bar = reinterpret_cast<uint64_t *>(smem);
    uint32_t *slot = reinterpret_cast<uint32_t *>(smem + 8);
    uint8_t *A = smem + 1024;         // [2 chunks][128 rows][16 B]: LBO 2048, SBO 128
    uint8_t *B = smem + 1024 + 4096;  // [2 chunks][16 rows][16 B]:  LBO 256,  SBO 128
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    auto aval = [](int m, int k) { return (float)(((m * 3 + k * 5) % 7) - 3); };
    auto bval = [](int n, int k) { return (float)(((n * 5 + k * 3) % 5) - 2); };
    for (int i = tid; i < 128 * K; i += 128) {
        const int m = i / K, k = i % K;
        const int off = (k / CPC) * 2048 + m * 16 + (k % CPC) * ESZ;
        if (KIND == 0) *reinterpret_cast<__nv_bfloat16 *>(A + off) = __float2bfloat16_rn(aval(m, k));
        else *reinterpret_cast<__nv_fp8_e4m3 *>(A + off) = __nv_fp8_e4m3(aval(m, k));
    }
    for (int i = tid; i < 16 * K; i += 128) {
        const int n = i / K, k = i % K;
        const int off = (k / CPC) * 256 + n * 16 + (k % CPC) * ESZ;
        if (KIND == 0) *reinterpret_cast<__nv_bfloat16 *>(B + off) = __float2bfloat16_rn(bval(n, k));
        else *reinterpret_cast<__nv_fp8_e4m3 *>(B + off) = __nv_fp8_e4m3(bval(n, k));
    }
    if (tid == 0) {
        mbar_init(bar, 1);
        fence_mbarrier_init();
    }
    if (warp == 0) {
        tmem_alloc(slot, 32);
        tmem_relinquish();
    }
    fence_proxy_async();  // generic-proxy smem writes -> visible to the tensor core
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tbase = *slot;
    if (tid == 0) {
        const uint64_t ad = smem_desc(smem_u32(A), 2048, 128);
        const uint64_t bd = smem_desc(smem_u32(B), 256, 128);
        umma<KIND>(tbase, ad, bd, instr_desc(128, 16, 0, 0) | (KIND == 0 ? (1u << 7) | (1u << 10) : 0u), 0u);
        umma_commit(bar);
    }
    const bool ok = mbar_wait_bounded(bar, 0, nullptr, WAIT_NS);
    tc_fence_after();
    float v[16];
    tmem_ld16(tbase + ((uint32_t)(warp * 32) << 16), v);
    int bad = ok ? 0 : 1000;
    const int m = warp * 32 + lane;
    for (int n = 0; n < 16; ++n) {
        float ref = 0.f;
        for (int k = 0; k < K; ++k) ref += aval(m, k) * bval(n, k);
        if (v[n] != ref) ++bad;
    }
    if (bad) atomicAdd(mismatches, bad);
    tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        tc_fence_after();
        tmem_dealloc(tbase, 32);
    }
}

// Convention probe for the 128-byte-swizzled K-major layout: A is 144 rows
// x 64 BF16 (128 B per row) stored with the swizzle TMA applies (16-byte unit
// u of row r lands at unit u ^ (r & 7) of a 1024-aligned buffer); B is 16 rows
// x 64.  For each row offset r0 = 0..7 the MMA chain (4 K-steps of 32 bytes)
// reads A from row r0 on, once with base offset 0 and once with base offset
// (start >> 7) & 7; out[mode * 8 + r0] = wrong accumulator elements.  Every
// address stays inside the 40 KB buffer whatever the hardware does with the
// base offset.
__global__ void __launch_bounds__(128, 1) sw128_probe_kernel(int *out) {
    extern __shared__ uint8_t smem_raw[];
    uint8_t *smem = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    uint64_t *bar = reinterpret_cast<uint64_t *>(smem);
    uint32_t *slot = reinterpret_cast<uint32_t *>(smem + 8);
    uint8_t *A = smem + 1024;             // 144 rows x 128 B = 18432 B
    uint8_t *B = smem + 1024 + 19456;     // 16 rows x 128 B, 1024-aligned
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    auto aval = [](int r, int k) { return (float)(((r * 7 + k * 3) % 9) - 4); };
    auto bval = [](int n, int k) { return (float)(((n * 3 + k * 5) % 7) - 3); };
    for (int i = tid; i < 144 * 64; i += 128) {
        const int r = i / 64, k = i % 64;
        const int unit = (k / 8) ^ (r & 7);
        *reinterpret_cast<__nv_bfloat16 *>(A + r * 128 + unit * 16 + (k % 8) * 2) = __float2bfloat16_rn(aval(r, k));
    }
    for (int i = tid; i < 16 * 64; i += 128) {
        const int n = i / 64, k = i % 64;
        const int unit = (k / 8) ^ (n & 7);
        *reinterpret_cast<__nv_bfloat16 *>(B + n * 128 + unit * 16 + (k % 8) * 2) = __float2bfloat16_rn(bval(n, k));
    }
    if (tid == 0) {
        mbar_init(bar, 1);
        fence_mbarrier_init();
    }
    if (warp == 0) {
        tmem_alloc(slot, 32);
        tmem_relinquish();
    }
    fence_proxy_async();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tbase = *slot;
    const uint32_t idesc = instr_desc(128, 16, 1, 1);
    for (int test = 0; test < 16; ++test) {
        const int mode = test / 8, r0 = test % 8;
        if (tid == 0) {
            for (int j = 0; j < 4; ++j) {
                const uint32_t as = smem_u32(A) + (uint32_t)(r0 * 128 + j * 32);
                const uint32_t bs = smem_u32(B) + (uint32_t)(j * 32);
                const uint64_t ad = smem_desc_sw128(as, mode ? ((as >> 7) & 7) : 0);
                const uint64_t bd = smem_desc_sw128(bs, mode ? ((bs >> 7) & 7) : 0);
                umma<0>(tbase, ad, bd, idesc, j ? 1u : 0u);
            }
            umma_commit(bar);
        }
        const bool ok = mbar_wait_bounded(bar, (uint32_t)(test & 1), nullptr, WAIT_NS);
        tc_fence_after();
        float v[16];
        tmem_ld16(tbase + ((uint32_t)(warp * 32) << 16), v);
        const int m = warp * 32 + lane;
        int bad = ok ? 0 : 1000;
        for (int n = 0; n < 16; ++n) {
            float ref = 0.f;
            for (int k = 0; k < 64; ++k) ref += aval(r0 + m, k) * bval(n, k);
            if (v[n] != ref) ++bad;
        }
        if (bad) atomicAdd(out + test, bad);
        tc_fence_before();
        __syncthreads();
        tc_fence_after();
    }
    if (warp == 0) {
        __syncwarp();
        tmem_dealloc(tbase, 32);
    }
}

// ---------------------------------------------------------------- host side

}  // namespace

// The driver's tensor-map encoder (looked up once).
PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        cudaDriverEntryPointQueryResult q;
        void *p = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    });
    return fn;
}

namespace {

// Output channels per CTA slice: the largest of 64/32/16 dividing cout_pad whose
// weights (k*k*cin_bytes per output channel) fit the resident budget.
int pick_ns(int cin_bytes, int cout_pad, int k) {
    const int per_n = k * k * cin_bytes;
    for (int ns : {64, 32, 16}) {
        if (cout_pad % ns == 0 && ns * per_n <= W_MAX) return ns;
    }
    return 16;
}

template <int IN_DT, int OUT_DT, int NS, int KS, int NCH, int EPI, int CBI, int CBO>
cudaError_t run(const CUtensorMap &map, TcParams p, cudaStream_t st) {
    constexpr int PXS = TM + KS - 1;
    constexpr uint32_t CREG = (KS * PXS * 128 + 1023u) & ~1023u;
    constexpr uint32_t STAGE_BYTES = CBI == 16 ? ((NCH * KS * PXS * 16 + 1023u) & ~1023u) : NCH * CREG;
    const uint32_t wround = (p.wbytes + 1023) & ~1023u;
    const int avail = SMEM_LIMIT - 1024 /*align slack*/ - SMEM_HDR - (int)wround;
    int stages = avail / (int)STAGE_BYTES;
    if (stages > 8) stages = 8;
    if (stages < 2) return cudaErrorInvalidConfiguration;
    p.stages = stages;
    // request at least 116 KB so one CTA occupies an SM (TMEM and scheduling assume it)
    int smem = 1024 + SMEM_HDR + (int)wround + stages * (int)STAGE_BYTES;
    if (smem < 118 * 1024) smem = 118 * 1024;
    auto kern = conv_tc_kernel<IN_DT, OUT_DT, NS, KS, NCH, EPI, CBI, CBO>;
    cudaError_t e = set_smem_limit<conv_tc_kernel<IN_DT, OUT_DT, NS, KS, NCH, EPI, CBI, CBO>>(smem);
    if (e != cudaSuccess) return e;
    const int tiles = ((p.W + TM - 1) / TM) * p.H * p.nimg;
    int sms = device_sm_count();
    int per_slice = sms / p.nslice;
    if (per_slice < 1) per_slice = 1;
    if (per_slice > tiles) per_slice = tiles;
    return launch_dependent(kern, per_slice * p.nslice, NTHREADS, smem, st, map, p);
}

using Runner = cudaError_t (*)(const CUtensorMap &, TcParams, cudaStream_t);

struct Variant {
    int in_dt, out_dt, ns, ks, nch, epi, cbi, cbo;
    Runner fn;
};

#define NVISR_V(I, O, NS_, KS_, NCH_, EPI_, CBI_, CBO_) \
    {I, O, NS_, KS_, NCH_, EPI_, CBI_, CBO_, &run<I, O, NS_, KS_, NCH_, EPI_, CBI_, CBO_>}
#define NVISR_V16(I, NS_, KS_, NCH_, EPI_, CBI_, CBO_) NVISR_V(I, I, NS_, KS_, NCH_, EPI_, CBI_, CBO_)
#define NVISR_VSET(I)                                                                                   \
    /* 64-channel (128-byte swizzled) inputs: bodies, tails, 1x1 blends, upsamplers */                  \
    NVISR_V16(I, 64, 3, 1, 0, 128, 128), NVISR_V16(I, 16, 3, 1, 1, 128, 16),                             \
    NVISR_V16(I, 64, 1, 1, 0, 128, 128), NVISR_V16(I, 64, 3, 1, 2, 128, 128),                           \
    NVISR_V16(I, 32, 3, 1, 0, 128, 16), NVISR_V16(I, 16, 3, 1, 0, 128, 16),                              \
    NVISR_V(I, DT_F32, 32, 3, 1, 0, 128, 16), NVISR_V(I, DT_F32, 16, 3, 1, 0, 128, 16),                 \
    /* 16-byte-chunk inputs (16 / 32 channels): heads, extract convs, narrow nets */                     \
    NVISR_V16(I, 64, 3, 2, 0, 16, 128), NVISR_V16(I, 64, 3, 4, 0, 16, 128),                              \
    NVISR_V16(I, 32, 3, 2, 0, 16, 16), NVISR_V16(I, 32, 3, 4, 0, 16, 16),                                \
    NVISR_V16(I, 16, 3, 2, 0, 16, 16), NVISR_V16(I, 16, 3, 4, 0, 16, 16), NVISR_V16(I, 16, 3, 4, 1, 16, 16), \
    /* float32 out from 16 / 32 channels: same-size output layers of narrow networks */                \
    NVISR_V(I, DT_F32, 16, 3, 2, 0, 16, 16), NVISR_V(I, DT_F32, 16, 3, 4, 0, 16, 16)

const Variant kVariants[] = {
    NVISR_VSET(DT_BF16),
    NVISR_VSET(DT_F16),
    // FP8 E4M3 operands (64-channel bodies, 16-byte chunks): BF16 trunk out, or FP8 out
    NVISR_V(DT_E4M3, DT_BF16, 64, 3, 4, 0, 16, 128), NVISR_V(DT_E4M3, DT_E4M3, 64, 3, 4, 0, 16, 16),
};

}  // namespace

int tc_nslice(int cin_pad, int cout_pad, int k, int dt) {
    return cout_pad / pick_ns(cin_pad * dtype_size(dt), cout_pad, k);
}

size_t tc_weight_bytes(int cin_pad, int cout_pad, int k, int dt) {
    return (size_t)k * k * cin_pad * dtype_size(dt) * cout_pad;
}

void prepare_weights_tc(const float *w, int cout, int cin, int k, int cin_pad, int cout_pad, int dt, float scale,
                        void *dst, bool sw128) {
    const int esz = dtype_size(dt);
    const int ns = pick_ns(cin_pad * esz, cout_pad, k);
    const int kk = k * k;
    uint8_t *out = static_cast<uint8_t *>(dst);
    const size_t total = tc_weight_bytes(cin_pad, cout_pad, k, dt);
    for (size_t i = 0; i < total; ++i) out[i] = 0;
    // no swizzle: [slice][tap][16-byte K chunk][n][16 B]
    // sw128:      [slice][tap][64-channel K chunk][n][128 B], 16-byte unit u of row n at u ^ (n & 7)
    const int cpc = sw128 ? 64 : 16 / esz;
    const int cb = cpc * esz;
    const int cin_chunks = cin_pad / cpc;
    for (int o = 0; o < cout; ++o) {
        const int sl = o / ns, n = o % ns;
        for (int c = 0; c < cin; ++c) {
            const int kc = c / cpc, e = c % cpc;
            for (int t = 0; t < kk; ++t) {
                const float v = w[((size_t)o * cin + c) * kk + t] * scale;
                size_t off = (size_t)sl * kk * cin_chunks * ns * cb + (((size_t)t * cin_chunks + kc) * ns + n) * cb;
                if (sw128) off += (size_t)(((e * esz / 16) ^ (n & 7)) * 16 + (e * esz) % 16);
                else off += (size_t)e * esz;
                if (dt == DT_BF16) {
                    __nv_bfloat16 h = __float2bfloat16_rn(v);
                    memcpy(out + off, &h, 2);
                } else if (dt == DT_F16) {
                    __half h = __float2half_rn(v);
                    memcpy(out + off, &h, 2);
                } else {
                    __nv_fp8_e4m3 h(v);
                    memcpy(out + off, &h, 1);
                }
            }
        }
    }
}

size_t tc_rows16_weight_bytes() { return (size_t)3 * 2 * 3 * 64 * 16; }

void prepare_weights_rows16(const float *w, int cin, int dt, void *dst) {
    uint8_t *out = static_cast<uint8_t *>(dst);
    memset(out, 0, tc_rows16_weight_bytes());
    // [kx][16-byte channel chunk kc][ky' = 2 - ky][64 out][8 channels], no swizzle
    for (int n = 0; n < 64; ++n)
        for (int c = 0; c < cin; ++c)
            for (int ky = 0; ky < 3; ++ky)
                for (int kx = 0; kx < 3; ++kx) {
                    const float v = w[((size_t)n * cin + c) * 9 + ky * 3 + kx];
                    const size_t row = (size_t)(2 - ky) * 64 + n;
                    const size_t off = (size_t)kx * 2 * 192 * 16 + (size_t)(c / 8) * 192 * 16 + row * 16 + (c % 8) * 2;
                    if (dt == DT_BF16) {
                        __nv_bfloat16 h = __float2bfloat16_rn(v);
                        memcpy(out + off, &h, 2);
                    } else {
                        __half h = __float2half_rn(v);
                        memcpy(out + off, &h, 2);
                    }
                }
}

size_t tc_rows_weight_bytes(int npr) { return (size_t)3 * 3 * npr * 128; }

void prepare_weights_rows(const float *w, int dt, void *dst, int cout, int npr) {
    uint8_t *out = static_cast<uint8_t *>(dst);
    memset(out, 0, tc_rows_weight_bytes(npr));
    for (int n = 0; n < cout; ++n)
        for (int c = 0; c < 64; ++c)
            for (int ky = 0; ky < 3; ++ky)
                for (int kx = 0; kx < 3; ++kx) {
                    const float v = w[((size_t)n * 64 + c) * 9 + ky * 3 + kx];
                    const size_t row = (size_t)(2 - ky) * npr + n;
                    const size_t off = (size_t)kx * 3 * npr * 128 + row * 128 + (((c / 8) ^ (n & 7)) * 16) + (c % 8) * 2;
                    if (dt == DT_BF16) {
                        __nv_bfloat16 h = __float2bfloat16_rn(v);
                        memcpy(out + off, &h, 2);
                    } else {
                        __half h = __float2half_rn(v);
                        memcpy(out + off, &h, 2);
                    }
                }
}

size_t tc_rows128_weight_bytes(int nslice) { return (size_t)nslice * 3 * 2 * 3 * 64 * 128; }

void prepare_weights_rows128(const float *w, int cout, int dt, void *dst) {
    const int nslice = (round_up(cout, 16) + 63) / 64;
    uint8_t *out = static_cast<uint8_t *>(dst);
    memset(out, 0, tc_rows128_weight_bytes(nslice));
    // [64-output slice][kx][64-channel chunk][ky' = 2 - ky][64 out][128 B swizzled]
    for (int o = 0; o < cout; ++o)
        for (int c = 0; c < 128; ++c)
            for (int ky = 0; ky < 3; ++ky)
                for (int kx = 0; kx < 3; ++kx) {
                    const float v = w[((size_t)o * 128 + c) * 9 + ky * 3 + kx];
                    const int sl = o / 64, n = o % 64, ch = c / 64, cc = c % 64;
                    const size_t row = (size_t)(2 - ky) * 64 + n;
                    const size_t off = (((size_t)sl * 3 + kx) * 2 + ch) * 3 * 64 * 128 + row * 128 +
                                       (((cc / 8) ^ (n & 7)) * 16) + (cc % 8) * 2;
                    if (dt == DT_BF16) {
                        __nv_bfloat16 h = __float2bfloat16_rn(v);
                        memcpy(out + off, &h, 2);
                    } else {
                        __half h = __float2half_rn(v);
                        memcpy(out + off, &h, 2);
                    }
                }
}

size_t tc_rows_f8_weight_bytes() { return (size_t)3 * 4 * 3 * 64 * 16; }

void prepare_weights_rows_f8(const float *w, float scale, void *dst) {
    uint8_t *out = static_cast<uint8_t *>(dst);
    memset(out, 0, tc_rows_f8_weight_bytes());
    // [kx][16-byte chunk kc][ky' = 2 - ky][64 out][16 channels], E4M3, no swizzle
    for (int n = 0; n < 64; ++n)
        for (int c = 0; c < 64; ++c)
            for (int ky = 0; ky < 3; ++ky)
                for (int kx = 0; kx < 3; ++kx) {
                    const float v = w[((size_t)n * 64 + c) * 9 + ky * 3 + kx] * scale;
                    const size_t row = (size_t)(2 - ky) * 64 + n;
                    const size_t off = ((size_t)kx * 4 + c / 16) * 192 * 16 + row * 16 + (c % 16);
                    const __nv_fp8_e4m3 q(v);
                    memcpy(out + off, &q, 1);
                }
}

void prepare_weights_rows_ps4(const float *w, int dt, void *dst) {
    // slice s = 2i + j: conv channels 4n + s (output channel n at shuffle offset (i, j))
    std::vector<float> ws((size_t)64 * 64 * 9);
    for (int sl = 0; sl < 4; ++sl) {
        for (int n = 0; n < 64; ++n)
            memcpy(ws.data() + (size_t)n * 64 * 9, w + (size_t)(4 * n + sl) * 64 * 9, sizeof(float) * 64 * 9);
        prepare_weights_rows(ws.data(), dt, static_cast<uint8_t *>(dst) + (size_t)sl * tc_rows_weight_bytes(64), 64, 64);
    }
}

namespace {

// Shared memory of the row kernel: the weights (72 KB for 64 input channels),
// the input-row ring, 2 output staging tiles (16-bit outputs) and, when the
// layer adds a residual, 2 residual tiles (without one, their room goes to
// deeper input prefetch).
inline int rows_stages(bool res, int *smem, int npr = 64, bool ps = false, int cin = 64, bool f32out = false,
                       bool f8 = false, int extra = 0) {
    const uint32_t nchk = f8 ? 4u : 2u;  // 16-byte chunks per pixel of the no-swizzle forms
    const bool sw = cin != 16 && !f8;
    const uint32_t ROWB = sw ? (((uint32_t)(cin / 64) * (TM + 2) * 128 + 1023u) & ~1023u)
                             : ((nchk * (TM + 2) * 16 + 1023u) & ~1023u);
    const uint32_t WB = sw ? 3 * 3 * (uint32_t)(cin / 64) * (uint32_t)npr * 128 : 3 * nchk * 3 * (uint32_t)npr * 16;
    // staging tiles: 16-bit outputs written by TMA stores, including the 64-channel
    // PixelShuffle slices (npr 64); the 16-channel shuffle tail stores directly
    const uint32_t TILES = (ps && npr != 64) || f32out ? 0u : (res ? 4u : 2u) * TM * 128;
    int stages = (SMEM_LIMIT - 1024 - SMEM_HDR - (int)WB - (int)TILES - extra) / (int)ROWB;
    if (stages > 8) stages = 8;
    *smem = 1024 + SMEM_HDR + (int)WB + stages * (int)ROWB + (int)TILES + extra;
    return stages;
}

template <int IN_DT, int OUT_DT, int CBO, int NPR = 64, bool PS = false, int CIN = 64>
cudaError_t run_rows(const CUtensorMap &map, const CUtensorMap &ymap, const CUtensorMap &rmap, TcParams p,
                     cudaStream_t st) {
    int smem;
    // the tuple head's float32 staging slots
    const int extra = CIN == 16 && p.ntup > 0 ? HEAD_NSL * 5 * (int)HEAD_FROW32 : 0;
    p.stages = rows_stages(p.res != nullptr, &smem, NPR, PS, CIN, false, IN_DT == DT_E4M3, extra);
    if (p.stages < 2) return cudaErrorInvalidConfiguration;
    auto kern = conv_rows_kernel<IN_DT, OUT_DT, CBO, false, NPR, PS, CIN>;
    cudaError_t e = set_smem_limit<conv_rows_kernel<IN_DT, OUT_DT, CBO, false, NPR, PS, CIN>>(smem);
    if (e != cudaSuccess) return e;
    RowPlan rp;
    rp.xtiles = (p.W + TM - 1) / TM;
    const int sms = device_sm_count();
    int bands = sms / (rp.xtiles * p.nimg);
    if (bands < 1) bands = 1;
    if (bands > p.H) bands = p.H;
    rp.rps = (p.H + bands - 1) / bands;
    rp.bands = (p.H + rp.rps - 1) / rp.rps;
    int grid = rp.xtiles * rp.bands * p.nimg;
    if (grid > sms) grid = sms;
    return launch_dependent(kern, grid, rows_threads(CIN, false), smem, st, map, ymap, rmap, p, rp, nullptr, 0);
}

// Row kernel over output-channel slices (p.nslice of 64): CTAs per slice =
// SMs / slices, each walking strips of one slice; the band height is the one
// that gives the fewest input rows per CTA (strips per CTA x (rows + 2 halo
// rows)).  Forms: 128 16-bit input channels (two 64-channel chunks) to float32
// 4-channel units; 64 -> 256 channels shuffled by PixelShuffle(2) into a
// blocked 16-bit tensor.
template <int IN_DT, int OUT_DT, int CBO, bool PS, int CIN>
cudaError_t run_rows_sliced(const CUtensorMap &map, const CUtensorMap &ymap, TcParams p, cudaStream_t st) {
    int smem;
    p.stages = rows_stages(false, &smem, 64, PS, CIN, OUT_DT == DT_F32);
    if (p.stages < 2) return cudaErrorInvalidConfiguration;
    auto kern = conv_rows_kernel<IN_DT, OUT_DT, CBO, false, 64, PS, CIN>;
    cudaError_t e = set_smem_limit<conv_rows_kernel<IN_DT, OUT_DT, CBO, false, 64, PS, CIN>>(smem);
    if (e != cudaSuccess) return e;
    const int ctas = std::max(1, device_sm_count() / p.nslice);
    RowPlan rp;
    rp.xtiles = (p.W + TM - 1) / TM;
    int best = 1 << 30;
    rp.rps = p.H;
    for (int bands = 1; bands <= p.H; ++bands) {
        const int rps = (p.H + bands - 1) / bands;
        const int strips = rp.xtiles * ((p.H + rps - 1) / rps) * p.nimg;
        const int per = (strips + ctas - 1) / ctas * (rps + 2);
        if (per < best) {
            best = per;
            rp.rps = rps;
        }
    }
    rp.bands = (p.H + rp.rps - 1) / rp.rps;
    const int strips = rp.xtiles * rp.bands * p.nimg;
    const int grid = std::min(ctas, strips) * p.nslice;
    return launch_dependent(kern, grid, rows_threads(CIN, false), smem, st, map, ymap, map, p, rp, nullptr, 0);
}

template <int IN_DT, int OUT_DT, int CBO>
cudaError_t run_rows_multi(const CUtensorMap &dummy, TcParams p, const RowProblem *dev_tab, int n, int total,
                           cudaStream_t st) {
    int smem;
    p.stages = rows_stages(p.res != nullptr, &smem);
    if (p.stages < 2) return cudaErrorInvalidConfiguration;
    auto kern = conv_rows_kernel<IN_DT, OUT_DT, CBO, true, 64, false, 64>;
    cudaError_t e = set_smem_limit<conv_rows_kernel<IN_DT, OUT_DT, CBO, true, 64, false, 64>>(smem);
    if (e != cudaSuccess) return e;
    RowPlan rp{};
    const int grid = std::min(total, device_sm_count());
    return launch_dependent(kern, grid, ROWS_THREADS, smem, st, dummy, dummy, dummy, p, rp, dev_tab, n);
}

// The row kernel's three tensor maps for one image set (x: 130-pixel row boxes
// with OOB zero fill; y and residual: 128-pixel row tiles).
cudaError_t encode_row_maps(const ConvArgs &a, CUtensorMap *map, CUtensorMap *ymap, CUtensorMap *rmap) {
    auto enc = encode_fn();
    if (!enc) return cudaErrorNotSupported;
    cuuint64_t dims[4] = {128, (cuuint64_t)a.W, (cuuint64_t)a.H, (cuuint64_t)a.nimg};
    cuuint64_t strides[3] = {128, (cuuint64_t)a.W * 128, (cuuint64_t)a.W * a.H * 128};
    cuuint32_t box[4] = {128, (cuuint32_t)(TM + 2), 1, 1};
    cuuint32_t tbox[4] = {128, (cuuint32_t)TM, 1, 1};
    cuuint32_t estr[4] = {1, 1, 1, 1};
    CUresult r = enc(map, CU_TENSOR_MAP_DATA_TYPE_UINT8, 4, const_cast<void *>(a.x), dims, strides, box, estr,
                     CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                     CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return cudaErrorInvalidValue;
    r = enc(ymap, CU_TENSOR_MAP_DATA_TYPE_UINT8, 4, a.y, dims, strides, tbox, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
            CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return cudaErrorInvalidValue;
    r = enc(rmap, CU_TENSOR_MAP_DATA_TYPE_UINT8, 4, const_cast<void *>(a.res ? a.res : a.y), dims, strides, tbox,
            estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return cudaErrorInvalidValue;
    return cudaSuccess;
}

TcParams rows_params(const ConvArgs &a) {
    TcParams p{};
    p.H = a.H; p.W = a.W; p.nimg = a.nimg; p.cin_chunks = 1;
    p.cout = 64; p.cout_pad = 64; p.ns = 64; p.nslice = 1;
    p.wts = static_cast<const uint8_t *>(a.w_rows);
    p.wbytes = (uint32_t)tc_rows_weight_bytes();
    p.bias = a.bias; p.act = a.act;
    p.res = static_cast<const uint8_t *>(a.res);
    p.y = static_cast<uint8_t *>(a.y);
    p.acc_scale = a.acc_scale; p.out_scale = a.out_scale; p.res_scale = 1.0f / a.out_scale;
    p.y2 = static_cast<uint8_t *>(a.y2); p.y2_scale = a.y2_scale; p.amax = a.amax;
    p.err = a.err;
    p.starve = test_starve();
    return p;
}

}  // namespace

bool rows_kernel_fits(const ConvArgs &a) {
    const int dt = a.in_dt;
    return a.w_rows && a.k == 3 && (dt == DT_BF16 || dt == DT_F16) && a.out_dt == dt && a.cin_pad == 64 &&
           a.cout_pad == 64 && a.cout == 64 && a.in_cpc == 64 && a.out_cpc == 64 && a.ps == 0;
}

// 3x3 layer from a 16-channel (two 16-byte chunks) 16-bit input to 64 channels.
bool rows_head_fits(const ConvArgs &a) {
    const int dt = a.in_dt;
    return a.w_rows && a.k == 3 && (dt == DT_BF16 || dt == DT_F16) && a.out_dt == dt && a.cin_pad == 16 &&
           a.in_cpc == 8 && a.cout_pad == 64 && a.cout == 64 && a.out_cpc == 64 && a.ps == 0 && !a.res;
}

// 3x3 layer from 128 16-bit channels (64-channel chunks) to <= 256 float32
// channels in 4-channel units (the offset/mask head of a deformable layer).
bool rows128_fits(const ConvArgs &a) {
    const int dt = a.in_dt;
    return a.w_rows && a.k == 3 && (dt == DT_BF16 || dt == DT_F16) && a.cin_pad == 128 && a.in_cpc == 64 &&
           a.out_dt == DT_F32 && a.out_cpc == 4 && a.cout_pad % 4 == 0 && a.cout_pad <= 256 && a.cout <= a.cout_pad &&
           a.ps == 0 && !a.res && !a.y2 && !a.amax && a.nimg == 1 && a.acc_scale == 1.f && a.out_scale == 1.f;
}

// FP8 64 -> 64 3x3 trunk layer: E4M3 input in 16-channel chunks; BF16 output (with
// an optional FP8 copy and residual), or an FP8-only output in 16-channel chunks.
bool rows_f8_fits(const ConvArgs &a) {
    const bool bf16_out = a.out_dt == DT_BF16 && a.out_cpc == 64;
    const bool f8_out = a.out_dt == DT_E4M3 && a.out_cpc == 16 && !a.res && !a.y2;
    return a.w_rows && a.k == 3 && a.in_dt == DT_E4M3 && a.cin_pad == 64 && a.in_cpc == 16 && a.cout == 64 &&
           a.cout_pad == 64 && a.ps == 0 && a.nimg == 1 && !a.amax && (bf16_out || f8_out);
}

// 64 -> 256 channels, PixelShuffle(2) into a blocked 64-channel 16-bit tensor.
bool rows_psb_fits(const ConvArgs &a) {
    const int dt = a.in_dt;
    return a.w_rows && a.k == 3 && (dt == DT_BF16 || dt == DT_F16) && a.out_dt == dt && a.cin_pad == 64 &&
           a.in_cpc == 64 && a.cout == 256 && a.cout_pad == 256 && a.ps == 2 && !a.ps_out && a.out_cpc == 64 &&
           !a.res && !a.y2 && !a.amax && a.nimg == 1 && a.acc_scale == 1.f && a.out_scale == 1.f;
}

// PixelShuffle(2) output layer with 64 input channels (<= 16 outputs, planar float32).
bool rows_ps_fits(const ConvArgs &a) {
    const int dt = a.in_dt;
    return a.w_rows && a.k == 3 && (dt == DT_BF16 || dt == DT_F16) && a.cin_pad == 64 && a.in_cpc == 64 &&
           a.cout_pad == 16 && a.cout <= 12 && a.cout % 4 == 0 && a.ps == 2 && a.ps_out && !a.res && !a.y2 &&
           !a.amax && a.nimg == 1;
}

cudaError_t launch_conv_rows_multi(const ConvArgs *args, int n, RowProblem *host_tab, RowProblem *dev_tab, int rps,
                                   cudaStream_t st, bool copy_table, bool launch) {
    if (n < 1) return cudaSuccess;
    const ConvArgs &a0 = args[0];
    for (int i = 0; i < n; ++i) {
        const ConvArgs &a = args[i];
        if (!rows_kernel_fits(a) || a.in_dt != a0.in_dt || a.w_rows != a0.w_rows || a.bias != a0.bias ||
            a.act != a0.act || (a.res != nullptr) != (a0.res != nullptr) || a.y2 || a.amax || a.acc_scale != 1.f ||
            a.out_scale != 1.f || a.nimg != 1)
            return cudaErrorInvalidValue;
    }
    int total = 0;
    for (int i = 0; i < n; ++i) {
        const ConvArgs &a = args[i];
        RowProblem &q = host_tab[i];
        cudaError_t e = encode_row_maps(a, &q.tmap, &q.ymap, &q.rmap);
        if (e != cudaSuccess) return e;
        q.H = a.H;
        q.W = a.W;
        q.xtiles = (a.W + TM - 1) / TM;
        q.rps = rps > 0 ? std::min(rps, a.H) : std::max(1, std::min(a.H, 64));
        q.strip0 = total;
        q.nstrips = q.xtiles * ((a.H + q.rps - 1) / q.rps);
        q.has_res = a.res != nullptr;
        q.pad_ = 0;
        total += q.nstrips;
    }
    if (copy_table) {
        cudaError_t e = cudaMemcpyAsync(dev_tab, host_tab, sizeof(RowProblem) * n, cudaMemcpyHostToDevice, st);
        if (e != cudaSuccess) return e;
    }
    if (!launch) return cudaSuccess;
    TcParams p = rows_params(a0);
    return a0.in_dt == DT_BF16 ? run_rows_multi<DT_BF16, DT_BF16, 128>(host_tab[0].tmap, p, dev_tab, n, total, st)
                               : run_rows_multi<DT_F16, DT_F16, 128>(host_tab[0].tmap, p, dev_tab, n, total, st);
}

cudaError_t launch_conv_tc(const ConvArgs &a, cudaStream_t st) {
    const int dt = a.in_dt;
    // 64 -> 64 3x3 layers with 64-channel 16-bit input and output: row-streaming kernel
    if (rows_kernel_fits(a)) {
        CUtensorMap map, ymap, rmap;
        cudaError_t e = encode_row_maps(a, &map, &ymap, &rmap);
        if (e != cudaSuccess) return e;
        const TcParams p = rows_params(a);
        return dt == DT_BF16 ? run_rows<DT_BF16, DT_BF16, 128>(map, ymap, rmap, p, st)
                             : run_rows<DT_F16, DT_F16, 128>(map, ymap, rmap, p, st);
    }
    if (rows_head_fits(a) && a.ring) {
        // the tuple head reading its ntup float32 frames from the ring: [slot][3][H][pitch]
        if (a.ntup < 1 || a.ntup > 5 || a.ring_pitch % 4) return cudaErrorInvalidValue;
        ConvArgs b = a;
        b.x = a.y;  // the 16-bit row map is not used by this form
        CUtensorMap map, ymap, rmap;
        cudaError_t e = encode_row_maps(b, &map, &ymap, &rmap);
        if (e != cudaSuccess) return e;
        auto enc = encode_fn();
        if (!enc) return cudaErrorNotSupported;
        cuuint64_t dims[4] = {(cuuint64_t)a.W, (cuuint64_t)a.H, 3, (cuuint64_t)a.ring_slots};
        cuuint64_t strides[3] = {(cuuint64_t)a.ring_pitch * 4, (cuuint64_t)a.ring_pitch * a.H * 4,
                                 (cuuint64_t)a.ring_pitch * a.H * 12};
        cuuint32_t box[4] = {136, (cuuint32_t)HEAD_RPB, 3, 1};
        cuuint32_t estr[4] = {1, 1, 1, 1};
        if (enc(&map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, const_cast<float *>(a.ring), dims, strides, box, estr,
                CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
            return cudaErrorInvalidValue;
        TcParams p = rows_params(a);
        p.wbytes = (uint32_t)tc_rows16_weight_bytes();
        p.ntup = a.ntup;
        for (int k = 0; k < a.ntup; ++k) p.tslot[k] = a.tslot[k];
        return dt == DT_BF16 ? run_rows<DT_BF16, DT_BF16, 128, 64, false, 16>(map, ymap, rmap, p, st)
                             : run_rows<DT_F16, DT_F16, 128, 64, false, 16>(map, ymap, rmap, p, st);
    }
    if (rows_head_fits(a)) {
        CUtensorMap map, ymap, rmap;
        cudaError_t e = encode_row_maps(a, &map, &ymap, &rmap);  // y (64 channels) and residual maps
        if (e != cudaSuccess) return e;
        auto enc = encode_fn();
        cuuint64_t dims[4] = {16, (cuuint64_t)a.W, (cuuint64_t)a.H, (cuuint64_t)(2 * a.nimg)};
        cuuint64_t strides[3] = {16, (cuuint64_t)a.W * 16, (cuuint64_t)a.W * a.H * 16};
        cuuint32_t box[4] = {16, (cuuint32_t)(TM + 2), 1, 2};
        cuuint32_t estr[4] = {1, 1, 1, 1};
        if (enc(&map, CU_TENSOR_MAP_DATA_TYPE_UINT8, 4, const_cast<void *>(a.x), dims, strides, box, estr,
                CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
            return cudaErrorInvalidValue;
        TcParams p = rows_params(a);
        p.wbytes = (uint32_t)tc_rows16_weight_bytes();
        return dt == DT_BF16 ? run_rows<DT_BF16, DT_BF16, 128, 64, false, 16>(map, ymap, rmap, p, st)
                             : run_rows<DT_F16, DT_F16, 128, 64, false, 16>(map, ymap, rmap, p, st);
    }
    if (rows128_fits(a)) {
        auto enc = encode_fn();
        if (!enc) return cudaErrorNotSupported;
        CUtensorMap map;
        cuuint64_t dims[4] = {128, (cuuint64_t)a.W, (cuuint64_t)a.H, (cuuint64_t)(2 * a.nimg)};
        cuuint64_t strides[3] = {128, (cuuint64_t)a.W * 128, (cuuint64_t)a.W * a.H * 128};
        cuuint32_t box[4] = {128, (cuuint32_t)(TM + 2), 1, 2};
        cuuint32_t estr[4] = {1, 1, 1, 1};
        if (enc(&map, CU_TENSOR_MAP_DATA_TYPE_UINT8, 4, const_cast<void *>(a.x), dims, strides, box, estr,
                CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
            return cudaErrorInvalidValue;
        TcParams p = rows_params(a);
        p.cout = a.cout;
        p.cout_pad = a.cout_pad;
        p.nslice = (a.cout_pad + 63) / 64;
        p.wbytes = (uint32_t)tc_rows128_weight_bytes(1);
        return dt == DT_BF16 ? run_rows_sliced<DT_BF16, DT_F32, 16, false, 128>(map, map, p, st)
                             : run_rows_sliced<DT_F16, DT_F32, 16, false, 128>(map, map, p, st);
    }
    if (rows_f8_fits(a)) {
        auto enc = encode_fn();
        if (!enc) return cudaErrorNotSupported;
        CUtensorMap map, ymap, rmap;
        cuuint64_t dims[4] = {16, (cuuint64_t)a.W, (cuuint64_t)a.H, (cuuint64_t)(4 * a.nimg)};
        cuuint64_t strides[3] = {16, (cuuint64_t)a.W * 16, (cuuint64_t)a.W * a.H * 16};
        cuuint32_t box[4] = {16, (cuuint32_t)(TM + 2), 1, 4};
        cuuint32_t estr[4] = {1, 1, 1, 1};
        if (enc(&map, CU_TENSOR_MAP_DATA_TYPE_UINT8, 4, const_cast<void *>(a.x), dims, strides, box, estr,
                CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
            return cudaErrorInvalidValue;
        TcParams p = rows_params(a);
        ConvArgs b = a;
        if (a.out_dt == DT_E4M3) {
            // FP8-only output: the FP8 copy path writes it; the 16-bit tile maps are unused
            p.no_main = 1;
            p.y2 = static_cast<uint8_t *>(a.y);
            p.y2_scale = a.out_scale;
            p.out_scale = 1.f;
            p.res_scale = 1.f;
            b.y = const_cast<void *>(b.res ? b.res : a.x);
        }
        b.x = b.y;  // the 16-bit row map is not used by this form
        cudaError_t e = encode_row_maps(b, &ymap, &ymap, &rmap);
        if (e != cudaSuccess) return e;
        return run_rows<DT_E4M3, DT_BF16, 128, 64, false, 64>(map, ymap, rmap, p, st);
    }
    if (rows_psb_fits(a)) {
        ConvArgs b = a;
        b.y = const_cast<void *>(a.x);  // the residual map is unused
        CUtensorMap map, ymap, rmap;
        cudaError_t e = encode_row_maps(b, &map, &ymap, &rmap);
        if (e != cudaSuccess) return e;
        // y: the shuffled 2H x 2W tensor of 128-byte pixel lines; a store box covers 128
        // pixels at a stride of 2 (one slice's pixels of one output row)
        auto enc = encode_fn();
        if (!enc) return cudaErrorNotSupported;
        {
            cuuint64_t dims[4] = {128, (cuuint64_t)(2 * a.W), (cuuint64_t)(2 * a.H), (cuuint64_t)a.nimg};
            cuuint64_t strides[3] = {128, (cuuint64_t)(2 * a.W) * 128, (cuuint64_t)(2 * a.W) * (2 * a.H) * 128};
            cuuint32_t box[4] = {128, (cuuint32_t)(2 * TM), 1, 1};
            cuuint32_t estr[4] = {1, 2, 1, 1};
            if (enc(&ymap, CU_TENSOR_MAP_DATA_TYPE_UINT8, 4, a.y, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                    CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                    CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
                return cudaErrorInvalidValue;
        }
        TcParams p = rows_params(a);
        p.cout = a.cout;
        p.cout_pad = a.cout_pad;
        p.nslice = 4;
        p.ps_act = a.ps_act;
        return dt == DT_BF16 ? run_rows_sliced<DT_BF16, DT_BF16, 128, true, 64>(map, ymap, p, st)
                             : run_rows_sliced<DT_F16, DT_F16, 128, true, 64>(map, ymap, p, st);
    }
    if (rows_ps_fits(a)) {
        ConvArgs b = a;
        b.y = const_cast<void *>(a.x);  // the shuffle epilogue stores directly; the y / residual maps are unused
        CUtensorMap map, ymap, rmap;
        cudaError_t e = encode_row_maps(b, &map, &ymap, &rmap);
        if (e != cudaSuccess) return e;
        TcParams p = rows_params(a);
        p.cout = a.cout;
        p.cout_pad = 16;
        p.ns = 16;
        p.wbytes = (uint32_t)tc_rows_weight_bytes(16);
        p.ps_out = a.ps_out;
        p.ps_pitch = a.ps_pitch;
        p.ps_act = a.ps_act;
        p.rq = a.rq;
        if (p.rq.on && a.cout != 12) return cudaErrorInvalidValue;  // requantise needs the 3 shuffled channels
        e = dt == DT_BF16 ? run_rows<DT_BF16, DT_BF16, 128, 16, true>(map, ymap, rmap, p, st)
                          : run_rows<DT_F16, DT_F16, 128, 16, true>(map, ymap, rmap, p, st);
        if (e != cudaSuccess || !p.rq.on) return e;
        return launch_rq_edge_fixup(p.rq, a.H, a.W, st);
    }
    if (dt == DT_F32) return cudaErrorInvalidValue;
    if (a.rq.on) return cudaErrorNotSupported;  // only the row kernel's shuffle tail requantises
    const int esz = dtype_size(dt);
    const int in_cpc = a.in_cpc ? a.in_cpc : 16 / esz;
    const int cbi = in_cpc * esz == 128 ? 128 : 16;
    if (in_cpc * esz != cbi || a.cin_pad % in_cpc) return cudaErrorInvalidValue;
    const int cin_chunks = a.cin_pad / in_cpc;
    const int ns = pick_ns(a.cin_pad * esz, a.cout_pad, a.k);
    // 16-byte chunks per stage: the largest built group (4 or 2) that divides the chunk count
    const int nch = cbi == 128 ? 1 : (cin_chunks % 4 == 0 ? 4 : 2);
    if (cin_chunks % nch || (cbi == 16 && nch % 2)) return cudaErrorInvalidValue;
    const int epi = a.ps > 0 ? (a.ps_out ? 1 : 2) : 0;
    const int odt = epi == 1 ? dt : a.out_dt;
    const int out_cpc = epi == 1 ? 16 / esz : (a.out_cpc ? a.out_cpc : 16 / dtype_size(odt));
    const int cbo = out_cpc * dtype_size(odt);
    if (cbo != 16 && cbo != 128) return cudaErrorInvalidValue;
    const Variant *v = nullptr;
    for (const Variant &c : kVariants)
        if (c.in_dt == dt && c.out_dt == odt && c.ns == ns && c.ks == a.k && c.nch == nch && c.epi == epi &&
            c.cbi == cbi && c.cbo == cbo)
            v = &c;
    if (!v) return cudaErrorNotSupported;
    auto enc = encode_fn();
    if (!enc) return cudaErrorNotSupported;
    // activation as a byte tensor: (chunk bytes, W, H, chunks of all images)
    CUtensorMap map;
    const int pxs = TM + a.k - 1;
    cuuint64_t dims[4] = {(cuuint64_t)cbi, (cuuint64_t)a.W, (cuuint64_t)a.H, (cuuint64_t)a.nimg * cin_chunks};
    cuuint64_t strides[3] = {(cuuint64_t)cbi, (cuuint64_t)a.W * cbi, (cuuint64_t)a.W * a.H * cbi};
    cuuint32_t box[4] = {(cuuint32_t)cbi, (cuuint32_t)pxs, (cuuint32_t)a.k, (cuuint32_t)(cbi == 128 ? 1 : nch)};
    cuuint32_t estr[4] = {1, 1, 1, 1};
    CUresult r = enc(&map, CU_TENSOR_MAP_DATA_TYPE_UINT8, 4, const_cast<void *>(a.x), dims, strides, box, estr,
                     CU_TENSOR_MAP_INTERLEAVE_NONE,
                     cbi == 128 ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_NONE,
                     CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return cudaErrorInvalidValue;
    TcParams p{};
    p.H = a.H; p.W = a.W; p.nimg = a.nimg; p.cin_chunks = cin_chunks;
    p.cout = a.cout; p.cout_pad = a.cout_pad; p.ns = ns; p.nslice = a.cout_pad / ns;
    p.wts = static_cast<const uint8_t *>(a.w);
    p.wbytes = (uint32_t)(a.k * a.k * a.cin_pad * esz * ns);
    p.bias = a.bias; p.act = a.act;
    p.res = static_cast<const uint8_t *>(a.res);
    p.y = static_cast<uint8_t *>(a.y);
    p.acc_scale = a.acc_scale; p.out_scale = a.out_scale; p.res_scale = 1.0f / a.out_scale;
    p.y2 = static_cast<uint8_t *>(a.y2); p.y2_scale = a.y2_scale; p.amax = a.amax;
    p.ps_out = a.ps_out; p.ps_pitch = a.ps_pitch; p.skip = a; p.ps_act = a.ps_act;
    p.err = a.err;
    p.starve = test_starve();
    return v->fn(map, p, st);
}

int tc_probe_sw128(int *dev_out16, cudaStream_t st) {
    const int smem = 44 * 1024;
    cudaFuncSetAttribute(sw128_probe_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    sw128_probe_kernel<<<1, 128, smem, st>>>(dev_out16);
    return (int)cudaGetLastError();
}

int tc_selftest(int kind, int *dev_mismatch, cudaStream_t st) {
    const int smem = 64 * 1024;
    if (kind == 0) {
        cudaFuncSetAttribute(mma_selftest_kernel<0>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        mma_selftest_kernel<0><<<1, 128, smem, st>>>(dev_mismatch);
    } else {
        cudaFuncSetAttribute(mma_selftest_kernel<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        mma_selftest_kernel<1><<<1, 128, smem, st>>>(dev_mismatch);
    }
    return (int)cudaGetLastError();
}

}  // namespace nvisr
