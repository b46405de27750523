// Residual block of the enhancement trunk, y = x + conv2(LeakyReLU(conv1(x) + b1)) + b2
// (Section 3.1: the networks NNVISR runs are stacks of such 3x3 blocks), both convs
// 64 -> 64 channels with zero padding, in one launch of 2-CTA clusters.
//
// The row-streaming scheme of the single-layer kernel (conv_tc.cu) runs twice, on the
// two SMs of a cluster:
//  * rank 0 (the conv1 CTA) TMA-loads rows of x, issues the stacked-tap MMAs of conv1
//    (one N = 192 MMA per (kx, K step) covers output rows r + 1, r, r - 1) into its TMEM
//    ring, and its epilogue turns each finished row into h = LeakyReLU(acc + b1), rounded
//    to the activation type, staged 128-byte swizzled (as the MMA reads it) and sent by one
//    bulk copy into a ring of h rows in rank 1's shared memory (distributed shared memory);
//  * rank 1 (the conv2 CTA) runs the same MMA scheme on those h rows with conv2's
//    weights, and its epilogue adds b2 and the residual x (a TMA load, an L2 hit: rank 0
//    read that row a few rows earlier) and stores y by TMA.
// h never reaches device memory.  Per block the DRAM traffic is x read once plus y
// written once, against x, h, h, x and y for two single-layer launches (at 1920 x 1080:
// 531 MB instead of 1327 MB), and the two layers' MMA streams run on two SMs at once.
//
// Tiles: conv1 computes the 128 h pixels [x0 - 1, x0 + 127) of a row (the MMA's M), which
// give conv2 the 126 outputs [x0, x0 + 126): column tiles are 126 pixels wide (x0 = 126 c)
// and conv2's two last accumulator lanes are discarded.  h pixels or rows outside the
// image are written as zero (conv2's zero padding).  Rows: the (image, column tile, row)
// sequence is cut into equal contiguous ranges, one per cluster; a range is one or more
// strips of output rows [ra, rb) of one column tile, for which conv1 produces h rows
// [ra - 1, rb] from x rows [ra - 2, rb + 1].
//
// Synchronisation between the two CTAs: rank 0's epilogue waits until rank 1's MMAs have
// released the h slot and the staging tile's previous row (tcgen05.commit multicast onto
// rank 0's barriers), stages the row and issues the copy, whose bytes complete the
// transaction count of rank 1's barrier of that slot (armed by rank 1 for each row).
// (Per-thread remote stores, each followed by a cluster-scope fence and release, measured
// 1.5 us per row: the round trips, not the MMAs, set the pace.)  Every wait is bounded in
// time; a CTA that gives up raises the abort flags of both CTAs and the error word.  Both
// CTAs end with two cluster barriers: between them each side waits for what the other has
// already started towards its shared memory (copies, MMA commits), counted in words the
// other side updates, so neither leaves while the other may still write into it.
#include <algorithm>
#include <mutex>

#include "common.cuh"
#include "sm100_ptx.cuh"
#include "tc_util.cuh"

namespace nvisr {

namespace {

constexpr int BT = 126;                   // output pixels of a column tile
constexpr int TMH = 128;                  // h pixels of a row tile (the MMA's M)
constexpr int PXS = TMH + 2;              // x pixels of a row box
constexpr int BTHREADS = 352;             // warps: 0 TMA, 1 MMA, 2-9 epilogue, 10 issuer waits
constexpr int NSLOT = 8;                  // accumulator rows in TMEM (64 columns each)
constexpr int HS = 5;                     // h rows in rank 1's ring
constexpr uint32_t AROW = PXS * 128;      // bytes of one 130-pixel row of 64 channels
constexpr uint32_t ROWB = 17408;          // its 1 KB-aligned slot
constexpr uint32_t WB = 3 * 3 * 64 * 128; // one conv's stacked weights [kx][2 - ky][64 out][128 B]
constexpr uint32_t WKX = 3 * 64 * 128;    // weights of one kx
constexpr uint32_t TILEB = TMH * 128;     // one output / residual row tile
constexpr uint32_t HDR = 1024;            // barriers, flags, bias
constexpr uint32_t REGION = HS * ROWB + 4 * TILEB;            // rank 1: h ring + 2 output + 2 residual tiles
constexpr int XST = 5;                    // rank 0: x stages, then 4 h staging tiles (2 per epilogue group)
static_assert(XST * ROWB + 4 * TILEB <= REGION, "rank 0's room");
constexpr int BLOCK_SMEM = 1024 + (int)(HDR + WB + REGION);   // + alignment slack
constexpr uint64_t WAIT_NS = 2000000000ull;
static_assert(BLOCK_SMEM <= 232448, "227 KB per CTA");
static_assert(XST >= 4, "x prefetch depth");

struct BlockParams {
    int H, W, nimg;
    int ncols;                 // column tiles per image: ceil(W / 126)
    const uint8_t *w1, *w2;    // stacked weights of conv1 and conv2
    const float *b1, *b2;      // biases [64]
    int *err;
    int starve;                // test drill: rank 0 loads no input, the pipeline waits run out
};

// MULTI: the images of several streams (one BlockProblem each, any sizes) share the launch;
// otherwise nimg images of one size stacked along the maps' outer dimension.
template <int DT, bool MULTI>
__global__ void __launch_bounds__(BTHREADS, 1)
    res_block_kernel(const __grid_constant__ CUtensorMap xmap,  // x: 130-pixel row boxes, OOB zero
                     const __grid_constant__ CUtensorMap rmap,  // x: 128-pixel row tiles (residual)
                     const __grid_constant__ CUtensorMap ymap,  // y: 126-pixel row tiles
                     const BlockParams p, const BlockProblem *__restrict__ probs, int nprob) {
    using TO = typename Elem<DT>::T;
    constexpr int AFMT = DT == DT_BF16 ? 1 : 0;
    extern __shared__ uint8_t smem_raw[];
    // same offset in both CTAs: the dynamic shared memory starts at the same address
    uint8_t *smem = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    uint64_t *full = reinterpret_cast<uint64_t *>(smem);  // rank 0: x row landed
    uint64_t *empty = full + 8;                           // rank 0: x stage read by the MMAs
    uint64_t *rowdone = full + 16;                        // accumulator row complete
    uint64_t *slotfree = full + 24;                       // accumulator row drained
    uint64_t *hfull = full + 32;                          // rank 1: h row written by rank 0
    uint64_t *hempty = full + 40;                         // rank 0: h slot read by rank 1's MMAs
    uint64_t *resfull = full + 48;                        // rank 1: residual tile per group
    uint64_t *wbar = full + 50;
    uint64_t *drain = full + 51;                          // the issuer's MMAs, after an abort
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(smem + 416);
    volatile int *abort = reinterpret_cast<volatile int *>(smem + 420);
    volatile int *grp_stop = reinterpret_cast<volatile int *>(smem + 424);
    int *ready = reinterpret_cast<int *>(smem + 432);
    int *h_issued = reinterpret_cast<int *>(smem + 436);    // rank 1: h copies rank 0 has started
    int *h_consumed = reinterpret_cast<int *>(smem + 440);  // rank 0: h rows rank 1's MMAs were issued on
    float *sbias = reinterpret_cast<float *>(smem + 512);
    uint8_t *wsm = smem + HDR;
    uint8_t *region = wsm + WB;        // rank 0: x stages; rank 1: h ring
    uint8_t *obuf = region + HS * ROWB;  // rank 1: output staging tile per group
    uint8_t *rbuf = obuf + 2 * TILEB;    // rank 1: residual tile per group
    uint8_t *stg = region + XST * ROWB;  // rank 0: h staging tiles [group][2]

    const uint32_t rank = cluster_ctarank();
    const bool first = rank == 0;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t npairs = cluster_count_x(), pair = cluster_id_x();
    const int64_t total = MULTI ? probs[nprob - 1].u0 + (int64_t)probs[nprob - 1].ncols * probs[nprob - 1].H
                                : (int64_t)p.nimg * p.ncols * p.H;
    const int64_t u_begin = total * pair / npairs, u_end = total * (pair + 1) / npairs;
    // the strip at position u of this cluster's range: problem (MULTI), image, column tile,
    // output rows [ra, rb)
    auto strip_at = [&](int64_t u, int &pi, int &img, int &col, int &ra, int &rb) {
        int64_t local = u, H = p.H;
        pi = 0;
        if (MULTI) {
            while (pi + 1 < nprob && u >= probs[pi + 1].u0) ++pi;
            local = u - probs[pi].u0;
            H = probs[pi].H;
        }
        const int64_t cg = local / H;
        ra = (int)(local - cg * H);
        rb = (int)min(H, (int64_t)ra + (u_end - u));
        img = MULTI ? 0 : (int)(cg / p.ncols);
        col = (int)(cg - (int64_t)img * p.ncols);
    };
    auto xmap_of = [&](int pi) { return MULTI ? &probs[pi].xmap : &xmap; };
    auto rmap_of = [&](int pi) { return MULTI ? &probs[pi].rmap : &rmap; };
    auto ymap_of = [&](int pi) { return MULTI ? &probs[pi].ymap : &ymap; };
    auto height_of = [&](int pi) { return MULTI ? probs[pi].H : p.H; };
    auto width_of = [&](int pi) { return MULTI ? probs[pi].W : p.W; };
    // rows this CTA's accumulators produce for a strip: h rows [ra - 1, rb + 1) (rank 0) or
    // output rows [ra, rb) (rank 1); its input rows run from oa - 1 to ob
    auto out_rows = [&](int ra, int rb, int &oa, int &ob) {
        oa = first ? ra - 1 : ra;
        ob = first ? rb + 1 : rb;
    };
    const uint32_t peer_abort = mapa_shared(smem_u32(const_cast<int *>(abort)), rank ^ 1u);
    auto fail = [&]() {
        *abort = 1;
        st_cluster_u32(peer_abort, 1u);
        if (p.err) atomicExch(p.err, DEVERR_TIMEOUT);
    };

    if (threadIdx.x == 0) {
        for (int k = 0; k < 8; ++k) {
            mbar_init(&full[k], 1);
            mbar_init(&empty[k], 1);
            mbar_init(&rowdone[k], 1);
            mbar_init(&slotfree[k], 128);
        }
        for (int k = 0; k < HS; ++k) {
            mbar_init(&hfull[k], 1);    // rank 1's arming (expect_tx) + the copy's bytes
            mbar_init(&hempty[k], 1);   // rank 1's MMA commit
        }
        mbar_init(&resfull[0], 1);
        mbar_init(&resfull[1], 1);
        mbar_init(wbar, 1);
        mbar_init(drain, 1);
        *abort = 0;
        grp_stop[0] = 0;
        grp_stop[1] = 0;
        *ready = 0;
        *h_issued = 0;
        *h_consumed = 0;
        fence_mbarrier_init();
        // weights are written once at filter creation: loaded before the wait on the previous kernel
        mbar_arrive_expect_tx(wbar, WB);
        const uint8_t *wsrc = first ? p.w1 : p.w2;
        for (uint32_t off = 0; off < WB; off += 32768u) bulk_load(wsm + off, wsrc + off, min(32768u, WB - off), wbar);
    }
    if (threadIdx.x >= 64 && threadIdx.x < 128) sbias[threadIdx.x - 64] = (first ? p.b1 : p.b2)[threadIdx.x - 64];
    if (!first && threadIdx.x >= 128 && threadIdx.x < 128 + HS * 16) {
        // h lines 128, 129 of every slot feed only the two discarded output pixels: zero
        const int t = threadIdx.x - 128;
        st_shared_u4(smem_u32(region + (t / 16) * ROWB + TMH * 128 + (t % 16) * 16), make_uint4(0u, 0u, 0u, 0u));
        fence_proxy_async();
    }
    if (warp == 1) {
        tmem_alloc(tmem_slot, 512);
        tmem_relinquish();
    }
    tc_fence_before();
    __syncthreads();
    cluster_sync_all();  // both CTAs' barriers are initialised before either arrives on the other's
    tc_fence_after();
    const uint32_t tmem_base = *tmem_slot;
    griddep_launch_dependents();
    griddep_wait();

    int w_done = 0, w_armed = 0;  // rank 1's wait warp: h rows landed / armed
    int i_rows = 0;               // rank 1's issuer: h rows whose MMAs it issued (and committed)
    if (warp == 0) {
        if (first && lane == 0) {
            // ---------------- producer (rank 0): x rows ra - 2 .. rb + 1 of each strip
            int gin = 0;
            bool ok = true;
            for (int64_t u = u_begin; u < u_end && ok && !p.starve;) {
                int pi, img, col, ra, rb;
                strip_at(u, pi, img, col, ra, rb);
                u += rb - ra;
                const int xb = col * BT - 2;  // box pixel 0 = h pixel col * BT - 1 minus one
                for (int r = ra - 2; r <= rb + 1; ++r, ++gin) {
                    const int s = gin % XST;
                    if (!mbar_wait_bounded(&empty[s], (uint32_t)((gin / XST) & 1) ^ 1u, abort, WAIT_NS)) {
                        fail();
                        ok = false;
                        break;
                    }
                    mbar_arrive_expect_tx(&full[s], AROW);
                    tma_load_4d(region + (size_t)s * ROWB, xmap_of(pi), &full[s], 0, xb, r, img);
                }
            }
            // copies still in flight after an early exit land before the CTA ends
            for (int k = 0; k < XST && k < gin; ++k) {
                const int idx = gin - 1 - k;
                mbar_wait_bounded(&full[idx % XST], (uint32_t)((idx / XST) & 1), nullptr, WAIT_NS);
            }
        }
        if (lane == 0) mbar_wait_bounded(wbar, 0, nullptr, WAIT_NS);
    } else if (warp == 1) {
        if (lane == 0) {
            // ---------------- MMA issuer (both ranks).  Input row r of a strip feeds the
            // CTA's accumulator rows r - 1 .. r + 1 (those inside [oa, ob)), which form one
            // run of contiguous TMEM slots or two where the ring wraps; row r + 1 gets its
            // first product (accumulate = 0) here.  The wait warp publishes how many input
            // rows are ready, so this thread makes no mbarrier waits while MMAs are queued.
            bool ok = mbar_wait_bounded(wbar, 0, abort, WAIT_NS);
            if (!ok) fail();
            const int S = first ? XST : HS;
            const uint64_t b_base = smem_desc_sw128(smem_u32(wsm), 0);
            const uint32_t id0 = instr_desc(TMH, 0, AFMT, AFMT);
            const uint32_t nstep = (uint32_t)(64 / 8) << 17;  // N += 64
            int s = 0, gout = 0, gin = 0, nready = 0, last_slot = -1;
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
                tc_fence_after();
                return true;
            };
            // (kx, K step) t: A advances one pixel (128 B) per kx and 32 bytes per K step inside
            // the swizzled line; B one kx block per kx
            auto a_off = [](int t) { return (uint64_t)(((t / 4) * 128 + (t % 4) * 32) >> 4); };
            auto b_off = [](int t) { return (uint64_t)(((t / 4) * WKX + (t % 4) * 32) >> 4); };
            for (int64_t u = u_begin; u < u_end && ok;) {
                int pi, img, col, ra, rb, oa, ob;
                strip_at(u, pi, img, col, ra, rb);
                u += rb - ra;
                out_rows(ra, rb, oa, ob);
                const int base = gout - oa;  // global accumulator-row index of row o is base + o
                for (int r = oa - 1; r <= ob; ++r) {
                    if (!await_row(gin)) {
                        ok = false;
                        break;
                    }
                    const int o_lo = max(r - 1, oa), o_hi = min(r + 1, ob - 1);
                    const bool fresh = r + 1 <= ob - 1;
                    const int sl = (base + r - 1) & (NSLOT - 1);
                    if (r - 1 >= oa && fresh && sl <= NSLOT - 3) {
                        // interior row whose three accumulator rows do not wrap the ring (6 of 8
                        // rows): one N = 192 run; the fresh row r + 1 starts at kx = 0, K step 0
                        const uint64_t a_base = smem_desc_sw128(smem_u32(region + (size_t)s * ROWB), 0);
                        const uint32_t md = tmem_base + (uint32_t)(sl * 64);
                        umma<0>(md, a_base, b_base, id0 + nstep * 2u, 1u);
                        umma<0>(md + 128u, a_base, b_base + (uint64_t)((2 * 64 * 128) >> 4), id0 + nstep, 0u);
#pragma unroll
                        for (int t = 1; t < 12; ++t) umma<0>(md, a_base + a_off(t), b_base + b_off(t), id0 + nstep * 3u, 1u);
                    } else if (o_lo <= o_hi) {
                        const uint64_t a_base = smem_desc_sw128(smem_u32(region + (size_t)s * ROWB), 0);
                        auto slot_of = [&](int o) { return (base + o) & (NSLOT - 1); };
                        auto bd_of = [&](int o) { return b_base + (uint64_t)(((o - r + 1) * 64 * 128) >> 4); };
                        const int sl0 = slot_of(o_lo);
                        const int len = o_hi - o_lo + 1;
                        const int m0 = min(len, NSLOT - sl0), m1 = len - m0;
                        const uint32_t md0 = tmem_base + (uint32_t)(sl0 * 64), md1 = tmem_base;
                        const uint32_t mi0 = id0 + nstep * (uint32_t)m0, mi1 = id0 + nstep * (uint32_t)max(m1, 1);
                        const uint64_t mb0 = bd_of(o_lo), mb1 = bd_of(o_lo + m0);
                        {
                            // first (kx, K step): the rows already started accumulate, the fresh row starts
                            const int old_hi = fresh ? min(r, o_hi) : o_hi;
                            const int olen = old_hi - o_lo + 1;
                            if (olen > 0) {
                                const int f0 = min(olen, m0), f1 = olen - f0;
                                umma<0>(md0, a_base, mb0, id0 + nstep * (uint32_t)f0, 1u);
                                if (f1 > 0) umma<0>(md1, a_base, mb1, id0 + nstep * (uint32_t)f1, 1u);
                            }
                            if (fresh)
                                umma<0>(tmem_base + (uint32_t)(slot_of(r + 1) * 64), a_base, bd_of(r + 1), id0 + nstep, 0u);
                        }
                        if (m1 == 0) {
#pragma unroll
                            for (int t = 1; t < 12; ++t) umma<0>(md0, a_base + a_off(t), mb0 + b_off(t), mi0, 1u);
                        } else {
#pragma unroll
                            for (int t = 1; t < 12; ++t) {
                                const uint64_t ad = a_base + a_off(t), boff = b_off(t);
                                umma<0>(md0, ad, mb0 + boff, mi0, 1u);
                                umma<0>(md1, ad, mb1 + boff, mi1, 1u);
                            }
                        }
                    }
                    // the input row's buffer is free once these MMAs have run: rank 0's x stage, or
                    // rank 1's h slot, released on rank 0's barrier of that slot
                    if (first) umma_commit(&empty[s]);
                    else umma_commit_multicast(&hempty[s], (uint16_t)1u);
                    if (r - 1 >= oa) {
                        const int i = base + r - 1;
                        umma_commit(&rowdone[i & (NSLOT - 1)]);
                        last_slot = i & (NSLOT - 1);
                        last_par = (uint32_t)((i >> 3) & 1);
                    }
                    if (++s == S) s = 0;
                    ++gin;
                }
                gout += ob - oa;
            }
            i_rows = gin;
            if (!ok) fail();
            if (last_slot >= 0) mbar_wait_bounded(&rowdone[last_slot], last_par, nullptr, WAIT_NS);
            if (*abort) {
                // an early exit may leave MMAs that no row commit covers
                umma_commit(drain);
                mbar_wait_bounded(drain, 0, nullptr, WAIT_NS);
            }
        }
    } else if (warp == 10) {
        if (lane == 0) {
            // ---------------- wait warp: for each input row in the issuer's order, wait until
            // the slot of its fresh accumulator row is drained and the row is in shared memory
            // (rank 0: the x row's TMA; rank 1: rank 0's h stores), then publish the count.
            const int S = first ? XST : HS;
            int s = 0, gout = 0, gin = 0;
            uint32_t ph = 0;
            bool ok = true;
            for (int64_t u = u_begin; u < u_end && ok;) {
                int pi, img, col, ra, rb, oa, ob;
                strip_at(u, pi, img, col, ra, rb);
                u += rb - ra;
                out_rows(ra, rb, oa, ob);
                const int base = gout - oa;
                for (int r = oa - 1; r <= ob; ++r) {
                    if (r + 1 <= ob - 1) {
                        const int i = base + r + 1;
                        if (!mbar_wait_bounded(&slotfree[i & (NSLOT - 1)], (uint32_t)((i >> 3) & 1) ^ 1u, abort,
                                               WAIT_NS)) {
                            ok = false;
                            break;
                        }
                    }
                    if (!first && gin >= w_armed) {
                        mbar_arrive_expect_tx(&hfull[s], TILEB);  // the copy of h row gin
                        w_armed = gin + 1;
                    }
                    const bool in = mbar_wait_bounded(first ? &full[s] : &hfull[s], ph, abort, WAIT_NS);
                    if (!in) {
                        ok = false;
                        break;
                    }
                    st_release_cta(ready, ++gin);
                    w_done = gin;
                    if (++s == S) {
                        s = 0;
                        ph ^= 1u;
                    }
                }
                gout += ob - oa;
            }
            if (!ok) fail();
        }
    } else if (first) {
        // ---------------- rank 0 epilogue: two groups of 4 warps (2-5, 6-9) on alternate h
        // rows; warp w reads TMEM lane quadrant w % 4 (pixel m), all 64 columns, stages the
        // pixel's 128-byte line, and the group leader copies the row into rank 1's h slot
        const int q = warp & 3;
        const int g = (warp - 2) >> 2;
        const int m = q * 32 + lane;
        const bool leader = warp == 2 + 4 * g && lane == 0;
        const int bar_id = 1 + g;
        const uint32_t h_remote = mapa_shared(smem_u32(region), 1u);
        const uint32_t hfull_remote = mapa_shared(smem_u32(hfull), 1u);
        const uint32_t issued_remote = mapa_shared(smem_u32(h_issued), 1u);
        // h row j has been read by rank 1's MMAs (its commit onto hempty)
        auto consumed = [&](int j) {
            return j < 0 || mbar_wait_bounded(&hempty[j % HS], (uint32_t)((j / HS) & 1), abort, WAIT_NS);
        };
        int gout = 0;
        bool ok = true;
        for (int64_t u = u_begin; u < u_end && ok;) {
            int pi, img, col, ra, rb;
            strip_at(u, pi, img, col, ra, rb);
            u += rb - ra;
            const int oa = ra - 1, ob = rb + 1;
            const int px = col * BT - 1 + m;
            const bool colok = px >= 0 && px < width_of(pi);
            const int Hs = height_of(pi);
            int o = oa + ((g - (gout & 1)) & 1);
            for (; o < ob; o += 2) {
                const int i = gout + (o - oa);
                const int slot = i & (NSLOT - 1), hs = i % HS;
                uint8_t *tile = stg + (size_t)(g * 2 + ((i >> 1) & 1)) * TILEB;
                bool w = mbar_wait_bounded(&rowdone[slot], (uint32_t)((i >> 3) & 1), abort, WAIT_NS);
                w = __all_sync(0xffffffffu, w);
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
                    mbar_arrive(&slotfree[slot]);
                } else {
#pragma unroll
                    for (int e = 0; e < 64; ++e) v[e] = 0.f;
                    if (lane == 0) {
                        fail();
                        grp_stop[g] = 1;
                    }
                }
                // bias and LeakyReLU(0.1) in packed f32x2 arithmetic (the single-layer kernel's)
#pragma unroll
                for (int e = 0; e < 64; e += 4) {
                    const float4 b = *reinterpret_cast<const float4 *>(sbias + e);
                    add_f32x2(v[e], v[e + 1], b.x, b.y);
                    add_f32x2(v[e + 2], v[e + 3], b.z, b.w);
                }
#pragma unroll
                for (int e = 0; e < 64; e += 2) {
                    float t0 = v[e], t1 = v[e + 1];
                    mul_f32x2(t0, t1, 0.1f, 0.1f);
                    v[e] = fmaxf(v[e], t0);
                    v[e + 1] = fmaxf(v[e + 1], t1);
                }
                const bool keep = colok && o >= 0 && o < Hs;  // else conv2's zero padding
                // the h slot's previous row (i - HS) and the staging tile's (i - 4) have been read
                bool wf = consumed(i - HS) && consumed(i - 4);
                wf = __all_sync(0xffffffffu, wf);
                if (!wf && lane == 0) {
                    fail();
                    grp_stop[g] = 1;
                }
                if (w && wf) {
                    uint8_t *line = tile + m * 128;
#pragma unroll
                    for (int uu = 0; uu < 8; ++uu) {
                        const int unit = uu ^ (m & 7);
                        uint4 ov = make_uint4(0u, 0u, 0u, 0u);
                        if (keep) {
                            ov.x = pack2<TO>(v[uu * 8 + 0], v[uu * 8 + 1]);
                            ov.y = pack2<TO>(v[uu * 8 + 2], v[uu * 8 + 3]);
                            ov.z = pack2<TO>(v[uu * 8 + 4], v[uu * 8 + 5]);
                            ov.w = pack2<TO>(v[uu * 8 + 6], v[uu * 8 + 7]);
                        }
                        *reinterpret_cast<uint4 *>(line + unit * 16) = ov;
                    }
                    fence_proxy_async();  // the staged row, before the copy reads it
                }
                if (leader && *abort) grp_stop[g] = 1;
                named_barrier(bar_id, 128);
                if (grp_stop[g]) {
                    ok = false;
                    break;
                }
                if (leader) {
                    bulk_copy_to_cluster(h_remote + (uint32_t)hs * ROWB, tile, TILEB, hfull_remote + (uint32_t)hs * 8u);
                    red_add_cluster(issued_remote, 1u);
                }
            }
            gout += ob - oa;
        }
    } else {
        // ---------------- rank 1 epilogue: bias + residual, staged 128-byte swizzled and
        // written by one TMA store per row (126 pixels); the residual arrives by TMA, issued
        // two rows ahead
        const int q = warp & 3;
        const int g = (warp - 2) >> 2;
        const int m = q * 32 + lane;
        const bool leader = warp == 2 + 4 * g && lane == 0;
        const int bar_id = 1 + g;
        uint8_t *ot = obuf + g * TILEB + m * 128;
        const uint8_t *rt = rbuf + g * TILEB + m * 128;
        int gout = 0;
        int res_loads = 0, last_res = -1;
        bool ok = true;
        for (int64_t u = u_begin; u < u_end && ok;) {
            int pi, img, col, ra, rb;
            strip_at(u, pi, img, col, ra, rb);
            u += rb - ra;
            const int x0 = col * BT;
            int o = ra + ((g - (gout & 1)) & 1);
            if (leader && o < rb) {
                mbar_arrive_expect_tx(&resfull[g], TILEB);
                tma_load_4d(rbuf + g * TILEB, rmap_of(pi), &resfull[g], 0, x0, o, img);
                last_res = res_loads++;
            }
            for (; o < rb; o += 2) {
                const int i = gout + (o - ra);
                const int slot = i & (NSLOT - 1);
                const int k = i >> 1;  // this group's row count: the phase of its residual barrier
                if (leader) bulk_wait_group_read<0>();  // the group's previous store has read its tile
                named_barrier(bar_id, 128);
                bool w = mbar_wait_bounded(&rowdone[slot], (uint32_t)((i >> 3) & 1), abort, WAIT_NS);
                w = __all_sync(0xffffffffu, w);
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
                    mbar_arrive(&slotfree[slot]);
                } else {
#pragma unroll
                    for (int e = 0; e < 64; ++e) v[e] = 0.f;
                    if (lane == 0) {
                        fail();
                        grp_stop[g] = 1;
                    }
                }
#pragma unroll
                for (int e = 0; e < 64; e += 4) {
                    const float4 b = *reinterpret_cast<const float4 *>(sbias + e);
                    add_f32x2(v[e], v[e + 1], b.x, b.y);
                    add_f32x2(v[e + 2], v[e + 3], b.z, b.w);
                }
                bool rw = mbar_wait_bounded(&resfull[g], (uint32_t)(k & 1), abort, WAIT_NS);
                rw = __all_sync(0xffffffffu, rw);
                if (!rw && lane == 0) {
                    fail();
                    grp_stop[g] = 1;
                }
#pragma unroll
                for (int uu = 0; uu < 8; ++uu) {
                    const int unit = uu ^ (m & 7);
                    const uint4 raw = *reinterpret_cast<const uint4 *>(rt + unit * 16);
                    const uint32_t wd[4] = {raw.x, raw.y, raw.z, raw.w};
#pragma unroll
                    for (int h = 0; h < 4; ++h) {
                        float r0, r1;
                        unpack2<TO>(wd[h], r0, r1);
                        add_f32x2(v[uu * 8 + 2 * h], v[uu * 8 + 2 * h + 1], r0, r1);
                    }
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
                fence_proxy_async();  // staging writes (and residual reads) before the async proxy
                if (leader && *abort) grp_stop[g] = 1;
                named_barrier(bar_id, 128);
                if (grp_stop[g]) {
                    ok = false;
                    break;
                }
                if (leader) {
                    tma_store_4d(ymap_of(pi), obuf + g * TILEB, 0, x0, o, img);
                    bulk_commit_group();
                    if (o + 2 < rb) {  // this group's next row; the tile's readers are done
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
    if (!first && warp == 1 && lane == 0) st_cluster_u32(mapa_shared(smem_u32(h_consumed), 0u), (uint32_t)i_rows);
    __syncthreads();
    cluster_sync_all();  // every copy and MMA commit towards either CTA has been issued; the counts are final
    if (!first && warp == 10 && lane == 0) {
        // h copies rank 0 started that this CTA has not waited for (after an early exit) land first
        const int issued = *h_issued;
        for (int j = w_done; j < issued; ++j) {
            const int s = j % HS;
            if (j >= w_armed) mbar_arrive_expect_tx(&hfull[s], TILEB);
            mbar_wait_bounded(&hfull[s], (uint32_t)((j / HS) & 1), nullptr, WAIT_NS);
        }
    }
    if (first && warp == 2 && lane == 0) {
        // rank 1's MMA commits onto this CTA's barriers have landed (the last one of each slot)
        const int n = *h_consumed;
        for (int j = max(0, n - HS); j < n; ++j)
            mbar_wait_bounded(&hempty[j % HS], (uint32_t)((j / HS) & 1), nullptr, WAIT_NS);
    }
    cluster_sync_all();  // neither CTA leaves while the other may still write into its shared memory
    if (warp == 1) {
        __syncwarp();
        tc_fence_after();
        tmem_dealloc(tmem_base, 512);
    }
}

// Clusters of this kernel that fit the device at once (one CTA per SM), looked up once per device.
template <int DT, bool MULTI>
int max_pairs() {
    static int cached[64] = {0};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) dev = 0;
    if (cached[dev] > 0) return cached[dev];
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = 2;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.gridDim = dim3(2 * std::max(1, device_sm_count() / 2));
    cfg.blockDim = dim3(BTHREADS);
    cfg.dynamicSmemBytes = BLOCK_SMEM;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    int n = 0;
    if (cudaOccupancyMaxActiveClusters(&n, res_block_kernel<DT, MULTI>, &cfg) != cudaSuccess || n < 1) {
        (void)cudaGetLastError();
        return 0;
    }
    cached[dev] = n;
    return n;
}

// units: output rows x column tiles of the launch (each cluster gets an equal range)
template <int DT, bool MULTI>
cudaError_t run_block(const CUtensorMap &xmap, const CUtensorMap &rmap, const CUtensorMap &ymap,
                      const BlockParams &p, const BlockProblem *probs, int nprob, int64_t units, cudaStream_t st) {
    cudaError_t e = set_smem_limit<res_block_kernel<DT, MULTI>>(BLOCK_SMEM);
    if (e != cudaSuccess) return e;
    int npairs = max_pairs<DT, MULTI>();
    if (npairs < 1) return cudaErrorInvalidConfiguration;
    // at least ~16 output rows per cluster: each strip costs conv1 two extra rows
    npairs = (int)std::max<int64_t>(1, std::min<int64_t>(npairs, units / 16));
    cudaLaunchAttribute at[2];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = 2;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    at[1].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[1].val.programmaticStreamSerializationAllowed = 1;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(2 * npairs);
    cfg.blockDim = dim3(BTHREADS);
    cfg.dynamicSmemBytes = BLOCK_SMEM;
    cfg.stream = st;
    cfg.attrs = at;
    cfg.numAttrs = 2;
    return cudaLaunchKernelEx(&cfg, res_block_kernel<DT, MULTI>, xmap, rmap, ymap, p, probs, nprob);
}

cudaError_t encode_block_map(CUtensorMap *map, const void *base, int W, int H, int nimg, int box_px) {
    auto enc = encode_fn();
    if (!enc) return cudaErrorNotSupported;
    cuuint64_t dims[4] = {128, (cuuint64_t)W, (cuuint64_t)H, (cuuint64_t)nimg};
    cuuint64_t strides[3] = {128, (cuuint64_t)W * 128, (cuuint64_t)W * H * 128};
    cuuint32_t box[4] = {128, (cuuint32_t)box_px, 1, 1};
    cuuint32_t estr[4] = {1, 1, 1, 1};
    const CUresult r = enc(map, CU_TENSOR_MAP_DATA_TYPE_UINT8, 4, const_cast<void *>(base), dims, strides, box, estr,
                           CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                           CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

cudaError_t encode_block_maps(const ConvArgs &c1, const ConvArgs &c2, CUtensorMap *xmap, CUtensorMap *rmap,
                              CUtensorMap *ymap) {
    cudaError_t e = encode_block_map(xmap, c1.x, c1.W, c1.H, c1.nimg, PXS);
    if (e == cudaSuccess) e = encode_block_map(rmap, c1.x, c1.W, c1.H, c1.nimg, TMH);
    if (e == cudaSuccess) e = encode_block_map(ymap, c2.y, c1.W, c1.H, c1.nimg, BT);
    return e;
}

BlockParams block_params(const ConvArgs &c1, const ConvArgs &c2) {
    BlockParams p{};
    p.H = c1.H;
    p.W = c1.W;
    p.nimg = c1.nimg;
    p.ncols = (c1.W + BT - 1) / BT;
    p.w1 = static_cast<const uint8_t *>(c1.w_rows);
    p.w2 = static_cast<const uint8_t *>(c2.w_rows);
    p.b1 = c1.bias;
    p.b2 = c2.bias;
    p.err = c1.err ? c1.err : c2.err;
    p.starve = test_starve();
    return p;
}

}  // namespace

bool res_block_fits(const ConvArgs &c1, const ConvArgs &c2) {
    if (!rows_kernel_fits(c1) || !rows_kernel_fits(c2)) return false;
    if (c2.in_dt != c1.in_dt || c1.nimg != c2.nimg || c1.H != c2.H || c1.W != c2.W || c1.nimg < 1) return false;
    if (c1.act != 1 || c1.res || c2.act != 0 || c2.res != c1.x || c2.x != c1.y) return false;
    if (c1.y2 || c2.y2 || c1.amax || c2.amax || c1.acc_scale != 1.f || c1.out_scale != 1.f || c2.acc_scale != 1.f ||
        c2.out_scale != 1.f)
        return false;
    // other clusters still read x (halo rows and columns) while y is written
    const size_t bytes = (size_t)c1.nimg * c1.H * c1.W * 128;
    const uint8_t *xb = static_cast<const uint8_t *>(c1.x), *yb = static_cast<const uint8_t *>(c2.y);
    return !(yb < xb + bytes && xb < yb + bytes);
}

cudaError_t launch_res_block(const ConvArgs &c1, const ConvArgs &c2, cudaStream_t st) {
    if (!res_block_fits(c1, c2)) return cudaErrorInvalidValue;
    CUtensorMap xmap, rmap, ymap;
    cudaError_t e = encode_block_maps(c1, c2, &xmap, &rmap, &ymap);
    if (e != cudaSuccess) return e;
    const BlockParams p = block_params(c1, c2);
    const int64_t units = (int64_t)p.nimg * p.ncols * p.H;
    return c1.in_dt == DT_BF16 ? run_block<DT_BF16, false>(xmap, rmap, ymap, p, nullptr, 0, units, st)
                               : run_block<DT_F16, false>(xmap, rmap, ymap, p, nullptr, 0, units, st);
}

cudaError_t launch_res_block_multi(const ConvArgs *c1, const ConvArgs *c2, int n, BlockProblem *host_tab,
                                   BlockProblem *dev_tab, cudaStream_t st, bool copy_table, bool launch) {
    if (n < 1) return cudaSuccess;
    for (int i = 0; i < n; ++i) {
        // one image each; the same weights, biases and dtype
        if (!res_block_fits(c1[i], c2[i]) || c1[i].nimg != 1 || c1[i].in_dt != c1[0].in_dt ||
            c1[i].w_rows != c1[0].w_rows || c2[i].w_rows != c2[0].w_rows || c1[i].bias != c1[0].bias ||
            c2[i].bias != c2[0].bias)
            return cudaErrorInvalidValue;
    }
    int64_t units = 0;
    for (int i = 0; i < n; ++i) {
        BlockProblem &q = host_tab[i];
        cudaError_t e = encode_block_maps(c1[i], c2[i], &q.xmap, &q.rmap, &q.ymap);
        if (e != cudaSuccess) return e;
        q.H = c1[i].H;
        q.W = c1[i].W;
        q.ncols = (c1[i].W + BT - 1) / BT;
        q.pad_ = 0;
        q.u0 = units;
        units += (int64_t)q.ncols * q.H;
    }
    if (copy_table) {
        cudaError_t e = cudaMemcpyAsync(dev_tab, host_tab, sizeof(BlockProblem) * n, cudaMemcpyHostToDevice, st);
        if (e != cudaSuccess) return e;
    }
    if (!launch) return cudaSuccess;
    const BlockParams p = block_params(c1[0], c2[0]);
    return c1[0].in_dt == DT_BF16
               ? run_block<DT_BF16, true>(host_tab[0].xmap, host_tab[0].rmap, host_tab[0].ymap, p, dev_tab, n, units, st)
               : run_block<DT_F16, true>(host_tab[0].xmap, host_tab[0].rmap, host_tab[0].ymap, p, dev_tab, n, units, st);
}

}  // namespace nvisr
