// Shared definitions of the CUDA path (internal; not part of the C ABI).
#pragma once

#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_fp8.h>
#include <stdint.h>

#include <string>
#include <utility>

#include "nvisr.h"

namespace nvisr {

// Element type of an activation tensor in the blocked layout.
enum DType : int { DT_F32 = 0, DT_BF16 = 1, DT_F16 = 2, DT_E4M3 = 3 };

inline int dtype_size(int dt) { return dt == DT_F32 ? 4 : (dt == DT_E4M3 ? 1 : 2); }
// Channels per 16-byte unit.
inline int chunk_channels(int dt) { return 16 / dtype_size(dt); }
// Channels per chunk of the blocked layout [C/cpc][H][W][cpc] of a tensor:
// 16-bit tensors whose padded channel count is a multiple of 64 use 64-channel
// (128-byte) chunks -- one 128-byte-swizzled TMA row per pixel -- and every
// other tensor uses 16-byte chunks.
inline int layout_cpc(int dt, int cpad) {
    if ((dt == DT_BF16 || dt == DT_F16) && cpad % 64 == 0) return 64;
    return chunk_channels(dt);
}
inline int round_up(int v, int m) { return (v + m - 1) / m * m; }
inline int64_t round_up64(int64_t v, int64_t m) { return (v + m - 1) / m * m; }

// Last error message (nvisr_last_error): kept per thread, and per engine for
// the calls an ErrScope marks as working on that engine.
void set_error(const std::string &msg);
struct ErrScope {
    explicit ErrScope(nvisr_engine *e);
    ~ErrScope();
    nvisr_engine *prev;
};
nvisr_status cuda_status(cudaError_t e, const char *where);

#define NVISR_TRY_CUDA(expr)                                                   \
    do {                                                                       \
        cudaError_t _e = (expr);                                               \
        if (_e != cudaSuccess) return ::nvisr::cuda_status(_e, #expr);         \
    } while (0)

// ---------------------------------------------------------------------------
// Kernel launchers (each returns the launch's cudaError_t).
// ---------------------------------------------------------------------------

// ingest: integer planes -> float32 planar R'G'B' (pitch in floats).
// yuv: the network works on Y'Cb'Cr' planes (no colour matrix in ingest / requantise).
cudaError_t launch_ingest(const nvisr_format &fmt, const void *y, int64_t py, const void *u,
                          int64_t pu, const void *v, int64_t pv, float *out, int64_t out_pitch,
                          cudaStream_t st, int yuv = 0);

// The network's skip path: the mean of up to two input frames (planar float32
// [3][h][pitch]) upsampled by an integer scale (1 nearest, 2 bilinear with
// align_corners = false and edge clamp), added to the network's residual.
struct SkipArgs {
    const float *src[2];
    int n;               // 0 = no skip
    int64_t pitch, plane;
    int h, w, scale, mode;
    int scale_y;         // vertical scale when it differs from scale (0 = scale)
};

// Requantisation fused into a 2 x 2 PixelShuffle output layer's epilogue: the layer's
// residual plus the bilinear x2 skip of one frame, R'G'B' -> Y'CbCr, chroma downsampling
// (4:2:0) by siting, range scale, round half to even, clamp, packed into integer planes.
// LEFT-sited 4:2:0 chroma at a 128-pixel strip's first column needs the previous strip's
// last column: the two CTAs leave their columns' values in `edge`, and
// launch_rq_edge_fixup finishes those samples.
struct FusedRq {
    int on;                   // 0: the layer writes planar float32 (no fusion)
    int wide;                 // samples of more than 8 bits (16-bit storage)
    int sub420;               // 4:2:0 (else 4:4:4)
    int loc;                  // chroma siting (nvisr_chroma_loc)
    float y_mul, y_add, c_mul, c_add, vmax;
    float kr, kg, kb, cb_s, cr_s;
    uint8_t *yp, *up, *vp;    // output planes
    int64_t py, pu, pv;       // their pitches in bytes
    const float *skip;        // skip frame, planar float32 [3][H][skip_pitch] (null: no skip)
    int64_t skip_pitch, skip_plane;
    float *edge;              // LEFT 4:2:0: 6 floats per (LR row, 128-pixel column tile)
};
// Colour constants of an output format for the fused form: false when the format or the
// network domain is not one it serves (transfer functions, Y'CbCr-domain networks, RGB planes).
bool fused_rq_format(const nvisr_format &f, int yuv, FusedRq *rq);
// Finishes the LEFT-sited 4:2:0 chroma samples at the first column of each 128-pixel tile
// after x = 0 (H low-resolution rows, W low-resolution columns).
cudaError_t launch_rq_edge_fixup(const FusedRq &rq, int H, int W, cudaStream_t st);
// Whether launch_rq_edge_fixup launches its kernel for this output (LEFT-sited 4:2:0, 2+ tiles).
bool rq_edge_fixup_runs(const FusedRq &rq, int W);

// A final layer's float32 output, blocked [cpad/4][H][W][4], PixelShuffled by (ry, rx) into
// planar [C / (ry*rx)][H*ry][dst_pitch]: dst[c][ry*y + i][rx*x + j] = src channel
// c*ry*rx + i*rx + j at (y, x).  C = 3 * ry * rx.
cudaError_t launch_shuffle_planar(const float *src, int H, int W, int ry, int rx, float *dst, int64_t dst_pitch,
                                  cudaStream_t st);

// requantise: float32 planar R'G'B' (+ skip) -> integer planes.
cudaError_t launch_requant(const nvisr_format &fmt, const float *in, int64_t in_pitch, void *y,
                           int64_t py, void *u, int64_t pu, void *v, int64_t pv, cudaStream_t st,
                           const SkipArgs *skip = nullptr, int yuv = 0);

// Up to 8 planar float32 frames of 3 channels each (tuple, frame-major
// channels) or one planar tensor of C channels -> blocked tensor of dtype dt
// with cpad channels (zero filled past the real channels).  scale multiplies
// every value before conversion (FP8 quantisation), and amax (optional)
// receives max |value| (before scaling) via atomicMax on its float bits.
struct PackArgs {
    const float *src[8];
    int nsrc;            // number of source tensors
    int ch_per_src;      // channels of each source
    int64_t src_pitch;   // floats between rows
    int64_t src_plane;   // floats between channels
    int H, W;
    void *dst;
    int cpad;
    int dt;
    int cpc;             // channels per chunk of dst (0 = one 16-byte unit)
    float scale;
    unsigned *amax;
};
cudaError_t launch_pack(const PackArgs &a, cudaStream_t st);
// Batched pack: n packs whose arguments (cpc set explicitly, same dtype) are in
// host_tab (for the grid) and, identically, in the device table dev_tab.
bool pack_rows_fits(const PackArgs &a);
cudaError_t launch_pack_table(const PackArgs *host_tab, const PackArgs *dev_tab, int n, cudaStream_t st);

// blocked tensor (cpc channels per chunk) -> planar float32 [C][H][W]
// (first C channels; value*scale).
cudaError_t launch_unpack(const void *src, int dt, int cpad, int cpc, int C, int H, int W, float scale,
                          float *dst, int64_t dst_pitch, cudaStream_t st);

// Convolution layer (3x3 or 1x1, stride 1, zero padding) on blocked tensors.
struct ConvArgs {
    const void *x;           // blocked input [cin_pad/cpc][H][W][cpc] per image
    int cin_pad;
    int in_cpc, out_cpc;     // channels per chunk of x and of y/res (0 = 16-byte units)
    int H, W;
    int nimg;                // images stacked along the outer dimension
    const void *w;           // prepared weights (kernel-specific layout)
    const void *w_rows;      // 3x3 with 64 input channels: weights for the row-streaming kernel (64 outputs,
                             // or <= 16 outputs shuffled into planar float32), or null
    const float *bias;       // [cout_pad] float32 (zero past cout)
    int cout, cout_pad, k;
    int act;                 // 0 none, 1 LeakyReLU(0.1)
    const void *res;         // blocked residual, same layout/dtype as y, or nullptr
    void *y;                 // blocked output [cout_pad/cpc][H][W][cpc]
    int in_dt, out_dt;       // dtypes of x and of y/res
    float acc_scale;         // multiplies the accumulator (FP8 dequant), 1 otherwise
    float out_scale;         // multiplies the stored value (FP8 quant of y), 1 otherwise
    void *y2;                // optional second output (FP8 copy of y), dtype E4M3
    float y2_scale;
    unsigned *amax;          // optional max |y| (float bits) for calibration
    // final layer: PixelShuffle(ps) into planar float32 + skip
    FusedRq rq;              // 2 x 2 shuffle tail (row kernel): requantise in the epilogue instead
    int ps;                  // 0: blocked store; r: pixel shuffle by r
    float *ps_out;           // planar float32 [cout/(r*r)][rH][rW] (final) or null
    int64_t ps_pitch;
    const float *skip_src[2];// planar float32 source frames of the skip (mean)
    int nskip;
    int64_t skip_pitch, skip_plane;
    int skip_mode;           // 0 none, 1 nearest, 2 bilinear
    int skip_scale;          // output size / skip frame size
    int skip_h, skip_w;      // skip frame size
    int ps_act;              // activation applied after the shuffle (blocked ps output)
    // tuple head only: read the tuple's ntup frames (float32 planar [3][H][ring_pitch] ring
    // slots tslot[] of ring) instead of a packed x
    const float *ring;
    int ring_slots, ntup;
    int64_t ring_pitch;
    int tslot[8];
    int *err;                // device error word (tensor-core kernels), may be null
};
cudaError_t launch_conv_simt(const ConvArgs &a, cudaStream_t st);
cudaError_t launch_conv_tc(const ConvArgs &a, cudaStream_t st);

// One image of a batched 64 -> 64 3x3 row-streaming launch: its tensor maps (in
// global memory, 64-byte aligned) and its strips [strip0, strip0 + nstrips).
struct RowProblem {  // aligned as its tensor maps (at least 64 bytes)
    CUtensorMap tmap, ymap, rmap;
    int H, W, xtiles, rps, strip0, nstrips, has_res, pad_;
};
// True when launch_conv_rows_multi takes layers of this shape.
bool rows_kernel_fits(const ConvArgs &a);
// 3x3 16-channel 16-bit head (packed tuple input, or the ring frames when a.ring is set)
bool rows_head_fits(const ConvArgs &a);
// One launch over n problems (same weights, bias, activation and dtypes; each
// its own x / y / res and size).  host_tab and dev_tab hold n RowProblem
// entries; the table is written to host_tab, copied to dev_tab on `st`, and
// must stay unchanged until the launch has run (a captured graph reuses it).
// rps = rows per strip (0 = automatic).  launch = false only fills (and copies) the table.
cudaError_t launch_conv_rows_multi(const ConvArgs *args, int n, RowProblem *host_tab, RowProblem *dev_tab, int rps,
                                   cudaStream_t st, bool copy_table = true, bool launch = true);

// Weight preparation (device buffers allocated by the caller).
// SIMT layout: [cin_pad][k*k][cout_pad] float32.
size_t simt_weight_bytes(int cin_pad, int cout_pad, int k);
void prepare_weights_simt(const float *w_oihw, int cout, int cin, int k, int cin_pad, int cout_pad,
                          float *dst_host);
// Tensor-core layout: canonical no-swizzle K-major core-matrix image per N slice.
size_t tc_weight_bytes(int cin_pad, int cout_pad, int k, int dt);
// sw128: 128-byte-swizzled image in 64-channel K chunks (for inputs stored with
// 64-channel chunks); otherwise the no-swizzle image in 16-byte K chunks.
void prepare_weights_tc(const float *w_oihw, int cout, int cin, int k, int cin_pad, int cout_pad,
                        int dt, float scale, void *dst_host, bool sw128);
int tc_nslice(int cin_pad, int cout_pad, int k, int dt);
// Row-streaming 64 -> 64 3x3 layout: [kx][2 - ky][64 out][128 B swizzled 64 in].
size_t tc_rows_weight_bytes(int npr = 64);
// Row-streaming image of a 3x3 layer from <= 16 input channels to 64:
// [kx][16-byte channel chunk][2 - ky][64 out][8 channels], no swizzle.
size_t tc_rows16_weight_bytes();
void prepare_weights_rows16(const float *w_oihw, int cin, int dt, void *dst_host);
// npr = 16: the PixelShuffle output form (cout <= 16 channels in 16 rows per tap).
void prepare_weights_rows(const float *w_oihw, int dt, void *dst_host, int cout = 64, int npr = 64);
// Row-streaming image of a 3x3 layer from 128 input channels to <= 256 outputs:
// [64-output slice][kx][64-channel chunk][2 - ky][64 out][128 B swizzled].
size_t tc_rows128_weight_bytes(int nslice);
void prepare_weights_rows128(const float *w_oihw, int cout, int dt, void *dst_host);
// 3x3 64 -> 256 layer followed by PixelShuffle(2): 4 row-streaming images of 64
// outputs (tc_rows_weight_bytes() each), image s holding conv channels 4n + s.
void prepare_weights_rows_ps4(const float *w_oihw, int dt, void *dst_host);
// FP8 row-streaming image of a 64 -> 64 3x3 layer (weights x scale, E4M3):
// [kx][16-byte chunk][2 - ky][64 out][16 channels], no swizzle.
size_t tc_rows_f8_weight_bytes();
void prepare_weights_rows_f8(const float *w_oihw, float scale, void *dst_host);

// DCN: x blocked (activation dtype); offsets and mask in one blocked float32
// tensor [om_cpad/4][H][W][4].  Channel order: torchvision's ([0, 18G) = (dy, dx)
// per (group, tap), [18G, 27G) = mask per (group, tap)), or tap-major (for tap
// k a block of 3G channels: (dy, dx) of each group, then each group's mask),
// which puts all of a tap's offsets and masks in 3G/4 adjacent 4-channel
// planes.  Masks are logits when mask_logits, else already in [0,1].
__host__ __device__ inline int dcn_off_channel(int g, int k, int G, bool tap_major) {
    return tap_major ? 3 * G * k + 2 * g : 2 * (g * 9 + k);
}
__host__ __device__ inline int dcn_mask_channel(int g, int k, int G, bool tap_major) {
    return tap_major ? 3 * G * k + 2 * G + g : 18 * G + g * 9 + k;
}
struct DcnArgs {
    const void *x;
    int cin_pad, H, W, groups;
    int x_cpc, y_cpc;        // channels per chunk of x and y (0 = 16-byte units)
    const float *om;
    int om_cpad;
    int om_tap_major;        // channel order of om (tap-major needs an even G)
    int mask_logits;
    const void *w;           // prepared weights (SIMT or TC layout, k = 3)
    const float *bias;
    int cout, cout_pad;
    void *y;
    int in_dt, out_dt;
    float acc_scale, out_scale;
    int *err;
    int starve;              // test drill: the gather loads nothing, the pipeline waits run out
};
cudaError_t launch_dcn_simt(const DcnArgs &a, cudaStream_t st);
cudaError_t launch_dcn_tc(const DcnArgs &a, cudaStream_t st);
// Copies a 16-bit activation from the blocked layout with x_cpc channels per
// chunk into 8-channel planes [cpad/8][H][W][8] (the DCN gather's layout).
cudaError_t launch_dcn_relayout8(const void *x, int cpad, int H, int W, int x_cpc, void *y, cudaStream_t st);

int device_sm_count();
// The driver's tensor-map encoder (cuTensorMapEncodeTiled), or null when it is missing.
PFN_cuTensorMapEncodeTiled_v12000 encode_fn();

// Residual block of a trunk in one launch (csrc/block_tc.cu): c1 = the block's first
// conv (64 -> 64 3x3, LeakyReLU, input x, output h), c2 = its second (64 -> 64 3x3, no
// activation, input h, residual x, output y).  h never reaches device memory: c1.y is not
// written.  fits: shapes, dtypes (BF16 / FP16, unit scales, one image set) and buffers
// allow it (y must not overlap x); launch returns cudaErrorInvalidValue otherwise.
bool res_block_fits(const ConvArgs &c1, const ConvArgs &c2);
cudaError_t launch_res_block(const ConvArgs &c1, const ConvArgs &c2, cudaStream_t st);
// One image of a batched block launch: its tensor maps (x as 130-pixel boxes, x as 128-pixel
// residual tiles, y as 126-pixel tiles; in global memory, 64-byte aligned), its size, and
// its first unit in the launch's (image, column tile, row) sequence.
struct alignas(64) BlockProblem {
    CUtensorMap xmap, rmap, ymap;
    int H, W, ncols, pad_;
    int64_t u0;
};
// One block launch over n images (c1[i], c2[i] as for launch_res_block; the same weights,
// biases and dtype; each its own x / y and size).  host_tab and dev_tab hold n entries; the
// table is written to host_tab, copied to dev_tab on `st` when copy_table, and must stay
// unchanged until the launch has run (a captured graph reuses it).  launch = false only
// fills (and copies) the table.
cudaError_t launch_res_block_multi(const ConvArgs *c1, const ConvArgs *c2, int n, BlockProblem *host_tab,
                                   BlockProblem *dev_tab, cudaStream_t st, bool copy_table, bool launch);

// Feature-pyramid resampling on blocked [C/cpc][H][W][cpc] tensors of dtype dt (x: H x W):
// up = false: 2x2 mean into (H/2) x (W/2) (H, W even); up = true: bilinear x2
// (align_corners = False, edge clamp) into 2H x 2W.
cudaError_t launch_resample2(bool up, int dt, const void *x, int xcpc, void *y, int ycpc, int C, int H, int W,
                             cudaStream_t st);

// Test drill of the calling thread (nvisr_test_starve): when set, the tensor-core
// kernels it launches load no input, so their first pipeline wait runs out.
int test_starve();

// Launches a tensor-core kernel with programmatic stream serialization, so that its CTAs may
// start (barriers, TMEM, weights) while the stream's previous kernel drains; the kernel waits
// (griddepcontrol.wait) for that kernel's completion before it touches activations.  Under
// stream capture the attribute becomes a programmatic edge of the graph.  Such a kernel reads
// nothing before that wait but data no kernel writes (weights and biases uploaded by copies).
template <typename... P, typename... A>
cudaError_t launch_dependent(void (*kern)(P...), dim3 grid, dim3 threads, int smem, cudaStream_t st, A &&...args) {
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = threads;
    cfg.dynamicSmemBytes = (size_t)smem;
    cfg.stream = st;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kern, std::forward<A>(args)...);
}

}  // namespace nvisr
