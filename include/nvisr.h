/*
 * nvisr.h -- C ABI of the GB300 frame-group video enhancement library.
 *
 * The library runs a video enhancement network over a stream of frames the
 * way NNVISR hosts one (arXiv 2308.03121): a filter is created from a network
 * description, the input/output pixel formats and the spatial / temporal
 * scale (Section 3.2, "End User Usage": one function, clip + parameters in,
 * enhanced clip out; scale factors and the Interpolation / Extra frame /
 * Double frame flags of Section 3.1 select the task); frames are pushed with
 * their scene-change property (Section 3.2) and enhanced frames are pulled in
 * presentation order, grouped within scenes by the rules of Section 3.3.
 *
 * Every stage runs in this library's CUDA kernels (sm_103a): ingest (integer
 * planes -> normalised float frame), 3x3 convolutions as implicit GEMM on the
 * tensor cores (BF16 / FP16 / FP8) or on FP32 SIMT lanes, modulated
 * deformable convolution (DCN v2, Section 3.1), and requantisation.
 *
 * Conventions for every call:
 *  - Every function returns an nvisr_status (void destroy calls excepted);
 *    nothing throws across the ABI.  nvisr_last_error(engine) gives a message
 *    for the most recent failure of a call on that engine (or on one of its
 *    filters, batches or servers); nvisr_last_error(NULL) the most recent
 *    failure of any call on this thread.
 *  - "device" pointers are CUDA device pointers of the engine's device;
 *    "host" pointers are ordinary (ideally pinned) host memory.  The caller
 *    owns every buffer it passes and keeps it alive for the call's duration.
 *  - Calls on one engine are not thread safe; use one engine per thread.
 */
#ifndef NVISR_H
#define NVISR_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define NVISR_ABI_VERSION 2

typedef enum nvisr_status {
    NVISR_OK = 0,
    NVISR_AGAIN = 1,             /* pull: no output ready yet; push more input */
    NVISR_FULL = 2,              /* push: ring full; pull first (backpressure) */
    NVISR_EOS = 3,               /* pull: all outputs of a flushed stream were returned */
    NVISR_INVALID_ARG = -1,
    NVISR_UNSUPPORTED_FORMAT = -2,
    NVISR_OUT_OF_MEMORY = -3,
    NVISR_OVER_BUDGET = -4,      /* the engine's HBM budget would be exceeded */
    NVISR_CUDA_ERROR = -5,
    NVISR_DEVICE_TIMEOUT = -6,   /* a bounded device-side wait expired */
    NVISR_BAD_NETWORK = -7,      /* malformed network description or weight blob */
    NVISR_INTERNAL = -8
} nvisr_status;

typedef enum nvisr_subsampling { NVISR_SUB_420 = 0, NVISR_SUB_444 = 1 } nvisr_subsampling;
typedef enum nvisr_range { NVISR_RANGE_LIMITED = 0, NVISR_RANGE_FULL = 1 } nvisr_range;
/* Colour matrix: BT.709, or BT.2020 non-constant luminance (same equations,
 * weights Kr 0.2627 / Kb 0.0593).  No transfer-function change is applied. */
/* Transfer of the coded R'G'B' signal.  NONE: the network sees the coded signal.  PQ
 * (SMPTE ST 2084) and HLG (BT.2100): the network sees linear light; ingest applies the
 * PQ EOTF (1.0 = 10000 cd/m^2) or the inverse HLG OETF after the matrix, requantise clamps
 * to [0, 1] and applies the inverse before it.  Only RGB-domain networks. */
typedef enum nvisr_transfer { NVISR_TRANSFER_NONE = 0, NVISR_TRANSFER_PQ = 1, NVISR_TRANSFER_HLG = 2 } nvisr_transfer;

/* NVISR_MATRIX_RGB: the three planes are R', G', B' (4:4:4 only), each with the luma range
 * equations and no matrix (Section 3.1: RGB I/O); it needs an RGB-domain network. */
typedef enum nvisr_matrix { NVISR_MATRIX_BT709 = 0, NVISR_MATRIX_BT2020 = 1, NVISR_MATRIX_RGB = 2 } nvisr_matrix;
/* Chroma siting of 4:2:0 planes: LEFT = ITU-T H.273 type 0 (co-sited
 * horizontally, between rows vertically), CENTER = type 1, POINT = replicate
 * on upsampling and 2x2 mean on downsampling. */
typedef enum nvisr_chroma_loc {
    NVISR_CHROMA_LEFT = 0, NVISR_CHROMA_CENTER = 1, NVISR_CHROMA_POINT = 2
} nvisr_chroma_loc;
/* Arithmetic of the network's contractions (convolution / DCN).  FP32 runs on
 * the SIMT lanes; the others on tcgen05 tensor cores with FP32 accumulation.
 * FP8 is E4M3 with per-tensor scales. */
typedef enum nvisr_precision {
    NVISR_PREC_FP32 = 0, NVISR_PREC_BF16 = 1, NVISR_PREC_FP16 = 2, NVISR_PREC_FP8 = 3
} nvisr_precision;

/* Integer YUV video format (Section 3.1: YUV / RGB I/O; colour-space aware).
 * Samples of bit_depth <= 8 are uint8, 9..16 are uint16 (low bits). */
typedef struct nvisr_format {
    int32_t width, height;       /* luma size in pixels */
    int32_t bit_depth;           /* 8, 10, 12 or 16 (more than 8: 16-bit samples) */
    int32_t subsampling;         /* nvisr_subsampling */
    int32_t range;               /* nvisr_range */
    int32_t matrix;              /* nvisr_matrix */
    int32_t chroma_loc;          /* nvisr_chroma_loc */
    int32_t transfer;            /* nvisr_transfer */
} nvisr_format;

/* Three planes Y, U (Cb), V (Cr), or R, G, B for NVISR_MATRIX_RGB.  pitch = bytes between rows. */
typedef struct nvisr_planes {
    void *data[3];
    int64_t pitch[3];
    int32_t on_device;           /* 1: device pointers, 0: host pointers */
    int32_t reserved;
} nvisr_planes;

/* Frame flags for nvisr_push. */
#define NVISR_FRAME_SCENE_CUT 1u /* this frame starts a new scene (cut before it) */

typedef struct nvisr_engine_desc {
    int32_t device;              /* CUDA device ordinal */
    int32_t max_filters;         /* 0 = unlimited */
    int64_t hbm_budget_bytes;    /* 0 = no budget beyond the device's memory */
    void *stream;                /* cudaStream_t to run on; NULL = engine creates one */
} nvisr_engine_desc;

typedef struct nvisr_filter_desc {
    const char *network_text;    /* "nvisr-net 1" description, NUL terminated */
    const float *weights;        /* host FP32 weight blob, in description order */
    int64_t weights_count;       /* number of floats in the blob */
    nvisr_format in_fmt;
    nvisr_format out_fmt;        /* width = scale_w x input width, height = scale_h x input height */
    int32_t scale_w, scale_h;    /* horizontal and vertical scale (Section 3.2); must match the
                                  * description's "scale sx [sy]".  Tuple networks: 2 x 2 (SR),
                                  * 1 x 1 (same-size enhancement, e.g. denoise), 1 x 2 or 2 x 1
                                  * (one-axis 2x, e.g. deinterlace); group networks: one scale */
    int32_t precision;           /* nvisr_precision */
    int32_t calib_frames;        /* FP8: frames whose activations set the scales (0 = 4) */
    uint32_t options;            /* NVISR_OPT_* bits (0 = defaults) */
} nvisr_filter_desc;

/* nvisr_filter_desc.options.  By default a tuple network with a 2 x 2
 * PixelShuffle output layer, on the tensor cores, with an RGB-domain network
 * and no transfer function, requantises inside that layer's epilogue (skip,
 * colour matrix, chroma downsampling, rounding and packing) instead of writing
 * float32 R'G'B' for a separate requantise kernel; the codes are the same.
 * NVISR_OPT_UNFUSED_OUTPUT keeps the separate kernel.
 * Likewise each residual block of a BF16 / FP16 trunk on the tensor cores
 * (conv 64 -> 64, LeakyReLU, conv 64 -> 64, + the block input, whose middle
 * tensor no other layer reads) runs as one launch that keeps the middle
 * tensor on chip (nvisr_resblock2d); the results are the same as two
 * launches.  NVISR_OPT_UNFUSED_BLOCKS runs the two layers as two launches.
 * NVISR_OPT_GUARD_BANDS surrounds every device buffer of the filter (ring,
 * staging planes, weights, activations) with two 4 KB guard bands of a known
 * byte pattern, which nvisr_filter_check_guards verifies: a check for kernels
 * that write outside their buffers (a debugging aid; it costs 8 KB per buffer
 * and a copy per check). */
enum { NVISR_OPT_UNFUSED_OUTPUT = 1, NVISR_OPT_UNFUSED_BLOCKS = 2, NVISR_OPT_GUARD_BANDS = 4 };

/* What an output frame is (nvisr_frame_info.kind). */
enum {
    NVISR_OUT_NETWORK = 0,       /* computed by the network */
    NVISR_OUT_PASSTHROUGH = 1    /* an input frame output as it is (Interpolation without Double frame) */
};

typedef struct nvisr_frame_info {
    int64_t index;               /* output frame index (presentation order) */
    int64_t src_first, src_last; /* input frames the output depends on */
    int32_t scene;               /* scene number of the output's source */
    int32_t kind;                /* NVISR_OUT_NETWORK or NVISR_OUT_PASSTHROUGH */
} nvisr_frame_info;

typedef struct nvisr_engine nvisr_engine;
typedef struct nvisr_filter nvisr_filter;

/* ----------------------------------------------------------------------------
 * Engine and filter (Section 3.2: create a filter from network + parameters;
 * frames in, enhanced frames out).
 * ------------------------------------------------------------------------- */

/* Create an engine on one GPU.  Owns the stream (unless given), the device
 * memory of every filter and the HBM budget.  *out receives the handle.
 * Errors: INVALID_ARG (NULL pointers, bad device), CUDA_ERROR. */
nvisr_status nvisr_engine_create(const nvisr_engine_desc *desc, nvisr_engine **out);

/* Destroy the engine and every filter it still owns. NULL is ignored. */
void nvisr_engine_destroy(nvisr_engine *engine);

/* The cudaStream_t the engine's work is enqueued on. */
void *nvisr_engine_stream(nvisr_engine *engine);

/* Device bytes currently held by the engine's filters. */
int64_t nvisr_engine_bytes_in_use(nvisr_engine *engine);

/* Create a filter: parse and check the network description (Section 3.1: the
 * network is consumed through a description of its graph), upload weights
 * converted to the precision's layout, allocate the frame ring and the
 * activations.  Device memory is charged to the engine's budget.
 * Errors: BAD_NETWORK, UNSUPPORTED_FORMAT, INVALID_ARG (scale/format mismatch),
 * OVER_BUDGET, OUT_OF_MEMORY, CUDA_ERROR. */
nvisr_status nvisr_filter_create(nvisr_engine *engine, const nvisr_filter_desc *desc,
                                 nvisr_filter **out);

/* Release a filter's device memory and handle. NULL is ignored. */
void nvisr_filter_destroy(nvisr_filter *filter);

/* Push the next input frame.  Host planes are copied to the device (on the
 * engine's copy stream) before the call returns and may be reused at once;
 * the ingest kernel that converts them into the filter's ring runs in stream
 * order on the engine's stream, as it does for device planes.
 * flags: NVISR_FRAME_SCENE_CUT marks the frame as the first of a new scene
 * (Section 3.2: scene changes arrive as a per-frame property).
 * Returns FULL when the ring holds no free slot (pull first), EOS after flush. */
nvisr_status nvisr_push(nvisr_filter *filter, const nvisr_planes *in, uint32_t flags);

/* Declare the end of the stream: the last scene closes and its tail outputs
 * become available (Section 3.3: the last frame is duplicated as needed). */
nvisr_status nvisr_flush(nvisr_filter *filter);

/* Produce the next output frame in presentation order into the caller's
 * planes (host or device).  Runs the network for the output's frame group if
 * it has not run yet.  Returns AGAIN if the group's input frames are not all
 * known yet, EOS once a flushed stream has returned every output.  For host
 * planes the call returns after the copy completes; while the copy runs (on
 * the engine's copy stream) the next ready output of a filter outside any
 * batch is already computed on the engine's stream.  Device planes are
 * written in stream order.
 * Group networks (Section 3.1 flags, Section 3.3 rules) consume n frames per
 * run and take n (+1 with Extra frame) frames, <= 8; the network computes n
 * outputs per run (2n with Double frame, <= 8).  Runs tile each scene by n;
 * frames past the scene end repeat its last frame; a run whose consumed
 * frames would pass the scene end is moved back to end there when the scene
 * holds n frames.  Every input frame gives 2 outputs with Interpolation or
 * Double frame (doubled frame rate), else 1, each emitted once.  With
 * Interpolation and without Double frame a frame's outputs are the frame
 * itself (kind NVISR_OUT_PASSTHROUGH: its planes copied unchanged when the
 * input and output formats are equal, else converted to the output format by
 * ingest and requantise) then the network output that follows it; such
 * filters need spatial scale 1.  info may be NULL. */
nvisr_status nvisr_pull(nvisr_filter *filter, nvisr_planes *out, nvisr_frame_info *info);

/* Number of outputs the filter can currently pull without more input. */
int64_t nvisr_filter_ready(nvisr_filter *filter);

/* Run every filter of the engine that has ready work, for up to max_outputs
 * outputs in total, leaving the results in their filters' output queues to be
 * pulled later (batched / serving mode).  *produced receives the count. */
nvisr_status nvisr_engine_step(nvisr_engine *engine, int32_t max_outputs, int32_t *produced);

/* Check a network description and blob size without a device (host only):
 * the same parse and validation nvisr_filter_create performs.  Returns OK or
 * BAD_NETWORK (message in nvisr_last_error). */
nvisr_status nvisr_network_check(const char *network_text, int64_t weights_count);

/* Per-kernel timing of a filter's work, recorded with CUDA events on the
 * engine's stream around every launch while enabled.  Kinds: */
enum {
    NVISR_K_INGEST = 0, NVISR_K_PACK = 1, NVISR_K_CONV_HEAD = 2, NVISR_K_CONV_BODY = 3,
    NVISR_K_CONV_TAIL = 4, NVISR_K_REQUANT = 5, NVISR_K_DCN = 6, NVISR_K_CONV_OTHER = 7,
    NVISR_K_RESAMPLE = 8,            /* feature-pyramid pool / up */
    NVISR_K_COUNT = 9
};
typedef struct nvisr_profile {
    double ms[NVISR_K_COUNT];        /* summed device time per kind */
    int64_t launches[NVISR_K_COUNT]; /* launches per kind */
} nvisr_profile;

/* Extract-stage cache of a two-frame group filter (Section 3.1: the extract
 * stage works on one frame, so a frame's features serve every run that takes
 * it): *hits counts frame slots whose features a run found computed by an
 * earlier run, *misses those it computed.  Both 0 for filters without the cache
 * (tuple networks, other group layouts). */
nvisr_status nvisr_filter_cache_stats(nvisr_filter *filter, int64_t *hits, int64_t *misses);

/* enable != 0 starts recording (clearing earlier totals); 0 stops. */
nvisr_status nvisr_filter_profile(nvisr_filter *filter, int32_t enable);
/* Wait for the recorded launches and return their totals since enabling. */
nvisr_status nvisr_filter_profile_read(nvisr_filter *filter, nvisr_profile *out);

const char *nvisr_status_string(nvisr_status status);
/* Message of the most recent failure on `engine` (calls on the engine or on its
 * filters, batches and servers), or, for NULL, of the calling thread's most
 * recent failed call (the only record for calls that take no engine: stage
 * entry points, host-only calls, a failed nvisr_engine_create).  The string is
 * owned by the library and valid until the next failing call of that kind. */
const char *nvisr_last_error(nvisr_engine *engine);

/* ----------------------------------------------------------------------------
 * Stage entry points (each runs one hot-path stage on caller-owned device
 * buffers, on the given cudaStream_t; used for per-stage parity tests).
 * ------------------------------------------------------------------------- */

/* Ingest: integer planes (device) -> R'G'B' float32 planar [3][H][W]
 * (row pitch out_pitch floats, channel stride out_pitch*H).  Range
 * normalisation (limited/full, 8/10 bit), chroma upsampling with the format's
 * siting (edges clamp), BT.709 Y'CbCr -> R'G'B', no clamping (Section 3.1:
 * YUV input converted for an RGB network). */
nvisr_status nvisr_ingest(const nvisr_format *fmt, const nvisr_planes *in, float *out_rgb,
                          int64_t out_pitch, void *stream);

/* Requantise: R'G'B' float32 planar [3][H][W] (row pitch in_pitch floats) ->
 * integer planes (device): BT.709 R'G'B' -> Y'CbCr, chroma downsampling,
 * range scaling, round half to even, clamp to [0, 2^b - 1] (Section 3.1:
 * YUV output). */
nvisr_status nvisr_requant(const nvisr_format *fmt, const float *in_rgb, int64_t in_pitch,
                           nvisr_planes *out, void *stream);

/* Frame-tuple source indices for a clip (Section 3.3: grouping within scenes;
 * sliding window of T frames, edge frames replicated at scene bounds).
 * flags[k] != 0: frame k starts a scene.  out receives nframes*T indices. */
nvisr_status nvisr_tuple_map(const uint8_t *flags, int32_t nframes, int32_t T, int32_t *out);

/* Group-model runs of one scene [s0, s1] (Section 3.1 flags, Section 3.3 rules):
 * runs consuming n frames and taking need = n (+1 with extra) frames;
 * out_inputs receives runs*need indices, out_skip the number of leading
 * consumed frames an earlier run covered and out_count the number the run
 * covers first (the counts add up to the scene's length).  *nruns receives the
 * run count; max_runs bounds the output arrays.  Host only. */
nvisr_status nvisr_group_runs(int32_t s0, int32_t s1, int32_t n, int32_t extra, int32_t max_runs,
                              int32_t *out_inputs, int32_t *out_skip, int32_t *out_count,
                              int32_t *nruns);

/* Every output of a group-network stream of nframes frames, in presentation
 * order, as nvisr_pull describes them after a flush (the filter's own
 * bookkeeping, run without a device): kind[o] (nvisr_frame_info.kind),
 * src_first[o], src_last[o] and net_k[o] (the network output index, -1 for a
 * passed-through frame).  flags[k] != 0: frame k starts a scene.  *nout
 * receives the output count; max_out bounds the arrays.  Host only. */
nvisr_status nvisr_group_outputs(const uint8_t *flags, int32_t nframes, int32_t n, int32_t extra,
                                 int32_t interp, int32_t dbl, int32_t max_out, int32_t *kind,
                                 int32_t *src_first, int32_t *src_last, int32_t *net_k,
                                 int32_t *nout);

/* Frame-store layout of Section 3.3, Figure 1 for a batch of b groups of n+1
 * frames: cell_frame[(n+1)*b] receives, per column-first address, the frame
 * index relative to the batch's first frame (-1 = unused cell); slot_start[n+1]
 * receives each input slot's first address; copy[2] the (src, dst) addresses
 * of the one copy that prepares the next batch in a store reused in place. */
nvisr_status nvisr_fig1_layout(int32_t n, int32_t b, int32_t *cell_frame, int32_t *slot_start,
                               int32_t *copy);

/* ----------------------------------------------------------------------------
 * Batched multi-stream stepping.
 *
 * A batch groups filters of one engine.  Each nvisr_batch_step computes the
 * next output of every member whose output is ready (its input frames have
 * been pushed, its previous output pulled); outputs are then pulled per
 * filter with nvisr_pull.  When the members run the same tuple network (equal
 * description text, weight blob and BF16/FP16 precision) the step shares its
 * launches across them, whatever their frame sizes and pixel formats:
 *  - the tuple packs of all participants run as one launch;
 *  - every 64->64 3x3 layer runs as one row-streaming launch over all
 *    participants' images (a table of per-image tensor maps and strips);
 *    the other layers run per participant;
 *  - the launch sequence of a set of participants is captured once as a CUDA
 *    graph and replayed on later steps with the same set;
 *  - the strip height of the shared launches is chosen per set by timing
 *    candidate heights on the set's first step (autotuner).
 * Other batches (mixed networks, FP32, FP8, group networks) step their
 * members one by one.  Ingest (push) and requantise (pull) stay per filter.
 * Destroy the batch before its filters.  Calls on one batch are not thread
 * safe.  Errors: INVALID_ARG (NULL, filters of another engine, duplicates),
 * CUDA_ERROR, INTERNAL (a member's tuple layout the batched pack cannot take).
 * ------------------------------------------------------------------------- */
typedef struct nvisr_batch nvisr_batch;
nvisr_status nvisr_batch_create(nvisr_engine *engine, nvisr_filter *const *filters, int32_t n,
                                nvisr_batch **out);
/* *produced (may be NULL) receives the number of outputs computed. */
nvisr_status nvisr_batch_step(nvisr_batch *batch, int32_t *produced);
/* Introspection: *shared = 1 when launches are shared, *graphs = CUDA graphs
 * captured so far, *rows_per_strip = the autotuned strip height of the most
 * recent participant set (0 before the first shared step).  Any may be NULL. */
nvisr_status nvisr_batch_info(nvisr_batch *batch, int32_t *shared, int32_t *graphs, int32_t *rows_per_strip);
void nvisr_batch_destroy(nvisr_batch *batch);

/* ----------------------------------------------------------------------------
 * Serving (continuous batching).
 *
 * A server owns the clips submitted to one engine.  A clip is one video
 * stream described like a filter (nvisr_filter_desc; the server copies the
 * description and the weights).  It waits in arrival order until it can be
 * created as a filter: fewer than max_active clips are active (0 = no limit)
 * and the engine's HBM budget holds its ring, activations and weights.  Every
 * nvisr_server_step first admits waiting clips, then steps each group of
 * active clips that run the same network as one batch (nvisr_batch): a clip
 * admitted while others are in flight joins the next step's shared launches.
 * Closing a clip frees its memory and admits waiting clips at once.
 * nvisr_server_push / _flush / _pull are nvisr_push / _flush / _pull on the
 * clip's filter and return AGAIN while the clip is still waiting.  Latency of
 * an output = the time its planes are written (pull of host planes; for device
 * planes the server waits for the engine stream) minus the push time of the
 * newest input frame it depends on; queueing delay = admission minus
 * submission.
 * Errors: INVALID_ARG (NULL, unknown clip), the filter and batch errors.
 * ------------------------------------------------------------------------- */
typedef struct nvisr_server nvisr_server;
typedef struct nvisr_server_stats_t {
    double latency_p50_ms, latency_p99_ms;  /* per output frame */
    double queue_p50_ms, queue_p99_ms;      /* per admitted clip */
    int64_t admitted, pending, active, completed, outputs;
    int64_t deferred_steps;                 /* admission attempts stopped by the HBM budget */
} nvisr_server_stats_t;
nvisr_status nvisr_server_create(nvisr_engine *engine, int32_t max_active, nvisr_server **out);
nvisr_status nvisr_server_submit(nvisr_server *server, const nvisr_filter_desc *desc, int64_t *clip);
nvisr_status nvisr_server_push(nvisr_server *server, int64_t clip, const nvisr_planes *in, uint32_t flags);
nvisr_status nvisr_server_flush(nvisr_server *server, int64_t clip);
/* *produced (may be NULL): outputs computed by this step over all clips. */
nvisr_status nvisr_server_step(nvisr_server *server, int32_t *produced);
nvisr_status nvisr_server_pull(nvisr_server *server, int64_t clip, nvisr_planes *out, nvisr_frame_info *info);
nvisr_status nvisr_server_close(nvisr_server *server, int64_t clip);
nvisr_status nvisr_server_stats(nvisr_server *server, nvisr_server_stats_t *out);
void nvisr_server_destroy(nvisr_server *server);

/* One 2-D convolution layer (Section 3.1 networks) on planar float32 tensors:
 * y[cout][H][W] = act(conv_k(x[cin][H][W]; w[cout][cin][k][k]) + b) (+ res),
 * stride 1, zero padding (k-1)/2, act 0 = none, 1 = LeakyReLU(0.1).  Runs the
 * precision's kernel (FP32 SIMT or tensor cores); the library converts x to
 * its internal layout in scratch device memory it allocates per call.
 * res may be NULL.  All pointers are device pointers. */
nvisr_status nvisr_conv2d(int32_t precision, const float *x, int32_t cin, int32_t h, int32_t w,
                          const float *weight, const float *bias, int32_t cout, int32_t k,
                          int32_t act, const float *res, float *y, void *stream);

/* Size of the fixed device area behind nvisr_conv2d_static (32 MiB per device). */
#define NVISR_CONV2D_STATIC_SCRATCH_BYTES (32 * 1024 * 1024)

/* nvisr_conv2d without any allocation.  The paper has no counterpart: this is
 * a library convenience for callers that must not allocate while they run
 * (device memory handed out in advance, or real-time work that cannot let
 * cudaFree synchronise the device).  Same arguments, results and error codes
 * as nvisr_conv2d, except:
 *  - every working buffer (blocked x, y and res, weight image, bias, error
 *    word) is carved from one static device array of
 *    NVISR_CONV2D_STATIC_SCRATCH_BYTES per device, set aside when the module
 *    loads; weights are laid out by device kernels, so nothing is staged on
 *    the host.  A problem that does not fit returns NVISR_OVER_BUDGET before
 *    any device work.  Need: (cin_pad + cout_pad * (res ? 2 : 1)) * H * W
 *    element bytes plus the weight image; 64 -> 64 channels with a residual
 *    fit ~43k pixels in FP32 and ~87k in BF16 / FP16;
 *  - precision is FP32, BF16 or FP16 (FP8 returns NVISR_UNSUPPORTED_FORMAT, an
 *    unknown precision NVISR_INVALID_ARG);
 *  - the area is shared by every call on a device, and keeps what the last
 *    call left in it (each call clears what must start at zero): calls that
 *    overlap in time on one device (several threads or streams) race and must
 *    be serialised by the caller;
 *  - the first call on each device (and again after the device's context is
 *    re-created, e.g. by cudaDeviceReset), made with that device current,
 *    looks up the area's address; make that first call before any stream
 *    capture.
 * Returns after synchronising `stream`: it reads the error word back. */
nvisr_status nvisr_conv2d_static(int32_t precision, const float *x, int32_t cin, int32_t h, int32_t w,
                                 const float *weight, const float *bias, int32_t cout, int32_t k,
                                 int32_t act, const float *res, float *y, void *stream);

/* Residual block of a trunk (Section 3.1: the networks are stacks of 3x3
 * convolutions with residual connections): y = x + conv2(LeakyReLU(conv1(x)
 * + b1)) + b2, both convs 64 -> 64 channels, 3x3, stride 1, zero padding 1,
 * LeakyReLU slope 0.1.  x, y: planar float32 [64][h][w]; w1, w2: [64][64][3][3]
 * (out, in, ky, kx); b1, b2: [64] or NULL (zero).  All pointers are device
 * pointers; y must not overlap x.  precision: BF16 or FP16 (activations and
 * operands in that type, FP32 accumulation; others return
 * NVISR_UNSUPPORTED_FORMAT).  fused != 0: one launch of 2-CTA clusters in
 * which one SM computes conv1 and writes its rows into the other SM's shared
 * memory, where conv2 reads them (the middle tensor never reaches device
 * memory); fused == 0: two launches of the single-layer row kernel.  Both
 * give the same values.  Scratch is allocated per call; returns after
 * synchronising `stream` (it reads the error word back: NVISR_DEVICE_TIMEOUT
 * if a device-side wait ran out). */
nvisr_status nvisr_resblock2d(int32_t precision, const float *x, int32_t h, int32_t w, const float *w1,
                              const float *b1, const float *w2, const float *b2, float *y, int32_t fused,
                              void *stream);

/* Modulated deformable convolution 3x3, DCN v2 as in torchvision's
 * deform_conv2d (Section 3.1): offsets [2*G*9][H][W] (dy, dx per group and
 * tap), mask [G*9][H][W] (already in [0,1]), stride 1, padding 1.  Planar
 * float32 device tensors; scratch allocated per call.  x must be finite: the
 * tensor-core gather skips the loads of corners whose bilinear weight is zero
 * (outside the image), and a skipped corner contributes weight x an earlier
 * sample, which is zero only for a finite sample. */
nvisr_status nvisr_dcn2d(int32_t precision, const float *x, int32_t cin, int32_t h, int32_t w,
                         const float *offsets, const float *mask, int32_t groups,
                         const float *weight, const float *bias, int32_t cout, float *y,
                         void *stream);

/* Checks the guard bands of a filter created with NVISR_OPT_GUARD_BANDS (no
 * counterpart in the paper).  Waits for the engine's streams, then reads every
 * band back: OK when all hold their pattern; otherwise NVISR_CUDA_ERROR, with
 * *bad = the number of buffers whose bands were overwritten and the first
 * such byte named in nvisr_last_error.  NVISR_INVALID_ARG for a filter
 * without guard bands. */
nvisr_status nvisr_filter_check_guards(nvisr_filter *f, int32_t *bad);

/* Test of the guard-band check (no counterpart in the paper): writes one byte
 * from the host (cudaMemset) into the band after the index-th guarded buffer
 * of the filter, so that the next nvisr_filter_check_guards reports it.
 * Allocated memory only; NVISR_INVALID_ARG for an index past the buffers. */
nvisr_status nvisr_test_poke_guard(nvisr_filter *f, int32_t index);

/* Fault drill for tests of the NVISR_DEVICE_TIMEOUT path (no counterpart in
 * the paper).  While on (on != 0), the tensor-core kernels (convolutions and
 * DCN) launched by the calling thread load no input, so their first pipeline
 * wait runs out after its time bound (2 s): the CTA raises its abort flag,
 * records the timeout in the engine's error word, lets its own copies and MMAs
 * finish, frees its TMEM and returns, and the call that reads the error word
 * returns NVISR_DEVICE_TIMEOUT.  Outputs of such calls are undefined.  0 turns
 * the drill off; later calls run normally.  Host only; always returns OK. */
nvisr_status nvisr_test_starve(int32_t on);

/* Tensor-core self test: one 128x16 MMA of BF16 (K = 16) and one of FP8 E4M3
 * (K = 32) small-integer operands through shared-memory descriptors, TMEM
 * and tcgen05.ld, compared with the exact products.  *mismatches_* receive
 * the number of wrong accumulator elements (0 = the descriptor conventions
 * hold).  Runs on the current device; allocates and frees a few bytes. */
nvisr_status nvisr_selftest(int32_t *mismatches_bf16, int32_t *mismatches_fp8);

/* Probe of the 128-byte-swizzled K-major operand convention the tensor-core
 * kernels rely on: an MMA chain reading A from row offsets 0..7 inside a
 * swizzle atom, with descriptor base offset 0 (out16[0..7]) and with base
 * offset (start >> 7) & 7 (out16[8..15]); each entry counts wrong accumulator
 * elements (0 = that convention reproduces the stored rows). */
nvisr_status nvisr_selftest_swizzle(int32_t *out16);

/* Library version / build information. */
int32_t nvisr_abi_version(void);
const char *nvisr_build_info(void);

#ifdef __cplusplus
}
#endif

#endif /* NVISR_H */
