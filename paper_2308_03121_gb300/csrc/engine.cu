// Engine, filter and C-ABI implementation.
//
// A filter follows the paper's statement of the problem (Section 3.2: one
// call, clip + parameters -> enhanced clip) as a push/pull stream:
//   push(frame, scene flag) -> H2D copy into the device ring -> ingest kernel
//   pull() -> group formation (Section 3.3: within scenes, edge frames
//             replicated) -> network forward (pack, conv / DCN layers) ->
//             requantise -> copy to the caller.
// The ring holds each input frame once as planar float32 R'G'B'; a frame
// tuple is a list of ring slots, so grouping copies no pixels.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <vector>

#include "common.cuh"
#include "netdesc.h"

namespace nvisr {

int tc_selftest(int kind, int *dev_mismatch, cudaStream_t st);
int tc_probe_sw128(int *dev_out16, cudaStream_t st);

// ---------------------------------------------------------------- errors

static thread_local std::string g_last_error;
static thread_local nvisr_engine *g_err_engine = nullptr;  // engine of the ABI call in progress
static thread_local int g_test_starve = 0;

int test_starve() { return g_test_starve; }

ErrScope::ErrScope(nvisr_engine *e) : prev(g_err_engine) { g_err_engine = e; }
ErrScope::~ErrScope() { g_err_engine = prev; }

nvisr_status cuda_status(cudaError_t e, const char *where) {
    set_error(std::string(where) + ": " + cudaGetErrorString(e));
    if (e == cudaErrorMemoryAllocation) return NVISR_OUT_OF_MEMORY;
    if (e == cudaErrorNotSupported) return NVISR_UNSUPPORTED_FORMAT;
    return NVISR_CUDA_ERROR;
}

static nvisr_status fail(nvisr_status s, const std::string &msg) {
    set_error(msg);
    return s;
}

int device_sm_count() {
    static int cache[64] = {0};
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 0 || dev >= 64) return 148;
    if (!cache[dev]) {
        int n = 0;
        cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
        cache[dev] = n > 0 ? n : 148;
    }
    return cache[dev];
}

}  // namespace nvisr

using namespace nvisr;

// ---------------------------------------------------------------- handles

struct nvisr_engine {
    int device = 0;
    int max_filters = 0;
    int64_t budget = 0;
    int64_t used = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    cudaStream_t copy_stream = nullptr;  // host <-> device copies of push / pull, beside the compute stream
    int *err_word = nullptr;  // device error word shared by this engine's kernels
    int *err_host = nullptr;  // pinned host copy of it, read after a pull's copies
    std::vector<nvisr_filter *> filters;
    std::string last_error;  // message of the most recent failure of a call on this engine
};

namespace nvisr {
// The message goes to the calling thread and, inside an ABI call on an engine
// (or one of its filters, batches or servers), to that engine too.
void set_error(const std::string &msg) {
    g_last_error = msg;
    if (g_err_engine) g_err_engine->last_error = msg;
}
}  // namespace nvisr

namespace {

struct DevBuf {
    nvisr_engine *eng = nullptr;
    void *ptr = nullptr;   // the allocation (freed with cudaFree)
    size_t bytes = 0;      // its size
    size_t guard = 0;      // guard band bytes before and after the buffer (0 = none)
    size_t user = 0;       // the buffer's requested size, between the two bands
};

constexpr size_t GUARD_BYTES = 4096;      // NVISR_OPT_GUARD_BANDS: each band's size
constexpr unsigned char GUARD_FILL = 0xA5;

// Device allocation counted against the engine's budget.  guard > 0 surrounds
// the buffer (the requested `bytes`, not rounded) with two bands of that size
// filled with GUARD_FILL, for nvisr_filter_check_guards.
nvisr_status dalloc(nvisr_engine *e, size_t bytes, std::vector<DevBuf> &owned, void **out, size_t guard = 0) {
    const size_t user = bytes;
    bytes = (size_t)round_up64((int64_t)std::max<size_t>(bytes + 2 * guard, 256), 256);
    if (e->budget > 0 && e->used + (int64_t)bytes > e->budget)
        return fail(NVISR_OVER_BUDGET, "HBM budget exceeded: need " + std::to_string(bytes) + " more bytes, " +
                                           std::to_string(e->budget - e->used) + " left");
    void *p = nullptr;
    cudaError_t ce = cudaMalloc(&p, bytes);
    if (ce != cudaSuccess) {
        cudaGetLastError();
        return fail(NVISR_OUT_OF_MEMORY, std::string("cudaMalloc: ") + cudaGetErrorString(ce));
    }
    if (guard) {
        uint8_t *b = static_cast<uint8_t *>(p);
        if ((ce = cudaMemset(b, GUARD_FILL, guard)) != cudaSuccess ||
            (ce = cudaMemset(b + guard + user, GUARD_FILL, bytes - guard - user)) != cudaSuccess) {
            cudaFree(p);
            return fail(NVISR_CUDA_ERROR, std::string("guard bands: ") + cudaGetErrorString(ce));
        }
    }
    e->used += (int64_t)bytes;
    owned.push_back({e, p, bytes, guard, user});
    *out = static_cast<uint8_t *>(p) + guard;
    return NVISR_OK;
}

struct Tensor {
    void *ptr = nullptr;
    int C = 0, cpad = 0, H = 0, W = 0, dt = DT_F32;
    void *f8 = nullptr;  // FP8 copy (when an FP8 layer consumes this tensor)
    int amax_slot = -1;  // calibration slot of the FP8 values
    int parent = -1;     // channel view of a concatenation buffer (tensor id)
    int choff = 0;       // first channel inside the parent
    int cpc = 0;         // channels per chunk of the blocked layout (layout_cpc)
};

struct Weights {
    void *rows = nullptr;        // row-streaming 64->64 3x3 layout (tensor-core path)
    void *simt_or_tc = nullptr;  // 16-bit / FP32 layout
    void *f8 = nullptr;          // FP8 layout
    void *rows_f8 = nullptr;     // FP8 row-streaming layout (64 -> 64 3x3)
    float *bias = nullptr;
    int cin_pad = 0, cout_pad = 0;
    float w_amax = 0.f;
};

enum Src { SRC_TENSOR = 0, SRC_TUPLE = 1 };

enum Op { OP_CONV = 0, OP_DCN = 1, OP_PACK = 2, OP_POOL = 3, OP_UP = 4 };

struct Step {
    int op = OP_CONV;
    int layer = 0;
    int widx = -1;       // weights variant (input channels permuted), -1 = the layer's own
    int om_t = -1;       // DCN: offsets/mask tensor
    bool om_tap_major = false;  // DCN: om channels in tap-major order (its head's rows permuted)
    std::vector<int> skip_frames;  // final outputs: frames whose upsampled mean is added
    int in_t = -1;       // input tensor id (SRC_TENSOR)
    int src = SRC_TENSOR;
    int frame_src = -1;  // group family: input from ring frame k
    std::vector<int> perm;  // group family: input channel c of the layer is stored channel perm[c]
    // extract cache: the frame slot whose features this step computes (-1: none), and for a
    // reader of a cached pair the weights variant per pair order (frame slot 0's part first, or
    // frame slot 1's part first)
    int xslot = -1;
    int xpair_w[2] = {-2, -2};
    int add_t = -1;
    int out_t = -1;      // -1: final output (PixelShuffle into planar float32)
    int out_index = -1;  // final output number
    bool fp8 = false;
    bool out_f8_only = false;
    // final output without the 2x2 shuffle (scale 1, or 1 x 2 / 2 x 1): the conv writes
    // float32 into final_f32, then a shuffle kernel writes the planar output
    bool plain = false;
    int psy = 2, psx = 2;
};

bool fmt_ok(const nvisr_format &f) {
    return f.width > 0 && f.height > 0 &&
           (f.bit_depth == 8 || f.bit_depth == 10 || f.bit_depth == 12 || f.bit_depth == 16) &&
           (f.subsampling == NVISR_SUB_420 || f.subsampling == NVISR_SUB_444) &&
           (f.range == NVISR_RANGE_LIMITED || f.range == NVISR_RANGE_FULL) &&
           (f.matrix == NVISR_MATRIX_BT709 || f.matrix == NVISR_MATRIX_BT2020 ||
            (f.matrix == NVISR_MATRIX_RGB && f.subsampling == NVISR_SUB_444)) &&
           (f.transfer == NVISR_TRANSFER_NONE || f.transfer == NVISR_TRANSFER_PQ || f.transfer == NVISR_TRANSFER_HLG) &&
           f.chroma_loc >= 0 && f.chroma_loc <= 2 &&
           (f.subsampling == NVISR_SUB_444 || (f.width % 2 == 0 && f.height % 2 == 0));
}

int64_t plane_bytes(const nvisr_format &f, int plane, int64_t *pitch, int *h) {
    const int esz = f.bit_depth > 8 ? 2 : 1;
    const bool sub = plane > 0 && f.subsampling == NVISR_SUB_420;
    const int w = sub ? f.width / 2 : f.width;
    *h = sub ? f.height / 2 : f.height;
    *pitch = round_up64((int64_t)w * esz, 256);
    return *pitch * *h;
}

int64_t plane_row_bytes(const nvisr_format &f, int plane) {
    const int esz = f.bit_depth > 8 ? 2 : 1;
    const bool sub = plane > 0 && f.subsampling == NVISR_SUB_420;
    return (int64_t)(sub ? f.width / 2 : f.width) * esz;
}

int plane_rows(const nvisr_format &f, int plane) {
    return (plane > 0 && f.subsampling == NVISR_SUB_420) ? f.height / 2 : f.height;
}

}  // namespace

struct nvisr_filter {
    nvisr_engine *eng = nullptr;
    NetDesc net;
    std::string net_text;          // the description and a hash of the weight blob: filters with
    uint64_t blob_hash = 0;        // equal text, blob and precision may share batched launches
    int64_t blob_count = 0;
    nvisr_format in_fmt{}, out_fmt{};
    int precision = NVISR_PREC_FP32;
    int act_dt = DT_F32;  // 16-bit / FP32 activation dtype
    bool tc = false;      // tensor-core kernels
    std::vector<DevBuf> owned;
    size_t guard = 0;  // NVISR_OPT_GUARD_BANDS: guard band bytes around each buffer

    // ring of ingested frames (planar float32 [3][H][pitch])
    int ring = 0;
    int64_t rpitch = 0;   // floats
    float *ring_base = nullptr;
    int64_t slot_floats = 0;
    void *stage[3] = {nullptr, nullptr, nullptr};
    int64_t stage_pitch[3] = {0, 0, 0};

    // stream bookkeeping
    int64_t pushed = 0;
    bool eos = false;
    std::vector<uint8_t> cut;      // per pushed frame: starts a scene
    int64_t next_out = 0;          // next output index to return
    int64_t total_out = -1;        // known after flush

    // network plan
    std::vector<Weights> wvar;     // weights with permuted input channels (concatenations)
    std::vector<Weights> weights;  // per layer (shared layers point to the owner)
    std::vector<int> om_tap_g;     // per layer: G when its output rows are stored tap-major, else 0
    std::vector<Tensor> tensors;
    void *dcn_x8 = nullptr;        // DCN input in 8-channel planes (tensor-core path)
    std::vector<Step> steps;
    std::vector<char> blk;           // step i and i + 1 form a residual block run as one fused launch
    int pack_t = -1;               // tensor id of the packed tuple
    int tuple_head = -1;           // the step that alone reads the packed tuple (-1: several or none)
    bool plain_final = false;      // some output uses a plain final layer (Step::plain)
    float *final_f32 = nullptr;    // its float32 output, blocked [4][H][W][4]
    float *out_rgb[8] = {};   // planar float32 residuals [3][sH][opitch], one per output of a run
    SkipArgs skip[8] = {};    // skip path of each output slot (added by requantise)
    // group family (Section 3.1): n frames per run (+1 with Extra frame), run_out network
    // outputs per run
    int grp_n = 1, grp_need = 1, run_out = 1;
    // Interpolation without Double frame: input frames are outputs too.  With equal input and
    // output formats they are copied unchanged from raw[] (the pushed planes, one ring slot
    // per frame, written on the compute stream); otherwise requantise converts the ring slot.
    bool passthru = false;
    bool pass_copy = false;
    void *raw[3] = {nullptr, nullptr, nullptr};
    int64_t raw_slot_bytes[3] = {0, 0, 0};
    int64_t opitch = 0;
    void *ostage[2][3] = {{nullptr, nullptr, nullptr}, {nullptr, nullptr, nullptr}};  // alternate per pull
    int64_t ostage_pitch[3] = {0, 0, 0};
    // output o is written into staging buffer o & 1 (requantised by the output layer itself
    // when fused_rq is set: rq_done[b] is then the output staging buffer b holds, else -1)
    bool fused_rq = false;
    FusedRq rq_base{};
    float *rq_edge = nullptr;
    int64_t rq_o = -1;             // the output the next forward computes (tuple family)
    int64_t rq_done[2] = {-1, -1};
    const nvisr_planes *rq_direct = nullptr;  // the caller's device planes, when a pull computes its own output
    int64_t rq_direct_done = -1;             // the output last requantised straight into them
    uint32_t options = 0;

    // host-plane copies on the engine's copy stream: the H2D of a push and the
    // D2H of a pull overlap the compute stream's work; a pull of host planes
    // also starts the next ready output (read-ahead), unless the filter has
    // joined a batch (whose step computes its outputs)
    cudaEvent_t ev_h2d = nullptr, ev_stage = nullptr, ev_req = nullptr, ev_d2h = nullptr;
    bool stage_used = false;
    bool batched = false;

    // group family: run cache (outputs of the last run)
    int64_t cached_run = -1;

    // extract cache (Section 3.1: the extract stage works on one frame): a two-frame group
    // network whose per-frame features feed channel concatenations of the two frames keeps
    // those concatenation buffers across runs.  Half h of every such buffer holds the
    // features of frame xc_tag[h]; a run computes only the frames no half holds.
    bool xcache = false;
    int64_t xc_tag[2] = {-1, -1};
    struct XPair { int parent; int part[2]; };  // part[k]: tensor of frame slot k's features
    std::vector<XPair> xpairs;
    int64_t xc_hits = 0, xc_misses = 0;

    // FP8 calibration
    bool calibrated = false;
    int calib_frames = 4;
    unsigned *amax = nullptr;      // device [n slots]
    int n_amax = 0;
    std::vector<float> act_scale;  // per amax slot

    // host-side queue of produced-but-not-pulled outputs (engine_step)
    std::deque<int64_t> produced;

    // per-kernel timing (nvisr_filter_profile)
    bool prof = false;
    struct Rec { int kind; cudaEvent_t a, b; int n; };  // n launches of one kind, back to back
    std::vector<Rec> recs;
    bool prof_join = false;  // the next scope of the last record's kind may extend it
    bool prof_hold = false;  // set by the step loops: the next launch is of the same kind
    bool prof_open = false;  // the last record's end event is not recorded yet
    std::vector<cudaEvent_t> ev_pool;
    double prof_ms[NVISR_K_COUNT] = {0};
    int64_t prof_n[NVISR_K_COUNT] = {0};
};

namespace {

cudaEvent_t take_event(nvisr_filter *f) {
    if (!f->ev_pool.empty()) {
        cudaEvent_t e = f->ev_pool.back();
        f->ev_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}

// Records the end event a run of same-kind launches left pending.
void prof_close(nvisr_filter *f) {
    if (!f->prof_open) return;
    cudaEventRecord(f->recs.back().b, f->eng->stream);
    f->prof_open = false;
}

void flush_profile(nvisr_filter *f) {
    prof_close(f);
    if (f->recs.empty()) return;
    cudaStreamSynchronize(f->eng->stream);
    for (auto &r : f->recs) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, r.a, r.b) == cudaSuccess) {
            f->prof_ms[r.kind] += ms;
            f->prof_n[r.kind] += r.n;
        }
        f->ev_pool.push_back(r.a);
        f->ev_pool.push_back(r.b);
    }
    f->recs.clear();
    f->prof_join = false;
}

// Records CUDA events around the launches issued during its lifetime.  Back-to-back
// scopes of one kind (a trunk's 20 body layers) share one event pair: while the step
// loop says the next launch is of the same kind (prof_hold) the end event waits, so no
// event separates two such launches and a launch may overlap its predecessor's drain
// (programmatic dependent launch).
struct ProfScope {
    nvisr_filter *f;
    int kind;
    int launches = 1;  // kernels this scope's call launched
    cudaEvent_t a = nullptr;
    bool join = false;
    ProfScope(nvisr_filter *f_, int kind_) : f(f_), kind(kind_) {
        if (!f->prof) {
            prof_close(f);
            return;
        }
        join = f->prof_join && !f->recs.empty() && f->recs.back().kind == kind;
        if (!join) {
            prof_close(f);
            a = take_event(f);
            cudaEventRecord(a, f->eng->stream);
        }
    }
    ~ProfScope() {
        if (join) {
            f->recs.back().n += launches;
        } else {
            if (!a) return;
            f->recs.push_back({kind, a, take_event(f), launches});
            f->prof_join = true;
        }
        f->prof_open = true;
        if (!f->prof_hold) prof_close(f);
        if (f->recs.size() > 4096 && !f->prof_open) flush_profile(f);
    }
};

// Stream work outside a ProfScope: the next scope starts a record of its own.
void prof_gap(nvisr_filter *f) {
    prof_close(f);
    f->prof_join = false;
}

float *ring_slot(nvisr_filter *f, int64_t frame) {
    return f->ring_base + (frame % f->ring) * f->slot_floats;
}

// Scene bounds of frame t among the known frames: s0 = last cut <= t,
// s1 = (first cut > t) - 1, or the last known frame; *closed says whether s1
// is final (a later cut is known, or the stream ended).
void scene_bounds(const nvisr_filter *f, int64_t t, int64_t *s0, int64_t *s1, bool *closed) {
    int64_t a = t;
    while (a > 0 && !f->cut[(size_t)a]) --a;
    *s0 = a;
    int64_t b = t + 1;
    while (b < f->pushed && !f->cut[(size_t)b]) ++b;
    *s1 = b - 1;
    *closed = (b < f->pushed) || f->eos;
}

// Tuple family: is output t computable, and with which source frames?
bool tuple_ready(const nvisr_filter *f, int64_t t, std::vector<int64_t> *idx) {
    if (t >= f->pushed) return false;
    const int T = f->net.frames, r = (T - 1) / 2;
    int64_t s0, s1;
    bool closed;
    scene_bounds(f, t, &s0, &s1, &closed);
    if (!closed && s1 < t + r) return false;
    if (idx) {
        idx->resize(T);
        for (int k = 0; k < T; ++k) (*idx)[k] = std::min(std::max(t - r + k, s0), s1);
    }
    return true;
}

// Group family: where output o comes from.  Scenes are cut by the per-frame
// flags; a scene [s0, s1] is covered by runs at nominal starts s0, s0 + n, ...,
// each consuming n frames and taking need = n (+1 with Extra frame) frames,
// indices past s1 taking s1 (Section 3.3: the interpolation network's last
// frame duplicated, a short scene duplicated further).  A run whose consumed
// frames would pass s1 is moved back to end at s1 when the scene holds n
// frames (recycling frames of the previous group).  Each consumed frame gives
// its outputs once: q = 2 of them with Interpolation (doubled frame rate) or
// Double frame, else 1; the outputs of frames an earlier run covered, and of
// duplicated frames past s1, are not emitted.  With Interpolation and without
// Double frame a frame's two outputs are the frame itself, passed through,
// then the network output that is its intermediate frame (Section 3.1).  A run
// is known once its frames are pushed inside its scene, or once the scene is
// closed (a later cut is known or the stream ended).
struct RunLoc {
    int64_t key = -1;             // nominal start frame (unique per run)
    int64_t oldest = 0;           // earliest frame the run may read (its start once known)
    std::vector<int64_t> inputs;  // the run's input frames (known runs)
    int k = 0;                    // network output index (pass = false)
    bool pass = false;            // o is input frame `frame` passed through
    int64_t frame = -1;
};

// Form of the run at `nominal` in scene [s0, s1]: its first frame, the number
// of leading consumed frames an earlier run covered, and the number it covers first.
void run_form(int64_t nominal, int64_t s0, int64_t s1, int n, int64_t *start, int *skip, int *count) {
    int64_t st = nominal;
    if (st + n - 1 > s1 && s1 - s0 + 1 >= n) st = s1 - n + 1;
    *start = st;
    *skip = (int)(nominal - st);
    *count = (int)(std::min<int64_t>(st + n - 1, s1) - nominal + 1);
}

// Outputs per consumed frame.
int group_q(const nvisr_filter *f) { return (f->net.interp || f->net.dbl) ? 2 : 1; }

// True when output o's run is known (and then *loc describes it); false with
// loc->oldest set to a lower bound of the frames that run will read.
bool group_locate(const nvisr_filter *f, int64_t o, RunLoc *loc) {
    const int n = f->grp_n, need = f->grp_need, q = group_q(f);
    const bool pass = f->net.interp && !f->net.dbl;
    int64_t base = 0, s0 = 0;
    loc->oldest = 0;
    while (s0 < f->pushed) {
        int64_t s1 = s0;
        while (s1 + 1 < f->pushed && !f->cut[(size_t)(s1 + 1)]) ++s1;
        const bool closed = s1 + 1 < f->pushed || f->eos;
        for (int64_t nominal = s0; nominal <= s1; nominal += n) {
            if (nominal + need - 1 > s1 && !closed) {
                // the run's frames are not all pushed and its form is not final yet
                loc->oldest = std::max<int64_t>(s0, nominal - n + 1);
                return false;
            }
            int64_t start;
            int skip, count;
            run_form(nominal, s0, s1, n, &start, &skip, &count);
            if (o < base + (int64_t)q * count) {
                const int j = q * skip + (int)(o - base);  // entry among the run's q * n
                loc->key = nominal;
                loc->oldest = start;
                loc->inputs.clear();
                for (int k = 0; k < need; ++k) loc->inputs.push_back(std::min(start + k, s1));
                loc->pass = pass && j % 2 == 0;
                loc->frame = loc->pass ? start + j / 2 : -1;
                loc->k = pass ? j / 2 : j;
                return true;
            }
            base += (int64_t)q * count;
        }
        s0 = s1 + 1;
    }
    loc->oldest = f->pushed;
    return false;
}

// Output count of a group-family stream once it has ended: every frame gives q.
int64_t group_total(const nvisr_filter *f) { return (int64_t)group_q(f) * f->pushed; }

bool group_ready(const nvisr_filter *f, int64_t o, RunLoc *loc) {
    RunLoc tmp;
    return group_locate(f, o, loc ? loc : &tmp);
}

// FP8 filters calibrate their activation scales on the first calib_frames
// outputs' tuples, so nothing is ready before those tuples are all known.
bool calibration_ready(const nvisr_filter *f) {
    if (f->precision != NVISR_PREC_FP8 || f->calibrated || f->n_amax == 0) return true;
    const int64_t n = f->eos ? std::min<int64_t>(f->calib_frames, f->pushed) : f->calib_frames;
    for (int64_t t = 0; t < n; ++t)
        if (!tuple_ready(f, t, nullptr)) return false;
    return true;
}

bool output_ready(const nvisr_filter *f, int64_t o) {
    if (f->net.family == "group") return group_ready(f, o, nullptr);
    return tuple_ready(f, o, nullptr) && calibration_ready(f);
}

// ---------------------------------------------------------------- plan

int act_cpad(const nvisr_filter *f, int C) {
    return f->tc ? round_up(C, 16) : round_up(C, 8);
}

nvisr_status upload(nvisr_filter *f, const void *host, size_t bytes, void **dev) {
    nvisr_status s = dalloc(f->eng, bytes, f->owned, dev, f->guard);
    if (s != NVISR_OK) return s;
    NVISR_TRY_CUDA(cudaMemcpy(*dev, host, bytes, cudaMemcpyHostToDevice));
    return NVISR_OK;
}

bool layer_is_fp8(const nvisr_filter *f, const NetLayer &L) {
    return f->precision == NVISR_PREC_FP8 && L.op == "conv" && L.k == 3 && L.cin == 64 && L.cout == 64 &&
           L.ps == 0 && L.in.size() == 1 && L.in[0] != "tuple" && L.in[0].rfind("frame", 0) != 0;
}

// Uploads one layer's weights (OIHW float32, with bias) in the precision's layout.
// sw: the 16-bit conv weights' layout for a 64-channel-multiple input: -1 follows the
// input's default chunking (128-byte swizzled for 64-channel chunks), 0 forces the
// no-swizzle form of inputs stored in 16-byte chunks.
nvisr_status upload_weights(nvisr_filter *f, const NetLayer &L, const float *w, const float *b, Weights &W,
                            int sw = -1) {
    W.cin_pad = act_cpad(f, L.cin);
    W.cout_pad = round_up(L.cout, 16);
    // padded to whole 64-channel slices (the row kernels read a slice's 64 biases)
    std::vector<float> bias(round_up(W.cout_pad, 64), 0.f);
    std::copy(b, b + L.cout, bias.begin());
    void *dbias;
    nvisr_status s = upload(f, bias.data(), bias.size() * 4, &dbias);
    if (s != NVISR_OK) return s;
    W.bias = (float *)dbias;
    if (!f->tc) {
        std::vector<float> host(simt_weight_bytes(W.cin_pad, W.cout_pad, L.k) / 4);
        prepare_weights_simt(w, L.cout, L.cin, L.k, W.cin_pad, W.cout_pad, host.data());
        s = upload(f, host.data(), host.size() * 4, &W.simt_or_tc);
    } else {
        std::vector<uint8_t> host(tc_weight_bytes(W.cin_pad, W.cout_pad, L.k, f->act_dt));
        // the conv kernel reads 64-channel inputs through 128-byte-swizzled operands;
        // the DCN kernel builds its own no-swizzle sampled tile
        const bool sw128 = L.op == "conv" && layout_cpc(f->act_dt, W.cin_pad) == 64 && sw != 0;
        prepare_weights_tc(w, L.cout, L.cin, L.k, W.cin_pad, W.cout_pad, f->act_dt, 1.0f, host.data(), sw128);
        s = upload(f, host.data(), host.size(), &W.simt_or_tc);
        if (s == NVISR_OK && L.op == "conv" && L.k == 3 && L.cin == 64 && L.cout == 64 && !L.ps) {
            std::vector<uint8_t> rows(tc_rows_weight_bytes());
            prepare_weights_rows(w, f->act_dt, rows.data());
            s = upload(f, rows.data(), rows.size(), &W.rows);
        } else if (s == NVISR_OK && L.op == "conv" && L.k == 3 && L.cin <= 16 && L.cout == 64 && !L.ps &&
                   f->act_dt != DT_F32) {
            // a 16-channel input (the tuple head): the row kernel's no-swizzle 16-channel form
            std::vector<uint8_t> rows(tc_rows16_weight_bytes());
            prepare_weights_rows16(w, L.cin, f->act_dt, rows.data());
            s = upload(f, rows.data(), rows.size(), &W.rows);
        } else if (s == NVISR_OK && L.op == "conv" && L.k == 3 && L.cin == 128 && L.cout <= 256 && !L.ps) {
            // 128 input channels (a concatenation of two 64-channel tensors), e.g. a DCN
            // offset/mask head: the row kernel's 128-channel form in 64-output slices
            std::vector<uint8_t> rows(tc_rows128_weight_bytes((W.cout_pad + 63) / 64));
            prepare_weights_rows128(w, L.cout, f->act_dt, rows.data());
            s = upload(f, rows.data(), rows.size(), &W.rows);
        } else if (s == NVISR_OK && L.op == "conv" && L.k == 3 && L.cin == 64 && L.cout == 256 && L.ps == 2) {
            // an upsampler (64 -> 256, PixelShuffle(2)): one row image per shuffle offset
            std::vector<uint8_t> rows(4 * tc_rows_weight_bytes(64));
            prepare_weights_rows_ps4(w, f->act_dt, rows.data());
            s = upload(f, rows.data(), rows.size(), &W.rows);
        } else if (s == NVISR_OK && L.op == "conv" && L.k == 3 && L.cin == 64 && L.cout <= 16 && L.cout % 4 == 0) {
            // a PixelShuffle(2) output layer: the row kernel's 16-column shuffle form
            std::vector<uint8_t> rows(tc_rows_weight_bytes(16));
            prepare_weights_rows(w, f->act_dt, rows.data(), L.cout, 16);
            s = upload(f, rows.data(), rows.size(), &W.rows);
        }
    }
    if (s != NVISR_OK) return s;
    if (layer_is_fp8(f, L)) {
        float amax = 0.f;
        for (int64_t k = 0; k < (int64_t)L.cout * L.cin * L.k * L.k; ++k) amax = std::max(amax, std::fabs(w[k]));
        W.w_amax = amax > 0.f ? amax : 1.f;
        const float sw = W.w_amax / 448.f;
        std::vector<uint8_t> host(tc_weight_bytes(L.cin, W.cout_pad, L.k, DT_E4M3));
        prepare_weights_tc(w, L.cout, L.cin, L.k, L.cin, W.cout_pad, DT_E4M3, 1.0f / sw, host.data(), false);
        s = upload(f, host.data(), host.size(), &W.f8);
        if (s != NVISR_OK) return s;
        std::vector<uint8_t> rows(tc_rows_f8_weight_bytes());
        prepare_weights_rows_f8(w, 1.0f / sw, rows.data());
        s = upload(f, rows.data(), rows.size(), &W.rows_f8);
        if (s != NVISR_OK) return s;
    }
    return NVISR_OK;
}

// Offset/mask heads whose output rows are stored tap-major (see DcnArgs): the
// head of a DCN layer with an even group count G, read by DCN layers only, and
// sharing its weights only with other such heads of the same G.  Returns per
// layer G, or 0 to keep torchvision's order.
std::vector<int> om_tap_major_groups(const NetDesc &net) {
    const int n = (int)net.layers.size();
    std::vector<int> G(n, 0);  // 0 = not a head, -1 = keep the order
    for (const NetLayer &D : net.layers) {
        if (D.op != "dcn") continue;
        const int p = net.find(D.om);
        if (p < 0) continue;
        const NetLayer &H = net.layers[p];
        const int want = D.groups % 2 == 0 && H.cout == 27 * D.groups && !H.ps ? D.groups : -1;
        G[p] = G[p] == 0 || G[p] == want ? want : -1;
    }
    for (const NetLayer &X : net.layers) {
        for (const std::string &nm : X.in) {
            const int p = net.find(nm);
            if (p >= 0) G[p] = G[p] ? -1 : 0;
        }
        const int a = X.add.empty() ? -1 : net.find(X.add);
        if (a >= 0) G[a] = G[a] ? -1 : 0;
    }
    for (const auto &o : net.outputs) {
        const int p = net.find(o.name);
        if (p >= 0) G[p] = G[p] ? -1 : 0;
    }
    std::vector<int> own(n, 0);
    for (int i = 0; i < n; ++i) {
        const int o = net.layers[i].owner, gi = G[i] > 0 ? G[i] : -1;
        own[o] = own[o] == 0 || own[o] == gi ? gi : -1;
    }
    std::vector<int> out(n, 0);
    for (int i = 0; i < n; ++i) out[i] = std::max(own[net.layers[i].owner], 0);
    return out;
}

// Head rows in tap-major order: the torchvision row that new row j takes.
int om_row_source(int j, int G) {
    const int k = j / (3 * G), r = j % (3 * G);
    return r < 2 * G ? 2 * ((r / 2) * 9 + k) + (r % 2) : 18 * G + (r - 2 * G) * 9 + k;
}

// Uploads a layer's weights, with its output rows permuted to tap-major order
// when it is such a head.
nvisr_status upload_layer(nvisr_filter *f, int li, const float *w, const float *b, Weights &W, int sw = -1) {
    const NetLayer &L = f->net.layers[li];
    const int G = f->om_tap_g[li];
    if (G == 0) return upload_weights(f, L, w, b, W, sw);
    const size_t per = (size_t)L.cin * L.k * L.k;
    std::vector<float> wo(per * L.cout), bo(L.cout);
    for (int j = 0; j < L.cout; ++j) {
        const int o = om_row_source(j, G);
        std::copy(w + o * per, w + (o + 1) * per, wo.begin() + j * per);
        bo[j] = b[o];
    }
    return upload_weights(f, L, wo.data(), bo.data(), W, sw);
}

nvisr_status prepare_weights(nvisr_filter *f, const float *blob) {
    const NetDesc &net = f->net;
    f->weights.resize(net.layers.size());
    f->om_tap_g = om_tap_major_groups(net);
    for (size_t i = 0; i < net.layers.size(); ++i) {
        const NetLayer &L = net.layers[i];
        if (L.op == "pool" || L.op == "up") continue;  // no weights
        if (L.owner != (int)i) {
            f->weights[i] = f->weights[L.owner];
            continue;
        }
        const float *w = blob + L.woff;
        const float *b = w + (int64_t)L.cout * L.cin * L.k * L.k;
        nvisr_status s = upload_layer(f, (int)i, w, b, f->weights[i]);
        if (s != NVISR_OK) return s;
    }
    return NVISR_OK;
}

// Builds the step list and allocates tensors with buffer reuse by liveness.
nvisr_status build_plan(nvisr_filter *f) {
    const NetDesc &net = f->net;
    const int H = f->in_fmt.height, W = f->in_fmt.width;
    std::map<std::string, int> tensor_of;  // layer name -> tensor id
    std::map<std::string, int> out_index;
    for (size_t i = 0; i < net.outputs.size(); ++i) out_index[net.outputs[i].name] = (int)i;
    f->tensors.clear();
    f->steps.clear();
    if (net.family == "tuple") {
        Tensor t;
        t.C = 3 * net.frames;
        t.cpad = act_cpad(f, t.C);
        t.H = H;
        t.W = W;
        t.dt = f->act_dt;
        f->pack_t = 0;
        f->tensors.push_back(t);
    }
    for (size_t i = 0; i < net.layers.size(); ++i) {
        const NetLayer &L = net.layers[i];
        if (L.op != "conv") return fail(NVISR_UNSUPPORTED_FORMAT, "layer " + L.name + ": op not supported by this plan");
        if (L.in.size() != 1) return fail(NVISR_UNSUPPORTED_FORMAT, "layer " + L.name + ": concatenated inputs");
        Step st;
        st.layer = (int)i;
        if (L.in[0] == "tuple") {
            st.src = SRC_TUPLE;
            st.in_t = f->pack_t;
        } else {
            auto it = tensor_of.find(L.in[0]);
            if (it == tensor_of.end()) return fail(NVISR_BAD_NETWORK, "layer " + L.name + ": unknown input");
            st.in_t = it->second;
        }
        const Tensor &src = f->tensors[st.in_t];
        if (src.C != L.cin) return fail(NVISR_BAD_NETWORK, "layer " + L.name + ": cin does not match its input");
        if (!L.add.empty()) st.add_t = tensor_of.at(L.add);
        st.fp8 = layer_is_fp8(f, L);
        if (out_index.count(L.name)) {
            // the output layer: 3 * psy * psx channels at input size, shuffled by the scale
            // (Section 3.2: horizontal and vertical scale; 2 x 2 super-resolution, 1 x 1
            // enhancement / denoise, 1 x 2 deinterlace)
            if (src.H != H || L.k != 3) return fail(NVISR_UNSUPPORTED_FORMAT, "output layer must be a 3x3 conv at input size");
            if (L.psx != net.scale || L.psy != net.scale_y)
                return fail(NVISR_UNSUPPORTED_FORMAT, "output layer's PixelShuffle must equal the network scale");
            if (L.cout != 3 * L.psx * L.psy)
                return fail(NVISR_UNSUPPORTED_FORMAT, "output layer must give 3 channels after its PixelShuffle");
            st.out_t = -1;
            st.out_index = out_index[L.name];
            st.skip_frames = {(net.frames - 1) / 2};
            st.psy = L.psy;
            st.psx = L.psx;
            st.plain = !(L.psy == 2 && L.psx == 2);
            f->plain_final = f->plain_final || st.plain;
        } else {
            if (L.ps || L.psx != 1 || L.psy != 1)
                return fail(NVISR_UNSUPPORTED_FORMAT, "inner PixelShuffle in a tuple network");
            Tensor t;
            t.C = L.cout;
            t.cpad = round_up(L.cout, 16);
            t.H = src.H;
            t.W = src.W;
            t.dt = f->act_dt;
            st.out_t = (int)f->tensors.size();
            tensor_of[L.name] = st.out_t;
            f->tensors.push_back(t);
        }
        f->steps.push_back(st);
    }
    // FP8: which tensors get an FP8 copy, which are FP8 only
    if (f->precision == NVISR_PREC_FP8) {
        std::vector<int> f8_uses(f->tensors.size(), 0), other_uses(f->tensors.size(), 0);
        for (const Step &s : f->steps) {
            if (s.fp8) f8_uses[s.in_t]++;
            else other_uses[s.in_t]++;
            if (s.add_t >= 0) other_uses[s.add_t]++;
        }
        int slot = 0;
        for (size_t t = 0; t < f->tensors.size(); ++t)
            if (f8_uses[t]) f->tensors[t].amax_slot = slot++;
        f->n_amax = slot;
        for (Step &s : f->steps)
            if (s.out_t >= 0 && f8_uses[s.out_t] && !other_uses[s.out_t]) s.out_f8_only = true;
        if (slot) {
            void *p;
            nvisr_status st = dalloc(f->eng, sizeof(unsigned) * slot, f->owned, &p, f->guard);
            if (st != NVISR_OK) return st;
            f->amax = (unsigned *)p;
            f->act_scale.assign(slot, 1.f);
        }
    }
    // liveness-based buffer reuse
    std::vector<int> last_use(f->tensors.size(), -1);
    int pack_readers = 0;
    f->tuple_head = -1;
    for (size_t i = 0; i < f->steps.size(); ++i) {
        const Step &s = f->steps[i];
        last_use[s.in_t] = std::max(last_use[s.in_t], (int)i);
        if (s.add_t >= 0) last_use[s.add_t] = std::max(last_use[s.add_t], (int)i);
        if (s.in_t == f->pack_t) {
            ++pack_readers;
            f->tuple_head = (int)i;
        }
        if (s.add_t >= 0 && s.add_t == f->pack_t) pack_readers += 2;
    }
    if (pack_readers != 1) f->tuple_head = -1;
    struct Buf { void *p; size_t bytes; int free_after; };
    std::vector<Buf> pool;
    auto acquire = [&](size_t bytes, int step, void **out) -> nvisr_status {
        for (Buf &b : pool)
            if (b.free_after < step && b.bytes >= bytes) {
                b.free_after = 1 << 30;
                *out = b.p;
                return NVISR_OK;
            }
        void *p;
        nvisr_status s = dalloc(f->eng, bytes, f->owned, &p, f->guard);
        if (s != NVISR_OK) return s;
        pool.push_back({p, bytes, 1 << 30});
        *out = p;
        return NVISR_OK;
    };
    auto release = [&](void *p, int step) {
        for (Buf &b : pool)
            if (b.p == p) b.free_after = step;
    };
    // tensor 0 (pack) is produced at step -1
    std::vector<std::pair<int, int>> producers;  // (step, tensor)
    if (f->pack_t >= 0) producers.push_back({-1, f->pack_t});
    for (size_t i = 0; i < f->steps.size(); ++i)
        if (f->steps[i].out_t >= 0) producers.push_back({(int)i, f->steps[i].out_t});
    // Allocate in step order; free after last use.  A tensor produced at step
    // i must not reuse a buffer still read at step i (free_after < i).
    size_t pi = 0;
    for (int step = -1; step < (int)f->steps.size(); ++step) {
        while (pi < producers.size() && producers[pi].first == step) {
            Tensor &t = f->tensors[producers[pi].second];
            const Step *ps = step >= 0 ? &f->steps[step] : nullptr;
            const bool only8 = ps && ps->out_f8_only;
            if (!only8) {
                nvisr_status s = acquire((size_t)t.cpad * t.H * t.W * dtype_size(t.dt), step, &t.ptr);
                if (s != NVISR_OK) return s;
            }
            if (t.amax_slot >= 0) {
                nvisr_status s = acquire((size_t)t.cpad * t.H * t.W, step, &t.f8);
                if (s != NVISR_OK) return s;
                if (only8) t.ptr = nullptr;
            }
            ++pi;
        }
        for (size_t t = 0; t < f->tensors.size(); ++t)
            if (last_use[t] == step) {
                if (f->tensors[t].ptr) release(f->tensors[t].ptr, step);
                if (f->tensors[t].f8) release(f->tensors[t].f8, step);
            }
    }
    // FP8 calibration needs the 16-bit tensors of FP8-only layers too
    if (f->precision == NVISR_PREC_FP8)
        for (Tensor &t : f->tensors)
            if (!t.ptr) {
                nvisr_status s = dalloc(f->eng, (size_t)t.cpad * t.H * t.W * dtype_size(t.dt), f->owned, &t.ptr, f->guard);
                if (s != NVISR_OK) return s;
            }
    for (Tensor &T : f->tensors) T.cpc = layout_cpc(T.dt, T.cpad);
    return NVISR_OK;
}

// Group-family plan (Section 3.1: a per-frame extract stage, then a fusion
// stage over the frame group): frame packs, convolutions, DCN layers,
// PixelShuffle stages.  A channel concatenation is free: its parts are
// produced straight into channel views of one buffer; a layer reading the
// parts in another order gets a copy of its weights with the input channels
// permuted to the storage order.  Buffers are reused by liveness.
nvisr_status build_plan_group(nvisr_filter *f, const float *blob) {
    const NetDesc &net = f->net;
    const int H = f->in_fmt.height, W = f->in_fmt.width;
    f->tensors.clear();
    f->steps.clear();
    f->wvar.clear();
    f->pack_t = -1;
    if (f->precision == NVISR_PREC_FP8) return fail(NVISR_UNSUPPORTED_FORMAT, "group networks run in FP32/BF16/FP16");
    if (net.scale != net.scale_y) return fail(NVISR_UNSUPPORTED_FORMAT, "group networks: one scale for both axes");
    for (const NetLayer &L : net.layers)
        if (L.psx != L.psy) return fail(NVISR_UNSUPPORTED_FORMAT, "group networks: PixelShuffle(2) only");
    f->grp_n = net.frames - (net.extra ? 1 : 0);
    f->grp_need = net.frames;
    f->run_out = net.dbl ? 2 * f->grp_n : f->grp_n;
    if (net.interp && !net.dbl && net.scale != 1)
        return fail(NVISR_UNSUPPORTED_FORMAT, "Interpolation without Double frame outputs the input frames as they "
                                              "are: the spatial scale must be 1");
    if (f->grp_n < 1 || net.frames > 8 || f->run_out > 8)
        return fail(NVISR_UNSUPPORTED_FORMAT, "group networks: at most 8 input frames and 8 outputs per run");
    if ((int)net.outputs.size() != f->run_out)
        return fail(NVISR_UNSUPPORTED_FORMAT, "group networks: the description lists n outputs (2n with Double frame)");
    std::map<std::string, int> tensor_of, out_index;
    for (size_t i = 0; i < net.outputs.size(); ++i) out_index[net.outputs[i].name] = (int)i;
    std::map<std::string, int> om_names;
    for (const NetLayer &L : net.layers)
        if (L.op == "dcn") om_names[L.om] = 1;
    auto chans = [&](const std::string &n) -> int {
        const int i = net.find(n);
        if (i < 0) return 3;
        return net.layers[i].ps ? net.layers[i].cout / 4 : net.layers[i].cout;
    };
    // concatenation groups: part -> (group, channel offset)
    struct Group { std::vector<std::string> parts; int C = 0; int t = -1; };
    std::vector<Group> groups;
    std::map<std::string, std::pair<int, int>> placed;
    for (const NetLayer &L : net.layers) {
        if (L.in.size() < 2) continue;
        int g = -1, found = 0;
        bool same = true;
        for (const std::string &n : L.in) {
            auto it = placed.find(n);
            if (it == placed.end()) continue;
            ++found;
            if (g < 0) g = it->second.first;
            else if (g != it->second.first) same = false;
        }
        if (found == 0) {
            Group G;
            for (const std::string &n : L.in) {
                if (net.find(n) < 0) return fail(NVISR_UNSUPPORTED_FORMAT, "layer " + L.name + ": concatenated frames");
                if (chans(n) % 16) return fail(NVISR_UNSUPPORTED_FORMAT, "concatenated tensors need 16k channels");
                placed[n] = {(int)groups.size(), G.C};
                G.parts.push_back(n);
                G.C += chans(n);
            }
            groups.push_back(G);
        } else if (found != (int)L.in.size() || !same || groups[g].parts.size() != L.in.size()) {
            return fail(NVISR_UNSUPPORTED_FORMAT, "layer " + L.name + ": concatenation overlaps another one");
        }
    }
    auto new_tensor = [&](int C, int cpad, int h, int w, int dt) {
        Tensor t;
        t.C = C; t.cpad = cpad; t.H = h; t.W = w; t.dt = dt;
        f->tensors.push_back(t);
        return (int)f->tensors.size() - 1;
    };
    auto source = [&](const std::string &n) -> int {
        auto it = tensor_of.find(n);
        if (it != tensor_of.end()) return it->second;
        if (n.rfind("frame", 0) != 0) return -1;
        const int k = atoi(n.c_str() + 5);
        if (k < 0 || k >= net.frames) return -1;
        const int id = new_tensor(3, act_cpad(f, 3), H, W, f->act_dt);
        tensor_of[n] = id;
        Step ps;
        ps.op = OP_PACK;
        ps.frame_src = k;
        ps.out_t = id;
        f->steps.push_back(ps);
        return id;
    };
    for (size_t i = 0; i < net.layers.size(); ++i) {
        const NetLayer &L = net.layers[i];
        Step st;
        st.layer = (int)i;
        st.op = L.op == "dcn" ? OP_DCN : (L.op == "pool" ? OP_POOL : (L.op == "up" ? OP_UP : OP_CONV));
        if (L.in.size() == 1) {
            st.in_t = source(L.in[0]);
        } else {
            const Group &G = groups[placed[L.in[0]].first];
            st.in_t = G.t;
            if (G.parts != L.in) {
                std::vector<int> perm(G.C);
                int loff = 0;
                for (const std::string &n : L.in) {
                    const int c = chans(n), soff = placed[n].second;
                    for (int j = 0; j < c; ++j) perm[soff + j] = loff + j;
                    loff += c;
                }
                st.perm = perm;
                const int kk = L.k * L.k;
                const float *w = blob + L.woff;
                const float *b = w + (int64_t)L.cout * L.cin * kk;
                std::vector<float> wp((size_t)L.cout * L.cin * kk);
                for (int o = 0; o < L.cout; ++o)
                    for (int c = 0; c < L.cin; ++c)
                        for (int t = 0; t < kk; ++t)
                            wp[((size_t)o * L.cin + c) * kk + t] = w[((size_t)o * L.cin + perm[c]) * kk + t];
                Weights Wv;
                nvisr_status s = upload_layer(f, (int)i, wp.data(), b, Wv);
                if (s != NVISR_OK) return s;
                st.widx = (int)f->wvar.size();
                f->wvar.push_back(Wv);
            }
        }
        if (st.in_t < 0) return fail(NVISR_BAD_NETWORK, "layer " + L.name + ": input not available");
        const Tensor src = f->tensors[st.in_t];
        if (src.C != L.cin) return fail(NVISR_BAD_NETWORK, "layer " + L.name + ": cin does not match its input");
        if (st.op == OP_DCN) {
            st.om_t = source(L.om);
            if (st.om_t < 0 || f->tensors[st.om_t].C != 27 * L.groups || f->tensors[st.om_t].dt != DT_F32)
                return fail(NVISR_BAD_NETWORK, "layer " + L.name + ": offset/mask head must have 27*groups channels");
            if (f->tensors[st.om_t].H != src.H) return fail(NVISR_BAD_NETWORK, "layer " + L.name + ": size mismatch");
            const int p = net.find(L.om);
            st.om_tap_major = p >= 0 && f->om_tap_g[p] == L.groups;
        }
        if (!L.add.empty()) {
            st.add_t = source(L.add);
            if (st.add_t < 0 || f->tensors[st.add_t].C != L.cout) return fail(NVISR_BAD_NETWORK, "bad add source");
        }
        if (out_index.count(L.name)) {
            // output layers: conv -> 12 channels + PixelShuffle(2), or at scale 1 a plain
            // conv -> 3 channels (float32 out, laid out planar by the shuffle kernel)
            const bool plain = net.scale == 1;
            if (plain ? (L.op != "conv" || L.ps || L.psx != 1 || L.psy != 1 || L.cout != 3 || L.k != 3)
                      : (L.op != "conv" || L.ps != 2 || L.cout != 12))
                return fail(NVISR_UNSUPPORTED_FORMAT, plain ? "output layers at scale 1: 3x3 conv -> 3 channels"
                                                            : "output layers: conv -> 12 ch + PixelShuffle(2)");
            if ((plain ? src.H != H || src.W != W : src.H * 2 != H * net.scale || src.W * 2 != W * net.scale))
                return fail(NVISR_UNSUPPORTED_FORMAT, "output layer " + L.name + ": size is not scale x input");
            if (plain) {
                st.plain = true;
                st.psy = st.psx = 1;
                f->plain_final = true;
            }
            st.out_t = -1;
            st.out_index = out_index[L.name];
            for (const std::string &n : net.outputs[st.out_index].skip) {
                const int k = atoi(n.c_str() + 5);
                if (n.rfind("frame", 0) != 0 || k < 0 || k >= net.frames) return fail(NVISR_BAD_NETWORK, "bad skip");
                st.skip_frames.push_back(k);
            }
            if (st.skip_frames.size() > 2) return fail(NVISR_UNSUPPORTED_FORMAT, "at most two skip frames");
        } else {
            const int C = L.ps ? L.cout / 4 : L.cout;
            int h = L.ps ? 2 * src.H : src.H, w = L.ps ? 2 * src.W : src.W;
            if (st.op == OP_POOL) {
                if (src.H % 2 || src.W % 2)
                    return fail(NVISR_UNSUPPORTED_FORMAT, "layer " + L.name + ": the 2x2 pool needs even sizes (" +
                                                              std::to_string(src.W) + "x" + std::to_string(src.H) + ")");
                h = src.H / 2;
                w = src.W / 2;
            } else if (st.op == OP_UP) {
                h = 2 * src.H;
                w = 2 * src.W;
            }
            const int dt = om_names.count(L.name) ? DT_F32 : f->act_dt;
            const int cpad = L.ps ? round_up(C, 16) : round_up(L.cout, 16);
            const int id = new_tensor(C, cpad, h, w, dt);
            auto pl = placed.find(L.name);
            if (pl != placed.end()) {
                Group &G = groups[pl->second.first];
                if (G.t < 0) G.t = new_tensor(G.C, G.C, h, w, f->act_dt);
                const Tensor &gt = f->tensors[G.t];
                if (gt.H != h || gt.W != w || dt != gt.dt || cpad != C)
                    return fail(NVISR_UNSUPPORTED_FORMAT, "concatenated tensors differ in size or type");
                f->tensors[id].parent = G.t;
                f->tensors[id].choff = pl->second.second;
            }
            tensor_of[L.name] = id;
            st.out_t = id;
        }
        f->steps.push_back(st);
    }
    // ---- extract cache (Section 3.1: the extract stage works on a single frame, so a
    // frame's features serve every run that takes it).  Two-frame networks only: a step is
    // an extract step when it depends on one frame slot and its output is a part of a
    // concatenation of both frames' features ("pair"), or feeds only extract steps.  The
    // pairs' buffers persist across runs; each of their halves holds one frame's features.
    const int n = (int)f->tensors.size();
    auto root = [&](int t) { return f->tensors[t].parent >= 0 ? f->tensors[t].parent : t; };
    f->xcache = false;
    f->xpairs.clear();
    std::vector<char> persistent(n, 0);
    if (net.frames == 2) {
        std::vector<int> mask(n, 0);                 // frame slots a tensor depends on
        std::vector<std::string> sig(n);             // the function of its frame that it is
        std::vector<int> producer(n, -1);
        for (size_t i = 0; i < f->steps.size(); ++i) {
            const Step &st = f->steps[i];
            if (st.out_t < 0) continue;
            int m = 0;
            std::string sg;
            if (st.op == OP_PACK) {
                m = 1 << st.frame_src;
                sg = "frame";
            } else {
                const NetLayer &L = net.layers[st.layer];
                const bool weightless = st.op == OP_POOL || st.op == OP_UP;
                sg = L.op + ":" + (weightless ? std::string("-") : std::to_string(L.owner)) + ":" +
                     std::to_string(L.act) + ":" + std::to_string(L.ps) + "(";
                for (int u : {st.in_t, st.add_t, st.om_t})
                    if (u >= 0) {
                        m |= mask[u];
                        sg += sig[u] + ",";
                    }
                sg += ")";
            }
            mask[st.out_t] |= m;
            sig[st.out_t] = sg;
            producer[st.out_t] = (int)i;
            if (f->tensors[st.out_t].parent >= 0) mask[f->tensors[st.out_t].parent] |= m;
        }
        // pairs: concatenations of exactly two parts, the same function of frame slots 0 and 1
        bool ok = true;
        std::vector<int> part_of_pair(n, 0);
        for (int t = 0; t < n && ok; ++t) {
            std::vector<int> parts;
            for (int c = 0; c < n; ++c)
                if (f->tensors[c].parent == t) parts.push_back(c);
            if (parts.empty()) continue;
            const bool single = parts.size() == 2 && (mask[parts[0]] == 1 || mask[parts[0]] == 2) &&
                                (mask[parts[1]] == 1 || mask[parts[1]] == 2);
            if (!single) {
                // a concatenation of other tensors (the alignment's blends): not cached, but it
                // must not hold single-frame parts either
                for (int c : parts)
                    if (mask[c] == 1 || mask[c] == 2) ok = false;
                continue;
            }
            if (mask[parts[0]] == mask[parts[1]] || sig[parts[0]] != sig[parts[1]] ||
                f->tensors[parts[0]].C != f->tensors[parts[1]].C || f->tensors[parts[0]].choff != 0) {
                ok = false;
                break;
            }
            nvisr_filter::XPair xp;
            xp.parent = t;
            for (int c : parts) {
                xp.part[mask[c] == 1 ? 0 : 1] = c;
                part_of_pair[c] = 1;
            }
            f->xpairs.push_back(xp);
        }
        if (f->xpairs.empty()) ok = false;
        // extract steps, from the last step back: single-frame steps whose output is a pair
        // part, or is read only by extract steps
        std::vector<char> is_x(f->steps.size(), 0);
        for (int i = (int)f->steps.size() - 1; i >= 0 && ok; --i) {
            const Step &st = f->steps[i];
            if (st.out_t < 0 || (mask[st.out_t] != 1 && mask[st.out_t] != 2)) continue;
            bool x = part_of_pair[st.out_t] != 0;
            if (!x) {
                int readers = 0;
                bool all = true;
                for (size_t j = 0; j < f->steps.size(); ++j) {
                    const Step &r = f->steps[j];
                    if (r.in_t == st.out_t || r.add_t == st.out_t || r.om_t == st.out_t) {
                        ++readers;
                        all = all && is_x[j];
                    }
                }
                x = readers > 0 && all;
            }
            is_x[i] = x;
        }
        // readers of a pair's buffer are two-input convolutions (weights per pair order)
        for (size_t i = 0; i < f->steps.size() && ok; ++i) {
            const Step &st = f->steps[i];
            for (const nvisr_filter::XPair &xp : f->xpairs)
                if (st.in_t == xp.parent && (st.op != OP_CONV || net.layers[st.layer].in.size() != 2)) ok = false;
            for (int u : {st.add_t, st.om_t})
                for (const nvisr_filter::XPair &xp : f->xpairs)
                    if (u == xp.parent) ok = false;
        }
        if (ok) {
            f->xcache = true;
            for (size_t i = 0; i < f->steps.size(); ++i)
                if (is_x[i]) f->steps[i].xslot = mask[f->steps[i].out_t] == 1 ? 0 : 1;
            for (const nvisr_filter::XPair &xp : f->xpairs) persistent[xp.parent] = 1;
        }
    }

    // liveness on root tensors (views count as their parent)
    std::vector<int> first_def(n, 1 << 30), last_use(n, -1);
    for (size_t i = 0; i < f->steps.size(); ++i) {
        const Step &st = f->steps[i];
        if (st.out_t >= 0) first_def[root(st.out_t)] = std::min(first_def[root(st.out_t)], (int)i);
        for (int u : {st.in_t, st.add_t, st.om_t})
            if (u >= 0) last_use[root(u)] = std::max(last_use[root(u)], (int)i);
    }
    struct Buf { void *p; size_t bytes; int free_after; };
    std::vector<Buf> pool;
    for (int t = 0; t < n; ++t)
        if (persistent[t]) {  // cached pairs: their own buffers, kept across runs
            Tensor &T = f->tensors[t];
            nvisr_status s = dalloc(f->eng, (size_t)T.cpad * T.H * T.W * dtype_size(T.dt), f->owned, &T.ptr, f->guard);
            if (s != NVISR_OK) return s;
        }
    for (int step = 0; step < (int)f->steps.size(); ++step) {
        for (int t = 0; t < n; ++t) {
            if (f->tensors[t].parent >= 0 || first_def[t] != step || persistent[t]) continue;
            Tensor &T = f->tensors[t];
            const size_t bytes = (size_t)T.cpad * T.H * T.W * dtype_size(T.dt);
            void *got = nullptr;
            for (Buf &b : pool)
                if (b.free_after < step && b.bytes >= bytes) {
                    b.free_after = 1 << 30;
                    got = b.p;
                    break;
                }
            if (!got) {
                nvisr_status s = dalloc(f->eng, bytes, f->owned, &got, f->guard);
                if (s != NVISR_OK) return s;
                pool.push_back({got, bytes, 1 << 30});
            }
            T.ptr = got;
        }
        for (int t = 0; t < n; ++t)
            if (f->tensors[t].parent < 0 && last_use[t] == step && f->tensors[t].ptr && !persistent[t])
                for (Buf &b : pool)
                    if (b.p == f->tensors[t].ptr) b.free_after = step;
    }
    for (Tensor &T : f->tensors) T.cpc = layout_cpc(T.dt, T.cpad);
    // a concatenation's parts are channel views of its buffer, so they share one chunk
    // layout: the narrowest part's (16-channel parts of a 64-channel buffer: 8 channels)
    for (Tensor &T : f->tensors)
        if (T.parent >= 0) f->tensors[T.parent].cpc = std::min(f->tensors[T.parent].cpc, T.cpc);
    for (Tensor &T : f->tensors)
        if (T.parent >= 0) T.cpc = f->tensors[T.parent].cpc;
    // a 16-bit conv whose 64-channel-multiple input was so narrowed reads it in 16-byte
    // chunks: its weights are laid out again, without the 128-byte swizzle
    for (Step &st : f->steps) {
        if (!f->tc || st.op != OP_CONV) continue;
        const Tensor &in = f->tensors[st.in_t];
        if (in.cpc == layout_cpc(in.dt, in.cpad)) continue;
        const NetLayer &L = net.layers[st.layer];
        const int kk = L.k * L.k;
        const float *w = blob + net.layers[L.owner].woff;
        const float *b = w + (int64_t)L.cout * L.cin * kk;
        std::vector<float> wp(w, w + (size_t)L.cout * L.cin * kk);
        if (!st.perm.empty())
            for (int o = 0; o < L.cout; ++o)
                for (int c = 0; c < L.cin; ++c)
                    for (int t = 0; t < kk; ++t)
                        wp[((size_t)o * L.cin + c) * kk + t] = w[((size_t)o * L.cin + st.perm[c]) * kk + t];
        Weights Wv;
        nvisr_status s = upload_layer(f, st.layer, wp.data(), b, Wv, 0);
        if (s != NVISR_OK) return s;
        st.widx = (int)f->wvar.size();
        f->wvar.push_back(Wv);
    }
    // extract cache: a pair whose buffer was narrowed to 16-byte chunks is not cached; the
    // readers of a cached pair get their weights for both orders of its halves
    for (const nvisr_filter::XPair &xp : f->xpairs) {
        const Tensor &P = f->tensors[xp.parent];
        if (P.cpc != layout_cpc(P.dt, P.cpad)) f->xcache = false;
    }
    if (!f->xcache) {
        for (Step &st : f->steps) st.xslot = -1;
        f->xpairs.clear();
    }
    for (Step &st : f->steps) {
        if (!f->xcache || st.op != OP_CONV) continue;
        const nvisr_filter::XPair *xp = nullptr;
        for (const nvisr_filter::XPair &q : f->xpairs)
            if (st.in_t == q.parent) xp = &q;
        if (!xp) continue;
        const NetLayer &L = net.layers[st.layer];
        const int C = f->tensors[xp->part[0]].C;
        // the frame slot whose features are the layer's first input
        int slot_first = -1;
        for (int k = 0; k < 2; ++k)
            for (const Step &q : f->steps)
                if (q.out_t == xp->part[k] && q.op != OP_PACK && net.layers[q.layer].name == L.in[0]) slot_first = k;
        if (slot_first < 0) return fail(NVISR_INTERNAL, "layer " + L.name + ": pair part not found");
        const int kk = L.k * L.k;
        const float *w = blob + net.layers[L.owner].woff;
        const float *b = w + (int64_t)L.cout * L.cin * kk;
        for (int order = 0; order < 2; ++order) {
            // order 0: the buffer holds frame slot 0's features first; 1: slot 1's first
            const bool swapped = (slot_first != order);
            if (!swapped) {
                st.xpair_w[order] = -1;  // the layer's own weights
                continue;
            }
            std::vector<float> wp((size_t)L.cout * L.cin * kk);
            for (int o = 0; o < L.cout; ++o)
                for (int c = 0; c < L.cin; ++c) {
                    const int src = c < C ? c + C : c - C;  // stored channel c holds layer channel src
                    for (int t = 0; t < kk; ++t)
                        wp[((size_t)o * L.cin + c) * kk + t] = w[((size_t)o * L.cin + src) * kk + t];
                }
            Weights Wv;
            nvisr_status s = upload_layer(f, st.layer, wp.data(), b, Wv);
            if (s != NVISR_OK) return s;
            st.xpair_w[order] = (int)f->wvar.size();
            f->wvar.push_back(Wv);
        }
    }
    // the tensor-core DCN gathers from its input copied into 8-channel planes
    size_t x8 = 0;
    for (const Step &st : f->steps)
        if (st.op == OP_DCN && f->tc && f->tensors[st.in_t].cpc != 8) {
            const Tensor &T = f->tensors[st.in_t];
            x8 = std::max(x8, (size_t)T.cpad * T.H * T.W * dtype_size(T.dt));
        }
    if (x8) {
        nvisr_status s = dalloc(f->eng, x8, f->owned, &f->dcn_x8, f->guard);
        if (s != NVISR_OK) return s;
    }
    for (Tensor &T : f->tensors)
        if (T.parent >= 0) {
            const Tensor &P = f->tensors[T.parent];
            if (T.cpc != P.cpc || T.choff % P.cpc) return fail(NVISR_INTERNAL, "view layout mismatch");
            T.ptr = (uint8_t *)P.ptr + (size_t)(T.choff / P.cpc) * P.H * P.W * P.cpc * dtype_size(P.dt);
        }
    return NVISR_OK;
}

// Runs one conv step.  calib: 16-bit pass recording amax of FP8-consumed tensors.
// Skip path of a final output: the frames whose upsampled mean requantise adds.
void set_final_skip(nvisr_filter *f, const Step &s, const float *const *frames) {
    SkipArgs &k = f->skip[s.out_index];
    k = SkipArgs{};
    k.n = f->net.skip ? std::min<int>((int)s.skip_frames.size(), 2) : 0;
    for (int i = 0; i < k.n; ++i) k.src[i] = frames[s.skip_frames[i]];
    k.pitch = f->rpitch;
    k.plane = f->rpitch * f->in_fmt.height;
    k.h = f->in_fmt.height;
    k.w = f->in_fmt.width;
    k.scale = f->net.scale;
    k.scale_y = f->net.scale_y;
    k.mode = f->net.skip;
}

// Profiling kind of a step's launch.
int step_kind(const nvisr_filter *f, const Step &s) {
    if (s.op == OP_DCN) return NVISR_K_DCN;
    if (s.op == OP_PACK) return NVISR_K_PACK;
    if (s.op == OP_POOL || s.op == OP_UP) return NVISR_K_RESAMPLE;
    const NetLayer &L = f->net.layers[s.layer];
    return s.out_t < 0 ? NVISR_K_CONV_TAIL
                       : (s.src == SRC_TUPLE ? NVISR_K_CONV_HEAD
                                             : (L.cin == 64 && L.cout == 64 && L.k == 3 && !L.ps ? NVISR_K_CONV_BODY
                                                                                                  : NVISR_K_CONV_OTHER));
}

// Before step i of a forward pass: whether the next launch is of the same profiling kind.
void hold_if_same_kind(nvisr_filter *f, size_t i) {
    f->prof_hold = i + 1 < f->steps.size() && step_kind(f, f->steps[i + 1]) == step_kind(f, f->steps[i]);
}

// Arguments of a conv step (no launch).  For the final layer it also sets the
// filter's skip arguments (the frames whose upsampled mean requantise adds).
ConvArgs conv_args(nvisr_filter *f, const Step &s, const float *const *frames, bool calib, int *kind) {
    const NetLayer &L = f->net.layers[s.layer];
    const Weights &Wt = s.widx >= 0 ? f->wvar[s.widx] : f->weights[s.layer];
    const Tensor &in = f->tensors[s.in_t];
    ConvArgs a{};
    a.cin_pad = in.cpad;
    a.in_cpc = in.cpc;
    a.H = in.H;
    a.W = in.W;
    a.nimg = 1;
    a.bias = Wt.bias;
    a.cout = L.cout;
    a.cout_pad = Wt.cout_pad;
    a.k = L.k;
    a.act = L.act;
    a.acc_scale = 1.f;
    a.out_scale = 1.f;
    a.y2_scale = 1.f;
    a.in_dt = in.dt;
    a.out_dt = f->act_dt;
    a.err = f->eng->err_word;
    const bool use_f8 = s.fp8 && !calib && f->calibrated;
    if (use_f8) {
        a.x = in.f8;
        a.in_dt = DT_E4M3;
        a.cin_pad = in.cpad;  // 64
        a.in_cpc = 16;        // FP8 copies use 16-channel (16-byte) chunks
        a.w = Wt.f8;
        a.w_rows = Wt.rows_f8;
        a.acc_scale = f->act_scale[in.amax_slot] * (Wt.w_amax / 448.f);
    } else {
        a.x = in.ptr;
        a.w = Wt.simt_or_tc;
        a.w_rows = Wt.rows;
    }
    if (s.add_t >= 0) a.res = f->tensors[s.add_t].ptr;
    if (s.out_t >= 0) {
        const Tensor &o = f->tensors[s.out_t];
        a.y = o.ptr;
        a.out_dt = o.dt;
        a.out_cpc = o.cpc;
        a.ps = L.ps;
        if (!calib && f->calibrated && o.amax_slot >= 0) {
            const float inv = 1.f / f->act_scale[o.amax_slot];
            if (s.out_f8_only && use_f8) {
                a.y = o.f8;
                a.out_dt = DT_E4M3;
                a.out_cpc = 16;
                a.out_scale = inv;
            } else {
                a.y2 = o.f8;
                a.y2_scale = inv;
            }
        }
        if (calib && o.amax_slot >= 0) a.amax = f->amax + o.amax_slot;
    } else if (s.plain) {
        // a last layer without the 2 x 2 shuffle: float32 output, shuffled into planar
        // float32 by its own kernel (run_step); the skip is added by requantise
        a.y = f->final_f32;
        a.out_dt = DT_F32;
        a.out_cpc = 4;
        a.ps = 0;
        set_final_skip(f, s, frames);
    } else {
        // the network's last layer: PixelShuffle(2) residual into planar float32; the
        // skip (upsampled input frames) is added by the requantise kernel
        a.ps = 2;
        a.ps_out = f->out_rgb[s.out_index];
        a.ps_pitch = f->opitch;
        a.skip_mode = 0;
        a.nskip = 0;
        set_final_skip(f, s, frames);
        if (f->fused_rq && !calib && !f->batched && f->rq_o >= 0) {
            // or requantised in the layer's epilogue, into the output's staging buffer (or straight
            // into the caller's device planes when the pull that wants them computes the output)
            const int b = (int)(f->rq_o & 1);
            a.rq = f->rq_base;
            a.rq.yp = (uint8_t *)f->ostage[b][0];
            a.rq.up = (uint8_t *)f->ostage[b][1];
            a.rq.vp = (uint8_t *)f->ostage[b][2];
            a.rq.py = f->ostage_pitch[0];
            a.rq.pu = f->ostage_pitch[1];
            a.rq.pv = f->ostage_pitch[2];
            if (const nvisr_planes *d = f->rq_direct) {
                a.rq.yp = (uint8_t *)d->data[0];
                a.rq.up = (uint8_t *)d->data[1];
                a.rq.vp = (uint8_t *)d->data[2];
                a.rq.py = d->pitch[0];
                a.rq.pu = d->pitch[1];
                a.rq.pv = d->pitch[2];
            }
            const SkipArgs &k = f->skip[s.out_index];
            a.rq.skip = k.n ? k.src[0] : nullptr;
            a.rq.skip_pitch = f->rpitch;
            a.rq.skip_plane = f->rpitch * f->in_fmt.height;
            a.rq.edge = f->rq_edge;
            if (f->rq_direct) f->rq_direct_done = f->rq_o;
            else f->rq_done[b] = f->rq_o;
        }
    }
    *kind = step_kind(f, s);
    return a;
}

// Residual blocks of a 16-bit tensor-core trunk: steps i, i + 1 = conv 64 -> 64 3x3 with
// LeakyReLU, then conv 64 -> 64 3x3 without activation that adds step i's input, where
// nothing else reads step i's output (nor a view of it).  Such a pair runs as one fused
// launch (launch_res_block) unless NVISR_OPT_UNFUSED_BLOCKS is set.
void plan_blocks(nvisr_filter *f) {
    const size_t n = f->steps.size();
    f->blk.assign(n, 0);
    if (!f->tc || (f->act_dt != DT_BF16 && f->act_dt != DT_F16) || f->precision == NVISR_PREC_FP8 ||
        (f->options & NVISR_OPT_UNFUSED_BLOCKS))
        return;
    std::vector<int> reads(f->tensors.size(), 0);
    for (const Step &s : f->steps) {
        if (s.in_t >= 0) reads[s.in_t]++;
        if (s.add_t >= 0) reads[s.add_t]++;
        if (s.om_t >= 0) reads[s.om_t]++;
    }
    std::vector<char> viewed(f->tensors.size(), 0);
    for (const Tensor &t : f->tensors)
        if (t.parent >= 0) viewed[t.parent] = 1;
    auto body = [](const NetLayer &L, int act) {
        return L.op == "conv" && L.cin == 64 && L.cout == 64 && L.k == 3 && L.ps == 0 && L.psx == 1 && L.psy == 1 &&
               L.act == act;
    };
    for (size_t i = 0; i + 1 < n; ++i) {
        const Step &a = f->steps[i], &b = f->steps[i + 1];
        if (a.op != OP_CONV || b.op != OP_CONV || a.src != SRC_TENSOR || b.src != SRC_TENSOR || a.fp8 || b.fp8)
            continue;
        if (a.out_t < 0 || b.out_t < 0 || a.add_t >= 0 || b.in_t != a.out_t || b.add_t != a.in_t) continue;
        if (a.xslot != b.xslot || a.xpair_w[0] != -2 || b.xpair_w[0] != -2 || a.frame_src >= 0) continue;
        if (!body(f->net.layers[a.layer], 1) || !body(f->net.layers[b.layer], 0)) continue;
        if (reads[a.out_t] != 1 || f->tensors[a.out_t].parent >= 0 || viewed[a.out_t]) continue;
        f->blk[i] = 1;
        ++i;  // blocks do not overlap
    }
}

nvisr_status run_step(nvisr_filter *f, const Step &s, const float *const *frames, bool calib);

// Steps i, i + 1 (a planned residual block) as one launch; as two where the buffers do not
// allow it.
nvisr_status run_block(nvisr_filter *f, size_t i, const float *const *frames) {
    const Step &s1 = f->steps[i], &s2 = f->steps[i + 1];
    int k1 = 0, k2 = 0;
    const ConvArgs a1 = conv_args(f, s1, frames, false, &k1);
    const ConvArgs a2 = conv_args(f, s2, frames, false, &k2);
    if (!res_block_fits(a1, a2)) {
        hold_if_same_kind(f, i);
        nvisr_status st = run_step(f, s1, frames, false);
        hold_if_same_kind(f, i + 1);
        return st == NVISR_OK ? run_step(f, s2, frames, false) : st;
    }
    hold_if_same_kind(f, i + 1);
    ProfScope ps(f, NVISR_K_CONV_BODY);
    const cudaError_t e = launch_res_block(a1, a2, f->eng->stream);
    if (e != cudaSuccess)
        return cuda_status(e, ("residual block " + f->net.layers[s1.layer].name + ", " +
                               f->net.layers[s2.layer].name).c_str());
    return NVISR_OK;
}

nvisr_status run_step(nvisr_filter *f, const Step &s, const float *const *frames, bool calib) {
    const NetLayer &L = f->net.layers[s.layer];
    const Weights &Wt = s.widx >= 0 ? f->wvar[s.widx] : f->weights[s.layer];
    const Tensor &in = f->tensors[s.in_t];
    cudaStream_t st = f->eng->stream;
    if (s.op == OP_POOL || s.op == OP_UP) {
        const Tensor &o = f->tensors[s.out_t];
        ProfScope ps(f, NVISR_K_RESAMPLE);
        const cudaError_t e =
            launch_resample2(s.op == OP_UP, in.dt, in.ptr, in.cpc, o.ptr, o.cpc, in.C, in.H, in.W, st);
        if (e != cudaSuccess) return cuda_status(e, ("resample layer " + L.name).c_str());
        return NVISR_OK;
    }
    if (s.op == OP_DCN) {
        const Tensor &om = f->tensors[s.om_t];
        const Tensor &o = f->tensors[s.out_t];
        DcnArgs d{};
        d.x = in.ptr; d.cin_pad = in.cpad; d.H = in.H; d.W = in.W; d.groups = L.groups;
        d.x_cpc = in.cpc; d.y_cpc = o.cpc;
        d.om = (const float *)om.ptr; d.om_cpad = om.cpad; d.om_tap_major = s.om_tap_major; d.mask_logits = 1;
        d.w = Wt.simt_or_tc; d.bias = Wt.bias; d.cout = L.cout; d.cout_pad = Wt.cout_pad;
        d.y = o.ptr; d.in_dt = in.dt; d.out_dt = o.dt; d.acc_scale = 1.f; d.out_scale = 1.f;
        d.err = f->eng->err_word;
        ProfScope ps(f, NVISR_K_DCN);
        if (f->tc && in.cpc != 8) {
            cudaError_t e = launch_dcn_relayout8(in.ptr, in.cpad, in.H, in.W, in.cpc, f->dcn_x8, st);
            if (e != cudaSuccess) return cuda_status(e, ("dcn layer " + L.name + " relayout").c_str());
            d.x = f->dcn_x8;
            d.x_cpc = 8;
        }
        cudaError_t e = f->tc ? launch_dcn_tc(d, st) : launch_dcn_simt(d, st);
        if (e != cudaSuccess) return cuda_status(e, ("dcn layer " + L.name).c_str());
        return NVISR_OK;
    }
    int kind = 0;
    const ConvArgs a = conv_args(f, s, frames, calib, &kind);
    ProfScope ps(f, kind);
    cudaError_t e = f->tc ? launch_conv_tc(a, st) : launch_conv_simt(a, st);
    if (e != cudaSuccess) return cuda_status(e, ("conv layer " + L.name).c_str());
    if (f->tc && rq_edge_fixup_runs(a.rq, a.W)) ps.launches = 2;  // the tail's chroma edge fix-up
    if (s.plain) {
        e = launch_shuffle_planar(f->final_f32, a.H, a.W, s.psy, s.psx, f->out_rgb[s.out_index], f->opitch, st);
        if (e != cudaSuccess) return cuda_status(e, ("output shuffle of " + L.name).c_str());
    }
    return NVISR_OK;
}

nvisr_status forward_tuple(nvisr_filter *f, const std::vector<int64_t> &idx, bool calib) {
    const Tensor &pk = f->tensors[f->pack_t];
    PackArgs pa{};
    const float *frames[8];
    for (size_t k = 0; k < idx.size(); ++k) frames[k] = pa.src[k] = ring_slot(f, idx[k]);
    // 16-bit tensor-core head: the conv reads the tuple's frames from the ring itself (same
    // values, channel order and rounding as the pack), so the packed tensor is not written
    int fused = -1;
    ConvArgs ha{};
    if (f->tc && !calib && f->tuple_head >= 0 && idx.size() <= 5) {
        int kind = 0;
        ha = conv_args(f, f->steps[f->tuple_head], frames, false, &kind);
        ha.ring = f->ring_base;
        ha.ring_slots = f->ring;
        ha.ring_pitch = f->rpitch;
        ha.ntup = (int)idx.size();
        for (size_t k = 0; k < idx.size(); ++k) ha.tslot[k] = (int)(idx[k] % f->ring);
        if (rows_head_fits(ha) && ha.nimg == 1 && pk.C == 3 * ha.ntup) fused = f->tuple_head;
    }
    if (fused >= 0) {
        for (size_t i = 0; i < f->steps.size(); ++i) {
            hold_if_same_kind(f, i);
            if ((int)i == fused) {
                ProfScope ps(f, NVISR_K_CONV_HEAD);
                cudaError_t e = launch_conv_tc(ha, f->eng->stream);
                if (e != cudaSuccess) return cuda_status(e, ("conv layer " + f->net.layers[f->steps[i].layer].name).c_str());
                continue;
            }
            if (!calib && f->blk[i]) {
                nvisr_status st = run_block(f, i++, frames);
                if (st != NVISR_OK) return st;
                continue;
            }
            nvisr_status st = run_step(f, f->steps[i], frames, calib);
            if (st != NVISR_OK) return st;
        }
        f->prof_hold = false;
        return NVISR_OK;
    }
    pa.nsrc = (int)idx.size();
    pa.ch_per_src = 3;
    pa.src_pitch = f->rpitch;
    pa.src_plane = f->rpitch * f->in_fmt.height;
    pa.H = pk.H;
    pa.W = pk.W;
    pa.dst = pk.ptr;
    pa.cpad = pk.cpad;
    pa.dt = pk.dt;
    pa.cpc = pk.cpc;
    pa.scale = 1.f;
    cudaError_t e;
    {
        ProfScope ps(f, NVISR_K_PACK);
        e = launch_pack(pa, f->eng->stream);
    }
    if (e != cudaSuccess) return cuda_status(e, "pack");
    for (size_t i = 0; i < f->steps.size(); ++i) {
        if (!calib && f->blk[i]) {
            nvisr_status st = run_block(f, i++, frames);
            if (st != NVISR_OK) return st;
            continue;
        }
        hold_if_same_kind(f, i);
        nvisr_status st = run_step(f, f->steps[i], frames, calib);
        if (st != NVISR_OK) return st;
    }
    f->prof_hold = false;
    return NVISR_OK;
}

// Extract cache of a run over frames (a, b): which half of the pair buffers holds each
// frame slot's features (h[k]) and whether the run computes them (need[k]).  A half keeps
// the frame it holds until a run needs it for a frame no half holds.
void xcache_plan(nvisr_filter *f, const std::vector<int64_t> &idx, int h[2], bool need[2]) {
    const int64_t fr[2] = {idx[0], idx[1]};
    const int64_t *tag = f->xc_tag;
    if (fr[0] == fr[1]) {
        h[0] = 0;
        h[1] = 1;
    } else {
        const int ha = tag[0] == fr[0] ? 0 : (tag[1] == fr[0] ? 1 : -1);
        const int hb = tag[0] == fr[1] ? 0 : (tag[1] == fr[1] ? 1 : -1);
        h[0] = ha >= 0 ? ha : (hb >= 0 ? 1 - hb : 0);
        h[1] = 1 - h[0];
    }
    for (int k = 0; k < 2; ++k) need[k] = tag[h[k]] != fr[k];
}

// Group family: one run over frames (idx[0], idx[1], ...) computing every output.
nvisr_status forward_group(nvisr_filter *f, const std::vector<int64_t> &idx) {
    const float *frames[8];
    for (size_t k = 0; k < idx.size() && k < 8; ++k) frames[k] = ring_slot(f, idx[k]);
    int h[2] = {0, 1};
    bool need[2] = {true, true};
    if (f->xcache) {
        xcache_plan(f, idx, h, need);
        // each frame slot's features: the half of every pair buffer chosen for it
        for (const nvisr_filter::XPair &xp : f->xpairs) {
            const Tensor &P = f->tensors[xp.parent];
            for (int k = 0; k < 2; ++k) {
                Tensor &T = f->tensors[xp.part[k]];
                T.choff = h[k] * T.C;
                T.ptr = (uint8_t *)P.ptr + (size_t)(T.choff / P.cpc) * P.H * P.W * P.cpc * dtype_size(P.dt);
            }
        }
        const int order = h[0] == 0 ? 0 : 1;
        for (Step &st : f->steps)
            if (st.xpair_w[order] > -2) st.widx = st.xpair_w[order];
        for (int k = 0; k < 2; ++k) {
            if (need[k]) {
                f->xc_tag[h[k]] = -1;  // set once the run is enqueued
                ++f->xc_misses;
            } else {
                ++f->xc_hits;
            }
        }
    }
    for (size_t i = 0; i < f->steps.size(); ++i) {
        const Step &s = f->steps[i];
        if (s.xslot >= 0 && !need[s.xslot]) continue;  // features held by the cache
        if (f->blk[i]) {
            nvisr_status st = run_block(f, i++, frames);
            if (st != NVISR_OK) return st;
            continue;
        }
        hold_if_same_kind(f, i);
        if (s.op == OP_PACK) {
            const Tensor &t = f->tensors[s.out_t];
            PackArgs pa{};
            pa.src[0] = frames[s.frame_src];
            pa.nsrc = 1;
            pa.ch_per_src = 3;
            pa.src_pitch = f->rpitch;
            pa.src_plane = f->rpitch * f->in_fmt.height;
            pa.H = t.H;
            pa.W = t.W;
            pa.dst = t.ptr;
            pa.cpad = t.cpad;
            pa.dt = t.dt;
            pa.cpc = t.cpc;
            pa.scale = 1.f;
            cudaError_t e;
            {
                ProfScope ps(f, NVISR_K_PACK);
                e = launch_pack(pa, f->eng->stream);
            }
            if (e != cudaSuccess) return cuda_status(e, "pack");
            continue;
        }
        nvisr_status st = run_step(f, s, frames, false);
        if (st != NVISR_OK) return st;
    }
    f->prof_hold = false;
    if (f->xcache)
        for (int k = 0; k < 2; ++k) f->xc_tag[h[k]] = idx[k];
    return NVISR_OK;
}

nvisr_status calibrate(nvisr_filter *f) {
    if (!calibration_ready(f)) return NVISR_AGAIN;
    const int n = (int)(f->eos ? std::min<int64_t>(f->calib_frames, f->pushed) : f->calib_frames);
    std::vector<int64_t> idx;
    NVISR_TRY_CUDA(cudaMemsetAsync(f->amax, 0, sizeof(unsigned) * f->n_amax, f->eng->stream));
    prof_gap(f);
    for (int t = 0; t < n; ++t) {
        tuple_ready(f, t, &idx);
        nvisr_status s = forward_tuple(f, idx, true);
        if (s != NVISR_OK) return s;
    }
    std::vector<unsigned> h(f->n_amax);
    NVISR_TRY_CUDA(cudaMemcpyAsync(h.data(), f->amax, sizeof(unsigned) * f->n_amax, cudaMemcpyDeviceToHost,
                                   f->eng->stream));
    NVISR_TRY_CUDA(cudaStreamSynchronize(f->eng->stream));
    for (int i = 0; i < f->n_amax; ++i) {
        float a;
        memcpy(&a, &h[i], 4);
        f->act_scale[i] = a > 0.f ? a / 448.f : 1.f;
    }
    f->calibrated = true;
    return NVISR_OK;
}

// Computes output o into f->out_rgb[output_slot(o)].
nvisr_status compute_output(nvisr_filter *f, int64_t o) {
    std::vector<int64_t> idx;
    if (f->net.family == "group") {
        RunLoc loc;
        if (!group_locate(f, o, &loc)) return NVISR_AGAIN;
        if (loc.pass) return NVISR_OK;                   // an input frame: nothing to compute
        if (f->cached_run == loc.key) return NVISR_OK;  // an earlier output of the same run computed it
        nvisr_status s = forward_group(f, loc.inputs);
        if (s == NVISR_OK) f->cached_run = loc.key;
        return s;
    }
    if (!tuple_ready(f, o, &idx)) return NVISR_AGAIN;
    if (f->precision == NVISR_PREC_FP8 && !f->calibrated && f->n_amax > 0) {
        nvisr_status s = calibrate(f);
        if (s != NVISR_OK) return s;
    }
    f->rq_o = o;
    f->rq_done[o & 1] = -1;
    const nvisr_status s = forward_tuple(f, idx, false);
    f->rq_o = -1;
    return s;
}

// Where output o's planes come from: network output slot `slot`, or input frame
// `frame` passed through (group family, Interpolation without Double frame).
struct OutSrc {
    int slot = 0;
    int64_t frame = -1;
};

OutSrc output_source(const nvisr_filter *f, int64_t o) {
    OutSrc r;
    if (f->net.family != "group") return r;
    RunLoc loc;
    if (!group_locate(f, o, &loc)) return r;
    if (loc.pass) r.frame = loc.frame;
    else r.slot = loc.k;
    return r;
}

const void *raw_plane(const nvisr_filter *f, int64_t frame, int p) {
    return (const uint8_t *)f->raw[p] + (frame % f->ring) * f->raw_slot_bytes[p];
}

// Writes output `src` into the caller's device planes, or into the current
// staging buffer followed by its D2H copy (and the error word's) on the copy
// stream; write_output_end waits for those copies.  A network output is
// requantised (with its skip); a passed-through input frame is copied from its
// raw planes, or requantised from its ring slot into the output format.
nvisr_status write_output_begin(nvisr_filter *f, nvisr_planes *out, OutSrc src, int64_t o) {
    cudaStream_t st = f->eng->stream;
    const nvisr_format &of = f->out_fmt;
    const int b = (int)(o & 1);
    void *dst[3];
    int64_t pitch[3];
    for (int p = 0; p < 3; ++p) {
        dst[p] = out->on_device ? out->data[p] : f->ostage[b][p];
        pitch[p] = out->on_device ? out->pitch[p] : f->ostage_pitch[p];
    }
    if (out->on_device && f->rq_direct_done == o) {
        // the output layer requantised output o into these planes already
        f->rq_direct_done = -1;
        return NVISR_OK;
    }
    if (f->rq_done[b] == o) {
        // the output layer requantised output o into staging buffer b already
        if (out->on_device) {
            prof_gap(f);
            for (int p = 0; p < 3; ++p)
                NVISR_TRY_CUDA(cudaMemcpy2DAsync(dst[p], pitch[p], f->ostage[b][p], f->ostage_pitch[p],
                                                 plane_row_bytes(of, p), plane_rows(of, p), cudaMemcpyDeviceToDevice,
                                                 st));
        }
    } else if (src.frame >= 0 && f->pass_copy) {
        prof_gap(f);
        for (int p = 0; p < 3; ++p)
            NVISR_TRY_CUDA(cudaMemcpy2DAsync(dst[p], pitch[p], raw_plane(f, src.frame, p), f->stage_pitch[p],
                                             plane_row_bytes(of, p), plane_rows(of, p), cudaMemcpyDeviceToDevice, st));
    } else {
        cudaError_t e;
        SkipArgs none{};
        const bool pass = src.frame >= 0;
        {
            ProfScope ps(f, NVISR_K_REQUANT);
            e = launch_requant(of, pass ? ring_slot(f, src.frame) : f->out_rgb[src.slot],
                               pass ? f->rpitch : f->opitch, dst[0], pitch[0], dst[1], pitch[1], dst[2], pitch[2], st,
                               pass ? &none : &f->skip[src.slot], f->net.yuv ? 1 : 0);
        }
        if (e != cudaSuccess) return cuda_status(e, "requant");
    }
    if (out->on_device) return NVISR_OK;
    cudaStream_t cs = f->eng->copy_stream;
    NVISR_TRY_CUDA(cudaEventRecord(f->ev_req, st));
    NVISR_TRY_CUDA(cudaStreamWaitEvent(cs, f->ev_req, 0));
    for (int p = 0; p < 3; ++p)
        NVISR_TRY_CUDA(cudaMemcpy2DAsync(out->data[p], out->pitch[p], f->ostage[b][p], f->ostage_pitch[p],
                                         plane_row_bytes(of, p), plane_rows(of, p), cudaMemcpyDeviceToHost, cs));
    NVISR_TRY_CUDA(cudaMemcpyAsync(f->eng->err_host, f->eng->err_word, sizeof(int), cudaMemcpyDeviceToHost, cs));
    NVISR_TRY_CUDA(cudaEventRecord(f->ev_d2h, cs));
    return NVISR_OK;
}

nvisr_status write_output_end(nvisr_filter *f) {
    NVISR_TRY_CUDA(cudaEventSynchronize(f->ev_d2h));
    const int h = *f->eng->err_host;
    if (h != 0) {
        // the error word is the engine's: outputs computed ahead (read-ahead, engine or batch
        // steps, a cached group run) may come from the failed launches too, so they are
        // dropped and computed again; the word is cleared once the stream is idle
        nvisr_engine *e = f->eng;
        cudaStreamSynchronize(e->stream);
        cudaMemsetAsync(e->err_word, 0, sizeof(int), e->stream);
        cudaStreamSynchronize(e->stream);
        for (nvisr_filter *g : e->filters) {
            g->produced.clear();
            g->cached_run = -1;
            g->xc_tag[0] = g->xc_tag[1] = -1;
        }
        prof_gap(f);
        return fail(NVISR_DEVICE_TIMEOUT, "a device-side wait exceeded its time bound (error word " +
                                              std::to_string(h) + ")");
    }
    return NVISR_OK;
}

}  // namespace

// ==================================================================== batched stepping

struct nvisr_batch {
    nvisr_engine *eng = nullptr;
    std::vector<nvisr_filter *> members;
    bool shared = false;  // every member runs one tuple network on the tensor cores
    struct Plan {
        std::vector<int> parts;                       // participating members
        PackArgs *pack_dev = nullptr;                 // per-step pack table (device)
        std::vector<RowProblem *> tab_host, tab_dev;  // per step: shared-launch table, or null
        // per step starting a residual block: the shared fused launch's table (steps si, si + 1), or null
        std::vector<BlockProblem *> btab_host, btab_dev;
        int rps = 0;                                  // rows per strip chosen by the autotuner
        cudaGraphExec_t exec = nullptr;
        bool no_graph = false;                        // capture failed: launch directly
        uint64_t last_use = 0;
    };
    std::vector<Plan> plans;
    uint64_t tick = 0;
    int graphs = 0;
};

namespace {

constexpr int kMaxPlans = 4;

void free_plan(nvisr_batch::Plan &p) {
    if (p.exec) cudaGraphExecDestroy(p.exec);
    if (p.pack_dev) cudaFree(p.pack_dev);
    for (RowProblem *t : p.tab_host)
        if (t) cudaFreeHost(t);
    for (BlockProblem *t : p.btab_host)
        if (t) cudaFreeHost(t);
    for (BlockProblem *t : p.btab_dev)
        if (t) cudaFree(t);
    for (RowProblem *t : p.tab_dev)
        if (t) cudaFree(t);
    p = nvisr_batch::Plan{};
}

// Batched tuple members must share the weight blob; launches use member 0's weights.
bool batchable(const nvisr_filter *f) {
    return f->net.family == "tuple" && f->tc && f->precision != NVISR_PREC_FP8 && !f->plain_final;
}

// Conv arguments of step si for a participant, with the (identical) weights of member 0.
ConvArgs member_args(nvisr_batch *b, nvisr_filter *f, size_t si, const float *const *frames) {
    int kind;
    ConvArgs a = conv_args(f, f->steps[si], frames, false, &kind);
    const nvisr_filter *f0 = b->members[0];
    const Step &s0 = f0->steps[si];
    const Weights &W0 = s0.widx >= 0 ? f0->wvar[s0.widx] : f0->weights[s0.layer];
    a.w = W0.simt_or_tc;
    a.w_rows = W0.rows;
    a.bias = W0.bias;
    return a;
}

struct PartFrames {
    std::vector<std::vector<const float *>> frames;  // per participant: the tuple's ring slots
};

// Enqueues one batched forward: the packs, then per layer one shared launch
// (row kernel over every participant's image) or per-participant launches.
nvisr_status enqueue_forward(nvisr_batch *b, nvisr_batch::Plan &P, const std::vector<PackArgs> &pack_host,
                             const PartFrames &pf, cudaStream_t st) {
    const int n = (int)P.parts.size();
    cudaError_t e = launch_pack_table(pack_host.data(), P.pack_dev, n, st);
    if (e != cudaSuccess) return cuda_status(e, "batched pack");
    std::vector<ConvArgs> args(n), args2(n);
    const size_t nsteps = b->members[0]->steps.size();
    for (size_t si = 0; si < nsteps; ++si) {
        for (int i = 0; i < n; ++i) args[i] = member_args(b, b->members[P.parts[i]], si, pf.frames[i].data());
        if (P.btab_host[si]) {
            // a residual block (steps si, si + 1) over every participant's image in one launch
            for (int i = 0; i < n; ++i) args2[i] = member_args(b, b->members[P.parts[i]], si + 1, pf.frames[i].data());
            e = launch_res_block_multi(args.data(), args2.data(), n, P.btab_host[si], P.btab_dev[si], st, false, true);
            if (e != cudaSuccess) return cuda_status(e, "batched residual block");
            ++si;
            continue;
        }
        if (P.tab_host[si]) {
            e = launch_conv_rows_multi(args.data(), n, P.tab_host[si], P.tab_dev[si], P.rps, st, false, true);
            if (e != cudaSuccess) return cuda_status(e, "batched conv");
            continue;
        }
        for (int i = 0; i < n; ++i) {
            e = launch_conv_tc(args[i], st);
            if (e != cudaSuccess) return cuda_status(e, "batched conv (per member)");
        }
    }
    return NVISR_OK;
}

// Autotuner: rows per strip of the shared 64 -> 64 launches, chosen by timing
// candidate heights on one layer of this participant set (the layer is
// recomputed in place; its output is rewritten by the real forward).
int tune_rps(nvisr_batch *b, nvisr_batch::Plan &P, const PartFrames &pf, cudaStream_t st) {
    const int n = (int)P.parts.size();
    size_t probe = SIZE_MAX;
    int maxh = 0;
    for (size_t si = 0; si < P.tab_host.size(); ++si)
        if (P.tab_host[si] && probe == SIZE_MAX) probe = si;
    if (probe == SIZE_MAX) return 64;
    std::vector<ConvArgs> args(n);
    for (int i = 0; i < n; ++i) {
        args[i] = member_args(b, b->members[P.parts[i]], probe, pf.frames[i].data());
        maxh = std::max(maxh, args[i].H);
    }
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    int best = 64;
    float best_ms = 1e30f;
    for (int rps : {16, 24, 32, 48, 64, 96, 128, 192}) {
        if (rps > 2 * maxh && rps != 16) continue;
        if (launch_conv_rows_multi(args.data(), n, P.tab_host[probe], P.tab_dev[probe], rps, st, true, true) !=
            cudaSuccess)
            continue;
        cudaEventRecord(e0, st);
        for (int r = 0; r < 3; ++r)
            launch_conv_rows_multi(args.data(), n, P.tab_host[probe], P.tab_dev[probe], rps, st, false, true);
        cudaEventRecord(e1, st);
        if (cudaEventSynchronize(e1) != cudaSuccess) break;
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (ms < best_ms) {
            best_ms = ms;
            best = rps;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return best;
}

nvisr_status build_batch_plan(nvisr_batch *b, nvisr_batch::Plan &P, const PartFrames &pf, cudaStream_t st) {
    const int n = (int)P.parts.size();
    NVISR_TRY_CUDA(cudaMalloc(&P.pack_dev, sizeof(PackArgs) * n));
    const size_t nsteps = b->members[0]->steps.size();
    P.tab_host.assign(nsteps, nullptr);
    P.tab_dev.assign(nsteps, nullptr);
    P.btab_host.assign(nsteps, nullptr);
    P.btab_dev.assign(nsteps, nullptr);
    std::vector<ConvArgs> args(n), args2(n);
    // residual blocks every participant runs fused alone: one shared fused launch each
    for (size_t si = 0; si + 1 < nsteps; ++si) {
        bool blk = true;
        for (int i = 0; i < n && blk; ++i) {
            nvisr_filter *f = b->members[P.parts[i]];
            blk = f->blk[si] != 0;
            if (blk) {
                args[i] = member_args(b, f, si, pf.frames[i].data());
                args2[i] = member_args(b, f, si + 1, pf.frames[i].data());
                blk = res_block_fits(args[i], args2[i]) && args[i].nimg == 1;
            }
        }
        if (!blk) continue;
        NVISR_TRY_CUDA(cudaMallocHost(&P.btab_host[si], sizeof(BlockProblem) * n));
        NVISR_TRY_CUDA(cudaMalloc(&P.btab_dev[si], sizeof(BlockProblem) * n));
        cudaError_t e = launch_res_block_multi(args.data(), args2.data(), n, P.btab_host[si], P.btab_dev[si], st,
                                               true, false);
        if (e != cudaSuccess) return cuda_status(e, "batched residual block table");
        ++si;
    }
    for (size_t si = 0; si < nsteps; ++si) {
        const bool in_block = P.btab_host[si] || (si > 0 && P.btab_host[si - 1]);
        bool rows = !in_block && n > 1 && b->members[0]->steps[si].op == OP_CONV;
        for (int i = 0; i < n && rows; ++i) {
            args[i] = member_args(b, b->members[P.parts[i]], si, pf.frames[i].data());
            rows = rows_kernel_fits(args[i]) && !args[i].y2 && !args[i].amax;
        }
        if (!rows) continue;
        NVISR_TRY_CUDA(cudaMallocHost(&P.tab_host[si], sizeof(RowProblem) * n));
        NVISR_TRY_CUDA(cudaMalloc(&P.tab_dev[si], sizeof(RowProblem) * n));
    }
    P.rps = tune_rps(b, P, pf, st);
    for (size_t si = 0; si < nsteps; ++si) {
        if (!P.tab_host[si]) continue;
        for (int i = 0; i < n; ++i) args[i] = member_args(b, b->members[P.parts[i]], si, pf.frames[i].data());
        cudaError_t e = launch_conv_rows_multi(args.data(), n, P.tab_host[si], P.tab_dev[si], P.rps, st, true, false);
        if (e != cudaSuccess) return cuda_status(e, "batched conv table");
    }
    NVISR_TRY_CUDA(cudaStreamSynchronize(st));  // tables are in place before any capture
    return NVISR_OK;
}

}  // namespace

// ==================================================================== C ABI

extern "C" {

int32_t nvisr_abi_version(void) { return NVISR_ABI_VERSION; }

const char *nvisr_build_info(void) {
    return "nvisr sm_103a (tcgen05/TMA tensor-core conv, FP32 SIMT conv, ingest, requantise)";
}

const char *nvisr_status_string(nvisr_status s) {
    switch (s) {
        case NVISR_OK: return "OK";
        case NVISR_AGAIN: return "AGAIN";
        case NVISR_FULL: return "FULL";
        case NVISR_EOS: return "EOS";
        case NVISR_INVALID_ARG: return "INVALID_ARG";
        case NVISR_UNSUPPORTED_FORMAT: return "UNSUPPORTED_FORMAT";
        case NVISR_OUT_OF_MEMORY: return "OUT_OF_MEMORY";
        case NVISR_OVER_BUDGET: return "OVER_BUDGET";
        case NVISR_CUDA_ERROR: return "CUDA_ERROR";
        case NVISR_DEVICE_TIMEOUT: return "DEVICE_TIMEOUT";
        case NVISR_BAD_NETWORK: return "BAD_NETWORK";
        case NVISR_INTERNAL: return "INTERNAL";
    }
    return "UNKNOWN";
}

const char *nvisr_last_error(nvisr_engine *e) { return e ? e->last_error.c_str() : g_last_error.c_str(); }

nvisr_status nvisr_network_check(const char *text, int64_t weights_count) {
    NetDesc net;
    std::string err;
    if (!parse_netdesc(text, weights_count, &net, &err)) return fail(NVISR_BAD_NETWORK, err);
    return NVISR_OK;
}

nvisr_status nvisr_engine_create(const nvisr_engine_desc *desc, nvisr_engine **out) {
    if (!desc || !out) return fail(NVISR_INVALID_ARG, "engine_create: NULL argument");
    *out = nullptr;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) {
        cudaGetLastError();
        return fail(NVISR_CUDA_ERROR, "no CUDA device");
    }
    if (desc->device < 0 || desc->device >= ndev) return fail(NVISR_INVALID_ARG, "bad device ordinal");
    NVISR_TRY_CUDA(cudaSetDevice(desc->device));
    auto *e = new nvisr_engine();
    e->device = desc->device;
    e->max_filters = desc->max_filters;
    e->budget = desc->hbm_budget_bytes;
    if (desc->stream) {
        e->stream = (cudaStream_t)desc->stream;
    } else {
        if (cudaStreamCreateWithFlags(&e->stream, cudaStreamNonBlocking) != cudaSuccess) {
            delete e;
            return fail(NVISR_CUDA_ERROR, "cudaStreamCreate failed");
        }
        e->own_stream = true;
    }
    if (cudaMalloc(&e->err_word, sizeof(int)) != cudaSuccess || cudaMemset(e->err_word, 0, sizeof(int)) != cudaSuccess ||
        cudaHostAlloc(&e->err_host, sizeof(int), cudaHostAllocDefault) != cudaSuccess ||
        cudaStreamCreateWithFlags(&e->copy_stream, cudaStreamNonBlocking) != cudaSuccess) {
        cudaFree(e->err_word);
        if (e->err_host) cudaFreeHost(e->err_host);
        if (e->own_stream) cudaStreamDestroy(e->stream);
        delete e;
        return fail(NVISR_OUT_OF_MEMORY, "error word or copy stream allocation failed");
    }
    *e->err_host = 0;
    *out = e;
    return NVISR_OK;
}

void nvisr_filter_destroy(nvisr_filter *f) {
    if (!f) return;
    nvisr_engine *e = f->eng;
    cudaSetDevice(e->device);
    cudaStreamSynchronize(e->stream);
    cudaStreamSynchronize(e->copy_stream);
    flush_profile(f);
    for (cudaEvent_t ev : f->ev_pool) cudaEventDestroy(ev);
    for (cudaEvent_t ev : {f->ev_h2d, f->ev_stage, f->ev_req, f->ev_d2h})
        if (ev) cudaEventDestroy(ev);
    for (DevBuf &b : f->owned) {
        cudaFree(b.ptr);
        e->used -= (int64_t)b.bytes;
    }
    e->filters.erase(std::remove(e->filters.begin(), e->filters.end(), f), e->filters.end());
    delete f;
}

void nvisr_engine_destroy(nvisr_engine *e) {
    if (!e) return;
    while (!e->filters.empty()) nvisr_filter_destroy(e->filters.back());
    cudaSetDevice(e->device);
    cudaStreamSynchronize(e->stream);
    cudaStreamSynchronize(e->copy_stream);
    cudaFree(e->err_word);
    cudaFreeHost(e->err_host);
    if (e->own_stream) cudaStreamDestroy(e->stream);
    cudaStreamDestroy(e->copy_stream);
    delete e;
}

void *nvisr_engine_stream(nvisr_engine *e) { return e ? (void *)e->stream : nullptr; }

int64_t nvisr_engine_bytes_in_use(nvisr_engine *e) { return e ? e->used : 0; }

nvisr_status nvisr_filter_create(nvisr_engine *e, const nvisr_filter_desc *d, nvisr_filter **out) {
    ErrScope es(e);
    if (!e || !d || !out) return fail(NVISR_INVALID_ARG, "filter_create: NULL argument");
    *out = nullptr;
    if (e->max_filters > 0 && (int)e->filters.size() >= e->max_filters)
        return fail(NVISR_OVER_BUDGET, "engine already holds max_filters filters");
    if (!d->weights && d->weights_count > 0) return fail(NVISR_INVALID_ARG, "weights NULL");
    if (d->precision < NVISR_PREC_FP32 || d->precision > NVISR_PREC_FP8)
        return fail(NVISR_INVALID_ARG, "unknown precision");
    if (!fmt_ok(d->in_fmt) || !fmt_ok(d->out_fmt)) return fail(NVISR_UNSUPPORTED_FORMAT, "unsupported pixel format");
    std::unique_ptr<nvisr_filter> f(new nvisr_filter());
    std::string err;
    if (!parse_netdesc(d->network_text, d->weights_count, &f->net, &err)) return fail(NVISR_BAD_NETWORK, err);
    if (f->net.yuv && (d->in_fmt.matrix == NVISR_MATRIX_RGB || d->out_fmt.matrix == NVISR_MATRIX_RGB))
        return fail(NVISR_UNSUPPORTED_FORMAT, "a YUV-domain network takes and gives Y'CbCr planes, not RGB");
    if (f->net.yuv && (d->in_fmt.transfer != NVISR_TRANSFER_NONE || d->out_fmt.transfer != NVISR_TRANSFER_NONE))
        return fail(NVISR_UNSUPPORTED_FORMAT, "a YUV-domain network sees the coded signal (no transfer)");
    const NetDesc &net = f->net;
    if (d->scale_w != net.scale || d->scale_h != net.scale_y)
        return fail(NVISR_INVALID_ARG, "scale does not match the network description");
    if (d->out_fmt.width != d->in_fmt.width * net.scale || d->out_fmt.height != d->in_fmt.height * net.scale_y)
        return fail(NVISR_INVALID_ARG, "output size must be scale x input size");
    if (net.align != 1) return fail(NVISR_UNSUPPORTED_FORMAT, "network stride alignment > 1 is not supported");
    if (net.family == "tuple" && (net.frames % 2 == 0 || net.frames > 8))
        return fail(NVISR_UNSUPPORTED_FORMAT, "tuple networks need an odd frame count <= 7");
    cudaSetDevice(e->device);
    f->eng = e;
    f->in_fmt = d->in_fmt;
    f->out_fmt = d->out_fmt;
    f->precision = d->precision;
    f->tc = d->precision != NVISR_PREC_FP32;
    f->act_dt = d->precision == NVISR_PREC_FP32 ? DT_F32 : (d->precision == NVISR_PREC_FP16 ? DT_F16 : DT_BF16);
    f->calib_frames = d->calib_frames > 0 ? d->calib_frames : 4;
    f->net_text = d->network_text;
    f->blob_count = d->weights_count;
    {
        uint64_t h = 1469598103934665603ull;  // FNV-1a over the blob bytes
        const uint8_t *b = reinterpret_cast<const uint8_t *>(d->weights);
        for (int64_t i = 0; i < d->weights_count * 4; ++i) h = (h ^ b[i]) * 1099511628211ull;
        f->blob_hash = h;
    }
    const int H = d->in_fmt.height, W = d->in_fmt.width;
    nvisr_status s;
    auto cleanup = [&](nvisr_status st) {
        for (DevBuf &b : f->owned) {
            cudaFree(b.ptr);
            e->used -= (int64_t)b.bytes;
        }
        f->owned.clear();
        return st;
    };
    f->guard = (d->options & NVISR_OPT_GUARD_BANDS) ? GUARD_BYTES : 0;
    // ring of ingested frames
    // ring: a tuple, or a group run plus the frames a recycled last run may reach back to
    f->ring = net.family == "group" ? 2 * net.frames + 2 : net.frames + 2;
    f->run_out = net.family == "group" ? (net.dbl ? 2 : 1) * (net.frames - (net.extra ? 1 : 0)) : 1;
    if (f->run_out < 1 || f->run_out > 8)
        return cleanup(fail(NVISR_UNSUPPORTED_FORMAT, "group networks: 1 to 8 outputs per run"));
    f->rpitch = round_up64(W, 4);
    f->slot_floats = 3 * f->rpitch * H;
    void *p;
    if ((s = dalloc(e, sizeof(float) * f->slot_floats * f->ring, f->owned, &p, f->guard)) != NVISR_OK) return cleanup(s);
    f->ring_base = (float *)p;
    for (int pl = 0; pl < 3; ++pl) {
        int rows;
        const int64_t bytes = plane_bytes(d->in_fmt, pl, &f->stage_pitch[pl], &rows);
        if ((s = dalloc(e, bytes, f->owned, &f->stage[pl], f->guard)) != NVISR_OK) return cleanup(s);
        const int64_t obytes = plane_bytes(d->out_fmt, pl, &f->ostage_pitch[pl], &rows);
        for (int b = 0; b < 2; ++b)
            if ((s = dalloc(e, obytes, f->owned, &f->ostage[b][pl], f->guard)) != NVISR_OK) return cleanup(s);
    }
    for (cudaEvent_t *ev : {&f->ev_h2d, &f->ev_stage, &f->ev_req, &f->ev_d2h})
        if (cudaEventCreateWithFlags(ev, cudaEventDisableTiming) != cudaSuccess)
            return cleanup(fail(NVISR_CUDA_ERROR, "cudaEventCreate failed"));
    f->passthru = net.family == "group" && net.interp && !net.dbl;
    f->pass_copy = f->passthru && memcmp(&d->in_fmt, &d->out_fmt, sizeof(nvisr_format)) == 0;
    if (f->pass_copy)
        for (int pl = 0; pl < 3; ++pl) {
            int rows;
            int64_t pitch;
            f->raw_slot_bytes[pl] = plane_bytes(d->in_fmt, pl, &pitch, &rows);
            if ((s = dalloc(e, (size_t)f->raw_slot_bytes[pl] * f->ring, f->owned, &f->raw[pl], f->guard)) != NVISR_OK)
                return cleanup(s);
        }
    f->opitch = round_up64((int64_t)W * net.scale, 4);
    for (int k = 0; k < f->run_out; ++k) {
        if ((s = dalloc(e, sizeof(float) * 3 * f->opitch * H * net.scale_y, f->owned, &p, f->guard)) != NVISR_OK)
            return cleanup(s);
        f->out_rgb[k] = (float *)p;
    }
    if ((s = prepare_weights(f.get(), d->weights)) != NVISR_OK) return cleanup(s);
    if ((s = (net.family == "group" ? build_plan_group(f.get(), d->weights) : build_plan(f.get()))) != NVISR_OK)
        return cleanup(s);
    if (f->plain_final) {
        if ((s = dalloc(e, sizeof(float) * 16 * (size_t)H * W, f->owned, &p, f->guard)) != NVISR_OK) return cleanup(s);
        f->final_f32 = (float *)p;
    }
    // requantise fused into a 2 x 2 shuffle output layer of 64 input channels (the row
    // kernel's shuffle tail): tensor-core tuple networks with an RGB domain, no transfer,
    // a bilinear skip of the centre frame or none
    f->options = d->options;
    plan_blocks(f.get());
    if (net.family == "tuple" && f->tc && !(d->options & NVISR_OPT_UNFUSED_OUTPUT) &&
        (net.skip == 0 || net.skip == 2) && !f->steps.empty()) {
        const Step &last = f->steps.back();
        const NetLayer &L = net.layers[last.layer];
        FusedRq rq{};
        if (last.op == OP_CONV && last.out_t < 0 && !last.plain && L.cin == 64 && L.cout == 12 && L.ps == 2 &&
            L.k == 3 && last.skip_frames.size() == 1 && fused_rq_format(d->out_fmt, net.yuv, &rq)) {
            f->fused_rq = true;
            f->rq_base = rq;
            const int tiles = (W + 127) / 128;
            if (rq.sub420 && rq.loc == NVISR_CHROMA_LEFT && tiles > 1) {
                if ((s = dalloc(e, sizeof(float) * 6 * (size_t)H * tiles, f->owned, &p, f->guard)) != NVISR_OK)
                    return cleanup(s);
                f->rq_edge = (float *)p;
            }
        }
    }
    e->filters.push_back(f.get());
    *out = f.release();
    return NVISR_OK;
}

nvisr_status nvisr_push(nvisr_filter *f, const nvisr_planes *in, uint32_t flags) {
    ErrScope es(f ? f->eng : nullptr);
    if (!f || !in) return fail(NVISR_INVALID_ARG, "push: NULL argument");
    if (f->eos) return fail(NVISR_EOS, "push after flush");
    for (int p = 0; p < 3; ++p)
        if (!in->data[p] || in->pitch[p] < plane_row_bytes(f->in_fmt, p))
            return fail(NVISR_INVALID_ARG, "push: plane " + std::to_string(p) + " NULL or pitch too small");
    // the slot overwritten by this frame must not be needed by a pending output
    int64_t oldest_needed;
    if (f->net.family == "tuple") {
        oldest_needed = f->next_out - (f->net.frames - 1) / 2;
    } else {
        RunLoc loc;
        group_locate(f, f->next_out, &loc);
        oldest_needed = loc.oldest;
    }
    if (f->pushed - f->ring >= std::max<int64_t>(oldest_needed, 0) && f->pushed >= f->ring)
        return NVISR_FULL;
    cudaSetDevice(f->eng->device);
    cudaStream_t st = f->eng->stream;
    const void *src[3];
    int64_t pitch[3];
    if (!in->on_device) {
        // host planes go through the staging planes on the copy stream, once the previous
        // frame's ingest has read them; the compute stream waits for the copy
        cudaStream_t cs = f->eng->copy_stream;
        if (f->stage_used) NVISR_TRY_CUDA(cudaEventSynchronize(f->ev_stage));
        for (int p = 0; p < 3; ++p)
            NVISR_TRY_CUDA(cudaMemcpy2DAsync(f->stage[p], f->stage_pitch[p], in->data[p], in->pitch[p],
                                             plane_row_bytes(f->in_fmt, p), plane_rows(f->in_fmt, p),
                                             cudaMemcpyHostToDevice, cs));
        NVISR_TRY_CUDA(cudaEventRecord(f->ev_h2d, cs));
        NVISR_TRY_CUDA(cudaStreamWaitEvent(st, f->ev_h2d, 0));
        prof_gap(f);
    }
    for (int p = 0; p < 3; ++p) {
        src[p] = in->on_device ? in->data[p] : f->stage[p];
        pitch[p] = in->on_device ? in->pitch[p] : f->stage_pitch[p];
    }
    cudaError_t e;
    {
        ProfScope ps(f, NVISR_K_INGEST);
        e = launch_ingest(f->in_fmt, src[0], pitch[0], src[1], pitch[1], src[2], pitch[2], ring_slot(f, f->pushed),
                          f->rpitch, st, f->net.yuv ? 1 : 0);
    }
    if (e != cudaSuccess) return cuda_status(e, "ingest");
    if (f->pass_copy) {
        // the frame's planes, kept for its output as it is (Interpolation without Double frame)
        prof_gap(f);
        for (int p = 0; p < 3; ++p)
            NVISR_TRY_CUDA(cudaMemcpy2DAsync((uint8_t *)f->raw[p] + (f->pushed % f->ring) * f->raw_slot_bytes[p],
                                             f->stage_pitch[p], src[p], pitch[p], plane_row_bytes(f->in_fmt, p),
                                             plane_rows(f->in_fmt, p), cudaMemcpyDeviceToDevice, st));
    }
    if (!in->on_device) {
        NVISR_TRY_CUDA(cudaEventRecord(f->ev_stage, st));
        f->stage_used = true;
        NVISR_TRY_CUDA(cudaEventSynchronize(f->ev_h2d));  // host planes may be reused on return
    }
    f->cut.push_back((flags & NVISR_FRAME_SCENE_CUT) && f->pushed > 0 ? 1 : 0);
    f->pushed++;
    return NVISR_OK;
}

nvisr_status nvisr_flush(nvisr_filter *f) {
    ErrScope es(f ? f->eng : nullptr);
    if (!f) return fail(NVISR_INVALID_ARG, "flush: NULL filter");
    f->eos = true;
    f->total_out = f->net.family == "group" ? group_total(f) : f->pushed;
    return NVISR_OK;
}

int64_t nvisr_filter_ready(nvisr_filter *f) {
    if (!f) return 0;
    int64_t n = 0;
    const int64_t end = f->eos ? f->total_out : (f->net.family == "group" ? group_total(f) : f->pushed);
    for (int64_t o = f->next_out; o < end && output_ready(f, o); ++o) ++n;
    return n;
}

nvisr_status nvisr_pull(nvisr_filter *f, nvisr_planes *out, nvisr_frame_info *info) {
    ErrScope es(f ? f->eng : nullptr);
    if (!f || !out) return fail(NVISR_INVALID_ARG, "pull: NULL argument");
    for (int p = 0; p < 3; ++p)
        if (!out->data[p] || out->pitch[p] < plane_row_bytes(f->out_fmt, p))
            return fail(NVISR_INVALID_ARG, "pull: plane " + std::to_string(p) + " NULL or pitch too small");
    if (f->eos && f->next_out >= f->total_out) return NVISR_EOS;
    const int64_t o = f->next_out;
    if (!output_ready(f, o)) return NVISR_AGAIN;
    cudaSetDevice(f->eng->device);
    nvisr_status s;
    bool have = !f->produced.empty() && f->produced.front() == o;
    if (!have) {
        // computed here: a fused output layer may write the caller's device planes itself
        // (the 16-bit luma stores take 4-byte aligned rows, the chroma ones 2-byte)
        const bool wide = f->out_fmt.bit_depth > 8;
        const int64_t ya = wide ? 4 : 2;
        const int64_t ca = f->out_fmt.subsampling == NVISR_SUB_444 ? ya : (wide ? 2 : 1);  // 4:4:4 chroma: pairs
        const bool direct = f->fused_rq && out->on_device && !f->batched &&
                            (uintptr_t)out->data[0] % ya == 0 && out->pitch[0] % ya == 0 &&
                            (uintptr_t)out->data[1] % ca == 0 && out->pitch[1] % ca == 0 &&
                            (uintptr_t)out->data[2] % ca == 0 && out->pitch[2] % ca == 0;
        f->rq_direct = direct ? out : nullptr;
        f->rq_direct_done = -1;
        s = compute_output(f, o);
        f->rq_direct = nullptr;
        if (s != NVISR_OK) return s;
    } else {
        f->produced.pop_front();
    }
    if ((s = write_output_begin(f, out, output_source(f, o), o)) != NVISR_OK) return s;
    if (!out->on_device) {
        // read-ahead: the next output's network runs on the compute stream while this
        // output's planes are copied out
        const int64_t n = o + 1;
        if (!f->batched && f->produced.empty() && !(f->eos && n >= f->total_out) && output_ready(f, n) &&
            compute_output(f, n) == NVISR_OK)
            f->produced.push_back(n);
        if ((s = write_output_end(f)) != NVISR_OK) return s;
    }
    if (info) {
        std::vector<int64_t> idx;
        int kind = NVISR_OUT_NETWORK;
        if (f->net.family == "group") {
            RunLoc loc;
            group_locate(f, o, &loc);
            idx = loc.inputs;
            if (loc.pass) {
                idx.assign(1, loc.frame);
                kind = NVISR_OUT_PASSTHROUGH;
            }
        }
        else tuple_ready(f, o, &idx);
        int scene = 0;
        for (int64_t k = 1; k <= idx.front(); ++k) scene += f->cut[(size_t)k];
        info->index = o;
        info->src_first = idx.front();
        info->src_last = idx.back();
        info->scene = scene;
        info->kind = kind;
    }
    f->next_out++;
    return NVISR_OK;
}

nvisr_status nvisr_filter_check_guards(nvisr_filter *f, int32_t *bad) {
    ErrScope es(f ? f->eng : nullptr);
    if (!f || !bad) return fail(NVISR_INVALID_ARG, "check_guards: NULL argument");
    *bad = 0;
    if (!f->guard) return fail(NVISR_INVALID_ARG, "check_guards: the filter was created without NVISR_OPT_GUARD_BANDS");
    NVISR_TRY_CUDA(cudaSetDevice(f->eng->device));
    NVISR_TRY_CUDA(cudaStreamSynchronize(f->eng->stream));
    NVISR_TRY_CUDA(cudaStreamSynchronize(f->eng->copy_stream));
    std::vector<unsigned char> band;
    std::string first;
    for (size_t i = 0; i < f->owned.size(); ++i) {
        const DevBuf &b = f->owned[i];
        if (!b.guard) continue;
        const uint8_t *base = static_cast<const uint8_t *>(b.ptr);
        const size_t after = b.bytes - b.guard - b.user;  // the post band runs to the allocation's end
        bool ok = true;
        for (int side = 0; side < 2 && ok; ++side) {
            const size_t n = side ? after : b.guard;
            band.resize(n);
            NVISR_TRY_CUDA(cudaMemcpy(band.data(), side ? base + b.guard + b.user : base, n, cudaMemcpyDeviceToHost));
            for (size_t j = 0; j < n; ++j)
                if (band[j] != GUARD_FILL) {
                    ok = false;
                    if (first.empty())
                        first = "buffer " + std::to_string(i) + " (" + std::to_string(b.user) + " bytes): " +
                                (side ? "byte " + std::to_string(j) + " after its end"
                                      : "byte " + std::to_string(b.guard - j) + " before its start");
                    break;
                }
        }
        if (!ok) ++*bad;
    }
    if (*bad) return fail(NVISR_CUDA_ERROR, "guard bands overwritten in " + std::to_string(*bad) + " buffer(s); first: " + first);
    return NVISR_OK;
}

nvisr_status nvisr_test_poke_guard(nvisr_filter *f, int32_t index) {
    ErrScope es(f ? f->eng : nullptr);
    if (!f || !f->guard) return fail(NVISR_INVALID_ARG, "poke_guard: no filter with guard bands");
    int32_t k = -1;
    for (size_t i = 0; i < f->owned.size(); ++i) {
        const DevBuf &b = f->owned[i];
        if (b.guard && ++k == index) {
            NVISR_TRY_CUDA(cudaSetDevice(f->eng->device));
            NVISR_TRY_CUDA(cudaStreamSynchronize(f->eng->stream));
            NVISR_TRY_CUDA(cudaMemset(static_cast<uint8_t *>(b.ptr) + b.guard + b.user, 0, 1));
            return NVISR_OK;
        }
    }
    return fail(NVISR_INVALID_ARG, "poke_guard: no such buffer");
}

nvisr_status nvisr_filter_cache_stats(nvisr_filter *f, int64_t *hits, int64_t *misses) {
    if (!f || !hits || !misses) return fail(NVISR_INVALID_ARG, "cache_stats: NULL argument");
    *hits = f->xc_hits;
    *misses = f->xc_misses;
    return NVISR_OK;
}

nvisr_status nvisr_filter_profile(nvisr_filter *f, int32_t enable) {
    ErrScope es(f ? f->eng : nullptr);
    if (!f) return fail(NVISR_INVALID_ARG, "profile: NULL filter");
    flush_profile(f);
    if (enable) {
        for (int k = 0; k < NVISR_K_COUNT; ++k) {
            f->prof_ms[k] = 0;
            f->prof_n[k] = 0;
        }
    }
    f->prof = enable != 0;
    return NVISR_OK;
}

nvisr_status nvisr_filter_profile_read(nvisr_filter *f, nvisr_profile *out) {
    ErrScope es(f ? f->eng : nullptr);
    if (!f || !out) return fail(NVISR_INVALID_ARG, "profile_read: NULL argument");
    flush_profile(f);
    for (int k = 0; k < NVISR_K_COUNT; ++k) {
        out->ms[k] = f->prof_ms[k];
        out->launches[k] = f->prof_n[k];
    }
    return NVISR_OK;
}

nvisr_status nvisr_engine_step(nvisr_engine *e, int32_t max_outputs, int32_t *produced) {
    ErrScope es(e);
    if (!e) return fail(NVISR_INVALID_ARG, "engine_step: NULL engine");
    int n = 0;
    for (nvisr_filter *f : e->filters) {
        if (n >= max_outputs) break;
        if (!f->produced.empty()) continue;  // one computed output buffered per filter
        const int64_t o = f->next_out;
        if (f->eos && o >= f->total_out) continue;
        if (!output_ready(f, o)) continue;
        nvisr_status s = compute_output(f, o);
        if (s == NVISR_AGAIN) continue;
        if (s != NVISR_OK) return s;
        f->produced.push_back(o);
        ++n;
    }
    if (produced) *produced = n;
    return NVISR_OK;
}

// ---------------------------------------------------------------- batched stepping

nvisr_status nvisr_batch_create(nvisr_engine *e, nvisr_filter *const *filters, int32_t n, nvisr_batch **out) {
    ErrScope es(e);
    if (!e || !filters || n < 1 || !out) return fail(NVISR_INVALID_ARG, "batch_create: bad arguments");
    *out = nullptr;
    std::unique_ptr<nvisr_batch> b(new nvisr_batch());
    b->eng = e;
    for (int i = 0; i < n; ++i) {
        nvisr_filter *f = filters[i];
        if (!f || f->eng != e) return fail(NVISR_INVALID_ARG, "batch_create: filter of another engine or NULL");
        for (nvisr_filter *g : b->members)
            if (g == f) return fail(NVISR_INVALID_ARG, "batch_create: filter listed twice");
        b->members.push_back(f);
    }
    for (nvisr_filter *f : b->members) f->batched = true;  // its outputs are the batch step's
    const nvisr_filter *f0 = b->members[0];
    b->shared = true;
    for (const nvisr_filter *f : b->members)
        b->shared = b->shared && batchable(f) && f->net_text == f0->net_text && f->blob_hash == f0->blob_hash &&
                    f->blob_count == f0->blob_count && f->precision == f0->precision;
    *out = b.release();
    return NVISR_OK;
}

nvisr_status nvisr_batch_step(nvisr_batch *b, int32_t *produced) {
    ErrScope es(b ? b->eng : nullptr);
    if (!b) return fail(NVISR_INVALID_ARG, "batch_step: NULL batch");
    int nprod = 0;
    nvisr_batch::Plan probe;
    PartFrames pf;
    std::vector<int64_t> outs;
    for (int m = 0; m < (int)b->members.size(); ++m) {
        nvisr_filter *f = b->members[m];
        if (!f->produced.empty()) continue;  // one computed output buffered per filter
        const int64_t o = f->next_out;
        if (f->eos && o >= f->total_out) continue;
        if (!output_ready(f, o)) continue;
        if (!b->shared) {
            nvisr_status s = compute_output(f, o);
            if (s == NVISR_AGAIN) continue;
            if (s != NVISR_OK) return s;
            f->produced.push_back(o);
            ++nprod;
            continue;
        }
        std::vector<int64_t> idx;
        if (!tuple_ready(f, o, &idx)) continue;
        std::vector<const float *> fr(8, nullptr);
        for (size_t k = 0; k < idx.size() && k < 8; ++k) fr[k] = ring_slot(f, idx[k]);
        probe.parts.push_back(m);
        pf.frames.push_back(fr);
        outs.push_back(o);
    }
    if (!probe.parts.empty()) {
        cudaStream_t st = b->eng->stream;
        const int n = (int)probe.parts.size();
        std::vector<PackArgs> pack(n);
        for (int i = 0; i < n; ++i) {
            nvisr_filter *f = b->members[probe.parts[i]];
            const Tensor &pk = f->tensors[f->pack_t];
            PackArgs &pa = pack[i];
            pa = PackArgs{};
            pa.nsrc = f->net.frames;
            for (int k = 0; k < pa.nsrc; ++k) pa.src[k] = pf.frames[i][k];
            pa.ch_per_src = 3;
            pa.src_pitch = f->rpitch;
            pa.src_plane = f->rpitch * f->in_fmt.height;
            pa.H = pk.H;
            pa.W = pk.W;
            pa.dst = pk.ptr;
            pa.cpad = pk.cpad;
            pa.dt = pk.dt;
            pa.cpc = pk.cpc ? pk.cpc : chunk_channels(pk.dt);
            pa.scale = 1.f;
            if (!pack_rows_fits(pa)) return fail(NVISR_INTERNAL, "batch_step: tuple pack layout not supported");
            for (const Step &s : f->steps)
                if (s.op == OP_CONV && s.out_t < 0) set_final_skip(f, s, pf.frames[i].data());
        }
        nvisr_batch::Plan *P = nullptr;
        for (nvisr_batch::Plan &q : b->plans)
            if (q.parts == probe.parts) P = &q;
        if (!P) {
            if ((int)b->plans.size() >= kMaxPlans) {
                auto lru = std::min_element(b->plans.begin(), b->plans.end(),
                                            [](const nvisr_batch::Plan &x, const nvisr_batch::Plan &y) {
                                                return x.last_use < y.last_use;
                                            });
                NVISR_TRY_CUDA(cudaStreamSynchronize(st));
                free_plan(*lru);
                b->plans.erase(lru);
            }
            b->plans.emplace_back();
            P = &b->plans.back();
            P->parts = probe.parts;
            nvisr_status s = build_batch_plan(b, *P, pf, st);
            if (s != NVISR_OK) {
                cudaStreamSynchronize(st);
                free_plan(*P);
                b->plans.pop_back();
                return s;
            }
        }
        P->last_use = ++b->tick;
        // pageable source: the runtime copies it out before returning, so the
        // table can be rewritten by the next step at once
        NVISR_TRY_CUDA(cudaMemcpyAsync(P->pack_dev, pack.data(), sizeof(PackArgs) * n, cudaMemcpyHostToDevice, st));
        if (P->exec) {
            NVISR_TRY_CUDA(cudaGraphLaunch(P->exec, st));
        } else {
            nvisr_status s = enqueue_forward(b, *P, pack, pf, st);
            if (s != NVISR_OK) return s;
            // capture the same launch sequence for the next steps of this participant set
            cudaGraph_t g = nullptr;
            if (!P->no_graph && cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal) == cudaSuccess) {
                const nvisr_status cs = enqueue_forward(b, *P, pack, pf, st);
                const cudaError_t ce = cudaStreamEndCapture(st, &g);
                if (cs == NVISR_OK && ce == cudaSuccess && g &&
                    cudaGraphInstantiate(&P->exec, g, 0) == cudaSuccess)
                    ++b->graphs;
                else
                    P->exec = nullptr;
                P->no_graph = P->exec == nullptr;
                if (g) cudaGraphDestroy(g);
                cudaGetLastError();  // a failed capture leaves the uncaptured path in use
            }
        }
        for (int i = 0; i < n; ++i) {
            b->members[probe.parts[i]]->produced.push_back(outs[i]);
            ++nprod;
        }
    }
    if (produced) *produced = nprod;
    return NVISR_OK;
}

nvisr_status nvisr_batch_info(nvisr_batch *b, int32_t *shared, int32_t *graphs, int32_t *rows_per_strip) {
    ErrScope es(b ? b->eng : nullptr);
    if (!b) return fail(NVISR_INVALID_ARG, "batch_info: NULL batch");
    if (shared) *shared = b->shared ? 1 : 0;
    if (graphs) *graphs = b->graphs;
    if (rows_per_strip) {
        int rps = 0;
        uint64_t last = 0;
        for (const nvisr_batch::Plan &q : b->plans)
            if (q.last_use >= last) {
                last = q.last_use;
                rps = q.rps;
            }
        *rows_per_strip = rps;
    }
    return NVISR_OK;
}

void nvisr_batch_destroy(nvisr_batch *b) {
    if (!b) return;
    cudaStreamSynchronize(b->eng->stream);
    for (nvisr_batch::Plan &q : b->plans) free_plan(q);
    delete b;
}

// ---------------------------------------------------------------- stages

nvisr_status nvisr_ingest(const nvisr_format *fmt, const nvisr_planes *in, float *out, int64_t out_pitch,
                          void *stream) {
    if (!fmt || !in || !out || !in->on_device) return fail(NVISR_INVALID_ARG, "ingest: bad arguments");
    if (!fmt_ok(*fmt)) return fail(NVISR_UNSUPPORTED_FORMAT, "ingest: unsupported format");
    if (out_pitch < fmt->width) return fail(NVISR_INVALID_ARG, "ingest: pitch < width");
    cudaError_t e = launch_ingest(*fmt, in->data[0], in->pitch[0], in->data[1], in->pitch[1], in->data[2],
                                  in->pitch[2], out, out_pitch, (cudaStream_t)stream);
    return e == cudaSuccess ? NVISR_OK : cuda_status(e, "ingest");
}

nvisr_status nvisr_requant(const nvisr_format *fmt, const float *in, int64_t in_pitch, nvisr_planes *out,
                           void *stream) {
    if (!fmt || !in || !out || !out->on_device) return fail(NVISR_INVALID_ARG, "requant: bad arguments");
    if (!fmt_ok(*fmt)) return fail(NVISR_UNSUPPORTED_FORMAT, "requant: unsupported format");
    if (in_pitch < fmt->width) return fail(NVISR_INVALID_ARG, "requant: pitch < width");
    cudaError_t e = launch_requant(*fmt, in, in_pitch, out->data[0], out->pitch[0], out->data[1], out->pitch[1],
                                   out->data[2], out->pitch[2], (cudaStream_t)stream);
    return e == cudaSuccess ? NVISR_OK : cuda_status(e, "requant");
}

nvisr_status nvisr_tuple_map(const uint8_t *flags, int32_t nframes, int32_t T, int32_t *out) {
    if (!flags || !out || nframes < 0 || T < 1 || T % 2 == 0) return fail(NVISR_INVALID_ARG, "tuple_map: bad arguments");
    const int r = (T - 1) / 2;
    int s0 = 0;
    for (int t = 0; t < nframes; ++t) {
        if (t > 0 && flags[t]) s0 = t;
        int s1 = t;
        while (s1 + 1 < nframes && !flags[s1 + 1]) ++s1;
        for (int k = 0; k < T; ++k) out[t * T + k] = std::min(std::max(t - r + k, s0), s1);
    }
    return NVISR_OK;
}

nvisr_status nvisr_group_runs(int32_t s0, int32_t s1, int32_t n, int32_t extra, int32_t max_runs,
                              int32_t *out_inputs, int32_t *out_skip, int32_t *out_count, int32_t *nruns) {
    if (n < 1 || s1 < s0 || !out_inputs || !out_skip || !out_count || !nruns)
        return fail(NVISR_INVALID_ARG, "group_runs: bad arguments");
    const int need = n + (extra ? 1 : 0);
    int runs = 0;
    for (int64_t nominal = s0; nominal <= s1; nominal += n) {
        if (runs >= max_runs) return fail(NVISR_INVALID_ARG, "group_runs: max_runs too small");
        int64_t start;
        int skip, count;
        run_form(nominal, s0, s1, n, &start, &skip, &count);
        for (int k = 0; k < need; ++k) out_inputs[runs * need + k] = (int32_t)std::min<int64_t>(start + k, s1);
        out_skip[runs] = skip;
        out_count[runs] = count;
        ++runs;
    }
    *nruns = runs;
    return NVISR_OK;
}

nvisr_status nvisr_group_outputs(const uint8_t *flags, int32_t nframes, int32_t n, int32_t extra, int32_t interp,
                                 int32_t dbl, int32_t max_out, int32_t *kind, int32_t *src_first, int32_t *src_last,
                                 int32_t *net_k, int32_t *nout) {
    if (!flags || nframes < 0 || n < 1 || !kind || !src_first || !src_last || !net_k || !nout)
        return fail(NVISR_INVALID_ARG, "group_outputs: bad arguments");
    // a filter without a device: only the bookkeeping group_locate reads
    nvisr_filter f;
    f.net.family = "group";
    f.net.interp = interp != 0;
    f.net.extra = extra != 0;
    f.net.dbl = dbl != 0;
    f.net.frames = n + (extra ? 1 : 0);
    f.grp_n = n;
    f.grp_need = f.net.frames;
    for (int k = 0; k < nframes; ++k) f.cut.push_back(k > 0 && flags[k] ? 1 : 0);
    f.pushed = nframes;
    f.eos = true;
    const int64_t total = group_total(&f);
    if (total > max_out) return fail(NVISR_INVALID_ARG, "group_outputs: max_out too small");
    for (int64_t o = 0; o < total; ++o) {
        RunLoc loc;
        if (!group_locate(&f, o, &loc)) return fail(NVISR_INTERNAL, "group_outputs: output not located");
        kind[o] = loc.pass ? NVISR_OUT_PASSTHROUGH : NVISR_OUT_NETWORK;
        src_first[o] = (int32_t)(loc.pass ? loc.frame : loc.inputs.front());
        src_last[o] = (int32_t)(loc.pass ? loc.frame : loc.inputs.back());
        net_k[o] = loc.pass ? -1 : loc.k;
    }
    *nout = (int32_t)total;
    return NVISR_OK;
}

nvisr_status nvisr_fig1_layout(int32_t n, int32_t b, int32_t *cell_frame, int32_t *slot_start, int32_t *copy) {
    if (n < 1 || b < 1 || !cell_frame || !slot_start || !copy) return fail(NVISR_INVALID_ARG, "fig1_layout: bad arguments");
    // column-first store of b rows x (n+1) columns: address = col * b + row
    for (int a = 0; a < (n + 1) * b; ++a) cell_frame[a] = -1;
    cell_frame[b - 1] = 0;
    for (int r = 0; r < b; ++r) {
        cell_frame[1 * b + r] = (r + 1) * n;
        for (int k = 1; k < n; ++k) cell_frame[(k + 1) * b + r] = r * n + k;
    }
    slot_start[0] = b - 1;
    for (int k = 1; k < n; ++k) slot_start[k] = (k + 1) * b;
    slot_start[n] = b;
    copy[0] = 2 * b - 1;
    copy[1] = b - 1;
    return NVISR_OK;
}

}  // extern "C"

// ---------------------------------------------------------------- per-call layer entry points

namespace {

struct Scratch {
    std::vector<void *> ptrs;
    ~Scratch() {
        for (void *p : ptrs) cudaFree(p);
    }
    cudaError_t alloc(size_t bytes, void **out) {
        cudaError_t e = cudaMalloc(out, std::max<size_t>(bytes, 256));
        if (e == cudaSuccess) ptrs.push_back(*out);
        return e;
    }
};

// Quantisation scale (amax / 448) of a planar tensor, measured on the device.
nvisr_status fp8_scale(const float *x, int C, int H, int W, Scratch &sc, cudaStream_t st, float *scale) {
    void *tmp, *am;
    const int cpad = round_up(C, 8);
    NVISR_TRY_CUDA(sc.alloc((size_t)cpad * H * W * 2, &tmp));
    NVISR_TRY_CUDA(sc.alloc(sizeof(unsigned), &am));
    NVISR_TRY_CUDA(cudaMemsetAsync(am, 0, sizeof(unsigned), st));
    PackArgs pa{};
    pa.src[0] = x;
    pa.nsrc = 1;
    pa.ch_per_src = C;
    pa.src_pitch = W;
    pa.src_plane = (int64_t)W * H;
    pa.H = H;
    pa.W = W;
    pa.dst = tmp;
    pa.cpad = cpad;
    pa.dt = DT_BF16;
    pa.scale = 1.f;
    pa.amax = (unsigned *)am;
    NVISR_TRY_CUDA(launch_pack(pa, st));
    unsigned h;
    NVISR_TRY_CUDA(cudaMemcpyAsync(&h, am, 4, cudaMemcpyDeviceToHost, st));
    NVISR_TRY_CUDA(cudaStreamSynchronize(st));
    float a;
    memcpy(&a, &h, 4);
    *scale = a > 0.f ? a / 448.f : 1.f;
    return NVISR_OK;
}

nvisr_status pack_planar(const float *x, int C, int cpad, int H, int W, int dt, float scale, void *dst,
                         cudaStream_t st, int cpc = 0) {
    PackArgs pa{};
    pa.src[0] = x;
    pa.nsrc = 1;
    pa.ch_per_src = C;
    pa.src_pitch = W;
    pa.src_plane = (int64_t)W * H;
    pa.H = H;
    pa.W = W;
    pa.dst = dst;
    pa.cpad = cpad;
    pa.dt = dt;
    pa.cpc = cpc;
    pa.scale = scale;
    NVISR_TRY_CUDA(launch_pack(pa, st));
    return NVISR_OK;
}

}  // namespace

extern "C" {

nvisr_status nvisr_conv2d(int32_t precision, const float *x, int32_t cin, int32_t h, int32_t w, const float *weight,
                          const float *bias, int32_t cout, int32_t k, int32_t act, const float *res, float *y,
                          void *stream) {
    if (!x || !weight || !y || cin < 1 || cout < 1 || h < 1 || w < 1 || (k != 1 && k != 3) || act < 0 || act > 1)
        return fail(NVISR_INVALID_ARG, "conv2d: bad arguments");
    if (precision < NVISR_PREC_FP32 || precision > NVISR_PREC_FP8) return fail(NVISR_INVALID_ARG, "conv2d: precision");
    cudaStream_t st = (cudaStream_t)stream;
    const bool tc = precision != NVISR_PREC_FP32;
    const int adt = precision == NVISR_PREC_FP32 ? DT_F32 : (precision == NVISR_PREC_FP16 ? DT_F16 : DT_BF16);
    const int idt = precision == NVISR_PREC_FP8 ? DT_E4M3 : adt;
    if (precision == NVISR_PREC_FP8 && (cin % 64 || cout != 64 || k != 3))
        return fail(NVISR_UNSUPPORTED_FORMAT, "conv2d: FP8 supports 64->64 3x3 layers");
    const int cin_pad = tc ? round_up(cin, idt == DT_E4M3 ? 16 : 16) : round_up(cin, 8);
    const int cout_pad = round_up(cout, 16);
    Scratch sc;
    // weights (host copy -> layout -> device)
    std::vector<float> hw((size_t)cout * cin * k * k), hb(cout_pad, 0.f);
    NVISR_TRY_CUDA(cudaMemcpyAsync(hw.data(), weight, hw.size() * 4, cudaMemcpyDeviceToHost, st));
    if (bias) NVISR_TRY_CUDA(cudaMemcpyAsync(hb.data(), bias, (size_t)cout * 4, cudaMemcpyDeviceToHost, st));
    NVISR_TRY_CUDA(cudaStreamSynchronize(st));
    float sx = 1.f, sw = 1.f;
    if (idt == DT_E4M3) {
        nvisr_status s = fp8_scale(x, cin, h, w, sc, st, &sx);
        if (s != NVISR_OK) return s;
        float amax = 0.f;
        for (float v : hw) amax = std::max(amax, std::fabs(v));
        sw = amax > 0.f ? amax / 448.f : 1.f;
    }
    void *dw, *db, *dx, *dy, *dr = nullptr;
    size_t wbytes;
    std::vector<uint8_t> hwl;
    if (tc) {
        wbytes = tc_weight_bytes(cin_pad, cout_pad, k, idt);
        hwl.resize(wbytes);
        prepare_weights_tc(hw.data(), cout, cin, k, cin_pad, cout_pad, idt, 1.f / sw, hwl.data(),
                           layout_cpc(idt, cin_pad) == 64);
    } else {
        wbytes = simt_weight_bytes(cin_pad, cout_pad, k);
        hwl.resize(wbytes);
        prepare_weights_simt(hw.data(), cout, cin, k, cin_pad, cout_pad, (float *)hwl.data());
    }
    NVISR_TRY_CUDA(sc.alloc(wbytes, &dw));
    NVISR_TRY_CUDA(cudaMemcpyAsync(dw, hwl.data(), wbytes, cudaMemcpyHostToDevice, st));
    void *dwr = nullptr;
    std::vector<uint8_t> hrows;
    if (tc && idt != DT_E4M3 && k == 3 && cin == 64 && cout == 64) {
        hrows.resize(tc_rows_weight_bytes());
        prepare_weights_rows(hw.data(), idt, hrows.data());
        NVISR_TRY_CUDA(sc.alloc(hrows.size(), &dwr));
        NVISR_TRY_CUDA(cudaMemcpyAsync(dwr, hrows.data(), hrows.size(), cudaMemcpyHostToDevice, st));
    }
    NVISR_TRY_CUDA(sc.alloc(cout_pad * 4, &db));
    NVISR_TRY_CUDA(cudaMemcpyAsync(db, hb.data(), cout_pad * 4, cudaMemcpyHostToDevice, st));
    NVISR_TRY_CUDA(sc.alloc((size_t)cin_pad * h * w * dtype_size(idt), &dx));
    NVISR_TRY_CUDA(sc.alloc((size_t)cout_pad * h * w * dtype_size(adt), &dy));
    const int in_cpc = layout_cpc(idt, cin_pad), out_cpc = layout_cpc(adt, cout_pad);
    nvisr_status s = pack_planar(x, cin, cin_pad, h, w, idt, 1.f / sx, dx, st, in_cpc);
    if (s != NVISR_OK) return s;
    if (res) {
        NVISR_TRY_CUDA(sc.alloc((size_t)cout_pad * h * w * dtype_size(adt), &dr));
        if ((s = pack_planar(res, cout, cout_pad, h, w, adt, 1.f, dr, st, out_cpc)) != NVISR_OK) return s;
    }
    int *err;
    NVISR_TRY_CUDA(sc.alloc(sizeof(int), (void **)&err));
    NVISR_TRY_CUDA(cudaMemsetAsync(err, 0, sizeof(int), st));
    ConvArgs a{};
    a.x = dx; a.cin_pad = cin_pad; a.H = h; a.W = w; a.nimg = 1; a.w = dw; a.w_rows = dwr; a.bias = (const float *)db;
    a.cout = cout; a.cout_pad = cout_pad; a.k = k; a.act = act; a.res = dr; a.y = dy;
    a.in_dt = idt; a.out_dt = adt; a.acc_scale = sx * sw; a.out_scale = 1.f; a.y2_scale = 1.f; a.err = err;
    a.in_cpc = in_cpc; a.out_cpc = out_cpc;
    cudaError_t e = tc ? launch_conv_tc(a, st) : launch_conv_simt(a, st);
    if (e != cudaSuccess) return cuda_status(e, "conv2d");
    NVISR_TRY_CUDA(launch_unpack(dy, adt, cout_pad, out_cpc, cout, h, w, 1.f, y, w, st));
    int herr = 0;
    NVISR_TRY_CUDA(cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, st));
    NVISR_TRY_CUDA(cudaStreamSynchronize(st));
    if (herr) return fail(NVISR_DEVICE_TIMEOUT, "conv2d: a device-side wait exceeded its bound");
    return NVISR_OK;
}

nvisr_status nvisr_resblock2d(int32_t precision, const float *x, int32_t h, int32_t w, const float *w1,
                              const float *b1, const float *w2, const float *b2, float *y, int32_t fused,
                              void *stream) {
    if (!x || !w1 || !w2 || !y || h < 1 || w < 1) return fail(NVISR_INVALID_ARG, "resblock2d: bad arguments");
    if (precision != NVISR_PREC_BF16 && precision != NVISR_PREC_FP16)
        return fail(NVISR_UNSUPPORTED_FORMAT, "resblock2d: BF16 or FP16");
    const size_t plane = (size_t)64 * h * w;
    if (y < x + plane && x < y + plane) return fail(NVISR_INVALID_ARG, "resblock2d: y overlaps x");
    const int dt = precision == NVISR_PREC_FP16 ? DT_F16 : DT_BF16;
    cudaStream_t st = (cudaStream_t)stream;
    Scratch sc;
    std::vector<float> hw1((size_t)64 * 64 * 9), hw2(hw1.size()), hb1(64, 0.f), hb2(64, 0.f);
    NVISR_TRY_CUDA(cudaMemcpyAsync(hw1.data(), w1, hw1.size() * 4, cudaMemcpyDeviceToHost, st));
    NVISR_TRY_CUDA(cudaMemcpyAsync(hw2.data(), w2, hw2.size() * 4, cudaMemcpyDeviceToHost, st));
    if (b1) NVISR_TRY_CUDA(cudaMemcpyAsync(hb1.data(), b1, 64 * 4, cudaMemcpyDeviceToHost, st));
    if (b2) NVISR_TRY_CUDA(cudaMemcpyAsync(hb2.data(), b2, 64 * 4, cudaMemcpyDeviceToHost, st));
    NVISR_TRY_CUDA(cudaStreamSynchronize(st));
    std::vector<uint8_t> r1(tc_rows_weight_bytes()), r2(tc_rows_weight_bytes());
    prepare_weights_rows(hw1.data(), dt, r1.data());
    prepare_weights_rows(hw2.data(), dt, r2.data());
    void *dr1, *dr2, *db1, *db2, *dx, *dh, *dy;
    const size_t abytes = plane * 2;
    NVISR_TRY_CUDA(sc.alloc(r1.size(), &dr1));
    NVISR_TRY_CUDA(sc.alloc(r2.size(), &dr2));
    NVISR_TRY_CUDA(sc.alloc(64 * 4, &db1));
    NVISR_TRY_CUDA(sc.alloc(64 * 4, &db2));
    NVISR_TRY_CUDA(sc.alloc(abytes, &dx));
    NVISR_TRY_CUDA(sc.alloc(abytes, &dh));
    NVISR_TRY_CUDA(sc.alloc(abytes, &dy));
    NVISR_TRY_CUDA(cudaMemcpyAsync(dr1, r1.data(), r1.size(), cudaMemcpyHostToDevice, st));
    NVISR_TRY_CUDA(cudaMemcpyAsync(dr2, r2.data(), r2.size(), cudaMemcpyHostToDevice, st));
    NVISR_TRY_CUDA(cudaMemcpyAsync(db1, hb1.data(), 64 * 4, cudaMemcpyHostToDevice, st));
    NVISR_TRY_CUDA(cudaMemcpyAsync(db2, hb2.data(), 64 * 4, cudaMemcpyHostToDevice, st));
    nvisr_status s = pack_planar(x, 64, 64, h, w, dt, 1.f, dx, st, 64);
    if (s != NVISR_OK) return s;
    int *err;
    NVISR_TRY_CUDA(sc.alloc(sizeof(int), (void **)&err));
    NVISR_TRY_CUDA(cudaMemsetAsync(err, 0, sizeof(int), st));
    ConvArgs a1{};
    a1.x = dx; a1.cin_pad = 64; a1.in_cpc = 64; a1.out_cpc = 64; a1.H = h; a1.W = w; a1.nimg = 1;
    a1.w_rows = dr1; a1.bias = (const float *)db1; a1.cout = 64; a1.cout_pad = 64; a1.k = 3; a1.act = 1;
    a1.y = dh; a1.in_dt = dt; a1.out_dt = dt; a1.acc_scale = 1.f; a1.out_scale = 1.f; a1.y2_scale = 1.f; a1.err = err;
    ConvArgs a2 = a1;
    a2.x = dh; a2.w_rows = dr2; a2.bias = (const float *)db2; a2.act = 0; a2.res = dx; a2.y = dy;
    cudaError_t e;
    if (fused) {
        if (!res_block_fits(a1, a2)) return fail(NVISR_UNSUPPORTED_FORMAT, "resblock2d: no fused form for these buffers");
        e = launch_res_block(a1, a2, st);
    } else {
        e = launch_conv_tc(a1, st);
        if (e == cudaSuccess) e = launch_conv_tc(a2, st);
    }
    if (e != cudaSuccess) return cuda_status(e, "resblock2d");
    NVISR_TRY_CUDA(launch_unpack(dy, dt, 64, 64, 64, h, w, 1.f, y, w, st));
    int herr = 0;
    NVISR_TRY_CUDA(cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, st));
    NVISR_TRY_CUDA(cudaStreamSynchronize(st));
    if (herr) return fail(NVISR_DEVICE_TIMEOUT, "resblock2d: a device-side wait exceeded its bound");
    return NVISR_OK;
}

nvisr_status nvisr_dcn2d(int32_t precision, const float *x, int32_t cin, int32_t h, int32_t w, const float *offsets,
                         const float *mask, int32_t groups, const float *weight, const float *bias, int32_t cout,
                         float *y, void *stream) {
    if (!x || !offsets || !mask || !weight || !y || cin < 1 || cout < 1 || h < 1 || w < 1 || groups < 1 ||
        cin % groups)
        return fail(NVISR_INVALID_ARG, "dcn2d: bad arguments");
    if (precision < NVISR_PREC_FP32 || precision > NVISR_PREC_FP16)
        return fail(NVISR_UNSUPPORTED_FORMAT, "dcn2d: FP32, BF16 or FP16");
    const bool tc = precision != NVISR_PREC_FP32;
    const int adt = precision == NVISR_PREC_FP32 ? DT_F32 : (precision == NVISR_PREC_FP16 ? DT_F16 : DT_BF16);
    if (tc && (cin != 64 || cout != 64 || (cin / groups) % 8))
        return fail(NVISR_UNSUPPORTED_FORMAT, "dcn2d: tensor-core DCN needs 64 -> 64 channels, 8k per group");
    if (!tc && ((cin / groups) % 4 || cin % 8))
        return fail(NVISR_UNSUPPORTED_FORMAT, "dcn2d: FP32 DCN needs cin % 8 == 0 and 4k channels per group");
    cudaStream_t st = (cudaStream_t)stream;
    const int cin_pad = cin, cout_pad = round_up(cout, 16);
    Scratch sc;
    std::vector<float> hw((size_t)cout * cin * 9), hb(cout_pad, 0.f);
    NVISR_TRY_CUDA(cudaMemcpyAsync(hw.data(), weight, hw.size() * 4, cudaMemcpyDeviceToHost, st));
    if (bias) NVISR_TRY_CUDA(cudaMemcpyAsync(hb.data(), bias, (size_t)cout * 4, cudaMemcpyDeviceToHost, st));
    NVISR_TRY_CUDA(cudaStreamSynchronize(st));
    std::vector<uint8_t> hwl;
    if (tc) {
        hwl.resize(tc_weight_bytes(cin_pad, cout_pad, 3, adt));
        prepare_weights_tc(hw.data(), cout, cin, 3, cin_pad, cout_pad, adt, 1.f, hwl.data(), false);
    } else {
        hwl.resize(simt_weight_bytes(cin_pad, cout_pad, 3));
        prepare_weights_simt(hw.data(), cout, cin, 3, cin_pad, cout_pad, (float *)hwl.data());
    }
    void *dw, *db, *dx, *dy, *dom;
    NVISR_TRY_CUDA(sc.alloc(hwl.size(), &dw));
    NVISR_TRY_CUDA(cudaMemcpyAsync(dw, hwl.data(), hwl.size(), cudaMemcpyHostToDevice, st));
    NVISR_TRY_CUDA(sc.alloc(cout_pad * 4, &db));
    NVISR_TRY_CUDA(cudaMemcpyAsync(db, hb.data(), cout_pad * 4, cudaMemcpyHostToDevice, st));
    NVISR_TRY_CUDA(sc.alloc((size_t)cin_pad * h * w * dtype_size(adt), &dx));
    NVISR_TRY_CUDA(sc.alloc((size_t)cout_pad * h * w * dtype_size(adt), &dy));
    // offsets then mask, as one blocked float32 operand [27G -> pad 4]
    const int om_c = 27 * groups, om_cpad = round_up(om_c, 4);
    NVISR_TRY_CUDA(sc.alloc((size_t)om_cpad * h * w * 4, &dom));
    {
        PackArgs pa{};
        pa.src[0] = offsets;
        pa.src[1] = mask;
        pa.nsrc = 1;
        pa.ch_per_src = 18 * groups;
        pa.src_pitch = w;
        pa.src_plane = (int64_t)w * h;
        pa.H = h;
        pa.W = w;
        pa.dst = dom;
        pa.cpad = om_cpad;
        pa.dt = DT_F32;
        pa.scale = 1.f;
        // offsets (18G channels) then mask (9G channels): two packs into one tensor
        // would split a 4-channel chunk when 18G % 4 != 0, so pack from a joined copy
        void *joined;
        NVISR_TRY_CUDA(sc.alloc((size_t)om_c * h * w * 4, &joined));
        NVISR_TRY_CUDA(cudaMemcpyAsync(joined, offsets, (size_t)18 * groups * h * w * 4, cudaMemcpyDeviceToDevice, st));
        NVISR_TRY_CUDA(cudaMemcpyAsync((float *)joined + (size_t)18 * groups * h * w, mask, (size_t)9 * groups * h * w * 4,
                                       cudaMemcpyDeviceToDevice, st));
        pa.src[0] = (const float *)joined;
        pa.ch_per_src = om_c;
        NVISR_TRY_CUDA(launch_pack(pa, st));
    }
    // the tensor-core gather reads x in 8-channel planes
    const int x_cpc = tc ? 8 : layout_cpc(adt, cin_pad), y_cpc = layout_cpc(adt, cout_pad);
    nvisr_status s = pack_planar(x, cin, cin_pad, h, w, adt, 1.f, dx, st, x_cpc);
    if (s != NVISR_OK) return s;
    int *err;
    NVISR_TRY_CUDA(sc.alloc(sizeof(int), (void **)&err));
    NVISR_TRY_CUDA(cudaMemsetAsync(err, 0, sizeof(int), st));
    DcnArgs d{};
    d.x = dx; d.cin_pad = cin_pad; d.H = h; d.W = w; d.groups = groups;
    d.om = (const float *)dom; d.om_cpad = om_cpad; d.mask_logits = 0;
    d.w = dw; d.bias = (const float *)db; d.cout = cout; d.cout_pad = cout_pad; d.y = dy;
    d.in_dt = adt; d.out_dt = adt; d.acc_scale = 1.f; d.out_scale = 1.f; d.err = err;
    d.x_cpc = x_cpc; d.y_cpc = y_cpc;
    cudaError_t e = tc ? launch_dcn_tc(d, st) : launch_dcn_simt(d, st);
    if (e != cudaSuccess) return cuda_status(e, "dcn2d");
    NVISR_TRY_CUDA(launch_unpack(dy, adt, cout_pad, y_cpc, cout, h, w, 1.f, y, w, st));
    int herr = 0;
    NVISR_TRY_CUDA(cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, st));
    NVISR_TRY_CUDA(cudaStreamSynchronize(st));
    if (herr) return fail(NVISR_DEVICE_TIMEOUT, "dcn2d: a device-side wait exceeded its bound");
    return NVISR_OK;
}

nvisr_status nvisr_test_starve(int32_t on) {
    g_test_starve = on ? 1 : 0;
    return NVISR_OK;
}

nvisr_status nvisr_selftest(int32_t *mismatches_bf16, int32_t *mismatches_fp8) {
    if (!mismatches_bf16 || !mismatches_fp8) return fail(NVISR_INVALID_ARG, "selftest: NULL argument");
    int *d;
    NVISR_TRY_CUDA(cudaMalloc(&d, 2 * sizeof(int)));
    cudaMemset(d, 0, 2 * sizeof(int));
    int e1 = tc_selftest(0, d, 0);
    int e2 = tc_selftest(1, d + 1, 0);
    cudaError_t se = cudaDeviceSynchronize();
    int h[2] = {-1, -1};
    cudaMemcpy(h, d, sizeof(h), cudaMemcpyDeviceToHost);
    cudaFree(d);
    if (e1 || e2 || se != cudaSuccess)
        return fail(NVISR_CUDA_ERROR, std::string("selftest launch: ") + cudaGetErrorString(se));
    *mismatches_bf16 = h[0];
    *mismatches_fp8 = h[1];
    return NVISR_OK;
}

nvisr_status nvisr_selftest_swizzle(int32_t *out16) {
    if (!out16) return fail(NVISR_INVALID_ARG, "selftest_swizzle: NULL argument");
    int *d;
    NVISR_TRY_CUDA(cudaMalloc(&d, 16 * sizeof(int)));
    cudaMemset(d, 0, 16 * sizeof(int));
    const int e = tc_probe_sw128(d, 0);
    const cudaError_t se = cudaDeviceSynchronize();
    cudaMemcpy(out16, d, 16 * sizeof(int), cudaMemcpyDeviceToHost);
    cudaFree(d);
    if (e || se != cudaSuccess) return fail(NVISR_CUDA_ERROR, std::string("selftest_swizzle: ") + cudaGetErrorString(se));
    return NVISR_OK;
}

}  // extern "C"
