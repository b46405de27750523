// Serving runtime: clips (one video stream each) are submitted at any time,
// admitted as filters while the engine's HBM budget and the slot count allow,
// and stepped together.  Clips that run the same network share batched
// launches (nvisr_batch), so a clip admitted while others are in flight joins
// the next step's shared launches instead of waiting for them to finish
// (continuous batching).  The server records, per output frame, the time from
// the push of the newest input frame it depends on to its pull, and per clip
// the time from submission to admission.
#include <algorithm>
#include <chrono>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <string>
#include <vector>

#include <cuda_runtime.h>

#include "nvisr.h"

namespace nvisr {
void set_error(const std::string &msg);
struct ErrScope {  // defined with the engine: errors of a call also go to its engine
    explicit ErrScope(nvisr_engine *e);
    ~ErrScope();
    nvisr_engine *prev;
};
}

struct nvisr_server {
    nvisr_engine *eng = nullptr;
    int max_active = 0;
    struct Clip {
        std::string text;
        std::vector<float> blob;
        nvisr_filter_desc desc{};
        nvisr_filter *f = nullptr;  // null while pending
        int group = -1;
        double t_submit = 0.0, t_admit = -1.0;
        std::vector<double> push_time;  // per pushed frame
    };
    struct Group {
        std::string key;  // network text + blob + precision: clips that can share launches
        std::vector<int64_t> members;
        nvisr_batch *batch = nullptr;
        bool dirty = true;
    };
    std::map<int64_t, Clip> clips;
    std::deque<int64_t> pending;
    std::vector<Group> groups;
    int64_t next_id = 0;
    int active = 0;
    int64_t admitted = 0, deferred_steps = 0, completed = 0, outputs = 0;
    std::vector<double> latency_ms, queue_ms;
};

namespace {

nvisr_status bad(const char *msg) {
    nvisr::set_error(msg);
    return NVISR_INVALID_ARG;
}

double now_s() {
    using namespace std::chrono;
    return duration<double>(steady_clock::now().time_since_epoch()).count();
}

std::string group_key(const nvisr_server::Clip &c) {
    std::string k = c.text;
    k += '\0';
    k.append(reinterpret_cast<const char *>(c.blob.data()), c.blob.size() * sizeof(float));
    k += static_cast<char>('0' + c.desc.precision);
    return k;
}

double percentile(std::vector<double> v, double q) {
    if (v.empty()) return 0.0;
    std::sort(v.begin(), v.end());
    const double pos = q * (double)(v.size() - 1);
    const size_t i = (size_t)pos;
    const double fr = pos - (double)i;
    return i + 1 < v.size() ? v[i] * (1.0 - fr) + v[i + 1] * fr : v[i];
}

void drop_batch(nvisr_server::Group &g) {
    if (g.batch) nvisr_batch_destroy(g.batch);
    g.batch = nullptr;
    g.dirty = true;
}

// Admit pending clips in arrival order while slots and the HBM budget allow.
nvisr_status admit(nvisr_server *s) {
    while (!s->pending.empty() && (s->max_active <= 0 || s->active < s->max_active)) {
        nvisr_server::Clip &c = s->clips[s->pending.front()];
        nvisr_filter *f = nullptr;
        const nvisr_status st = nvisr_filter_create(s->eng, &c.desc, &f);
        if (st == NVISR_OVER_BUDGET || st == NVISR_OUT_OF_MEMORY) {
            ++s->deferred_steps;  // waits for a finishing clip to free memory
            break;
        }
        if (st != NVISR_OK) return st;
        c.f = f;
        c.t_admit = now_s();
        s->queue_ms.push_back((c.t_admit - c.t_submit) * 1e3);
        const std::string key = group_key(c);
        int gi = -1;
        for (size_t i = 0; i < s->groups.size(); ++i)
            if (s->groups[i].key == key) gi = (int)i;
        if (gi < 0) {
            s->groups.emplace_back();
            s->groups.back().key = key;
            gi = (int)s->groups.size() - 1;
        }
        c.group = gi;
        s->groups[gi].members.push_back(s->pending.front());
        drop_batch(s->groups[gi]);
        s->pending.pop_front();
        ++s->active;
        ++s->admitted;
    }
    return NVISR_OK;
}

}  // namespace

extern "C" {

nvisr_status nvisr_server_create(nvisr_engine *engine, int32_t max_active, nvisr_server **out) {
    nvisr::ErrScope es(engine);
    if (!engine || !out) return bad("server_create: NULL argument");
    nvisr_server *s = new nvisr_server();
    s->eng = engine;
    s->max_active = max_active;
    *out = s;
    return NVISR_OK;
}

nvisr_status nvisr_server_submit(nvisr_server *s, const nvisr_filter_desc *desc, int64_t *clip) {
    nvisr::ErrScope es(s ? s->eng : nullptr);
    if (!s || !desc || !clip || !desc->network_text || (!desc->weights && desc->weights_count > 0))
        return bad("server_submit: bad arguments");
    const int64_t id = s->next_id++;
    nvisr_server::Clip &c = s->clips[id];
    c.text = desc->network_text;
    c.blob.assign(desc->weights, desc->weights + desc->weights_count);
    c.desc = *desc;
    c.desc.network_text = c.text.c_str();
    c.desc.weights = c.blob.data();
    c.t_submit = now_s();
    s->pending.push_back(id);
    *clip = id;
    return admit(s);
}

nvisr_status nvisr_server_push(nvisr_server *s, int64_t clip, const nvisr_planes *in, uint32_t flags) {
    nvisr::ErrScope es(s ? s->eng : nullptr);
    if (!s) return bad("server: NULL server");
    auto it = s->clips.find(clip);
    if (it == s->clips.end()) return bad("server: unknown clip");
    nvisr_server::Clip &c = it->second;
    if (!c.f) return NVISR_AGAIN;  // not admitted yet
    const nvisr_status st = nvisr_push(c.f, in, flags);
    if (st == NVISR_OK) c.push_time.push_back(now_s());
    return st;
}

nvisr_status nvisr_server_flush(nvisr_server *s, int64_t clip) {
    nvisr::ErrScope es(s ? s->eng : nullptr);
    if (!s) return bad("server: NULL server");
    auto it = s->clips.find(clip);
    if (it == s->clips.end()) return bad("server: unknown clip");
    if (!it->second.f) return NVISR_AGAIN;
    return nvisr_flush(it->second.f);
}

nvisr_status nvisr_server_step(nvisr_server *s, int32_t *produced) {
    nvisr::ErrScope es(s ? s->eng : nullptr);
    if (!s) return bad("server: NULL server");
    nvisr_status st = admit(s);
    if (st != NVISR_OK) return st;
    int total = 0;
    for (nvisr_server::Group &g : s->groups) {
        if (g.members.empty()) continue;
        if (g.dirty || !g.batch) {
            std::vector<nvisr_filter *> fs;
            for (int64_t id : g.members) fs.push_back(s->clips[id].f);
            if ((st = nvisr_batch_create(s->eng, fs.data(), (int32_t)fs.size(), &g.batch)) != NVISR_OK) return st;
            g.dirty = false;
        }
        int32_t n = 0;
        if ((st = nvisr_batch_step(g.batch, &n)) != NVISR_OK) return st;
        total += n;
    }
    if (produced) *produced = total;
    return NVISR_OK;
}

nvisr_status nvisr_server_pull(nvisr_server *s, int64_t clip, nvisr_planes *out, nvisr_frame_info *info) {
    nvisr::ErrScope es(s ? s->eng : nullptr);
    if (!s) return bad("server: NULL server");
    auto it = s->clips.find(clip);
    if (it == s->clips.end()) return bad("server: unknown clip");
    nvisr_server::Clip &c = it->second;
    if (!c.f) return NVISR_AGAIN;
    nvisr_frame_info fi{};
    const nvisr_status st = nvisr_pull(c.f, out, &fi);
    if (st == NVISR_OK && out->on_device) {
        // device planes are written in stream order: the output is ready once the stream gets there
        const cudaError_t e = cudaStreamSynchronize((cudaStream_t)nvisr_engine_stream(s->eng));
        if (e != cudaSuccess) return NVISR_CUDA_ERROR;
    }
    if (st == NVISR_OK) {
        if (fi.src_last >= 0 && fi.src_last < (int64_t)c.push_time.size())
            s->latency_ms.push_back((now_s() - c.push_time[(size_t)fi.src_last]) * 1e3);
        ++s->outputs;
        if (info) *info = fi;
    }
    return st;
}

nvisr_status nvisr_server_close(nvisr_server *s, int64_t clip) {
    nvisr::ErrScope es(s ? s->eng : nullptr);
    if (!s) return bad("server: NULL server");
    auto it = s->clips.find(clip);
    if (it == s->clips.end()) return bad("server: unknown clip");
    nvisr_server::Clip &c = it->second;
    if (c.f) {
        nvisr_server::Group &g = s->groups[(size_t)c.group];
        drop_batch(g);
        g.members.erase(std::remove(g.members.begin(), g.members.end(), clip), g.members.end());
        nvisr_filter_destroy(c.f);
        --s->active;
        ++s->completed;
    } else {
        s->pending.erase(std::remove(s->pending.begin(), s->pending.end(), clip), s->pending.end());
    }
    s->clips.erase(it);
    return admit(s);  // the freed memory may let waiting clips in
}

nvisr_status nvisr_server_stats(nvisr_server *s, nvisr_server_stats_t *out) {
    nvisr::ErrScope es(s ? s->eng : nullptr);
    if (!s || !out) return bad("server_stats: NULL argument");
    std::memset(out, 0, sizeof(*out));
    out->latency_p50_ms = percentile(s->latency_ms, 0.50);
    out->latency_p99_ms = percentile(s->latency_ms, 0.99);
    out->queue_p50_ms = percentile(s->queue_ms, 0.50);
    out->queue_p99_ms = percentile(s->queue_ms, 0.99);
    out->admitted = s->admitted;
    out->pending = (int64_t)s->pending.size();
    out->active = s->active;
    out->completed = s->completed;
    out->outputs = s->outputs;
    out->deferred_steps = s->deferred_steps;
    return NVISR_OK;
}

void nvisr_server_destroy(nvisr_server *s) {
    if (!s) return;
    for (nvisr_server::Group &g : s->groups) drop_batch(g);
    for (auto &kv : s->clips)
        if (kv.second.f) nvisr_filter_destroy(kv.second.f);
    delete s;
}

}  // extern "C"
