// Continuous-batching request server over rmdec handles (see include/rmdec_serve.h).
//
// One worker thread owns all CUDA work. Requests wait in a FIFO until they can be admitted:
// a batch is the longest FIFO run of queued requests of the oldest request's code (up to
// max_batch_frames), admitted when a CUDA stream is free and the device arena has room for
// the batch's LLRs and outputs. A batch's requests are copied into one contiguous arena
// block, decoded with a single rmdec_decode launch and copied back, all on the batch's stream,
// so copies and decodes of different batches overlap on the device. A completion event per
// batch retires its requests and frees its arena block, which admits the next requests.
//
// With fuse_codes, codes that can share a grouped launch (include/rmdec_group.h: p-FHT-FSCL
// decoders of one list size, up to 16 per family) form a family. When the oldest request is
// smaller than one full wave of its code's own launch, the batch is the FIFO run of the
// family's requests of that kind: they are laid out code by code in the arena and decoded by
// one rmdec_group_decode call with one segment per code. Larger requests are batched per
// code as without fusing.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include "../../include/rmdec.h"
#include "../../include/rmdec_group.h"
#include "../../include/rmdec_serve.h"
#include "rmdec_internal.h"

namespace {

using Clock = std::chrono::steady_clock;

struct Request {
    uint64_t id = 0;
    int code = 0;
    const void* llr = nullptr;
    int64_t frames = 0;
    uint32_t* out = nullptr;
    Clock::time_point t_submit, t_done;
    bool done = false;
    rmdec_status status = RMDEC_OK;
};

struct Batch {
    int code = 0;
    int stream = 0;
    std::vector<Request*> reqs;
    int64_t frames = 0;
    size_t offset = 0, bytes = 0;
    cudaEvent_t ev = nullptr;
    bool failed = false;
};

// First-fit allocator over the arena with coalescing frees (offsets aligned to 256 bytes).
class Arena {
   public:
    void reset(size_t bytes) {
        free_.clear();
        free_[0] = bytes;
    }
    bool alloc(size_t bytes, size_t* off) {
        bytes = (bytes + 255) / 256 * 256;
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second >= bytes) {
                *off = it->first;
                const size_t rest = it->second - bytes, at = it->first + bytes;
                free_.erase(it);
                if (rest) free_[at] = rest;
                return true;
            }
        }
        return false;
    }
    void release(size_t off, size_t bytes) {
        bytes = (bytes + 255) / 256 * 256;
        auto it = free_.emplace(off, bytes).first;
        auto nx = std::next(it);
        if (nx != free_.end() && it->first + it->second == nx->first) {
            it->second += nx->second;
            free_.erase(nx);
        }
        if (it != free_.begin()) {
            auto pv = std::prev(it);
            if (pv->first + pv->second == it->first) {
                pv->second += it->second;
                free_.erase(it);
            }
        }
    }

   private:
    std::map<size_t, size_t> free_;
};

size_t align256(size_t b) { return (b + 255) / 256 * 256; }

}  // namespace

struct rmdec_server {
    rmdec_server_config cfg{};
    int device = 0;
    void* arena_ptr = nullptr;
    Arena arena;
    std::vector<cudaStream_t> streams;
    std::vector<bool> stream_busy;
    struct Code {
        rmdec_t h;
        size_t in_bpf, out_bpf;
        int family;  // -1: decoded alone
        int member;  // index within the family's group
        int64_t wave = -1;  // frames that fill the GPU in the code's own launch (-1: not known yet)
    };
    struct Family {
        int L = 0;
        std::vector<int> codes;
        rmdec_group_t grp = nullptr;
        bool stale = true;  // group must be (re)created with the current member list
    };
    std::vector<Code> codes;
    std::vector<Family> families;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<Request*> pending;
    std::map<uint64_t, Request*> requests;
    std::vector<Batch*> inflight;
    std::thread worker;
    bool stop = false;
    uint64_t next_id = 1;
    int64_t n_submitted = 0, n_completed = 0, frames_completed = 0, n_batches = 0, n_cancelled = 0;
    // latencies of the most recent kLatWindow completed requests (a ring), and the maximum
    // over all of them: the record stays bounded on a long-running server
    static constexpr size_t kLatWindow = size_t(1) << 16;
    std::vector<double> latencies;
    size_t lat_next = 0;
    double lat_max = 0.0;
    bool have_first = false;
    Clock::time_point t_first, t_last;
    std::string err;

    rmdec_status fail(rmdec_status st, const char* fmt, ...) {
        char buf[512];
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(buf, sizeof buf, fmt, ap);
        va_end(ap);
        err = buf;
        return st;
    }

    // Retires finished batches. Called with mu held.
    void reap() {
        for (size_t i = 0; i < inflight.size();) {
            Batch* b = inflight[i];
            const cudaError_t e = cudaEventQuery(b->ev);
            if (e == cudaErrorNotReady) {
                ++i;
                continue;
            }
            const auto now = Clock::now();
            for (Request* r : b->reqs) {
                r->done = true;
                r->t_done = now;
                r->status = (e == cudaSuccess && !b->failed) ? RMDEC_OK : RMDEC_ECUDA;
                const double us = std::chrono::duration<double, std::micro>(now - r->t_submit).count();
                if (latencies.size() < kLatWindow)
                    latencies.push_back(us);
                else
                    latencies[lat_next] = us;
                lat_next = (lat_next + 1) % kLatWindow;
                lat_max = std::max(lat_max, us);
                n_completed++;
                frames_completed += r->frames;
            }
            t_last = now;
            arena.release(b->offset, b->bytes);
            stream_busy[b->stream] = false;
            cudaEventDestroy(b->ev);
            delete b;
            inflight.erase(inflight.begin() + i);
            cv_done.notify_all();
        }
    }

    // Forms and launches at most one batch. Called with mu held; returns true if launched.
    bool launch_one(std::unique_lock<std::mutex>& lk) {
        if (pending.empty()) return false;
        int sidx = -1;
        for (int i = 0; i < (int)streams.size(); i++)
            if (!stream_busy[i]) {
                sidx = i;
                break;
            }
        if (sidx < 0) return false;
        const int code = pending.front()->code;
        const int fam = codes[code].family;
        if (fam >= 0 && families[fam].stale) {
            Family& F = families[fam];
            if (F.grp) rmdec_group_destroy(F.grp);
            F.grp = nullptr;
            std::vector<rmdec_t> hs;
            for (int ci : F.codes) hs.push_back(codes[ci].h);
            if (rmdec_group_create(&F.grp, hs.data(), (int)hs.size()) != RMDEC_OK) F.grp = nullptr;
            F.stale = false;
        }
        // Requests that fill the GPU on their own gain nothing from sharing a launch and would
        // hold up the small ones batched with them: only requests below their code's wave are
        // fused; a large oldest request starts a batch of its own code as without fusing.
        auto small = [&](const Request* r) {
            Code& c = codes[r->code];
            if (c.wave < 0) {
                rmdec_host::MemberInfo mi;
                c.wave = rmdec_host::member_info(c.h, true, &mi) == RMDEC_OK ? mi.wave : 0;
            }
            return r->frames < c.wave;
        };
        const bool fused = fam >= 0 && families[fam].grp && small(pending.front());
        // FIFO run of the oldest request's code (or, fused, of its family's small requests),
        // capped by max_batch_frames and by the whole arena: a batch larger than the arena
        // could never be admitted, even with nothing in flight (the oldest request alone always
        // fits, submit checks that)
        std::vector<Request*> take;
        int64_t frames = 0;
        std::vector<std::pair<int, int64_t>> code_frames;  // per code, in order of first appearance
        auto bytes_with = [&](const Request* r) {
            size_t b = 0;
            bool seen = false;
            for (const auto& cf : code_frames) {
                const int64_t f = cf.second + (cf.first == r->code ? r->frames : 0);
                seen = seen || cf.first == r->code;
                b += align256((size_t)f * codes[cf.first].in_bpf) + align256((size_t)f * codes[cf.first].out_bpf);
            }
            if (!seen)
                b += align256((size_t)r->frames * codes[r->code].in_bpf) + align256((size_t)r->frames * codes[r->code].out_bpf);
            return b;
        };
        for (Request* r : pending) {
            if (fused ? (codes[r->code].family != fam || !small(r)) : r->code != code) continue;
            if (frames + r->frames > cfg.max_batch_frames || bytes_with(r) > (size_t)cfg.arena_bytes) break;
            auto it = std::find_if(code_frames.begin(), code_frames.end(), [&](const auto& cf) { return cf.first == r->code; });
            if (it == code_frames.end())
                code_frames.emplace_back(r->code, r->frames);
            else
                it->second += r->frames;
            take.push_back(r);
            frames += r->frames;
        }
        if (take.empty()) return false;
        const double waited = std::chrono::duration<double, std::micro>(Clock::now() - take.front()->t_submit).count();
        if (frames < cfg.min_batch_frames && waited < (double)cfg.max_wait_us && !inflight.empty()) return false;
        // arena layout: per code in the batch (in order of first appearance), its requests'
        // LLRs, then their output words
        struct Part {
            int code;
            int64_t frames = 0;
            size_t in_off = 0, out_off = 0;
        };
        std::vector<Part> parts;
        for (Request* r : take) {
            auto it = std::find_if(parts.begin(), parts.end(), [&](const Part& p) { return p.code == r->code; });
            if (it == parts.end()) {
                parts.push_back(Part{r->code});
                it = parts.end() - 1;
            }
            it->frames += r->frames;
        }
        size_t bytes = 0;
        for (Part& p : parts) {
            p.in_off = bytes;
            bytes += align256((size_t)p.frames * codes[p.code].in_bpf);
            p.out_off = bytes;
            bytes += align256((size_t)p.frames * codes[p.code].out_bpf);
        }
        size_t off = 0;
        if (!arena.alloc(bytes, &off)) return false;  // admission waits for memory
        for (Request* r : take) pending.erase(std::find(pending.begin(), pending.end(), r));
        Batch* b = new Batch;
        b->code = code;
        b->stream = sidx;
        b->reqs = take;
        b->frames = frames;
        b->offset = off;
        b->bytes = bytes;
        stream_busy[sidx] = true;
        n_batches++;
        rmdec_group_t grp = fused ? families[fam].grp : nullptr;
        lk.unlock();
        cudaStream_t st = streams[sidx];
        nvtxRangePushA(grp ? "rmdec_server_batch_fused" : "rmdec_server_batch");
        uint8_t* base = static_cast<uint8_t*>(arena_ptr) + off;
        bool ok = true;
        std::vector<int64_t> at(parts.size(), 0);  // frames placed so far per part
        std::vector<size_t> req_part(take.size());
        std::vector<int64_t> req_at(take.size());
        for (size_t q = 0; q < take.size(); q++) {
            Request* r = take[q];
            const size_t pi = std::find_if(parts.begin(), parts.end(), [&](const Part& p) { return p.code == r->code; }) - parts.begin();
            req_part[q] = pi;
            req_at[q] = at[pi];
            const Code& c = codes[r->code];
            ok &= cudaMemcpyAsync(base + parts[pi].in_off + (size_t)at[pi] * c.in_bpf, r->llr, (size_t)r->frames * c.in_bpf,
                                  cudaMemcpyHostToDevice, st) == cudaSuccess;
            at[pi] += r->frames;
        }
        if (grp) {
            std::vector<rmdec_segment> segs;
            for (const Part& p : parts)
                segs.push_back(rmdec_segment{codes[p.code].member, base + p.in_off, p.frames,
                                             reinterpret_cast<uint32_t*>(base + p.out_off)});
            ok &= rmdec_group_decode(grp, segs.data(), (int)segs.size(), st) == RMDEC_OK;
        } else {
            for (const Part& p : parts)
                ok &= rmdec_decode(codes[p.code].h, base + p.in_off, p.frames, reinterpret_cast<uint32_t*>(base + p.out_off),
                                   st) == RMDEC_OK;
        }
        for (size_t q = 0; q < take.size(); q++) {
            Request* r = take[q];
            const Part& p = parts[req_part[q]];
            const Code& c = codes[r->code];
            ok &= cudaMemcpyAsync(r->out, base + p.out_off + (size_t)req_at[q] * c.out_bpf, (size_t)r->frames * c.out_bpf,
                                  cudaMemcpyDeviceToHost, st) == cudaSuccess;
        }
        cudaEventCreateWithFlags(&b->ev, cudaEventDisableTiming);
        cudaEventRecord(b->ev, st);
        nvtxRangePop();
        b->failed = !ok;
        lk.lock();
        inflight.push_back(b);
        return true;
    }

    void run() {
        cudaSetDevice(device);
        std::unique_lock<std::mutex> lk(mu);
        for (;;) {
            reap();
            bool launched = false;
            while (launch_one(lk)) launched = true;
            if (stop && inflight.empty()) break;
            if (launched) continue;
            // idle: wake on a new submission, or poll completions / batching deadlines
            cv_work.wait_for(lk, std::chrono::microseconds(inflight.empty() && pending.empty() ? 2000 : 20));
        }
    }
};

namespace {
thread_local std::string g_server_error;
}

extern "C" {

rmdec_status rmdec_server_create(rmdec_server_t* out, const rmdec_server_config* cfg) {
    if (!out || !cfg) {
        g_server_error = "null argument";
        return RMDEC_EINVAL;
    }
    *out = nullptr;
    if (cfg->n_streams < 1 || cfg->n_streams > 16 || cfg->arena_bytes <= 0 || cfg->max_batch_frames < 1 ||
        cfg->min_batch_frames < 0 || cfg->max_wait_us < 0 || cfg->fuse_codes < 0 || cfg->fuse_codes > 1) {
        g_server_error = "bad server configuration";
        return RMDEC_EINVAL;
    }
    rmdec_server* s = new (std::nothrow) rmdec_server;
    if (!s) return RMDEC_ENOMEM;
    s->cfg = *cfg;
    cudaError_t e = cudaGetDevice(&s->device);
    if (e != cudaSuccess) {
        g_server_error = std::string("no CUDA device: ") + cudaGetErrorString(e);
        delete s;
        return RMDEC_EDEVICE;
    }
    if ((e = rmdec_host::device_alloc(&s->arena_ptr, (size_t)cfg->arena_bytes)) != cudaSuccess) {
        g_server_error = std::string("arena allocation: ") + cudaGetErrorString(e);
        delete s;
        return RMDEC_ENOMEM;
    }
    s->arena.reset((size_t)cfg->arena_bytes);
    s->streams.resize(cfg->n_streams);
    s->stream_busy.assign(cfg->n_streams, false);
    for (auto& st : s->streams) cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
    s->worker = std::thread([s] { s->run(); });
    *out = s;
    return RMDEC_OK;
}

rmdec_status rmdec_server_add_decoder(rmdec_server_t s, rmdec_t h, int* code_id) {
    if (!s || !h || !code_id) return RMDEC_EINVAL;
    int n = 0, k = 0;
    if (rmdec_info(h, &n, &k, nullptr) != RMDEC_OK) return s->fail(RMDEC_EINVAL, "bad decoder handle");
    rmdec_host::MemberInfo mi;
    if (rmdec_host::member_info(h, false, &mi) != RMDEC_OK) return s->fail(RMDEC_EINVAL, "bad decoder handle");
    std::lock_guard<std::mutex> g(s->mu);
    const int id = (int)s->codes.size();
    int fam = -1, member = 0;
    if (s->cfg.fuse_codes && mi.algo == 0 && mi.m <= 9 && mi.r <= 3 && mi.hadamard == 0 && (mi.L == 1 || mi.L == 2 || mi.L == 4 || mi.L == 8)) {
        for (int f = 0; f < (int)s->families.size(); f++)
            if (s->families[f].L == mi.L && s->families[f].codes.size() < 16) fam = f;
        if (fam < 0) {
            s->families.emplace_back();
            fam = (int)s->families.size() - 1;
            s->families[fam].L = mi.L;
        }
        member = (int)s->families[fam].codes.size();
        s->families[fam].codes.push_back(id);
        s->families[fam].stale = true;
    }
    s->codes.push_back({h, (size_t)n * rmdec_host::llr_elem_bytes_of(h), (size_t)((k + 31) / 32) * 4, fam, member});
    *code_id = id;
    return RMDEC_OK;
}

rmdec_status rmdec_server_submit(rmdec_server_t s, int code_id, const void* llr_host, int64_t n_frames,
                                 uint32_t* bits_out_host, uint64_t* request) {
    if (!s || !request) return RMDEC_EINVAL;
    std::lock_guard<std::mutex> g(s->mu);
    if (code_id < 0 || code_id >= (int)s->codes.size()) return s->fail(RMDEC_EINVAL, "unknown code %d", code_id);
    if (n_frames < 1 || !llr_host || !bits_out_host) return s->fail(RMDEC_EINVAL, "bad request buffers");
    const auto& c = s->codes[code_id];
    if (n_frames > s->cfg.max_batch_frames ||
        align256((size_t)n_frames * c.in_bpf) + align256((size_t)n_frames * c.out_bpf) > (size_t)s->cfg.arena_bytes)
        return s->fail(RMDEC_EINVAL, "request of %lld frames exceeds the batch or arena limit", (long long)n_frames);
    Request* r = new Request;
    r->id = s->next_id++;
    r->code = code_id;
    r->llr = llr_host;
    r->frames = n_frames;
    r->out = bits_out_host;
    r->t_submit = Clock::now();
    if (!s->have_first) {
        s->have_first = true;
        s->t_first = r->t_submit;
    }
    s->pending.push_back(r);
    s->requests[r->id] = r;
    s->n_submitted++;
    *request = r->id;
    s->cv_work.notify_one();
    return RMDEC_OK;
}

rmdec_status rmdec_server_poll(rmdec_server_t s, uint64_t request, int64_t timeout_us, double* latency_us) {
    if (!s) return RMDEC_EINVAL;
    std::unique_lock<std::mutex> lk(s->mu);
    auto it = s->requests.find(request);
    if (it == s->requests.end()) return s->fail(RMDEC_EINVAL, "unknown request %llu", (unsigned long long)request);
    Request* r = it->second;
    if (!r->done && timeout_us > 0)
        s->cv_done.wait_for(lk, std::chrono::microseconds(timeout_us), [r] { return r->done; });
    if (!r->done) return timeout_us > 0 ? RMDEC_ETIMEDOUT : RMDEC_EBUSY;
    if (latency_us) *latency_us = std::chrono::duration<double, std::micro>(r->t_done - r->t_submit).count();
    const rmdec_status st = r->status;
    s->requests.erase(it);
    delete r;
    return st;
}

rmdec_status rmdec_server_cancel(rmdec_server_t s, uint64_t request) {
    if (!s) return RMDEC_EINVAL;
    std::lock_guard<std::mutex> g(s->mu);
    auto it = s->requests.find(request);
    if (it == s->requests.end()) return s->fail(RMDEC_EINVAL, "unknown request %llu", (unsigned long long)request);
    Request* r = it->second;
    auto pit = std::find(s->pending.begin(), s->pending.end(), r);
    if (pit == s->pending.end())
        return s->fail(RMDEC_EBUSY, "request %llu was already admitted", (unsigned long long)request);
    s->pending.erase(pit);
    r->done = true;
    r->status = RMDEC_ECANCELED;
    r->t_done = Clock::now();
    s->n_cancelled++;
    s->cv_done.notify_all();
    return RMDEC_OK;
}

rmdec_status rmdec_server_stats_get(rmdec_server_t s, rmdec_server_stats* out) {
    if (!s || !out) return RMDEC_EINVAL;
    std::unique_lock<std::mutex> g(s->mu);
    memset(out, 0, sizeof *out);
    out->submitted = s->n_submitted;
    out->completed = s->n_completed;
    out->frames_completed = s->frames_completed;
    out->batches = s->n_batches;
    out->queued = (int64_t)s->pending.size();
    out->cancelled = s->n_cancelled;
    int64_t inf = 0;
    for (Batch* b : s->inflight) inf += (int64_t)b->reqs.size();
    out->in_flight = inf;
    if (s->have_first && s->n_completed)
        out->busy_seconds = std::chrono::duration<double>(s->t_last - s->t_first).count();
    std::vector<double> l = s->latencies;
    out->latency_max_us = s->lat_max;
    g.unlock();  // sort outside the lock: the worker keeps admitting and retiring meanwhile
    if (!l.empty()) {
        std::sort(l.begin(), l.end());
        auto pct = [&](double q) { return l[std::min(l.size() - 1, (size_t)(q * (double)(l.size() - 1) + 0.5))]; };
        out->latency_p50_us = pct(0.50);
        out->latency_p99_us = pct(0.99);
    }
    return RMDEC_OK;
}

void rmdec_server_destroy(rmdec_server_t s) {
    if (!s) return;
    {
        std::lock_guard<std::mutex> g(s->mu);
        s->stop = true;
        for (Request* r : s->pending) {
            s->requests.erase(r->id);
            delete r;
        }
        s->pending.clear();
        s->cv_work.notify_all();
    }
    if (s->worker.joinable()) s->worker.join();
    for (auto& kv : s->requests) delete kv.second;
    for (auto& st : s->streams) cudaStreamDestroy(st);
    for (auto& f : s->families)
        if (f.grp) rmdec_group_destroy(f.grp);
    if (s->arena_ptr) cudaFree(s->arena_ptr);
    delete s;
}

const char* rmdec_server_last_error(rmdec_server_t s) {
    if (!s) return g_server_error.c_str();
    return s->err.c_str();
}

}  // extern "C"
