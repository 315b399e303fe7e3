// Serving loop: circuits arrive over time, are admitted while device memory
// (state bytes) and execution slots allow, run concurrently with everything
// already on the GPU, and report latency stamps.  The paper simulates one
// circuit at a time; requests share nothing, so each runs on its own stream
// (or, for states that fit one CTA, together with the other small requests
// admitted in the same step in one one-CTA-per-circuit launch).  A request's
// kernels depend only on its own circuit, so its result is the same alone
// and in any mix.
//
// One worker thread owns the server's streams: it releases timed
// submissions, admits requests in arrival order (first-fit allocation in one
// device arena of the byte budget), issues their programs, polls completion
// events and publishes results.  The programs themselves (pass planning,
// block composition, descriptors: about half a millisecond of host time for
// a 277-gate request) are built by a pool of builder threads as soon as a
// request is admitted, so that one host thread's planning does not cap the
// number of requests served per second.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <new>
#include <thread>
#include <unordered_map>
#include <vector>

#include "qd_internal.cuh"
#include "qd_program.h"
#include "qd_runtime.h"

using namespace qd;

namespace {

using Clock = std::chrono::steady_clock;

// First-fit allocator over [0, cap) with coalescing of freed blocks.
class RangeAlloc {
  public:
    void reset(size_t cap) {
        free_.clear();
        if (cap) free_[0] = cap;
    }
    bool alloc(size_t n, size_t& off) {
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second >= n) {
                off = it->first;
                const size_t rest = it->second - n;
                const size_t start = it->first + n;
                free_.erase(it);
                if (rest) free_[start] = rest;
                return true;
            }
        }
        return false;
    }
    void release(size_t off, size_t n) {
        auto it = free_.emplace(off, n).first;
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

struct Request {
    uint64_t id;
    int32_t keep;
    double release;  // server-clock time it becomes visible (its arrival)
    Layout L;
    std::vector<qd_gate_desc> descs;
    std::vector<double> mats;
    std::vector<HGate> G;
    bool small;
    int dmax;
    size_t off, bytes;
    double t_admit, t_done;
    double norm;
    int32_t status;
    Program prog;                // built by a builder thread after admission
    std::atomic<int> built{0};   // 0 pending, 1 built, 2 failed
};

struct Slot {  // runs one non-small request at a time
    cudaStream_t stream;
    cudaEvent_t done;
    Arena arena;
    double* partials;
    double* dnorm;
    double* hnorm;  // pinned
    std::shared_ptr<Request> req;
    bool issued = false;
};

// The one-CTA program of a group of small requests, built by a builder thread.
struct GroupBuild {
    std::vector<std::shared_ptr<Request>> reqs;
    Program prog;
    size_t o3 = 0, o5 = 0;
    int n3 = 0, n5 = 0;
    uint32_t m3 = 1, m5 = 1;
    std::atomic<int> built{0};  // 0 pending, 1 built, 2 failed
};

struct Lane {  // runs one group of small requests at a time
    cudaStream_t stream;
    cudaEvent_t done;
    Arena arena;
    double* dnorms;
    double* hnorms;  // pinned
    std::vector<std::shared_ptr<Request>> reqs;
    std::shared_ptr<GroupBuild> gb;
    bool issued = false;
};

// A build task: a non-small request's program, or a small-request group's.
struct BuildTask {
    std::shared_ptr<Request> req;
    std::shared_ptr<GroupBuild> group;
};

constexpr int kLanes = 4;

}  // namespace

struct qd_server {
    int32_t prec;
    int device;
    size_t budget;
    int max_group;
    int64_t small_max;
    FuseCfg cfg;
    char* arena_dev;
    RangeAlloc ralloc;
    std::vector<Slot> slots;
    Lane lanes[kLanes];
    Clock::time_point t0;

    std::mutex mu;
    std::condition_variable cv;
    std::deque<std::shared_ptr<Request>> submitted;  // by release time order of submission
    std::vector<qd_request_result> results;
    std::unordered_map<uint64_t, std::shared_ptr<Request>> kept;
    uint64_t next_id = 1;
    uint64_t n_submitted = 0, n_done = 0;
    std::atomic<bool> stop{false};
    std::thread worker;

    std::mutex bmu;  // builder pool
    std::condition_variable bcv;
    std::deque<BuildTask> bq;
    bool bstop = false;
    std::vector<std::thread> builders;

    double now() const { return std::chrono::duration<double>(Clock::now() - t0).count(); }
};

namespace {

size_t state_bytes(const qd_server* s, int64_t D) {
    return (((size_t)D * (s->prec == QD_C64 ? 8 : 16)) + 255) & ~(size_t)255;
}

void publish(qd_server* s, const std::shared_ptr<Request>& r) {
    qd_request_result out{};
    out.id = r->id;
    out.status = r->status;
    out.kept = (r->keep && r->status == QD_OK) ? 1 : 0;
    out.num_amplitudes = r->L.D;
    out.norm = r->norm;
    out.t_arrival = r->release;
    out.t_admit = r->t_admit;
    out.t_done = r->t_done;
    std::lock_guard<std::mutex> lk(s->mu);
    s->results.push_back(out);
    if (out.kept) s->kept[r->id] = r;
    s->n_done++;
    s->cv.notify_all();
}

// Builder thread: host-side construction of programs (no stream work).
template <typename R>
void builder_loop(qd_server* s) {
    cudaSetDevice(s->device);
    while (true) {
        BuildTask t;
        {
            std::unique_lock<std::mutex> lk(s->bmu);
            s->bcv.wait(lk, [&] { return s->bstop || !s->bq.empty(); });
            if (s->bq.empty()) return;  // stopping and nothing left
            t = std::move(s->bq.front());
            s->bq.pop_front();
        }
        int ok = 1;
        try {
            if (t.req) {
                Request& r = *t.req;
                build_program<R>(r.L, s->arena_dev + r.off, r.G, s->cfg, true, r.prog);
            } else {
                GroupBuild& g = *t.group;
                std::vector<SmallTask> t3, t5;
                for (size_t i = 0; i < g.reqs.size(); ++i) {
                    const Request& r = *g.reqs[i];
                    SmallTask st{};
                    st.psi_off = r.off;
                    st.D = (uint32_t)r.L.D;
                    st.norm_index = (uint32_t)i;
                    st.chunk_off = put_small_chunks<R>(r.L, r.G, s->cfg, g.prog, &st.nchunks);
                    if (r.dmax <= 3) {
                        t3.push_back(st);
                        g.m3 = std::max(g.m3, st.D);
                    } else {
                        t5.push_back(st);
                        g.m5 = std::max(g.m5, st.D);
                    }
                }
                g.o3 = t3.empty() ? 0 : g.prog.put(t3.data(), sizeof(SmallTask) * t3.size());
                g.o5 = t5.empty() ? 0 : g.prog.put(t5.data(), sizeof(SmallTask) * t5.size());
                g.n3 = (int)t3.size();
                g.n5 = (int)t5.size();
            }
        } catch (...) {
            ok = 2;
        }
        if (t.req) t.req->built.store(ok, std::memory_order_release);
        else t.group->built.store(ok, std::memory_order_release);
    }
}

void enqueue_build(qd_server* s, BuildTask t) {
    {
        std::lock_guard<std::mutex> lk(s->bmu);
        s->bq.push_back(std::move(t));
    }
    s->bcv.notify_one();
}

template <typename R>
bool issue_big(qd_server* s, Slot& sl, const std::shared_ptr<Request>& r) {
    NvtxRange nvtx_("served request");
    const Program& prog = r->prog;
    if (sl.arena.upload(prog.desc.data(), prog.desc.size(), sl.stream) != QD_OK) return false;
    if (issue(prog, static_cast<const char*>(sl.arena.dev), sl.stream) != QD_OK) return false;
    if (launch_norm<R>(s->arena_dev + r->off, r->L.D, sl.partials, reduce_blocks(r->L.D), sl.dnorm, sl.stream) !=
        cudaSuccess)
        return false;
    if (cudaMemcpyAsync(sl.hnorm, sl.dnorm, sizeof(double), cudaMemcpyDeviceToHost, sl.stream) != cudaSuccess)
        return false;
    return cudaEventRecord(sl.done, sl.stream) == cudaSuccess;
}

template <typename R>
bool issue_small(qd_server* s, Lane& ln) {
    NvtxRange nvtx_("served small-request group");
    const GroupBuild& g = *ln.gb;
    if (ln.arena.upload(g.prog.desc.data(), g.prog.desc.size(), ln.stream) != QD_OK) return false;
    const char* base = static_cast<const char*>(ln.arena.dev);
    if (launch_batch_small<R>(reinterpret_cast<const SmallTask*>(base + g.o3), g.n3, 3, g.m3, s->arena_dev, base,
                              ln.dnorms, ln.stream) != cudaSuccess)
        return false;
    if (launch_batch_small<R>(reinterpret_cast<const SmallTask*>(base + g.o5), g.n5, 5, g.m5, s->arena_dev, base,
                              ln.dnorms, ln.stream) != cudaSuccess)
        return false;
    if (cudaMemcpyAsync(ln.hnorms, ln.dnorms, sizeof(double) * ln.reqs.size(), cudaMemcpyDeviceToHost,
                        ln.stream) != cudaSuccess)
        return false;
    return cudaEventRecord(ln.done, ln.stream) == cudaSuccess;
}

template <typename R>
void worker_loop(qd_server* s) {
    cudaSetDevice(s->device);
    std::deque<std::shared_ptr<Request>> pending;  // released, waiting for admission (FIFO)
    std::vector<std::shared_ptr<Request>> timed;   // submitted with a future release time
    while (true) {
        {
            std::unique_lock<std::mutex> lk(s->mu);
            while (!s->submitted.empty()) {
                std::shared_ptr<Request> r = s->submitted.front();
                s->submitted.pop_front();
                if (r->status == -1) {  // qd_server_release: give a kept state's bytes back
                    s->ralloc.release(r->off, r->bytes);
                    continue;
                }
                timed.push_back(r);
            }
        }
        const double now = s->now();
        // release arrivals whose time has come, in release order
        std::stable_sort(timed.begin(), timed.end(),
                         [](const std::shared_ptr<Request>& a, const std::shared_ptr<Request>& b) {
                             return a->release < b->release;
                         });
        size_t nrel = 0;
        while (nrel < timed.size() && timed[nrel]->release <= now) ++nrel;
        for (size_t i = 0; i < nrel; ++i) pending.push_back(timed[i]);
        timed.erase(timed.begin(), timed.begin() + (long)nrel);

        bool progressed = nrel > 0;
        // admission in arrival order
        int free_lane = -1;
        for (int l = 0; l < kLanes; ++l)
            if (s->lanes[l].reqs.empty()) {
                free_lane = l;
                break;
            }
        std::vector<std::shared_ptr<Request>> group;
        while (!pending.empty()) {
            std::shared_ptr<Request> r = pending.front();
            int slot = -1;
            if (r->small) {
                if (free_lane < 0 || (int)group.size() >= s->max_group) break;
            } else {
                for (size_t k = 0; k < s->slots.size(); ++k)
                    if (!s->slots[k].req) {
                        slot = (int)k;
                        break;
                    }
                if (slot < 0) break;
            }
            size_t off = 0;
            if (!s->ralloc.alloc(r->bytes, off)) break;  // wait for memory to free up
            pending.pop_front();
            r->off = off;
            r->t_admit = s->now();
            progressed = true;
            if (r->small) {
                group.push_back(r);
            } else {
                Slot& sl = s->slots[(size_t)slot];
                sl.req = r;
                sl.issued = false;
                enqueue_build(s, BuildTask{r, nullptr});
            }
        }
        if (!group.empty()) {
            Lane& ln = s->lanes[free_lane];
            ln.reqs = group;
            ln.gb = std::make_shared<GroupBuild>();
            ln.gb->reqs = group;
            ln.issued = false;
            enqueue_build(s, BuildTask{nullptr, ln.gb});
        }
        // issue what the builders have finished
        for (Slot& sl : s->slots) {
            if (!sl.req || sl.issued) continue;
            const int b = sl.req->built.load(std::memory_order_acquire);
            if (b == 0) continue;
            sl.issued = true;
            progressed = true;
            if (b == 2) {
                sl.req->status = QD_ERR_OOM;  // host failure while building
            } else if (!issue_big<R>(s, sl, sl.req)) {
                cudaGetLastError();
                sl.req->status = QD_ERR_CUDA;
            }
            sl.req->prog = Program();  // descriptors uploaded, launches issued
        }
        for (Lane& ln : s->lanes) {
            if (ln.reqs.empty() || ln.issued) continue;
            const int b = ln.gb->built.load(std::memory_order_acquire);
            if (b == 0) continue;
            ln.issued = true;
            progressed = true;
            if (b == 2) {
                for (auto& r : ln.reqs) r->status = QD_ERR_OOM;
            } else if (!issue_small<R>(s, ln)) {
                cudaGetLastError();
                for (auto& r : ln.reqs) r->status = QD_ERR_CUDA;
            }
            ln.gb.reset();
        }
        // completions
        for (Slot& sl : s->slots) {
            if (!sl.req || !sl.issued) continue;
            const cudaError_t q = sl.req->status == QD_OK ? cudaEventQuery(sl.done) : cudaSuccess;
            if (q == cudaErrorNotReady) continue;
            std::shared_ptr<Request> r = sl.req;
            sl.req.reset();
            r->t_done = s->now();
            if (q != cudaSuccess) r->status = QD_ERR_CUDA;
            if (r->status == QD_OK) r->norm = *sl.hnorm;
            if (!(r->keep && r->status == QD_OK)) s->ralloc.release(r->off, r->bytes);
            publish(s, r);
            progressed = true;
        }
        for (Lane& ln : s->lanes) {
            if (ln.reqs.empty() || !ln.issued) continue;
            const bool failed = ln.reqs[0]->status != QD_OK;
            const cudaError_t q = failed ? cudaSuccess : cudaEventQuery(ln.done);
            if (q == cudaErrorNotReady) continue;
            const double t = s->now();
            for (size_t i = 0; i < ln.reqs.size(); ++i) {
                std::shared_ptr<Request> r = ln.reqs[i];
                r->t_done = t;
                if (q != cudaSuccess) r->status = QD_ERR_CUDA;
                if (r->status == QD_OK) r->norm = ln.hnorms[i];
                if (!(r->keep && r->status == QD_OK)) s->ralloc.release(r->off, r->bytes);
                publish(s, r);
            }
            ln.reqs.clear();
            progressed = true;
        }
        bool busy = !pending.empty() || !timed.empty();
        for (const Slot& sl : s->slots) busy = busy || (bool)sl.req;
        for (const Lane& ln : s->lanes) busy = busy || !ln.reqs.empty();
        if (s->stop.load() && !busy) {
            std::lock_guard<std::mutex> lk(s->mu);
            if (s->submitted.empty()) break;
        }
        if (!busy) {
            std::unique_lock<std::mutex> lk(s->mu);
            s->cv.wait_for(lk, std::chrono::milliseconds(2), [&] { return !s->submitted.empty() || s->stop.load(); });
        } else if (!progressed) {
            std::this_thread::sleep_for(std::chrono::microseconds(20));
        }
    }
}

void destroy_server(qd_server* s) {
    if (!s) return;
    if (s->worker.joinable()) {
        s->stop.store(true);
        s->cv.notify_all();
        s->worker.join();
    }
    {
        std::lock_guard<std::mutex> lk(s->bmu);
        s->bstop = true;
    }
    s->bcv.notify_all();
    for (std::thread& t : s->builders)
        if (t.joinable()) t.join();
    cudaDeviceSynchronize();
    for (Slot& sl : s->slots) {
        if (sl.stream) cudaStreamDestroy(sl.stream);
        if (sl.done) cudaEventDestroy(sl.done);
        sl.arena.release();
        if (sl.partials) cudaFree(sl.partials);
        if (sl.dnorm) cudaFree(sl.dnorm);
        if (sl.hnorm) cudaFreeHost(sl.hnorm);
    }
    for (Lane& ln : s->lanes) {
        if (ln.stream) cudaStreamDestroy(ln.stream);
        if (ln.done) cudaEventDestroy(ln.done);
        ln.arena.release();
        if (ln.dnorms) cudaFree(ln.dnorms);
        if (ln.hnorms) cudaFreeHost(ln.hnorms);
    }
    if (s->arena_dev) cudaFree(s->arena_dev);
    delete s;
}

}  // namespace

extern "C" {

qd_status qd_server_create(int32_t prec, const qd_server_opts* opts, qd_server** out) {
    try {
        if (!out) return fail(QD_ERR_ARG, "out is NULL");
        if (prec != QD_C64 && prec != QD_C128) return fail(QD_ERR_ARG, "unknown precision %d", prec);
        qd_server* s = new (std::nothrow) qd_server();
        if (!s) return fail(QD_ERR_OOM, "host allocation failed");
        s->prec = prec;
        s->budget = (opts && opts->hbm_budget_bytes) ? (size_t)opts->hbm_budget_bytes : ((size_t)8 << 30);
        const int nslots = (opts && opts->max_slots > 0) ? std::min(opts->max_slots, 256) : 16;
        s->max_group = (opts && opts->max_group > 0) ? opts->max_group : 1024;
        s->small_max = (opts && opts->small_max_amps > 0) ? opts->small_max_amps : (prec == QD_C64 ? 8192 : 4096);
        qd_fusion_opts fo{};
        if (opts) fo = opts->fusion;
        s->cfg = fuse_cfg(&fo, prec);
        qd_status rc = check_cfg(s->cfg, prec);
        if (rc == QD_OK && s->small_max > tile_limit(prec))
            rc = fail(QD_ERR_UNSUPPORTED, "small-request tile above shared memory");
        if (rc != QD_OK) {
            delete s;
            return rc;
        }
        s->arena_dev = nullptr;
        s->t0 = Clock::now();
        cudaGetDevice(&s->device);
        cudaError_t e = cudaMalloc(reinterpret_cast<void**>(&s->arena_dev), s->budget);
        if (e != cudaSuccess) {
            s->arena_dev = nullptr;
            destroy_server(s);
            return fail(QD_ERR_OOM, "server state arena of %zu bytes: %s", s->budget, cudaGetErrorString(e));
        }
        s->ralloc.reset(s->budget);
        s->slots.resize((size_t)nslots);
        for (Slot& sl : s->slots) {
            e = cudaStreamCreateWithFlags(&sl.stream, cudaStreamNonBlocking);
            if (e == cudaSuccess) e = cudaEventCreateWithFlags(&sl.done, cudaEventDisableTiming);
            if (e == cudaSuccess) e = cudaMalloc(&sl.partials, sizeof(double) * 2 * 1024);
            if (e == cudaSuccess) e = cudaMalloc(&sl.dnorm, sizeof(double));
            if (e == cudaSuccess) e = cudaMallocHost(&sl.hnorm, sizeof(double));
            if (e != cudaSuccess) break;
        }
        for (Lane& ln : s->lanes) {
            if (e != cudaSuccess) break;
            e = cudaStreamCreateWithFlags(&ln.stream, cudaStreamNonBlocking);
            if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ln.done, cudaEventDisableTiming);
            if (e == cudaSuccess) e = cudaMalloc(&ln.dnorms, sizeof(double) * (size_t)s->max_group);
            if (e == cudaSuccess) e = cudaMallocHost(&ln.hnorms, sizeof(double) * (size_t)s->max_group);
        }
        if (e != cudaSuccess) {
            destroy_server(s);
            return fail(QD_ERR_CUDA, "server set-up: %s", cudaGetErrorString(e));
        }
        tc_status_ptr();  // resolved once here, before builder threads may ask for it
        const unsigned hw = std::thread::hardware_concurrency();
        const int nb = (int)std::max(1u, std::min(8u, hw > 2 ? hw - 2 : 1u));
        for (int i = 0; i < nb; ++i)
            s->builders.emplace_back(prec == QD_C64 ? std::thread(builder_loop<float>, s)
                                                    : std::thread(builder_loop<double>, s));
        s->worker = prec == QD_C64 ? std::thread(worker_loop<float>, s) : std::thread(worker_loop<double>, s);
        *out = s;
        return QD_OK;
    } catch (...) {
        return fail(QD_ERR_OOM, "host exception in qd_server_create");
    }
}

qd_status qd_server_submit_at(qd_server* s, const qd_circuit* c, int32_t keep_state, double release_time,
                              uint64_t* id_out) {
    try {
        if (!s || !c) return fail(QD_ERR_ARG, "server or circuit is NULL");
        auto r = std::make_shared<Request>();
        qd_status rc = make_layout(c->dims, c->n_wires, r->L);
        if (rc != QD_OK) return rc;
        if (c->n_gates < 0 || (c->n_gates > 0 && (!c->gates || !c->matrices)))
            return fail(QD_ERR_ARG, "bad gate list");
        r->descs.assign(c->gates, c->gates + c->n_gates);
        int64_t nmat = 0;
        for (const qd_gate_desc& g : r->descs) {
            int64_t P = 1;
            for (int m = 0; m < g.n_wires && m < QD_MAX_GATE_WIRES; ++m)
                if (g.wires[m] >= 0 && g.wires[m] < r->L.n) P *= r->L.dims[g.wires[m]];
            nmat = std::max(nmat, g.matrix_offset + P * P);
        }
        r->mats.assign(c->matrices, c->matrices + 2 * nmat);
        rc = load_gates(r->L, s->prec, r->descs.data(), (int32_t)r->descs.size(), r->mats.data(), r->G);
        if (rc != QD_OK) return rc;
        r->bytes = state_bytes(s, r->L.D);
        if (r->bytes > s->budget)
            return fail(QD_ERR_UNSUPPORTED, "state of %zu bytes exceeds the server budget of %zu", r->bytes, s->budget);
        r->small = small_eligible(r->L, r->G, s->small_max, &r->dmax);
        r->keep = keep_state;
        r->status = QD_OK;
        r->norm = 0.0;
        std::lock_guard<std::mutex> lk(s->mu);
        r->id = s->next_id++;
        r->release = release_time < 0 ? s->now() : release_time;
        s->submitted.push_back(r);
        s->n_submitted++;
        s->cv.notify_all();
        if (id_out) *id_out = r->id;
        return QD_OK;
    } catch (...) {
        return fail(QD_ERR_OOM, "host exception in qd_server_submit");
    }
}

qd_status qd_server_submit(qd_server* s, const qd_circuit* c, int32_t keep_state, uint64_t* id_out) {
    return qd_server_submit_at(s, c, keep_state, -1.0, id_out);
}

qd_status qd_server_poll(qd_server* s, qd_request_result* out, int32_t max, int32_t* n_out) {
    if (!s || !n_out || (max > 0 && !out)) return fail(QD_ERR_ARG, "bad poll arguments");
    std::lock_guard<std::mutex> lk(s->mu);
    const int32_t n = (int32_t)std::min<size_t>((size_t)std::max(max, 0), s->results.size());
    for (int32_t i = 0; i < n; ++i) out[i] = s->results[(size_t)i];
    s->results.erase(s->results.begin(), s->results.begin() + n);
    *n_out = n;
    return QD_OK;
}

qd_status qd_server_drain(qd_server* s, double timeout_s) {
    if (!s) return fail(QD_ERR_ARG, "server is NULL");
    std::unique_lock<std::mutex> lk(s->mu);
    const bool ok = s->cv.wait_for(lk, std::chrono::duration<double>(timeout_s),
                                   [&] { return s->n_done == s->n_submitted; });
    if (!ok) return fail(QD_ERR_TIMEOUT, "%llu of %llu requests finished before the timeout",
                         (unsigned long long)s->n_done, (unsigned long long)s->n_submitted);
    return QD_OK;
}

qd_status qd_server_now(qd_server* s, double* t) {
    if (!s || !t) return fail(QD_ERR_ARG, "server or out is NULL");
    *t = s->now();
    return QD_OK;
}

qd_status qd_server_get_amplitudes(qd_server* s, uint64_t id, double* host) {
    if (!s || !host) return fail(QD_ERR_ARG, "server or out is NULL");
    std::shared_ptr<Request> r;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        auto it = s->kept.find(id);
        if (it == s->kept.end()) return fail(QD_ERR_ARG, "request %llu has no kept state", (unsigned long long)id);
        r = it->second;
    }
    const size_t D = (size_t)r->L.D;
    const char* src = s->arena_dev + r->off;
    // the request finished (its event completed) before it was published
    if (s->prec == QD_C128) {
        QD_CUDA(cudaMemcpy(host, src, D * 16, cudaMemcpyDeviceToHost), "server download");
    } else {
        float* raw = reinterpret_cast<float*>(reinterpret_cast<char*>(host) + D * 8);
        QD_CUDA(cudaMemcpy(raw, src, D * 8, cudaMemcpyDeviceToHost), "server download");
        for (size_t e = 0; e < 2 * D; ++e) host[e] = (double)raw[e];
    }
    return QD_OK;
}

qd_status qd_server_release(qd_server* s, uint64_t id) {
    if (!s) return fail(QD_ERR_ARG, "server is NULL");
    std::shared_ptr<Request> r;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        auto it = s->kept.find(id);
        if (it == s->kept.end()) return fail(QD_ERR_ARG, "request %llu has no kept state", (unsigned long long)id);
        r = it->second;
        s->kept.erase(it);
    }
    // The allocator belongs to the worker thread: hand the block back through
    // a released request with no work.
    auto rel = std::make_shared<Request>();
    rel->off = r->off;
    rel->bytes = r->bytes;
    rel->id = 0;
    rel->status = -1;  // marker: free only
    std::lock_guard<std::mutex> lk(s->mu);
    s->submitted.push_back(rel);
    s->cv.notify_all();
    return QD_OK;
}

qd_status qd_server_destroy(qd_server* s) {
    destroy_server(s);
    return QD_OK;
}

}  // extern "C"
