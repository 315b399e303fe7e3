// C ABI of libqudit.so (declared in include/qudit.h): state objects, exact
// gate classification, planning of the class enumeration and kernel
// dispatch.  Host code only; the kernels live in qd_kernels.cu.
#include <nvtx3/nvToolsExt.h>
#include <atomic>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "qd_internal.cuh"
#include "qd_runtime.h"
#include "qudit.h"

namespace qd {

static std::atomic<uint64_t> g_launches{0};
void count_launch(int n) { g_launches.fetch_add((uint64_t)n, std::memory_order_relaxed); }
static std::atomic<uint64_t> g_uploaded{0};
void count_upload(size_t bytes) { g_uploaded.fetch_add((uint64_t)bytes, std::memory_order_relaxed); }

static thread_local std::string g_err;

NvtxRange::NvtxRange(const char* name) { nvtxRangePushA(name); }
NvtxRange::~NvtxRange() { nvtxRangePop(); }

qd_status fail(qd_status st, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_err = buf;
    return st;
}

void set_last_error(const char* msg) { g_err = msg ? msg : ""; }

qd_status cuda_fail(cudaError_t e, const char* what) {
    return fail(QD_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}


qd_status make_layout(const int32_t* dims, int32_t n, Layout& L) {
    if (!dims) return fail(QD_ERR_ARG, "dims is NULL");
    if (n < 1 || n > QD_MAX_WIRES) return fail(QD_ERR_ARG, "number of wires %d outside [1, %d]", n, QD_MAX_WIRES);
    L.n = n;
    int64_t D = 1;
    for (int i = 0; i < n; ++i) {
        if (dims[i] < 2 || dims[i] > QD_MAX_DIM)
            return fail(QD_ERR_ARG, "dimension of wire %d is %d, outside [2, %d]", i, dims[i], QD_MAX_DIM);
        L.dims[i] = dims[i];
        L.b[i] = D;
        if (D > ((int64_t)1 << 44) / dims[i])
            return fail(QD_ERR_ARG, "state of more than 2^44 amplitudes");
        D *= dims[i];
    }
    L.b[n] = D;
    L.D = D;
    return QD_OK;
}

size_t amp_bytes(int32_t prec) { return prec == QD_C64 ? 8 : 16; }

// ---------------------------------------------------------------------------
// Planning
// ---------------------------------------------------------------------------

void build_map(const Layout& L, const int32_t* ins_w, const int64_t* ins_v, int m, IndexMap& map,
                      uint64_t& classes) {
    // sort inserted wires ascending (m <= kMaxInserted, insertion sort)
    int w[kMaxInserted];
    int64_t v[kMaxInserted];
    for (int i = 0; i < m; ++i) { w[i] = ins_w[i]; v[i] = ins_v[i]; }
    for (int i = 1; i < m; ++i)
        for (int k = i; k > 0 && w[k - 1] > w[k]; --k) {
            std::swap(w[k - 1], w[k]);
            std::swap(v[k - 1], v[k]);
        }
    map.m = m;
    map.fixed = 0;
    uint64_t prod = 1;
    for (int i = 0; i < m; ++i) {
        map.fixed += (uint64_t)v[i] * (uint64_t)L.b[w[i]];
        prod *= (uint64_t)L.dims[w[i]];
        if (i == 0) {
            map.seg[0].init((uint64_t)L.b[w[0]]);
            map.off[0] = 1;
        } else {
            map.seg[i].init((uint64_t)(L.b[w[i]] / L.b[w[i - 1] + 1]));
            map.off[i] = (uint64_t)L.b[w[i - 1] + 1];
        }
    }
    map.off[m] = (uint64_t)L.b[w[m - 1] + 1];
    classes = (uint64_t)L.D / prod;
}

qd_status make_plan(const Layout& L, int32_t prec, const int32_t* wires, int32_t k, const double* U,
                           const int32_t* cw, const int32_t* cv, int32_t nc, Plan& p) {
    if (prec != QD_C64 && prec != QD_C128) return fail(QD_ERR_ARG, "unknown precision %d", prec);
    if (!wires || !U) return fail(QD_ERR_ARG, "wires or matrix is NULL");
    if (k < 1 || k > L.n) return fail(QD_ERR_ARG, "gate acts on %d wires of %d", k, L.n);
    if (nc < 0 || nc > QD_MAX_CONTROLS) return fail(QD_ERR_ARG, "%d controls outside [0, %d]", nc, QD_MAX_CONTROLS);
    if (nc > 0 && (!cw || !cv)) return fail(QD_ERR_ARG, "control lists are NULL");
    if (k + nc > L.n) return fail(QD_ERR_ARG, "gate wires plus controls exceed the wire count");
    p.D = (uint64_t)L.D;
    bool used[kMaxWires] = {false};
    int64_t P = 1;
    for (int i = 0; i < k; ++i) {
        if (wires[i] < 0 || wires[i] >= L.n) return fail(QD_ERR_ARG, "gate wire %d out of range", wires[i]);
        if (used[wires[i]]) return fail(QD_ERR_ARG, "gate wire %d listed twice", wires[i]);
        used[wires[i]] = true;
        P *= L.dims[wires[i]];
        if (P > QD_MAX_GATE_DIM) return fail(QD_ERR_UNSUPPORTED, "gate dimension above %d", QD_MAX_GATE_DIM);
    }
    for (int i = 0; i < nc; ++i) {
        if (cw[i] < 0 || cw[i] >= L.n) return fail(QD_ERR_ARG, "control wire %d out of range", cw[i]);
        if (used[cw[i]]) return fail(QD_ERR_ARG, "control wire %d repeats a gate or control wire", cw[i]);
        if (cv[i] < 0 || cv[i] >= L.dims[cw[i]])
            return fail(QD_ERR_ARG, "control value %d of wire %d outside [0, %d)", cv[i], cw[i], L.dims[cw[i]]);
        used[cw[i]] = true;
    }
    int32_t ins_w[kMaxInserted];
    int64_t ins_v[kMaxInserted];
    int m = 0;
    for (int i = 0; i < k; ++i) { ins_w[m] = wires[i]; ins_v[m] = 0; ++m; }
    for (int i = 0; i < nc; ++i) { ins_w[m] = cw[i]; ins_v[m] = cv[i]; ++m; }
    build_map(L, ins_w, ins_v, m, p.map, p.classes);
    int64_t run = L.D;
    for (int i = 0; i < m; ++i) run = L.b[ins_w[i]] < run ? L.b[ins_w[i]] : run;
    p.run = run;
    p.P = (int)P;

    if (k == 1 && P <= kMaxSmallD) {
        const int d = (int)P;
        p.family = 0;
        p.d = d;
        p.bt = L.b[wires[0]];
        auto re = [&](int r, int c) { return U[2 * (r * d + c)]; };
        auto im = [&](int r, int c) { return U[2 * (r * d + c) + 1]; };
        auto nz = [&](int r, int c) { return re(r, c) != 0.0 || im(r, c) != 0.0; };
        auto one = [&](int r, int c) { return re(r, c) == 1.0 && im(r, c) == 0.0; };
        bool diag = true;
        for (int r = 0; r < d; ++r)
            for (int c = 0; c < d; ++c)
                if (r != c && nz(r, c)) diag = false;
        bool perm = true;
        int src[kMaxSmallD];
        bool col_used[kMaxSmallD] = {false};
        for (int r = 0; r < d && perm; ++r) {
            int cnt = 0;
            for (int c = 0; c < d; ++c)
                if (nz(r, c)) { ++cnt; src[r] = c; }
            if (cnt != 1 || col_used[src[r]]) perm = false;
            else col_used[src[r]] = true;
        }
        p.lmask = p.smask = 0;
        p.pure = false;
        for (int r = 0; r < kMaxSmallD; ++r) p.perm[r] = r < d ? r : 0;
        if (diag) {
            p.kind = kDiag;
            for (int r = 0; r < d; ++r)
                if (!one(r, r)) p.lmask |= 1u << r;
            p.smask = p.lmask;
        } else if (perm) {
            p.kind = kPerm;
            p.pure = true;
            for (int r = 0; r < d; ++r) {
                p.perm[r] = src[r];
                if (!one(r, src[r])) p.pure = false;
                if (src[r] != r || !one(r, src[r])) {
                    p.smask |= 1u << r;
                    p.lmask |= 1u << src[r];
                }
            }
        } else {
            p.kind = kDense;
            p.lmask = p.smask = (1u << d) - 1u;
        }
        p.vec = (prec == QD_C64 && (run % 2) == 0) ? 2 : 1;
    } else {
        p.family = 1;
        p.kind = kDense;
        p.vec = 1;
        p.d = 0;
        p.bt = 0;
        p.lmask = p.smask = 0;
        p.pure = false;
        for (int r = 0; r < P; ++r) {
            uint64_t o = 0;
            int rem = r;
            for (int i = 0; i < k; ++i) {
                o += (uint64_t)(rem % L.dims[wires[i]]) * (uint64_t)L.b[wires[i]];
                rem /= L.dims[wires[i]];
            }
            p.off[r] = o;
        }
    }
    return QD_OK;
}

}  // namespace qd

using namespace qd;

// ---------------------------------------------------------------------------
// State object
// ---------------------------------------------------------------------------

static qd_status init_state_common(qd_state* st) {
    QD_CUDA(cudaGetDevice(&st->device), "cudaGetDevice");
    int maxd = 2;
    for (int i = 0; i < st->L.n; ++i) maxd = st->L.dims[i] > maxd ? st->L.dims[i] : maxd;
    st->nb = reduce_blocks(st->L.D);
    cudaError_t e = cudaMalloc(&st->partials, sizeof(double) * 2 * (size_t)st->nb * maxd);
    if (e != cudaSuccess) return fail(QD_ERR_OOM, "reduction workspace: %s", cudaGetErrorString(e));
    e = cudaMalloc(&st->dev_out, sizeof(double) * kMaxGateDim);
    if (e != cudaSuccess) return fail(QD_ERR_OOM, "readout buffer: %s", cudaGetErrorString(e));
    e = cudaMallocHost(&st->host_out, sizeof(double) * kMaxGateDim);
    if (e != cudaSuccess) return fail(QD_ERR_OOM, "pinned readout buffer: %s", cudaGetErrorString(e));
    const size_t slot = amp_bytes(st->prec) * kMaxGateDim * kMaxGateDim;
    e = cudaMalloc(&st->ring_dev, slot * kRingSlots);
    if (e != cudaSuccess) return fail(QD_ERR_OOM, "matrix ring: %s", cudaGetErrorString(e));
    e = cudaMallocHost(&st->ring_host, slot * kRingSlots);
    if (e != cudaSuccess) return fail(QD_ERR_OOM, "pinned matrix ring: %s", cudaGetErrorString(e));
    for (int i = 0; i < kRingSlots; ++i) {
        QD_CUDA(cudaEventCreateWithFlags(&st->ring_ev[i], cudaEventDisableTiming), "cudaEventCreate");
        st->ring_ev_live[i] = true;
    }
    return QD_OK;
}

static void free_state(qd_state* st) {
    if (!st) return;
    cudaStreamSynchronize(st->stream);
    if (st->owns && st->psi) cudaFree(st->psi);
    if (st->partials) cudaFree(st->partials);
    if (st->dev_out) cudaFree(st->dev_out);
    if (st->host_out) cudaFreeHost(st->host_out);
    if (st->ring_dev) cudaFree(st->ring_dev);
    if (st->ring_host) cudaFreeHost(st->ring_host);
    for (int i = 0; i < kRingSlots; ++i)
        if (st->ring_ev_live[i]) cudaEventDestroy(st->ring_ev[i]);
    if (st->arena) {
        st->arena[0].release();
        st->arena[1].release();
        delete[] st->arena;
    }
    delete st->pend;
    delete st->lazy;
    qd::circuit_cache_free(st->ccache);
    delete st;
}

static qd_state* new_state() {
    qd_state* st = new (std::nothrow) qd_state;
    if (!st) return nullptr;
    std::memset(static_cast<void*>(st), 0, sizeof(qd_state));
    return st;
}

template <typename R>
static qd_status reset_impl(qd_state* st) {
    cudaError_t e = launch_set_basis<R>(st->psi, st->L.D, 0, st->stream);
    if (e != cudaSuccess) return cuda_fail(e, "reset");
    return QD_OK;
}

static qd_status reset_state(qd_state* st) {
    return st->prec == QD_C64 ? reset_impl<float>(st) : reset_impl<double>(st);
}

// ---------------------------------------------------------------------------
// Gate dispatch
// ---------------------------------------------------------------------------
template <typename R, int DT>
static cudaError_t run_gate1(qd_state* st, const Plan& p, const double* U) {
    using T2 = typename Cplx<R>::T2;
    Gate1Args<R, DT> a;
    std::memset(static_cast<void*>(&a), 0, sizeof a);
    a.psi = reinterpret_cast<T2*>(st->psi);
    a.D = p.D - g_bounds_shrink;
    a.n_elems = p.classes / (uint64_t)p.vec;
    a.bt = (uint64_t)p.bt;
    a.map = p.map;
    a.kind = p.kind;
    a.lmask = p.lmask;
    a.smask = p.smask;
    a.pure_perm = p.pure ? 1u : 0u;
    for (int r = 0; r < DT; ++r) a.perm[r] = p.perm[r];
    for (int i = 0; i < DT * DT; ++i) {
        a.U[i].x = (R)U[2 * i];
        a.U[i].y = (R)U[2 * i + 1];
    }
    if (p.vec == 2) {
        if constexpr (sizeof(R) == 4) return launch_gate1<R, DT, 2>(a, st->stream);
    }
    return launch_gate1<R, DT, 1>(a, st->stream);
}

template <typename R, int DT>
static cudaError_t run_gate1_scan(qd_state* st, const Plan& p, const double* U, const ScanControls& c) {
    using T2 = typename Cplx<R>::T2;
    Gate1Args<R, DT> a;
    std::memset(static_cast<void*>(&a), 0, sizeof a);
    a.psi = reinterpret_cast<T2*>(st->psi);
    a.D = p.D - g_bounds_shrink;
    a.n_elems = p.classes;  // one class per thread
    a.bt = (uint64_t)p.bt;
    a.map = p.map;
    a.kind = p.kind;
    a.lmask = p.lmask;
    a.smask = p.smask;
    a.pure_perm = p.pure ? 1u : 0u;
    for (int r = 0; r < DT; ++r) a.perm[r] = p.perm[r];
    for (int i = 0; i < DT * DT; ++i) {
        a.U[i].x = (R)U[2 * i];
        a.U[i].y = (R)U[2 * i + 1];
    }
    return launch_gate1_scan<R, DT>(a, c, st->stream);
}

template <typename R>
static cudaError_t dispatch_gate1_scan(qd_state* st, const Plan& p, const double* U, const ScanControls& c) {
    switch (p.d) {
        case 2: return run_gate1_scan<R, 2>(st, p, U, c);
        case 3: return run_gate1_scan<R, 3>(st, p, U, c);
        case 4: return run_gate1_scan<R, 4>(st, p, U, c);
        case 5: return run_gate1_scan<R, 5>(st, p, U, c);
        case 6: return run_gate1_scan<R, 6>(st, p, U, c);
        case 7: return run_gate1_scan<R, 7>(st, p, U, c);
        case 8: return run_gate1_scan<R, 8>(st, p, U, c);
        default: return cudaErrorInvalidValue;
    }
}

template <typename R>
static cudaError_t dispatch_gate1(qd_state* st, const Plan& p, const double* U) {
    switch (p.d) {
        case 2: return run_gate1<R, 2>(st, p, U);
        case 3: return run_gate1<R, 3>(st, p, U);
        case 4: return run_gate1<R, 4>(st, p, U);
        case 5: return run_gate1<R, 5>(st, p, U);
        case 6: return run_gate1<R, 6>(st, p, U);
        case 7: return run_gate1<R, 7>(st, p, U);
        case 8: return run_gate1<R, 8>(st, p, U);
        default: return cudaErrorInvalidValue;
    }
}

template <typename R>
static qd_status run_tile(qd_state* st, const Plan& p, const double* U) {
    using T2 = typename Cplx<R>::T2;
    const int P = p.P;
    const size_t slot_bytes = sizeof(T2) * kMaxGateDim * kMaxGateDim;
    const int s = st->ring_next;
    st->ring_next = (s + 1) % kRingSlots;
    QD_CUDA(cudaEventSynchronize(st->ring_ev[s]), "matrix ring wait");
    T2* h = reinterpret_cast<T2*>(static_cast<char*>(st->ring_host) + slot_bytes * s);
    T2* dptr = reinterpret_cast<T2*>(static_cast<char*>(st->ring_dev) + slot_bytes * s);
    for (int i = 0; i < P * P; ++i) {
        h[i].x = (R)U[2 * i];
        h[i].y = (R)U[2 * i + 1];
    }
    QD_CUDA(cudaMemcpyAsync(dptr, h, sizeof(T2) * P * P, cudaMemcpyHostToDevice, st->stream), "matrix upload");
    count_upload(sizeof(T2) * P * P);
    QD_CUDA(cudaEventRecord(st->ring_ev[s], st->stream), "matrix ring record");
    GateTileArgs<R> a;
    std::memset(static_cast<void*>(&a), 0, sizeof a);
    a.psi = reinterpret_cast<T2*>(st->psi);
    a.D = p.D - g_bounds_shrink;
    a.U = dptr;
    a.n_classes = p.classes;
    a.map = p.map;
    a.P = P;
    a.Q = 64;
    for (int r = 0; r < P; ++r) a.off[r] = p.off[r];
    cudaError_t e = launch_gate_tile<R>(a, st->stream, (int)gate_tile_smem<R>(P, a.Q));
    if (e != cudaSuccess) return cuda_fail(e, "tile gate kernel");
    return QD_OK;
}

// Deferred fusion: copy a validated gate into the state's queue.
static qd_status enqueue(qd_state* st, const int32_t* wires, int32_t k, const double* U, const int32_t* cw,
                         const int32_t* cv, int32_t nc, int P) {
    if (k > QD_MAX_GATE_WIRES || nc > QD_MAX_CONTROLS) return fail(QD_ERR_UNSUPPORTED, "gate too wide to queue");
    if (!st->pend) st->pend = new Pending();
    qd_gate_desc g;
    std::memset(&g, 0, sizeof g);
    g.n_wires = k;
    g.n_ctrl = nc;
    for (int i = 0; i < k; ++i) g.wires[i] = wires[i];
    for (int i = 0; i < nc; ++i) {
        g.ctrl_wires[i] = cw[i];
        g.ctrl_vals[i] = cv[i];
    }
    g.matrix_offset = (int64_t)(st->pend->mats.size() / 2);
    st->pend->gates.push_back(g);
    st->pend->mats.insert(st->pend->mats.end(), U, U + 2 * (size_t)P * P);
    if (st->pend->gates.size() >= kMaxPending) return flush_pending(st);
    return QD_OK;
}

qd_status qd::flush_pending(qd_state* st) {
    if (!st->pend || st->pend->gates.empty()) return QD_OK;
    Pending q;
    std::swap(q.gates, st->pend->gates);
    std::swap(q.mats, st->pend->mats);
    qd_fusion_opts o;
    std::memset(&o, 0, sizeof o);
    o.mode = QD_FUSE_BLOCK;
    o.block_dim = st->fuse_dim;
    o.tc_mode = st->tc_mode;
    return run_circuit(st, q.gates.data(), (int32_t)q.gates.size(), q.mats.data(), &o);
}

static void drop_pending(qd_state* st) {
    if (st->pend) {
        st->pend->gates.clear();
        st->pend->mats.clear();
    }
}

#define QD_FLUSH(st)                                \
    do {                                            \
        const qd_status f_ = ::qd::flush_pending(st); \
        if (f_ != QD_OK) return f_;                 \
    } while (0)

// queued gates, then the lazy frame: the device buffer holds the logical state
#define QD_MATERIALIZE(st)                            \
    do {                                              \
        QD_FLUSH(st);                                 \
        const qd_status m_ = ::qd::materialize(st);   \
        if (m_ != QD_OK) return m_;                   \
    } while (0)

// ---------------------------------------------------------------------------
// Lazy permutations and phases (qd_set_lazy).  The frame (sigma, phi) of
// each wire makes psi_L[x] = prod_w phi_w[x_w] psi_P[sigma(x)]:
//   - an uncontrolled single-wire gate with one unit-modulus entry per row
//     and column (X_{+a}, Z_d, S, T, their products: U[y, pi(y)]) only
//     updates the frame: sigma_w <- sigma_w o pi, phi_w[y] <- U[y, pi(y)]
//     phi_w[pi(y)]; no launch, no traffic;
//   - any other gate on wires W runs in the physical frame: control values
//     v -> sigma_c(v); U_phys[sigma_W(r), sigma_W(c)] = U[r, c] phi_W(c), and
//     phi_w = 1 for w in W afterwards (a controlled gate first applies the
//     phases of W as a diagonal gate: its unmatched classes keep them);
//   - materialize() applies psi[x] <- phi_w[x_w] psi[x with x_w -> sigma_w(x_w)]
//     on every touched wire (one monomial pass each) and resets the frame.
// ---------------------------------------------------------------------------
static bool unit_monomial(const double* U, int d, int* pi) {
    for (int r = 0; r < d; ++r) {
        int cnt = 0;
        for (int c = 0; c < d; ++c) {
            const double re = U[2 * (r * d + c)], im = U[2 * (r * d + c) + 1];
            if (re != 0.0 || im != 0.0) {
                ++cnt;
                pi[r] = c;
                if (std::fabs(std::sqrt(re * re + im * im) - 1.0) > 1e-12) return false;
            }
        }
        if (cnt != 1) return false;
    }
    bool seen[QD_MAX_DIM] = {false};
    for (int r = 0; r < d; ++r) {
        if (seen[pi[r]]) return false;
        seen[pi[r]] = true;
    }
    return true;
}

static void lazy_reset(LazyFrame& f, const Layout& L) {
    f.sigma.assign(L.n, {});
    f.phi.assign(L.n, {});
    f.touched.assign(L.n, 0);
    for (int w = 0; w < L.n; ++w) {
        f.sigma[w].resize(L.dims[w]);
        f.phi[w].assign(2 * (size_t)L.dims[w], 0.0);
        for (int y = 0; y < L.dims[w]; ++y) {
            f.sigma[w][y] = y;
            f.phi[w][2 * y] = 1.0;
        }
    }
}

static qd_status apply_now(qd_state* st, const int32_t* wires, int32_t k, const double* U, const int32_t* cw,
                           const int32_t* cv, int32_t nc);

qd_status qd::materialize(qd_state* st) {
    if (!st->lazy) return QD_OK;
    LazyFrame& f = *st->lazy;
    for (int w = 0; w < st->L.n; ++w) {
        if (!f.touched[w]) continue;
        const int d = st->L.dims[w];
        std::vector<double> M(2 * (size_t)d * d, 0.0);
        for (int r = 0; r < d; ++r) {
            M[2 * (r * d + f.sigma[w][r])] = f.phi[w][2 * r];
            M[2 * (r * d + f.sigma[w][r]) + 1] = f.phi[w][2 * r + 1];
        }
        const int32_t ww = w;
        const qd_status rc = apply_now(st, &ww, 1, M.data(), nullptr, nullptr, 0);
        if (rc != QD_OK) return rc;
        for (int y = 0; y < d; ++y) {
            f.sigma[w][y] = y;
            f.phi[w][2 * y] = 1.0;
            f.phi[w][2 * y + 1] = 0.0;
        }
        f.touched[w] = 0;
    }
    return QD_OK;
}

qd_status qd::apply_any(qd_state* st, const int32_t* wires, int32_t k, const double* U, const int32_t* cw,
                        const int32_t* cv, int32_t nc) {
    if (!st) return fail(QD_ERR_ARG, "state is NULL");
    if (!st->lazy || st->fuse_dim >= 2) return apply_now(st, wires, k, U, cw, cv, nc);
    Plan p;  // validation of the gate as given
    qd_status rc = make_plan(st->L, st->prec, wires, k, U, cw, cv, nc, p);
    if (rc != QD_OK) return rc;
    LazyFrame& f = *st->lazy;
    if (k == 1 && nc == 0) {
        const int w = wires[0], d = st->L.dims[w];
        int pi[QD_MAX_DIM];
        if (unit_monomial(U, d, pi)) {
            std::vector<int32_t> s2(d);
            std::vector<double> p2(2 * (size_t)d);
            for (int y = 0; y < d; ++y) {
                s2[y] = f.sigma[w][pi[y]];
                const double ur = U[2 * (y * d + pi[y])], ui = U[2 * (y * d + pi[y]) + 1];
                const double fr = f.phi[w][2 * pi[y]], fi = f.phi[w][2 * pi[y] + 1];
                p2[2 * y] = ur * fr - ui * fi;
                p2[2 * y + 1] = ur * fi + ui * fr;
            }
            f.sigma[w] = s2;
            f.phi[w] = p2;
            f.touched[w] = 1;
            return QD_OK;
        }
    }
    // run in the physical frame.  A controlled gate leaves the classes whose
    // controls are not met untouched, so the phases of its target wires
    // cannot be absorbed into its matrix: they are applied first, as a
    // diagonal gate in the physical frame.
    if (nc > 0) {
        for (int j = 0; j < k; ++j) {
            const int w = wires[j], d = st->L.dims[w];
            bool unit = true;
            for (int y = 0; y < d; ++y) unit = unit && f.phi[w][2 * y] == 1.0 && f.phi[w][2 * y + 1] == 0.0;
            if (unit) continue;
            std::vector<double> Dg(2 * (size_t)d * d, 0.0);
            for (int y = 0; y < d; ++y) {
                const int py = f.sigma[w][y];
                Dg[2 * ((size_t)py * d + py)] = f.phi[w][2 * y];
                Dg[2 * ((size_t)py * d + py) + 1] = f.phi[w][2 * y + 1];
            }
            const int32_t ww = w;
            rc = apply_now(st, &ww, 1, Dg.data(), nullptr, nullptr, 0);
            if (rc != QD_OK) return rc;
            for (int y = 0; y < d; ++y) {
                f.phi[w][2 * y] = 1.0;
                f.phi[w][2 * y + 1] = 0.0;
            }
        }
    }
    int P = 1;
    int dw[QD_MAX_GATE_WIRES];
    for (int j = 0; j < k; ++j) {
        dw[j] = st->L.dims[wires[j]];
        P *= dw[j];
    }
    std::vector<int> phys(P);
    std::vector<double> ph(2 * (size_t)P);
    for (int i = 0; i < P; ++i) {  // local index -> physical local index, phase of its digits
        int rem = i, o = 0, s = 1;
        double pr = 1.0, pim = 0.0;
        for (int j = 0; j < k; ++j) {
            const int x = rem % dw[j];
            rem /= dw[j];
            o += f.sigma[wires[j]][x] * s;
            s *= dw[j];
            const double fr = f.phi[wires[j]][2 * x], fi = f.phi[wires[j]][2 * x + 1];
            const double t = pr * fr - pim * fi;
            pim = pr * fi + pim * fr;
            pr = t;
        }
        phys[i] = o;
        ph[2 * i] = pr;
        ph[2 * i + 1] = pim;
    }
    std::vector<double> U2(2 * (size_t)P * P);
    for (int r = 0; r < P; ++r)
        for (int c = 0; c < P; ++c) {
            const double ur = U[2 * (r * P + c)], ui = U[2 * (r * P + c) + 1];
            const size_t o = 2 * ((size_t)phys[r] * P + phys[c]);
            U2[o] = ur * ph[2 * c] - ui * ph[2 * c + 1];
            U2[o + 1] = ur * ph[2 * c + 1] + ui * ph[2 * c];
        }
    std::vector<int32_t> cv2(nc > 0 ? nc : 1);
    for (int m = 0; m < nc; ++m) cv2[m] = f.sigma[cw[m]][cv[m]];
    rc = apply_now(st, wires, k, U2.data(), cw, nc > 0 ? cv2.data() : cv, nc);
    if (rc != QD_OK) return rc;
    for (int j = 0; j < k; ++j) {  // the wires' phases now live in the state
        const int w = wires[j];
        for (int y = 0; y < dw[j]; ++y) {
            f.phi[w][2 * y] = 1.0;
            f.phi[w][2 * y + 1] = 0.0;
        }
        bool id = true;
        for (int y = 0; y < dw[j]; ++y) id = id && f.sigma[w][y] == y;
        f.touched[w] = id ? 0 : 1;
    }
    return QD_OK;
}

static qd_status apply_now(qd_state* st, const int32_t* wires, int32_t k, const double* U, const int32_t* cw,
                           const int32_t* cv, int32_t nc) {
    if (!st) return fail(QD_ERR_ARG, "state is NULL");
    Plan p;
    qd_status rc = make_plan(st->L, st->prec, wires, k, U, cw, cv, nc, p);
    if (rc != QD_OK) return rc;
    if (p.classes == 0) return QD_OK;
    if (st->fuse_dim >= 2) return enqueue(st, wires, k, U, cw, cv, nc, p.P);
    if (p.family == 0) {
        if (p.smask == 0) return QD_OK;  // identity
        cudaError_t e = st->prec == QD_C64 ? dispatch_gate1<float>(st, p, U) : dispatch_gate1<double>(st, p, U);
        if (e != cudaSuccess) return cuda_fail(e, "gate kernel");
        return QD_OK;
    }
    if (st->prec == QD_C64 && st->tc_mode != QD_TC_OFF &&
        (p.P >= kTcMinP || (st->tc_mode == QD_TC_BF16X3 && nc == 0 && p.P >= kRingMinP))) {
        // tensor-core block: through the circuit path (descriptor upload + launch)
        qd_gate_desc g{};
        g.n_wires = k;
        g.n_ctrl = nc;
        for (int i = 0; i < k; ++i) g.wires[i] = wires[i];
        for (int i = 0; i < nc; ++i) {
            g.ctrl_wires[i] = cw[i];
            g.ctrl_vals[i] = cv[i];
        }
        g.matrix_offset = 0;
        qd_fusion_opts o;
        std::memset(&o, 0, sizeof o);
        o.mode = QD_FUSE_OFF;
        o.tc_mode = st->tc_mode;
        return run_circuit(st, &g, 1, U, &o);
    }
    return st->prec == QD_C64 ? run_tile<float>(st, p, U) : run_tile<double>(st, p, U);
}

// ---------------------------------------------------------------------------
// Readout helpers
// ---------------------------------------------------------------------------
static qd_status check_device_status(qd_state* st) {
    const int32_t e = tc_status_take(st->stream);
    if (e != 0) return fail(QD_ERR_TIMEOUT, "a tensor-core kernel gave up waiting for its MMAs (status %d)", e);
    return QD_OK;
}

qd_status qd::read_out(qd_state* st, int count, double* host) {
    QD_CUDA(cudaMemcpyAsync(st->host_out, st->dev_out, sizeof(double) * count, cudaMemcpyDeviceToHost, st->stream),
            "readout copy");
    QD_CUDA(cudaStreamSynchronize(st->stream), "readout sync");
    qd_status rc = check_device_status(st);
    if (rc != QD_OK) return rc;
    std::memcpy(host, st->host_out, sizeof(double) * count);
    return QD_OK;
}

#define QD_GUARD_BEGIN try {
#define QD_GUARD_END                                                 \
    }                                                                \
    catch (const std::bad_alloc&) { return fail(QD_ERR_OOM, "host allocation failed"); } \
    catch (...) { return fail(QD_ERR_ARG, "unexpected host exception"); }

extern "C" {

qd_status qd_state_create(const int32_t* dims, int32_t n, int32_t prec, void* stream, qd_state** out) {
    QD_GUARD_BEGIN
    if (!out) return fail(QD_ERR_ARG, "out is NULL");
    if (prec != QD_C64 && prec != QD_C128) return fail(QD_ERR_ARG, "unknown precision %d", prec);
    Layout L;
    qd_status rc = make_layout(dims, n, L);
    if (rc != QD_OK) return rc;
    qd_state* st = new_state();
    if (!st) return fail(QD_ERR_OOM, "host allocation failed");
    st->L = L;
    st->prec = prec;
    st->stream = reinterpret_cast<cudaStream_t>(stream);
    st->owns = true;
    st->bytes = (size_t)L.D * amp_bytes(prec);
    cudaError_t e = cudaMalloc(&st->psi, st->bytes);
    if (e != cudaSuccess) {
        st->psi = nullptr;
        free_state(st);
        return fail(QD_ERR_OOM, "state of %zu bytes: %s", (size_t)L.D * amp_bytes(prec), cudaGetErrorString(e));
    }
    rc = init_state_common(st);
    if (rc == QD_OK) rc = reset_state(st);
    if (rc != QD_OK) {
        std::string msg = g_err;
        free_state(st);
        g_err = msg;
        return rc;
    }
    *out = st;
    return QD_OK;
    QD_GUARD_END
}

qd_status qd_state_wrap(void* dev_ptr, size_t bytes, const int32_t* dims, int32_t n, int32_t prec, void* stream,
                        qd_state** out) {
    QD_GUARD_BEGIN
    if (!out || !dev_ptr) return fail(QD_ERR_ARG, "out or dev_ptr is NULL");
    if (prec != QD_C64 && prec != QD_C128) return fail(QD_ERR_ARG, "unknown precision %d", prec);
    if (reinterpret_cast<uintptr_t>(dev_ptr) % 16 != 0) return fail(QD_ERR_ARG, "dev_ptr is not 16-byte aligned");
    Layout L;
    qd_status rc = make_layout(dims, n, L);
    if (rc != QD_OK) return rc;
    if (bytes < (size_t)L.D * amp_bytes(prec))
        return fail(QD_ERR_ARG, "buffer of %zu bytes is smaller than %lld amplitudes", bytes, (long long)L.D);
    qd_state* st = new_state();
    if (!st) return fail(QD_ERR_OOM, "host allocation failed");
    st->L = L;
    st->prec = prec;
    st->stream = reinterpret_cast<cudaStream_t>(stream);
    st->owns = false;
    st->psi = dev_ptr;
    st->bytes = (size_t)L.D * amp_bytes(prec);
    rc = init_state_common(st);
    if (rc != QD_OK) {
        std::string msg = g_err;
        free_state(st);
        g_err = msg;
        return rc;
    }
    *out = st;
    return QD_OK;
    QD_GUARD_END
}

qd_status qd_state_destroy(qd_state* st) {
    QD_GUARD_BEGIN
    free_state(st);
    return QD_OK;
    QD_GUARD_END
}

qd_status qd_state_reset(qd_state* st) {
    QD_GUARD_BEGIN
    if (!st) return fail(QD_ERR_ARG, "state is NULL");
    drop_pending(st);
    if (st->lazy) lazy_reset(*st->lazy, st->L);
    return reset_state(st);
    QD_GUARD_END
}

qd_status qd_state_set_stream(qd_state* st, void* stream) {
    QD_GUARD_BEGIN
    if (!st) return fail(QD_ERR_ARG, "state is NULL");
    QD_MATERIALIZE(st);
    QD_CUDA(cudaStreamSynchronize(st->stream), "stream switch");
    st->stream = reinterpret_cast<cudaStream_t>(stream);
    return QD_OK;
    QD_GUARD_END
}

qd_status qd_state_info(const qd_state* st, int64_t* num_amplitudes, int32_t* num_wires, int32_t* prec) {
    if (!st) return fail(QD_ERR_ARG, "state is NULL");
    if (num_amplitudes) *num_amplitudes = st->L.D;
    if (num_wires) *num_wires = st->L.n;
    if (prec) *prec = st->prec;
    return QD_OK;
}

qd_status qd_state_device_ptr(const qd_state* st, void** dev_ptr) {
    QD_GUARD_BEGIN
    if (!st || !dev_ptr) return fail(QD_ERR_ARG, "state or out is NULL");
    QD_MATERIALIZE(const_cast<qd_state*>(st));  // queued gates and the lazy frame are the state's pending content
    *dev_ptr = st->psi;
    return QD_OK;
    QD_GUARD_END
}

qd_status qd_state_set_amplitudes(qd_state* st, const double* host) {
    QD_GUARD_BEGIN
    if (!st || !host) return fail(QD_ERR_ARG, "state or host buffer is NULL");
    drop_pending(st);
    if (st->lazy) lazy_reset(*st->lazy, st->L);
    const size_t D = (size_t)st->L.D;
    if (st->prec == QD_C128) {
        QD_CUDA(cudaMemcpyAsync(st->psi, host, D * 16, cudaMemcpyHostToDevice, st->stream), "upload");
    } else {
        std::vector<float> tmp(2 * D);
        for (size_t i = 0; i < 2 * D; ++i) tmp[i] = (float)host[i];
        QD_CUDA(cudaMemcpyAsync(st->psi, tmp.data(), D * 8, cudaMemcpyHostToDevice, st->stream), "upload");
        QD_CUDA(cudaStreamSynchronize(st->stream), "upload sync");
    }
    QD_CUDA(cudaStreamSynchronize(st->stream), "upload sync");
    return QD_OK;
    QD_GUARD_END
}

qd_status qd_state_get_amplitudes(qd_state* st, double* host) {
    QD_GUARD_BEGIN
    if (!st || !host) return fail(QD_ERR_ARG, "state or host buffer is NULL");
    QD_MATERIALIZE(st);
    const size_t D = (size_t)st->L.D;
    if (st->prec == QD_C128) {
        QD_CUDA(cudaMemcpyAsync(host, st->psi, D * 16, cudaMemcpyDeviceToHost, st->stream), "download");
        QD_CUDA(cudaStreamSynchronize(st->stream), "download sync");
    } else {
        // raw binary32 pairs into the upper half of the caller's buffer, then
        // widen front to back: element e is written at byte 8e and read from
        // byte 8D + 4e, which is never behind the write position.
        float* raw = reinterpret_cast<float*>(reinterpret_cast<char*>(host) + D * 8);
        QD_CUDA(cudaMemcpyAsync(raw, st->psi, D * 8, cudaMemcpyDeviceToHost, st->stream), "download");
        QD_CUDA(cudaStreamSynchronize(st->stream), "download sync");
        for (size_t e = 0; e < 2 * D; ++e) host[e] = (double)raw[e];
    }
    return QD_OK;
    QD_GUARD_END
}

static qd_status wire_move_args(qd_state* st, int32_t wire, const void* buf, int64_t& lo, int64_t& d, int64_t& hi) {
    if (!st || !buf) return fail(QD_ERR_ARG, "state or device buffer is NULL");
    if (wire < 0 || wire >= st->L.n) return fail(QD_ERR_ARG, "wire %d out of range [0, %d)", wire, st->L.n);
    const uintptr_t b = reinterpret_cast<uintptr_t>(buf), p = reinterpret_cast<uintptr_t>(st->psi);
    if (b % 16 != 0) return fail(QD_ERR_ARG, "device buffer is not 16-byte aligned");
    if (b < p + st->bytes && p < b + st->bytes) return fail(QD_ERR_ARG, "device buffer overlaps the state");
    lo = st->L.b[wire];
    d = st->L.dims[wire];
    hi = st->L.D / (lo * d);
    return QD_OK;
}

qd_status qd_state_wire_to_top(qd_state* st, int32_t wire, void* dev_out) {
    QD_GUARD_BEGIN
    int64_t lo, d, hi;
    qd_status rc = wire_move_args(st, wire, dev_out, lo, d, hi);
    if (rc != QD_OK) return rc;
    QD_MATERIALIZE(st);
    cudaError_t e = st->prec == QD_C64 ? launch_wire_move<float>(st->psi, dev_out, lo, d, hi, true, st->stream)
                                       : launch_wire_move<double>(st->psi, dev_out, lo, d, hi, true, st->stream);
    if (e != cudaSuccess) return cuda_fail(e, "wire move kernel");
    return QD_OK;
    QD_GUARD_END
}

qd_status qd_state_wire_from_top(qd_state* st, int32_t wire, const void* dev_in) {
    QD_GUARD_BEGIN
    int64_t lo, d, hi;
    qd_status rc = wire_move_args(st, wire, dev_in, lo, d, hi);
    if (rc != QD_OK) return rc;
    drop_pending(st);  // the state is overwritten, as by qd_state_set_amplitudes
    if (st->lazy) lazy_reset(*st->lazy, st->L);
    cudaError_t e = st->prec == QD_C64 ? launch_wire_move<float>(dev_in, st->psi, lo, d, hi, false, st->stream)
                                       : launch_wire_move<double>(dev_in, st->psi, lo, d, hi, false, st->stream);
    if (e != cudaSuccess) return cuda_fail(e, "wire move kernel");
    return QD_OK;
    QD_GUARD_END
}

// Checkpoint file: a 64-byte header (magic "QDSTATE1", precision, number of
// wires, the dims as int32 after it, then D), then the raw amplitudes.
// Copies go through a pinned staging buffer of at most 256 MiB, so no
// host buffer of the state's size is needed.
static constexpr char kCkptMagic[8] = {'Q', 'D', 'S', 'T', 'A', 'T', 'E', '1'};
static constexpr size_t kCkptChunk = (size_t)256 << 20;

qd_status qd_bounds_status(int64_t* first_bad_index, int32_t* checks_compiled) {
    const uint64_t v[3] = {bounds_take_kernels(), bounds_take_fusion(), bounds_take_tc()};
    uint64_t bad = 0;
    for (uint64_t x : v)
        if (x && !bad) bad = x;
    if (first_bad_index) *first_bad_index = bad ? (int64_t)(bad - 1) : -1;
    if (checks_compiled) *checks_compiled = QD_BOUNDS;
    if (bad) return fail(QD_ERR_DEVICE, "a kernel formed the index %llu outside its buffer (access skipped)",
                         (unsigned long long)(bad - 1));
    return QD_OK;
}

qd_status qd_test_set_bounds_shrink(int64_t amplitudes) {
    if (amplitudes < 0) return fail(QD_ERR_ARG, "negative shrink");
    g_bounds_shrink = (uint64_t)amplitudes;
    return QD_OK;
}

qd_status qd_state_save(qd_state* st, const char* path) {
    QD_GUARD_BEGIN
    if (!st || !path) return fail(QD_ERR_ARG, "state or path is NULL");
    QD_MATERIALIZE(st);
    FILE* f = std::fopen(path, "wb");
    if (!f) return fail(QD_ERR_ARG, "cannot open %s for writing", path);
    int64_t hdr[8] = {0};
    std::memcpy(hdr, kCkptMagic, 8);
    hdr[1] = st->prec;
    hdr[2] = st->L.n;
    hdr[3] = st->L.D;
    bool ok = std::fwrite(hdr, sizeof hdr, 1, f) == 1 &&
              std::fwrite(st->L.dims, sizeof(int32_t), (size_t)st->L.n, f) == (size_t)st->L.n;
    void* stage = nullptr;
    const size_t chunk = st->bytes < kCkptChunk ? st->bytes : kCkptChunk;
    if (ok && cudaMallocHost(&stage, chunk) != cudaSuccess) {
        std::fclose(f);
        return fail(QD_ERR_OOM, "checkpoint staging buffer");
    }
    for (size_t o = 0; ok && o < st->bytes; o += chunk) {
        const size_t n = st->bytes - o < chunk ? st->bytes - o : chunk;
        ok = cudaMemcpyAsync(stage, static_cast<char*>(st->psi) + o, n, cudaMemcpyDeviceToHost, st->stream) ==
                 cudaSuccess &&
             cudaStreamSynchronize(st->stream) == cudaSuccess && std::fwrite(stage, 1, n, f) == n;
    }
    if (stage) cudaFreeHost(stage);
    ok = (std::fclose(f) == 0) && ok;
    if (!ok) return fail(QD_ERR_CUDA, "checkpoint of the state to %s failed", path);
    return QD_OK;
    QD_GUARD_END
}

qd_status qd_state_load(qd_state* st, const char* path) {
    QD_GUARD_BEGIN
    if (!st || !path) return fail(QD_ERR_ARG, "state or path is NULL");
    FILE* f = std::fopen(path, "rb");
    if (!f) return fail(QD_ERR_ARG, "cannot open %s", path);
    int64_t hdr[8];
    std::vector<int32_t> dims((size_t)st->L.n);
    bool ok = std::fread(hdr, sizeof hdr, 1, f) == 1 && std::memcmp(hdr, kCkptMagic, 8) == 0 &&
              hdr[1] == st->prec && hdr[2] == st->L.n && hdr[3] == st->L.D &&
              std::fread(dims.data(), sizeof(int32_t), dims.size(), f) == dims.size() &&
              std::memcmp(dims.data(), st->L.dims, sizeof(int32_t) * dims.size()) == 0;
    if (!ok) {
        std::fclose(f);
        return fail(QD_ERR_ARG, "%s is not a checkpoint of a state with these dims and precision", path);
    }
    drop_pending(st);  // the state is overwritten, as by qd_state_set_amplitudes
    if (st->lazy) lazy_reset(*st->lazy, st->L);
    void* stage = nullptr;
    const size_t chunk = st->bytes < kCkptChunk ? st->bytes : kCkptChunk;
    if (cudaMallocHost(&stage, chunk) != cudaSuccess) {
        std::fclose(f);
        return fail(QD_ERR_OOM, "checkpoint staging buffer");
    }
    for (size_t o = 0; ok && o < st->bytes; o += chunk) {
        const size_t n = st->bytes - o < chunk ? st->bytes - o : chunk;
        ok = cudaStreamSynchronize(st->stream) == cudaSuccess && std::fread(stage, 1, n, f) == n &&
             cudaMemcpyAsync(static_cast<char*>(st->psi) + o, stage, n, cudaMemcpyHostToDevice, st->stream) ==
                 cudaSuccess;
    }
    ok = cudaStreamSynchronize(st->stream) == cudaSuccess && ok;
    cudaFreeHost(stage);
    std::fclose(f);
    if (!ok) return fail(QD_ERR_ARG, "reading the checkpoint %s failed (short file or copy error)", path);
    return QD_OK;
    QD_GUARD_END
}

qd_status qd_state_get_raw(qd_state* st, void* host, size_t bytes) {
    QD_GUARD_BEGIN
    if (!st || !host) return fail(QD_ERR_ARG, "state or host buffer is NULL");
    QD_MATERIALIZE(st);
    if (bytes < st->bytes) return fail(QD_ERR_ARG, "host buffer of %zu bytes < %zu", bytes, st->bytes);
    QD_CUDA(cudaMemcpyAsync(host, st->psi, st->bytes, cudaMemcpyDeviceToHost, st->stream), "download");
    QD_CUDA(cudaStreamSynchronize(st->stream), "download sync");
    return QD_OK;
    QD_GUARD_END
}

qd_status qd_state_get_raw_async(qd_state* st, void* host, size_t bytes) {
    QD_GUARD_BEGIN
    if (!st || !host) return fail(QD_ERR_ARG, "state or host buffer is NULL");
    QD_MATERIALIZE(st);
    if (bytes < st->bytes) return fail(QD_ERR_ARG, "host buffer of %zu bytes < %zu", bytes, st->bytes);
    QD_CUDA(cudaMemcpyAsync(host, st->psi, st->bytes, cudaMemcpyDeviceToHost, st->stream), "download");
    return QD_OK;
    QD_GUARD_END
}

qd_status qd_apply_gate(qd_state* st, int32_t target, const double* U) {
    qd::NvtxRange nvtx_("qd_apply_gate");
    QD_GUARD_BEGIN
    return apply_any(st, &target, 1, U, nullptr, nullptr, 0);
    QD_GUARD_END
}

qd_status qd_apply_controlled(qd_state* st, int32_t target, const double* U, const int32_t* cw,
                              const int32_t* cv, int32_t nc) {
    qd::NvtxRange nvtx_("qd_apply_controlled");
    QD_GUARD_BEGIN
    return apply_any(st, &target, 1, U, cw, cv, nc);
    QD_GUARD_END
}

qd_status qd_apply_multi(qd_state* st, const int32_t* wires, int32_t k, const double* U, const int32_t* cw,
                         const int32_t* cv, int32_t nc) {
    qd::NvtxRange nvtx_("qd_apply_multi");
    QD_GUARD_BEGIN
    return apply_any(st, wires, k, U, cw, cv, nc);
    QD_GUARD_END
}

qd_status qd_norm(qd_state* st, double* out) {
    qd::NvtxRange nvtx_("qd_norm");
    QD_GUARD_BEGIN
    if (!st || !out) return fail(QD_ERR_ARG, "state or out is NULL");
    QD_FLUSH(st);
    cudaError_t e = st->prec == QD_C64
                        ? launch_norm<float>(st->psi, st->L.D, st->partials, st->nb, st->dev_out, st->stream)
                        : launch_norm<double>(st->psi, st->L.D, st->partials, st->nb, st->dev_out, st->stream);
    if (e != cudaSuccess) return cuda_fail(e, "norm kernel");
    return read_out(st, 1, out);
    QD_GUARD_END
}

qd_status qd_probabilities_device(qd_state* st, double* dev_out) {
    QD_GUARD_BEGIN
    if (!st || !dev_out) return fail(QD_ERR_ARG, "state or out is NULL");
    QD_MATERIALIZE(st);
    if (reinterpret_cast<uintptr_t>(dev_out) % 8 != 0) return fail(QD_ERR_ARG, "dev_out is not 8-byte aligned");
    cudaError_t e = st->prec == QD_C64 ? launch_probs<float>(st->psi, st->L.D, dev_out, st->stream)
                                       : launch_probs<double>(st->psi, st->L.D, dev_out, st->stream);
    if (e != cudaSuccess) return cuda_fail(e, "probability kernel");
    return QD_OK;
    QD_GUARD_END
}

qd_status qd_probabilities(qd_state* st, double* host_out) {
    QD_GUARD_BEGIN
    if (!st || !host_out) return fail(QD_ERR_ARG, "state or out is NULL");
    QD_MATERIALIZE(st);
    double* tmp = nullptr;
    const size_t bytes = sizeof(double) * (size_t)st->L.D;
    cudaError_t e = cudaMallocAsync(reinterpret_cast<void**>(&tmp), bytes, st->stream);
    if (e != cudaSuccess) return fail(QD_ERR_OOM, "probability buffer: %s", cudaGetErrorString(e));
    e = st->prec == QD_C64 ? launch_probs<float>(st->psi, st->L.D, tmp, st->stream)
                           : launch_probs<double>(st->psi, st->L.D, tmp, st->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(host_out, tmp, bytes, cudaMemcpyDeviceToHost, st->stream);
    cudaFreeAsync(tmp, st->stream);
    if (e != cudaSuccess) return cuda_fail(e, "probabilities");
    QD_CUDA(cudaStreamSynchronize(st->stream), "probabilities sync");
    return QD_OK;
    QD_GUARD_END
}

qd_status qd_marginal(qd_state* st, int32_t wire, double* host_out) {
    QD_GUARD_BEGIN
    if (!st || !host_out) return fail(QD_ERR_ARG, "state or out is NULL");
    QD_FLUSH(st);
    if (wire < 0 || wire >= st->L.n) return fail(QD_ERR_ARG, "wire %d out of range", wire);
    IndexMap map;
    uint64_t classes;
    const int32_t w = wire;
    const int64_t v = 0;
    build_map(st->L, &w, &v, 1, map, classes);
    const int d = st->L.dims[wire];
    cudaError_t e = st->prec == QD_C64
                        ? launch_marginal<float>(st->psi, map, classes, (uint64_t)st->L.b[wire], d, st->partials,
                                                 st->nb, st->dev_out, st->stream)
                        : launch_marginal<double>(st->psi, map, classes, (uint64_t)st->L.b[wire], d, st->partials,
                                                  st->nb, st->dev_out, st->stream);
    if (e != cudaSuccess) return cuda_fail(e, "marginal kernel");
    const qd_status rc = read_out(st, d, host_out);
    if (rc != QD_OK || !st->lazy || !st->lazy->touched[wire]) return rc;
    // logical digit k sits at physical digit sigma(k); phases do not change probabilities
    std::vector<double> phys(host_out, host_out + d);
    for (int k2 = 0; k2 < d; ++k2) host_out[k2] = phys[st->lazy->sigma[wire][k2]];
    return QD_OK;
    QD_GUARD_END
}

qd_status qd_synchronize(qd_state* st) {
    QD_GUARD_BEGIN
    if (!st) return fail(QD_ERR_ARG, "state is NULL");
    QD_FLUSH(st);
    QD_CUDA(cudaStreamSynchronize(st->stream), "synchronize");
    return check_device_status(st);
    QD_GUARD_END
}

qd_status qd_apply_controlled_scan(qd_state* st, int32_t target, const double* U, const int32_t* cw,
                                   const int32_t* cv, int32_t nc) {
    QD_GUARD_BEGIN
    if (!st) return fail(QD_ERR_ARG, "state is NULL");
    QD_MATERIALIZE(st);  // queued gates and the lazy frame come first
    Plan full;  // validates the gate and its controls exactly as qd_apply_controlled does
    qd_status rc = make_plan(st->L, st->prec, &target, 1, U, cw, cv, nc, full);
    if (rc != QD_OK) return rc;
    if (full.family != 0) return fail(QD_ERR_UNSUPPORTED, "scan formulation: single wires of dimension <= 8");
    if (full.classes == 0 || full.smask == 0) return QD_OK;
    Plan p;  // every class of the target wire
    rc = make_plan(st->L, st->prec, &target, 1, U, nullptr, nullptr, 0, p);
    if (rc != QD_OK) return rc;
    ScanControls c;
    std::memset(static_cast<void*>(&c), 0, sizeof c);
    c.m = nc;
    for (int m = 0; m < nc; ++m) {
        c.stride[m].init((uint64_t)st->L.b[cw[m]]);
        c.dim[m].init((uint64_t)st->L.dims[cw[m]]);
        c.val[m] = (uint64_t)cv[m];
    }
    cudaError_t e = st->prec == QD_C64 ? dispatch_gate1_scan<float>(st, p, U, c) : dispatch_gate1_scan<double>(st, p, U, c);
    if (e != cudaSuccess) return cuda_fail(e, "scan gate kernel");
    return QD_OK;
    QD_GUARD_END
}

qd_status qd_set_fusion(qd_state* st, int32_t max_block_dim, int32_t tc_mode) {
    QD_GUARD_BEGIN
    if (!st) return fail(QD_ERR_ARG, "state is NULL");
    if (tc_mode != QD_TC_TF32X3 && tc_mode != QD_TC_BF16X3 && tc_mode != QD_TC_OFF)
        return fail(QD_ERR_ARG, "unknown tc_mode %d", tc_mode);
    // gates already queued run with the settings they were queued under
    QD_MATERIALIZE(st);
    st->fuse_dim = max_block_dim <= 1 ? 0 : (max_block_dim > QD_MAX_GATE_DIM ? QD_MAX_GATE_DIM : max_block_dim);
    st->tc_mode = tc_mode;
    return QD_OK;
    QD_GUARD_END
}

qd_status qd_set_lazy(qd_state* st, int32_t enable) {
    QD_GUARD_BEGIN
    if (!st) return fail(QD_ERR_ARG, "state is NULL");
    if (enable) {
        if (!st->lazy) {
            QD_FLUSH(st);
            st->lazy = new LazyFrame();
            lazy_reset(*st->lazy, st->L);
        }
        return QD_OK;
    }
    QD_MATERIALIZE(st);
    delete st->lazy;
    st->lazy = nullptr;
    return QD_OK;
    QD_GUARD_END
}

qd_status qd_flush(qd_state* st) {
    QD_GUARD_BEGIN
    if (!st) return fail(QD_ERR_ARG, "state is NULL");
    return flush_pending(st);
    QD_GUARD_END
}

const char* qd_last_error(void) { return g_err.c_str(); }

uint64_t qd_launch_count(void) { return g_launches.load(std::memory_order_relaxed); }

uint64_t qd_bytes_uploaded(void) { return g_uploaded.load(std::memory_order_relaxed); }

const char* qd_version(void) { return "qudit-gb300 0.1 (sm_103a)"; }

qd_status qd_plan_gate(const int32_t* dims, int32_t n, int32_t prec, const int32_t* wires, int32_t k,
                       const double* U, const int32_t* cw, const int32_t* cv, int32_t nc, qd_plan_info* out) {
    QD_GUARD_BEGIN
    if (!out) return fail(QD_ERR_ARG, "out is NULL");
    Layout L;
    qd_status rc = make_layout(dims, n, L);
    if (rc != QD_OK) return rc;
    Plan p;
    rc = make_plan(L, prec, wires, k, U, cw, cv, nc, p);
    if (rc != QD_OK) return rc;
    out->family = p.family;
    out->kind = p.kind;
    out->vec = p.vec;
    int rows = 0;
    for (int r = 0; r < 32; ++r) rows += (p.smask >> r) & 1u;
    out->touched_rows = p.family == 0 ? rows : p.P;
    out->classes = (int64_t)p.classes;
    out->run = p.run;
    return QD_OK;
    QD_GUARD_END
}

qd_status qd_selftest_host(int32_t trials) {
    QD_GUARD_BEGIN
    uint64_t s = 0x9E3779B97F4A7C15ull;
    auto rnd = [&]() {  // xorshift64*
        s ^= s >> 12;
        s ^= s << 25;
        s ^= s >> 27;
        return s * 0x2545F4914F6CDD1Dull;
    };
    // 1. division by invariant integers
    for (int t = 0; t < trials; ++t) {
        uint64_t d = 1 + rnd() % ((t % 3 == 0) ? 7 : (t % 3 == 1) ? 100000 : (1ull << 40));
        FastDiv f(d);
        const uint64_t ns[6] = {0, 1, d - 1, d, rnd() % (1ull << 45), (1ull << 45) - 1};
        for (uint64_t n : ns)
            if (f.div(n) != n / d)
                return fail(QD_ERR_ARG, "fast division %llu / %llu wrong", (unsigned long long)n, (unsigned long long)d);
    }
    // 2. class enumeration: map(g) visits exactly the indices whose inserted
    //    digits equal their fixed values, in increasing order.
    for (int t = 0; t < trials; ++t) {
        Layout L;
        int32_t dims[6];
        const int n = 2 + (int)(rnd() % 5);
        for (int i = 0; i < n; ++i) dims[i] = 2 + (int)(rnd() % 4);
        if (make_layout(dims, n, L) != QD_OK) return QD_ERR_ARG;
        const int m = 1 + (int)(rnd() % (uint64_t)(n - 1));
        int32_t w[6];
        int64_t v[6];
        int cnt = 0;
        for (int i = 0; i < n && cnt < m; ++i)
            if (rnd() % 2 == 0 || n - i == m - cnt) { w[cnt] = i; v[cnt] = (int64_t)(rnd() % (uint64_t)dims[i]); ++cnt; }
        IndexMap map;
        uint64_t classes;
        build_map(L, w, v, cnt, map, classes);
        uint64_t g = 0;
        for (int64_t j = 0; j < L.D; ++j) {
            bool match = true;
            for (int i = 0; i < cnt; ++i)
                if ((j / L.b[w[i]]) % L.dims[w[i]] != v[i]) match = false;
            if (!match) continue;
            if (g >= classes || map.map(g) != (uint64_t)j)
                return fail(QD_ERR_ARG, "class enumeration wrong at g=%llu", (unsigned long long)g);
            ++g;
        }
        if (g != classes) return fail(QD_ERR_ARG, "class count wrong");
    }
    return QD_OK;
    QD_GUARD_END
}

}  // extern "C"
