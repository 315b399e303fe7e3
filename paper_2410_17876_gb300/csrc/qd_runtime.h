// Host-side internals shared by the runtime translation units (C ABI,
// fusion planner): error reporting, layout and gate planning, the state
// object and the per-gate dispatcher.
#pragma once

#include <cuda_runtime.h>

#include <vector>

#include "qd_internal.cuh"
#include "qudit.h"

namespace qd {

qd_status fail(qd_status st, const char* fmt, ...);
qd_status cuda_fail(cudaError_t e, const char* what);
void set_last_error(const char* msg);

#define QD_CUDA(call, what)                                     \
    do {                                                        \
        cudaError_t e_ = (call);                                \
        if (e_ != cudaSuccess) return ::qd::cuda_fail(e_, what); \
    } while (0)

qd_status make_layout(const int32_t* dims, int32_t n, Layout& L);

// NVTX range for the lifetime of the object (API calls, fused passes, batch
// layers, served requests); costs one call through a function pointer when
// no profiler is attached.
struct NvtxRange {
    explicit NvtxRange(const char* name);
    ~NvtxRange();
    NvtxRange(const NvtxRange&) = delete;
    NvtxRange& operator=(const NvtxRange&) = delete;
};

// Device buffer plus pinned staging for kernel descriptors.  upload() waits
// until the previous upload from the staging buffer has completed before
// overwriting it, grows both buffers when needed (after synchronising the
// stream), and issues one asynchronous copy on the stream.
struct Arena {
    void* dev = nullptr;
    void* host = nullptr;
    size_t cap = 0;
    cudaEvent_t ev{};
    bool ev_live = false;
    qd_status upload(const void* bytes, size_t n, cudaStream_t s);
    void release();
};
size_t amp_bytes(int32_t prec);

// Plan of one gate for the per-gate kernels.
struct Plan {
    int family;   // 0 = per-class register kernel, 1 = shared-memory tile kernel
    int kind;
    int vec;
    int d;        // single-wire dimension (family 0)
    int P;
    uint32_t lmask, smask;
    bool pure;
    int perm[kMaxSmallD];
    int64_t bt;
    IndexMap map;
    uint64_t classes;
    uint64_t D;   // amplitudes of the state
    int64_t run;
    uint64_t off[kMaxGateDim];
};

// Gates queued by deferred fusion: descriptors and their matrices (2 P^2
// doubles each, at matrix_offset complex entries).
struct Pending {
    std::vector<qd_gate_desc> gates;
    std::vector<double> mats;
};
constexpr size_t kMaxPending = 4096;

// Lazy permutations and phases of the per-gate path: the logical state is
// psi_L[x] = prod_w phi_w[x_w] * psi_P[sigma(x)], sigma acting digit by digit
// (sigma_w a permutation of wire w's digits, phi_w unit-modulus phases).
struct LazyFrame {
    std::vector<std::vector<int32_t>> sigma;  // per wire, indexed by logical digit
    std::vector<std::vector<double>> phi;     // per wire, interleaved (re, im) per logical digit
    std::vector<char> touched;                // wire's sigma / phi differ from the identity
};

void build_map(const Layout& L, const int32_t* ins_w, const int64_t* ins_v, int m, IndexMap& map,
               uint64_t& classes);
qd_status make_plan(const Layout& L, int32_t prec, const int32_t* wires, int32_t k, const double* U,
                    const int32_t* cw, const int32_t* cv, int32_t nc, Plan& p);

}  // namespace qd

namespace qd {
struct CircuitCache;
}

static constexpr int kRingSlots = 8;

struct qd_state {
    qd::Layout L;
    int32_t prec;
    void* psi;
    bool owns;
    size_t bytes;
    cudaStream_t stream;
    int device;
    int nb;              // reduction blocks
    double* partials;    // nb * 2 * max_dim doubles
    double* dev_out;     // kMaxGateDim doubles
    double* host_out;    // pinned, kMaxGateDim doubles
    void* ring_dev;      // kRingSlots matrices of P*P complex (P <= 64)
    void* ring_host;     // pinned staging
    cudaEvent_t ring_ev[kRingSlots];
    bool ring_ev_live[kRingSlots];
    int ring_next;
    qd::Arena* arena;    // two descriptor arenas of circuit calls (device + pinned staging), alternating
    int32_t tc_mode;     // QD_TC_*: complex64 gates of 17..64 dimensions (0 = QD_TC_TF32X3)
    int32_t fuse_dim;    // deferred fusion: largest composed block (< 2: off)
    qd::Pending* pend;   // gates queued by deferred fusion
    qd::LazyFrame* lazy; // lazy permutations and phases (NULL: off)
    qd::CircuitCache* ccache;  // the last circuit of qd_apply_circuit, built once when it repeats
};

namespace qd {
void circuit_cache_free(CircuitCache* c);
qd_status run_circuit(qd_state* st, const qd_gate_desc* gates, int32_t n_gates, const double* matrices,
                      const qd_fusion_opts* opts);
qd_status flush_pending(qd_state* st);
qd_status materialize(qd_state* st);  // apply the lazy frame to the device state (no-op when off or identity)
qd_status apply_any(qd_state* st, const int32_t* wires, int32_t k, const double* U, const int32_t* cw,
                    const int32_t* cv, int32_t nc);
qd_status read_out(qd_state* st, int count, double* host);
// Host-to-device bytes of gate data (descriptors and matrices) copied so far.
void count_upload(size_t bytes);
}  // namespace qd
