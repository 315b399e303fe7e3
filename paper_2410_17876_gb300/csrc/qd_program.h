// Circuit programs shared by the circuit, batch and serving entry points:
// validated gates, fusion settings, the launches of a circuit with their
// descriptors, and the one-CTA small-circuit kernel's task records.
#pragma once

#include <cstring>
#include <functional>
#include <vector>

#include "qd_internal.cuh"
#include "qd_runtime.h"

namespace qd {

struct HGate {
    int k, nc, P;
    int wires[QD_MAX_GATE_WIRES];
    int cw[QD_MAX_CONTROLS], cv[QD_MAX_CONTROLS];
    const double* U;
    Plan plan;
    bool diag, fusable;
    bool unitary;  // U^H U = I to 1e-10 (binary64); blocks of unitary gates are unitary
    uint64_t tmask, cmask;
};

struct FuseCfg {
    int mode;
    int64_t Tmax;
    int min_gates;
    int64_t min_row;
    int block_dim;  // largest composed block inside a pass (< 4: no composition)
    int tc_mode;    // QD_TC_*: complex64 blocks of 17..64 dimensions
    bool runs;      // complex64 tile passes: runs of single-wire gates may be applied in registers
};

int64_t tile_limit(int32_t prec);
FuseCfg fuse_cfg(const qd_fusion_opts* o, int32_t prec);
qd_status check_cfg(const FuseCfg& cfg, int32_t prec);

// Validate and classify a circuit's gates (QD_ERR_ARG / UNSUPPORTED naming the gate).
qd_status load_gates(const Layout& L, int32_t prec, const qd_gate_desc* gates, int32_t n, const double* matrices,
                     std::vector<HGate>& out);

using Op = std::function<cudaError_t(cudaStream_t, const char*)>;

struct Program {
    std::vector<char> desc;
    std::vector<Op> ops;
    size_t reserve(size_t n) {
        const size_t o = (desc.size() + 255) & ~(size_t)255;
        desc.resize(o + n);
        return o;
    }
    size_t put(const void* p, size_t n) {
        const size_t o = reserve(n);
        std::memcpy(desc.data() + o, p, n);
        return o;
    }
};

// Ops of a whole circuit on the state at psi: optional reset to |0...0>,
// then the planned passes in order (no CUDA call is made here).
template <typename R>
void build_program(const Layout& L, void* psi, const std::vector<HGate>& G, const FuseCfg& cfg, bool reset_first,
                   Program& prog);

// Issue a program's launches on stream s; its descriptors are at base.
qd_status issue(const Program& prog, const char* base, cudaStream_t s);

// One small circuit of a batch (whole state in one CTA).
struct SmallTask {
    uint64_t psi_off;     // byte offset of the state in the batch's state arena
    uint64_t chunk_off;   // byte offset of its first chunk in the descriptor arena
    uint32_t D;           // amplitudes
    uint32_t nchunks;
    uint32_t norm_index;  // slot of its squared norm
    uint32_t pad_;
};

// A circuit runs whole in one CTA when its state fits (D <= small_max) and
// every gate can join a fused pass; *dmax receives its largest wire dimension.
bool small_eligible(const Layout& L, const std::vector<HGate>& G, int64_t small_max, int* dmax);

// Append the circuit's one-CTA chunks to prog; returns the first chunk's
// offset and sets *nchunks.
template <typename R>
size_t put_small_chunks(const Layout& L, const std::vector<HGate>& G, const FuseCfg& cfg, Program& prog,
                        uint32_t* nchunks);

// Launch the one-CTA kernel over ntasks small circuits (tasks in device memory).
template <typename R>
cudaError_t launch_batch_small(const SmallTask* tasks, int ntasks, int dmax, uint32_t max_d, char* state_base,
                               const char* desc_base, double* norms, cudaStream_t s);

}  // namespace qd
