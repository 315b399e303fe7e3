// Internal declarations shared by the library's translation units.
//
// Index arithmetic.  A gate on wires W with controls C visits the classes
// of amplitudes that differ only in the digits of W (section "Superposition
// gates": block size b_i = prod_{t<i} d_t, repetitions prod_{t>i} d_t).
// Instead of scanning all D indices for the control condition
// floor(j / b_c) mod d_c = v_c (section "Controlled and Multi-Controlled
// Gates"), the digits of W (set to 0) and of C (set to v_c) are *inserted*
// into a free index g that counts only the visited classes:
//
//   inserted wires sorted p_0 < ... < p_{m-1};
//   g = g_0 + seg_0 * (g_1 + seg_1 * (... g_m)),  seg_0 = b_{p_0},
//       seg_i = b_{p_i} / b_{p_{i-1}+1};
//   j(g) = fixed + g_0 + sum_{i>=1} g_i * b_{p_{i-1}+1},
//       fixed = sum over controls of v_c * b_c.
//
// The divisions by the invariant seg_i use the round-up multiply-high method
// of Granlund and Montgomery, "Division by invariant integers using
// multiplication" (PLDI 1994), section 4.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include <memory>
#include <vector>

#ifndef QD_HD
#define QD_HD __host__ __device__ __forceinline__
#endif

// Bounds-checked build (QD_BOUNDS=1; a debug build in place of a memory
// sanitizer).  The gate kernels check every global index they form against
// the size of the buffer it indexes.  An index outside records the first
// such index (plus one) in a device word of its translation unit and the
// access is skipped: no trap, no assert.  qd_bounds_status reads and clears
// the words.  The regular build compiles the checks out.
#ifndef QD_BOUNDS
#define QD_BOUNDS 0
#endif

namespace qd {

namespace {
#if QD_BOUNDS
__device__ unsigned long long g_bounds_bad = 0ull;
__device__ __forceinline__ bool in_bounds(uint64_t i, uint64_t n) {
    if (i < n) return true;
    atomicCAS(&g_bounds_bad, 0ull, (unsigned long long)i + 1ull);
    return false;
}
#else
__device__ __forceinline__ constexpr bool in_bounds(uint64_t, uint64_t) { return true; }
#endif
}  // namespace

// Host side of one translation unit's bounds word: 0, or 1 + the first index
// found outside its buffer; cleared on read (0 in the regular build).
#if QD_BOUNDS
#define QD_DEFINE_BOUNDS_TAKE(fname)                                                              \
    uint64_t fname() {                                                                            \
        unsigned long long v = 0ull, z = 0ull;                                                    \
        if (cudaMemcpyFromSymbol(&v, g_bounds_bad, sizeof v) != cudaSuccess) return 0;            \
        if (v) cudaMemcpyToSymbol(g_bounds_bad, &z, sizeof z);                                    \
        return (uint64_t)v;                                                                       \
    }
#else
#define QD_DEFINE_BOUNDS_TAKE(fname) \
    uint64_t fname() { return 0; }
#endif
uint64_t bounds_take_kernels();
uint64_t bounds_take_fusion();
uint64_t bounds_take_tc();
// Amplitudes the bounds-checked build hides from the end of every buffer
// (a testing hook: accesses there are then reported and skipped).
extern uint64_t g_bounds_shrink;

constexpr int kMaxWires = 48;
constexpr int kMaxInserted = 24;  // gate wires (<= 6 for P <= 64) + controls (<= 16)
constexpr int kMaxGateDim = 64;
constexpr int kMaxSmallD = 8;     // single-wire gates up to this dimension use the register kernel

QD_HD uint64_t umulhi64(uint64_t a, uint64_t b) {
#ifdef __CUDA_ARCH__
    return __umul64hi(a, b);
#else
    return (uint64_t)(((unsigned __int128)a * (unsigned __int128)b) >> 64);
#endif
}

// Unsigned 64-bit division by an invariant divisor d >= 1.
struct FastDiv {
    uint64_t d;
    uint64_t mul;
    uint32_t s1, s2;

    FastDiv() = default;
    __host__ explicit FastDiv(uint64_t div) { init(div); }
    // Valid for 1 <= div <= 2^62 (indices here stay far below that).
    __host__ void init(uint64_t div) {
        d = div;
        int l = 0;
        while (((uint64_t)1 << l) < div) ++l;  // l = ceil(log2 d)
        // mul = floor(2^64 (2^l - d) / d) + 1, which fits in 64 bits
        const unsigned __int128 num = ((unsigned __int128)(((uint64_t)1 << l) - div)) << 64;
        mul = (uint64_t)(num / div) + 1;
        s1 = l < 1 ? l : 1;
        s2 = l > 1 ? l - 1 : 0;
    }
    QD_HD uint64_t div(uint64_t n) const {
        const uint64_t t = umulhi64(mul, n);
        return (t + ((n - t) >> s1)) >> s2;
    }
    QD_HD void divmod(uint64_t n, uint64_t& q, uint64_t& r) const {
        q = div(n);
        r = n - q * d;
    }
};

// Unsigned 32-bit division by an invariant divisor (same method, N = 32).
struct FastDiv32 {
    uint32_t d, mul, s1, s2;
    __host__ void init(uint32_t div) {
        d = div;
        int l = 0;
        while (l < 32 && ((uint64_t)1 << l) < div) ++l;
        mul = (uint32_t)(((((uint64_t)1 << l) - div) << 32) / div + 1);
        s1 = l < 1 ? l : 1;
        s2 = l > 1 ? l - 1 : 0;
    }
    __device__ __forceinline__ uint32_t div(uint32_t n) const {
        const uint32_t t = __umulhi(mul, n);
        return (t + ((n - t) >> s1)) >> s2;
    }
};

// Free class index -> basis index of the class's member with all gate digits 0.
struct IndexMap {
    int32_t m;                   // number of inserted wires
    uint64_t fixed;              // sum of control values * strides
    FastDiv seg[kMaxInserted];   // seg[0..m-1]
    uint64_t off[kMaxInserted + 1];
    QD_HD uint64_t map(uint64_t g) const {
        uint64_t j = fixed;
        uint64_t r = g;
#pragma unroll 1
        for (int i = 0; i < m; ++i) {
            uint64_t q, rem;
            seg[i].divmod(r, q, rem);
            j += rem * off[i];
            r = q;
        }
        return j + r * off[m];
    }
};

// Host-side description of the state layout.
struct Layout {
    int32_t n;
    int32_t dims[kMaxWires];
    int64_t b[kMaxWires + 1];  // b[w] = prod_{t<w} d_t, b[n] = D
    int64_t D;
};

// Kinds a gate matrix is classified into (exactly, in binary64).
enum GateKind : int32_t { kDense = 0, kDiag = 1, kPerm = 2 };

template <typename R> struct Cplx;
template <> struct Cplx<float> { using T2 = float2; };
template <> struct Cplx<double> { using T2 = double2; };

// Arguments of the per-class register kernel (single wire, d <= kMaxSmallD).
template <typename R, int DT>
struct Gate1Args {
    using T2 = typename Cplx<R>::T2;
    T2* psi;
    uint64_t D;           // amplitudes of the state (bounds-checked build)
    uint64_t n_elems;     // classes / vec
    uint64_t bt;          // stride of the target wire (distance between class members)
    IndexMap map;
    int32_t kind;
    uint32_t lmask;       // rows loaded
    uint32_t smask;       // rows stored
    uint32_t pure_perm;   // permutation entries are all exactly 1
    int32_t perm[DT];     // kPerm: source row of each output row
    T2 U[DT * DT];
};

// Control tests of the scanning formulation: digit m of index j is
// (j / stride[m]) mod dim[m].d, compared with val[m].
struct ScanControls {
    int32_t m;
    FastDiv stride[kMaxInserted];
    FastDiv dim[kMaxInserted];
    uint64_t val[kMaxInserted];
};

// Arguments of the shared-memory tile kernel (any gate with P <= 64).
template <typename R>
struct GateTileArgs {
    using T2 = typename Cplx<R>::T2;
    T2* psi;
    uint64_t D;           // amplitudes of the state (bounds-checked build)
    const T2* U;          // device, P x P row-major
    uint64_t n_classes;
    IndexMap map;
    int32_t P;
    int32_t Q;            // classes per tile
    uint64_t off[kMaxGateDim];  // member offsets of local row r
};

// Launchers (qd_kernels.cu).  All return a cudaError_t of the launch.
template <typename R, int DT, int VEC>
cudaError_t launch_gate1(const Gate1Args<R, DT>& a, cudaStream_t s);
template <typename R, int DT>
cudaError_t launch_gate1_scan(const Gate1Args<R, DT>& a, const ScanControls& c, cudaStream_t s);
template <typename R>
cudaError_t launch_gate_tile(const GateTileArgs<R>& a, cudaStream_t s, int smem_bytes);
template <typename R>
size_t gate_tile_smem(int P, int Q);

template <typename R>
cudaError_t launch_set_basis(void* psi, int64_t D, int64_t index, cudaStream_t s);
template <typename R>
cudaError_t launch_norm(const void* psi, int64_t D, double* partials, int nblocks, double* dev_out,
                        cudaStream_t s);
template <typename R>
cudaError_t launch_probs(const void* psi, int64_t D, double* out, cudaStream_t s);
template <typename R>
cudaError_t launch_marginal(const void* psi, const IndexMap& map, uint64_t n_per_digit,
                            uint64_t stride, int d, double* partials, int nblocks, double* dev_out,
                            cudaStream_t s);
template <typename R>
cudaError_t launch_widen(const void* psi, int64_t D, double* out, cudaStream_t s);
template <typename R>
cudaError_t launch_narrow(const double* in, int64_t D, void* psi, cudaStream_t s);

// Tensor-core path for composed blocks (qd_tc.cu, complex64 only).
size_t block_tc_operand_bytes();
void block_tc_pack(const double* U, int P, int tc_mode, void* out);
cudaError_t launch_block_tc(float2* psi, uint64_t D, const void* a_ops, int tc_mode, bool renorm, uint64_t n_classes,
                            const IndexMap& map, int P, const uint64_t* off, cudaStream_t s);
bool block_is_unitary(const double* U, int P, double tol);
// BF16x3 blocks without controls through the ring of tiles: the kernel's
// arguments for a block on `wires` (k wires, the gate's order) with the
// P x P matrix U, and its B operand (to be uploaded); nullptr where the
// block does not suit that kernel (the register-staged one then runs).
struct BlockRing;
std::shared_ptr<const BlockRing> block_ring_prepare(const Layout& L, float2* psi, const int32_t* wires, int k,
                                                    int P, const double* U, bool renorm,
                                                    std::vector<unsigned char>& b_ops);
cudaError_t launch_block_ring(const BlockRing& r, const void* b_ops, cudaStream_t s);
int32_t tc_status_take(cudaStream_t s);
int32_t* tc_status_ptr();  // device status word shared by the kernels with bounded waits
constexpr int kTcMinP = 17;  // complex64 blocks of at least this dimension go to the tensor cores
constexpr int kRingMinP = 9;  // BF16x3: blocks without controls of at least this dimension, through the tile ring

int reduce_blocks(int64_t D);

// Norms of many states in two launches (batches), each state's result the
// bits launch_norm gives it: nb = reduce_blocks(D) partial blocks starting
// at partial pair part_off, the sum written to norms[out_index].
struct NormEntry {
    const void* psi;
    int64_t D;
    uint32_t nb;
    uint32_t a16;        // complex64 amplitudes 16-byte aligned
    uint64_t part_off;
    uint32_t out_index;
    uint32_t pad_;
};
template <typename R>
cudaError_t launch_norm_batch(const NormEntry* entries, const uint64_t* block_prefix, int32_t n,
                              uint64_t total_blocks, double* partials, double* norms, cudaStream_t s);
// Set many states to |0...0> in one launch: chunk_prefix[e] = chunks of
// kBasisChunkAmps amplitudes before entry e.
constexpr int64_t kBasisChunkAmps = 1 << 16;
template <typename R>
cudaError_t launch_basis_batch(const NormEntry* entries, const uint64_t* chunk_prefix, int32_t n,
                               uint64_t total_chunks, cudaStream_t s);

// Move one wire to the most significant digit (to_top) or back: with lo =
// b_w, d = d_w, hi = D / (lo d), index (h d + y) lo + l of the state is index
// (y hi + h) lo + l of the moved copy.  Out of place (src != dst).
template <typename R>
cudaError_t launch_wire_move(const void* src, void* dst, int64_t lo, int64_t d, int64_t hi, bool to_top,
                             cudaStream_t s);

void count_launch(int n = 1);

}  // namespace qd
