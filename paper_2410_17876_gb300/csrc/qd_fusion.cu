// Circuits and gate fusion: a host planner that groups consecutive gates into
// passes over a cached wire set, and the kernel that applies one pass.
//
// A pass with cached wire set S (the lowest wires 0..L-1, whose amplitudes are
// contiguous, plus the high wires its gates act on) treats the state as
// D / prod_{w in S} d_w independent tiles: a tile holds the amplitudes whose
// digits outside S are fixed.  Every gate whose target wires lie in S maps
// each tile onto itself (its classes, section "Superposition gates", never
// leave a tile), and a control outside S has one digit per tile, so the
// condition of section "Controlled and Multi-Controlled Gates" is evaluated
// once per tile.  A CTA loads a tile into shared memory, applies the pass's
// gates in order, and writes the tile back: one HBM round trip for the whole
// pass instead of one per gate.
#include <algorithm>
#include <cstring>
#include <functional>
#include <new>
#include <string>
#include <vector>

#include "qd_internal.cuh"
#include "qd_program.h"
#include "qd_tc_common.cuh"
#include "qd_runtime.h"

namespace qd {

constexpr int kMaxFusedD = 5;      // single-wire gates up to this dimension join fused passes
constexpr int kMaxTileCtrl = 7;    // controls of a fused gate (inside or outside the tile)
constexpr int kMaxLocalIns = 1 + kMaxTileCtrl;
constexpr int kMaxPassGates = 64;  // gates per fused pass (their descriptors live in shared memory)
constexpr size_t kPlanWindow = 256;  // remaining gates examined when a pass's wire set is chosen
constexpr int kMaxRows = 2048;

// Class enumeration inside a tile (local index space of S), 32-bit.
struct __align__(16) LocalMap {
    int32_t m;
    uint32_t fixed;
    uint32_t pad_[2];
    FastDiv32 seg[kMaxLocalIns];
    uint32_t off[kMaxLocalIns + 4];
    __device__ __forceinline__ uint32_t map(uint32_t g) const {
        uint32_t j = fixed, r = g;
        for (int i = 0; i < m; ++i) {
            const uint32_t q = seg[i].div(r);
            j += (r - q * seg[i].d) * off[i];
            r = q;
        }
        return j + r * off[m];
    }
};

constexpr int kMaxBlock = 16;       // largest composed block on CUDA cores (product of its wires' dimensions)
constexpr int kMaxTcBlock = 32;     // complex64: blocks of 17..32 dimensions run on the tensor cores inside tiles
constexpr uint8_t kTcBlock = 3;     // FGate kind of such a block
constexpr uint8_t kRun = 4;         // FGate kind of a run of single-wire gates applied in registers
constexpr int kMaxRunGates = 16;    // gates per run
constexpr int kMaxChunkGates = 64;  // gate records per chunk
constexpr int kPoolEntries = 2048;  // matrix entries per chunk (complex, in the state's precision)

// One gate or composed block inside a chunk.  Built on the host, staged in
// shared memory by every CTA that applies the chunk.
//   single = 1: one wire of dimension P = d (in-tile controls inserted in map;
//               lst/step give the one-division enumeration when m == 1);
//   single = 0: a dense / diagonal / monomial P x P block over several wires,
//               members of a class at base + off[r].
struct __align__(16) FGate {
    LocalMap map;
    uint32_t nclasses;
    uint32_t lst, step;
    uint32_t u_off;  // matrix: entries [u_off, u_off + PP * PP) of the chunk pool, row-major, PP columns
    uint8_t P, PP, kind, single;
    uint8_t n_out, pure, unitary, nsub;
    uint16_t lmask, smask;
    uint32_t op_off;  // kTcBlock: byte offset of the B operand (hi | lo, 32 KB) from the descriptor base
    uint8_t out_w[8], out_v[8];  // controls outside the tile: global wire, value
    uint16_t off[kMaxTcBlock];
    // kRun: the block's wire dimensions (shape id), and per gate the position
    // of its target among the block's wires, the members it acts on (its
    // in-block controls met) and its d x d matrix in the chunk pool
    uint8_t shape, pad1[3];
    uint8_t sub_pos[kMaxRunGates];
    uint16_t sub_mask[kMaxRunGates];
    uint16_t sub_u[kMaxRunGates];
};

// Chunk header; the chunk is [header][ngates FGate][npool matrix entries], 16-byte aligned.
struct __align__(16) ChunkHdr {
    uint32_t ngates, npool, bytes, pad;
};

template <typename R>
__host__ __device__ inline size_t chunk_bytes(uint32_t ngates, uint32_t npool) {
    return sizeof(ChunkHdr) + sizeof(FGate) * (size_t)ngates + sizeof(typename Cplx<R>::T2) * (size_t)npool;
}
template <typename R>
__host__ __device__ inline size_t chunk_smem_max() {
    return (chunk_bytes<R>(kMaxChunkGates, kPoolEntries) + 15) & ~(size_t)15;
}

template <typename R>
struct FusedArgs {
    using T2 = typename Cplx<R>::T2;
    T2* psi;
    const char* chunks;  // first chunk (device)
    int32_t nchunks;
    uint32_t T;      // tile amplitudes
    uint32_t bL;     // contiguous run (row) length
    uint32_t rows;   // rows per tile
    int32_t vec2;    // complex64 with even rows: 16-byte accesses
    FastDiv32 bLdiv;
    uint64_t ntiles;
    int32_t nfree;   // wires outside S, ascending
    int32_t free_w[kMaxWires];
    uint32_t free_d[kMaxWires];
    FastDiv32 free_div[kMaxWires];  // division by free_d (tile indices are below 2^32)
    uint64_t free_b[kMaxWires];
    const uint64_t* rowoff;  // device, rows entries: offset of each row from the tile base
    int32_t* status;         // tensor-core kernel: QD_ERR_TIMEOUT if a bounded wait gave up
    uint32_t stage;          // bytes of the pass's largest chunk: k_fused_tile's shared-memory stage
    uint32_t first_bytes;    // bytes of the first chunk (staged by k_fused_tile with the row offsets)
    const char* desc_base;   // the program's descriptors (tensor-core operands)
};

// A tile pass of one circuit in a batch's device-side layer queue: the
// fields of FusedArgs that a tile needs, with the descriptors given as byte
// offsets into the batch's descriptor blob and at most kLayerMaxFree wires
// outside the tile.
constexpr int kLayerMaxFree = 16;
template <typename R>
struct __align__(16) LayerEntry {
    using T2 = typename Cplx<R>::T2;
    T2* psi;
    uint64_t chunks_off, rows_off;
    int32_t nchunks;
    uint32_t T, bL, rows;
    int32_t vec2;
    FastDiv32 bLdiv;
    uint64_t ntiles;
    int32_t nfree;
    int32_t free_w[kLayerMaxFree];
    uint32_t free_d[kLayerMaxFree];
    FastDiv32 free_div[kLayerMaxFree];
    uint64_t free_b[kLayerMaxFree];
    uint32_t stage, first_bytes;
};


namespace {

template <typename T2> __device__ __forceinline__ T2 fcmul(const T2& u, const T2& x) {
    T2 r;
    r.x = u.x * x.x - u.y * x.y;
    r.y = u.x * x.y + u.y * x.x;
    return r;
}
template <typename T2> __device__ __forceinline__ void fcmac(T2& acc, const T2& u, const T2& x) {
    acc.x = fma(u.x, x.x, acc.x);
    acc.x = fma(-u.y, x.y, acc.x);
    acc.y = fma(u.x, x.y, acc.y);
    acc.y = fma(u.y, x.x, acc.y);
}

// Small fixed-size arrays, indexed only by unrolled loop counters so that
// they stay in registers.
template <typename T, int N>
struct Arr {
    T v[N];
};

// y = G x for one class held in registers.  Monomial (permutation) gates run
// as dense ones: their zero entries contribute exact zeros, and a pure
// permutation's unit entries move values exactly.  Selecting x_{pi(r)} by a
// data-dependent index instead is compiled into a local-memory copy of the
// class -- for the whole kernel, whichever gate kind runs -- which made every
// qutrit gate of a tile pass five times slower than a qubit gate (measured:
// 99 vs 17 us per gate on 26.9M amplitudes).
template <typename T2, int DT>
__device__ __forceinline__ Arr<T2, DT> class_math(const Arr<T2, DT> x, int kind, const Arr<T2, DT * DT> u) {
    Arr<T2, DT> y;
    if (kind != kDiag) {
#pragma unroll
        for (int r = 0; r < DT; ++r) {
            T2 acc = fcmul(u.v[r * DT], x.v[0]);
#pragma unroll
            for (int k = 1; k < DT; ++k) fcmac(acc, u.v[r * DT + k], x.v[k]);
            y.v[r] = acc;
        }
    } else {
#pragma unroll
        for (int r = 0; r < DT; ++r) y.v[r] = fcmul(u.v[r * DT + r], x.v[r]);
    }
    return y;
}

// Apply one single-wire gate of dimension DT to the tile in shared memory.
// Matrix and masks are loop invariants read once per gate from the staged
// chunk.  With no control inside the tile (m == 1) a class index
// c = hi * lst + lo has base hi * lst * d + lo (one division); complex64 with
// an even local stride processes two adjacent classes with 16-byte accesses.
template <typename R, int DT>
__device__ __forceinline__ void tile_gate(typename Cplx<R>::T2* tile, const FGate& G,
                                          const typename Cplx<R>::T2* pool) {
    using T2 = typename Cplx<R>::T2;
    const int kind = G.kind;
    const uint32_t lmask = G.lmask, smask = G.smask, lst = G.lst, nc = G.nclasses;
    Arr<T2, DT * DT> u;
    const T2* gu = pool + G.u_off;
#pragma unroll
    for (int r = 0; r < DT; ++r)
#pragma unroll
        for (int k = 0; k < DT; ++k) u.v[r * DT + k] = gu[r * G.PP + k];
    if (G.map.m == 1) {
        const FastDiv32 f = G.map.seg[0];
        const uint32_t step = G.step;
        if constexpr (sizeof(R) == 4) {
            if ((lst & 1u) == 0) {
                for (uint32_t c = 2 * threadIdx.x; c < nc; c += 2 * blockDim.x) {
                    const uint32_t hi = f.div(c);
                    const uint32_t b = hi * step + (c - hi * lst);
                    Arr<T2, DT> x0, x1;
#pragma unroll
                    for (int k = 0; k < DT; ++k) {
                        float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
                        if (lmask >> k & 1u) v = *reinterpret_cast<const float4*>(tile + b + k * lst);
                        x0.v[k] = make_float2(v.x, v.y);
                        x1.v[k] = make_float2(v.z, v.w);
                    }
                    const Arr<T2, DT> y0 = class_math<T2, DT>(x0, kind, u);
                    const Arr<T2, DT> y1 = class_math<T2, DT>(x1, kind, u);
#pragma unroll
                    for (int r = 0; r < DT; ++r)
                        if (smask >> r & 1u)
                            *reinterpret_cast<float4*>(tile + b + r * lst) =
                                make_float4(y0.v[r].x, y0.v[r].y, y1.v[r].x, y1.v[r].y);
                }
                return;
            }
            if (DT == 2 && lst == 1) {  // the class is two adjacent amplitudes
                for (uint32_t c = threadIdx.x; c < nc; c += blockDim.x) {
                    const float4 v = *reinterpret_cast<const float4*>(tile + 2 * c);
                    Arr<T2, DT> x;
                    x.v[0] = make_float2(v.x, v.y);
                    x.v[DT - 1] = make_float2(v.z, v.w);
                    const Arr<T2, DT> y = class_math<T2, DT>(x, kind, u);
                    if (smask == 3u)
                        *reinterpret_cast<float4*>(tile + 2 * c) = make_float4(y.v[0].x, y.v[0].y, y.v[DT - 1].x,
                                                                               y.v[DT - 1].y);
                    else
#pragma unroll
                        for (int r = 0; r < DT; ++r)
                            if (smask >> r & 1u) tile[2 * c + r] = y.v[r];
                }
                return;
            }
        }
        for (uint32_t c = threadIdx.x; c < nc; c += blockDim.x) {
            const uint32_t hi = f.div(c);
            const uint32_t b = hi * step + (c - hi * lst);
            Arr<T2, DT> x;
#pragma unroll
            for (int k = 0; k < DT; ++k) {
                x.v[k].x = 0;
                x.v[k].y = 0;
                if (lmask >> k & 1u) x.v[k] = tile[b + k * lst];
            }
            const Arr<T2, DT> y = class_math<T2, DT>(x, kind, u);
#pragma unroll
            for (int r = 0; r < DT; ++r)
                if (smask >> r & 1u) tile[b + r * lst] = y.v[r];
        }
    } else {
        for (uint32_t c = threadIdx.x; c < nc; c += blockDim.x) {
            const uint32_t b = G.map.map(c);
            Arr<T2, DT> x;
#pragma unroll
            for (int k = 0; k < DT; ++k) {
                x.v[k].x = 0;
                x.v[k].y = 0;
                if (lmask >> k & 1u) x.v[k] = tile[b + k * lst];
            }
            const Arr<T2, DT> y = class_math<T2, DT>(x, kind, u);
#pragma unroll
            for (int r = 0; r < DT; ++r)
                if (smask >> r & 1u) tile[b + r * lst] = y.v[r];
        }
    }
}

// Dense (or monomial) composed block, one class per thread: the class's
// members are gathered into registers (padded rows masked out) before the
// first store; each output row is accumulated from the matrix row in the
// staged pool, read by all threads at the same address (a broadcast) -- for
// complex64 two adjacent entries per 16-byte load.
template <typename R, int PP>
__device__ __forceinline__ void block_dense(typename Cplx<R>::T2* tile, const FGate& G,
                                            const typename Cplx<R>::T2* M, const uint32_t (&off)[PP]) {
    using T2 = typename Cplx<R>::T2;
    const uint32_t nc = G.nclasses, lmask = G.lmask, smask = G.smask;
    for (uint32_t c = threadIdx.x; c < nc; c += blockDim.x) {
        const uint32_t b = G.map.map(c);
        T2 x[PP];
#pragma unroll
        for (int k = 0; k < PP; ++k) {
            x[k].x = 0;
            x[k].y = 0;
            if (lmask >> k & 1u) x[k] = tile[b + off[k]];
        }
#pragma unroll
        for (int r = 0; r < PP; ++r) {
            if (!(smask >> r & 1u)) continue;
            const T2* Mr = M + r * PP;
            T2 a;
            a.x = a.y = 0;
            if constexpr (sizeof(R) == 4 && PP % 2 == 0) {
#pragma unroll
                for (int k = 0; k < PP; k += 2) {
                    const float4 m2 = *reinterpret_cast<const float4*>(Mr + k);
                    fcmac(a, make_float2(m2.x, m2.y), x[k]);
                    fcmac(a, make_float2(m2.z, m2.w), x[k + 1]);
                }
            } else {
#pragma unroll
                for (int k = 0; k < PP; ++k) fcmac(a, Mr[k], x[k]);
            }
            tile[b + off[r]] = a;
        }
    }
}

// Apply one composed block (P <= PP) to the tile, one class per thread.
// Dense and monomial blocks (the latter run as dense ones, see class_math)
// through block_dense; diagonal blocks scale each member.  Measured
// alternatives that were slower on the benchmark circuit's passes: two
// classes per thread (their registers cost more than the matrix loads they
// share: 8-dimensional blocks 53 vs 48 us per 26.9M amplitudes); all rows of
// one or two classes accumulated as outer products over the inputs (20-28%
// slower); monomial blocks gathered from the tile by source address
// (register pressure of the whole kernel).
template <typename R, int PP>
__device__ __forceinline__ void block_gate(typename Cplx<R>::T2* tile, const FGate& G,
                                           const typename Cplx<R>::T2* pool) {
    using T2 = typename Cplx<R>::T2;
    const uint32_t nc = G.nclasses, lmask = G.lmask, smask = G.smask;
    uint32_t off[PP];
#pragma unroll
    for (int r = 0; r < PP; ++r) off[r] = G.off[r];
    const T2* M = pool + G.u_off;
    if (G.kind != kDiag) {
        block_dense<R, PP>(tile, G, M, off);
        return;
    }
    for (uint32_t c = threadIdx.x; c < nc; c += blockDim.x) {
        const uint32_t b0 = G.map.map(c);
        T2 x0[PP];
#pragma unroll
        for (int k = 0; k < PP; ++k) {
            x0[k].x = 0;
            x0[k].y = 0;
            if (lmask >> k & 1u) x0[k] = tile[b0 + off[k]];
        }
#pragma unroll
        for (int r = 0; r < PP; ++r)
            if (smask >> r & 1u) tile[b0 + off[r]] = fcmul(M[r * PP + r], x0[r]);
    }
}

// Runs of single-wire gates applied in registers (complex64).  A class of
// the block's wires (three or four qubit wires: 8 or 16 members) is
// gathered once; each gate of the run then updates the members in
// registers -- d x d products on the groups of members that differ only in
// the gate's target digit, skipping groups its controls exclude -- and the
// class is written back once.  One shared-memory sweep for the whole run,
// and each gate's own arithmetic instead of the composed P x P product.
// Member m of a class has digit (m / stride_j) % d_j on block wire j, the
// first wire least significant.  Every register index is a compile-time
// constant: the gate's position selects an instantiation.
template <int D0, int D1, int D2, int D3>
struct RunShape {
    static constexpr int P = D0 * D1 * D2 * D3;
    static constexpr int nw = 1 + (D1 > 1) + (D2 > 1) + (D3 > 1);
    static constexpr int dim(int j) { return j == 0 ? D0 : j == 1 ? D1 : j == 2 ? D2 : D3; }
    static constexpr int stride(int j) { return j == 0 ? 1 : j == 1 ? D0 : j == 2 ? D0 * D1 : D0 * D1 * D2; }
};

template <typename S, int J>
__device__ __forceinline__ void run_apply(float2 (&x)[S::P], const float2* U, uint32_t mask) {
    constexpr int D = S::dim(J), ST = S::stride(J);
    float2 u[D * D];
#pragma unroll
    for (int i = 0; i < D * D; ++i) u[i] = U[i];
#pragma unroll
    for (int m = 0; m < S::P; ++m) {
        if ((m / ST) % D != 0) continue;  // group base: target digit 0
        uint32_t gm = 0;
#pragma unroll
        for (int k = 0; k < D; ++k) gm |= 1u << (m + k * ST);
        if (!(mask & gm)) continue;  // the gate's controls exclude this group (uniform across threads)
        float2 y[D];
#pragma unroll
        for (int r = 0; r < D; ++r) {
            float2 acc = fcmul(u[r * D], x[m]);
#pragma unroll
            for (int k = 1; k < D; ++k) fcmac(acc, u[r * D + k], x[m + k * ST]);
            y[r] = acc;
        }
#pragma unroll
        for (int r = 0; r < D; ++r) x[m + r * ST] = y[r];
    }
}

template <typename S>
__device__ __forceinline__ void run_block(float2* tile, const FGate& G, const float2* pool) {
    const uint16_t* off = G.off;  // read from the staged record at each use: registers go to the class
    const uint32_t nc = G.nclasses;
    const int ns = G.nsub;
    for (uint32_t c = threadIdx.x; c < nc; c += blockDim.x) {
        const uint32_t b = G.map.map(c);
        float2 x[S::P];
#pragma unroll
        for (int k = 0; k < S::P; ++k) x[k] = tile[b + off[k]];
        for (int s = 0; s < ns; ++s) {
            const float2* U = pool + G.sub_u[s];
            const uint32_t mask = G.sub_mask[s];
            switch (G.sub_pos[s]) {
                case 0: run_apply<S, 0>(x, U, mask); break;
                case 1:
                    if constexpr (S::nw > 1) run_apply<S, 1>(x, U, mask);
                    break;
                case 2:
                    if constexpr (S::nw > 2) run_apply<S, 2>(x, U, mask);
                    break;
                default:
                    if constexpr (S::nw > 3) run_apply<S, 3>(x, U, mask);
                    break;
            }
        }
#pragma unroll
        for (int r = 0; r < S::P; ++r) tile[b + off[r]] = x[r];
    }
}

// Shape ids of runs (wire dimensions, first wire least significant).  Only
// qubit blocks of three and four wires: on the benchmark circuit the cost
// model picks runs almost only there, and every further shape enlarges the
// kernel (instruction-fetch stalls; measured 0.7% slower with nine shapes).
constexpr int kRunShapes = 2;
__host__ __device__ constexpr int run_shape_dims(int id, int j) {
    constexpr int t[kRunShapes][4] = {{2, 2, 2, 1}, {2, 2, 2, 2}};
    return t[id][j];
}

__device__ __forceinline__ void run_dispatch(float2* tile, const FGate& G, const float2* pool) {
    switch (G.shape) {
        case 0: run_block<RunShape<2, 2, 2, 1>>(tile, G, pool); break;
        default: run_block<RunShape<2, 2, 2, 2>>(tile, G, pool); break;
    }
}

// Tensor-core blocks inside a tile (complex64, blocks of 17..32 dimensions).
// For 128 classes at a time the block is the contraction
//     Y (128 x 64) = X (128 x 64) . B^T,  B = [[Re U, -Im U], [Im U, Re U]]
// with the members' real parts at K = 0..31 and imaginary parts at 32..63
// (zero-padded beyond P), outputs likewise along N.  X is staged from the
// tile into tensor memory (tcgen05.st, lane = class) as TF32 hi / lo parts;
// B (hi | lo, 32 KB, K-major) comes from the program's descriptors into
// shared memory; one thread issues 3 x 8 MMAs (M = 128, N = 64, K = 8,
// A_hi B_hi + A_hi B_lo + A_lo B_hi) into the accumulator, commits to an
// mbarrier, and every thread waits (bounded).  The epilogue reads its
// outputs back (tcgen05.ld), restores each class's 2-norm when the block is
// unitary (the tensor cores' FP32 accumulation is biased toward zero) and
// writes them into the tile.  Tensor memory: A_hi [0, 64), A_lo [64, 128),
// D [128, 192).  256 threads: thread t handles class t % 128 of the group,
// members / outputs 16 (t / 128) .. + 15.
struct TcTileCtx {
    uint32_t tm;      // tensor memory base
    uint32_t mbar;    // shared address of the MMA mbarrier
    uint32_t phase;   // its next phase parity
    float* sB;        // shared: B_hi | B_lo (2 x 64 x 64 floats)
    const char* desc; // the program's descriptors (global)
    float2* s_nin;    // shared [2][128]: input squared norms (s, c parts), two halves per class
    float2* s_nout;   // shared [2][128]
};
constexpr uint32_t kTileTcOpBytes = 2u * 64u * 64u * 4u;

__device__ bool tile_tc_block(float2* tile, const FGate& G, TcTileCtx& c) {
    const int tid = threadIdx.x, warp = tid >> 5;
    {
        const uint4* src = reinterpret_cast<const uint4*>(c.desc + G.op_off);
        uint4* dst = reinterpret_cast<uint4*>(c.sB);
        for (int i = tid; i < (int)(kTileTcOpBytes / 16); i += blockDim.x) dst[i] = src[i];
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    const int row = tid & 127, half = tid >> 7;
    const uint32_t lanes = (uint32_t)(32 * (warp & 3)) << 16;
    const int P = G.P;
    const uint32_t nc = G.nclasses;
    const uint32_t idesc = tc_idesc(2u);  // TF32, M = 128, N = 64
    for (uint32_t g0 = 0; g0 < nc; g0 += 128) {
        const uint32_t cls = g0 + (uint32_t)row;
        const bool valid = cls < nc;
        const uint32_t base = valid ? G.map.map(cls) : 0u;
        NormAcc pn;
        {
            float xr[16], xi[16], h[16], l[16];
#pragma unroll
            for (int i = 0; i < 16; ++i) {
                const int r = 16 * half + i;
                const float2 v = (valid && r < P) ? tile[base + G.off[r]] : make_float2(0.f, 0.f);
                xr[i] = v.x;
                xi[i] = v.y;
                pn.add_sq(v.x);
                pn.add_sq(v.y);
            }
#pragma unroll
            for (int i = 0; i < 16; ++i) {
                h[i] = tf32_hi(xr[i]);
                l[i] = xr[i] - h[i];
            }
            tmem_st16(c.tm + lanes + 16u * half, h);
            tmem_st16(c.tm + lanes + 64u + 16u * half, l);
#pragma unroll
            for (int i = 0; i < 16; ++i) {
                h[i] = tf32_hi(xi[i]);
                l[i] = xi[i] - h[i];
            }
            tmem_st16(c.tm + lanes + 32u + 16u * half, h);
            tmem_st16(c.tm + lanes + 96u + 16u * half, l);
        }
        c.s_nin[half * 128 + row] = make_float2(pn.s, pn.c);
        asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncthreads();  // every member gathered before any output is written back
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        if (tid == 0) {
            const uint32_t lbo = (64 / 8) * 128;  // bytes between core matrices along K (64 rows)
            const uint64_t bd0 = smem_desc(smem_u32(c.sB), lbo, 128);
            constexpr uint64_t kStep = 2 * (64 / 8) * 128 / 16;  // one k-step: two core matrices, 16-byte units
            constexpr uint64_t kLo = (64u * 64u * 4u) >> 4;        // B_lo
#pragma unroll
            for (int term = 0; term < 3; ++term) {
                const uint32_t a0 = c.tm + (term == 2 ? 64u : 0u);         // A_lo for the third product
                const uint64_t b0 = bd0 + (term == 1 ? kLo : 0);            // B_lo for the second
#pragma unroll
                for (int ks = 0; ks < 8; ++ks)
                    mma_tf32_ta(c.tm + 128u, a0 + 8u * (uint32_t)ks, b0 + (uint64_t)ks * kStep, idesc,
                                (term | ks) != 0 ? 1u : 0u);
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(c.mbar)
                         : "memory");
        }
        const bool ok = mbar_wait(c.mbar, c.phase);
        c.phase ^= 1u;
        if (__syncthreads_or(!ok)) return false;
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        float yr[16], yi[16];
        tmem_ld16(c.tm + lanes + 128u + 16u * half, yr);
        tmem_ld16(c.tm + lanes + 160u + 16u * half, yi);
        NormAcc po;
#pragma unroll
        for (int i = 0; i < 16; ++i) {
            po.add_sq(yr[i]);
            po.add_sq(yi[i]);
        }
        c.s_nout[half * 128 + row] = make_float2(po.s, po.c);
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncthreads();
        float cc = 0.f;
        if (G.unitary) {
            // as in the whole-state kernel: y <- y (1 + c), c = sqrt(ni / no) - 1
            const float2 a0 = c.s_nin[row], a1 = c.s_nin[128 + row];
            const float2 b0 = c.s_nout[row], b1 = c.s_nout[128 + row];
            NormFF ni, no;
            ni.add(a0.x, a0.y);
            ni.add(a1.x, a1.y);
            no.add(b0.x, b0.y);
            no.add(b1.x, b1.y);
            cc = norm_fix(ni, no);
        }
        if (valid) {
#pragma unroll
            for (int i = 0; i < 16; ++i) {
                const int r = 16 * half + i;
                if (r < P) tile[base + G.off[r]] = make_float2(fmaf(yr[i], cc, yr[i]), fmaf(yi[i], cc, yi[i]));
            }
        }
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncthreads();  // the next group reuses tensor memory and the norm arrays
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    }
    return true;
}

// Apply a list of chunks to a tile in shared memory.  stage: shared memory
// for one chunk; odig: digits of the wires outside the tile (fused passes);
// tc: tensor-core context (TC = true: complex64 tiles with kTcBlock gates);
// first_staged: the caller has already staged the first chunk.
// Returns false (the same on every thread) if a tensor-core wait gave up.
template <typename R, int DMAX, bool TC = false>
__device__ __forceinline__ bool apply_chunks(typename Cplx<R>::T2* tile, const char* chunk, int nchunks,
                                             unsigned char* stage, const int32_t* odig, TcTileCtx* tc = nullptr,
                                             bool first_staged = false) {
    using T2 = typename Cplx<R>::T2;
    for (int ci = 0; ci < nchunks; ++ci) {
        const ChunkHdr h = *reinterpret_cast<const ChunkHdr*>(chunk);
        __syncthreads();  // the previous chunk is done with the stage
        if (!(first_staged && ci == 0)) {
            // every 16-byte piece in flight at once (cp.async), then wait
            const uint32_t d0 = static_cast<uint32_t>(__cvta_generic_to_shared(stage));
            for (uint32_t i = threadIdx.x; i < h.bytes / 16; i += blockDim.x)
                asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(d0 + 16u * i), "l"(chunk + 16u * i));
            asm volatile("cp.async.wait_all;" ::: "memory");
        }
        __syncthreads();
        const FGate* gates = reinterpret_cast<const FGate*>(stage + sizeof(ChunkHdr));
        const T2* pool = reinterpret_cast<const T2*>(stage + sizeof(ChunkHdr) + sizeof(FGate) * h.ngates);
        for (uint32_t gi = 0; gi < h.ngates; ++gi) {
            const FGate& G = gates[gi];
            if (odig) {
                bool ok = true;
                for (int c = 0; c < G.n_out; ++c) ok = ok && (odig[G.out_w[c]] == (int32_t)G.out_v[c]);
                if (!ok) continue;  // uniform across the CTA
            }
            if constexpr (TC && sizeof(R) == 4) {
                if (G.kind == kTcBlock) {
                    if (!tile_tc_block(reinterpret_cast<float2*>(tile), G, *tc)) return false;
                    continue;  // tile_tc_block ends with a barrier
                }
            }
            if constexpr (sizeof(R) == 4) {
                if (G.kind == kRun) {
                    run_dispatch(reinterpret_cast<float2*>(tile), G, reinterpret_cast<const float2*>(pool));
                    __syncthreads();
                    continue;
                }
            }
            if (G.single) {
                if (G.P == 2) tile_gate<R, 2>(tile, G, pool);
                else if (DMAX == 3 || G.P == 3) tile_gate<R, 3>(tile, G, pool);
                else if (G.P == 4) tile_gate<R, (DMAX > 3 ? 4 : 3)>(tile, G, pool);
                else tile_gate<R, DMAX>(tile, G, pool);
            } else {
                switch (G.PP) {
                    case 4: block_gate<R, 4>(tile, G, pool); break;
                    case 6: block_gate<R, 6>(tile, G, pool); break;
                    case 8: block_gate<R, 8>(tile, G, pool); break;
                    case 9: block_gate<R, 9>(tile, G, pool); break;
                    case 12: block_gate<R, 12>(tile, G, pool); break;
                    default: block_gate<R, 16>(tile, G, pool); break;
                }
            }
            __syncthreads();
        }
        chunk += h.bytes;
    }
    return true;
}

// Load tile at g (rows of bL amplitudes at the offsets srow) into shared
// memory with cp.async: every 16-byte piece (8-byte for complex64 with odd
// rows) of a thread is in flight at once.  Staged through registers, each
// load would wait for the previous shared-memory store, which the compiler
// cannot move past the next row-offset read (both are shared memory): one
// load in flight per thread, the fixed cost of a pass.  The caller's next
// barrier publishes the other threads' pieces.
template <typename R, typename A>
__device__ __forceinline__ void tile_load_async(typename Cplx<R>::T2* tile, const typename Cplx<R>::T2* g,
                                                const uint64_t* srow, const A& a) {
    constexpr uint32_t kEl = sizeof(typename Cplx<R>::T2);
    const uint32_t s0 = static_cast<uint32_t>(__cvta_generic_to_shared(tile));
    const uint64_t gbase = (uint64_t)(g - a.psi), lim = (uint64_t)a.ntiles * a.T;  // bounds-checked build
    if (kEl == 16 || a.vec2) {
        constexpr uint32_t per = 16 / kEl;
        for (uint32_t e = per * threadIdx.x; e < a.T; e += per * blockDim.x) {
            const uint32_t r = a.bLdiv.div(e);
            if (!in_bounds(gbase + srow[r] + (e - r * a.bL) + per - 1, lim)) continue;
            asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(s0 + e * kEl),
                         "l"(g + srow[r] + (e - r * a.bL)));
        }
    } else {
        for (uint32_t e = threadIdx.x; e < a.T; e += blockDim.x) {
            const uint32_t r = a.bLdiv.div(e);
            if (!in_bounds(gbase + srow[r] + (e - r * a.bL), lim)) continue;
            asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(s0 + e * kEl),
                         "l"(g + srow[r] + (e - r * a.bL)));
        }
    }
    asm volatile("cp.async.wait_all;" ::: "memory");
}

__host__ __device__ inline size_t fused_rows_bytes(uint32_t rows) { return ((size_t)rows * 8 + 15) & ~(size_t)15; }

// One tile of a pass: the row offsets and the first chunk are staged while
// thread 0 derives the tile's base index and outside digits, the tile is
// loaded, the pass's chunks are applied, the tile is stored.  `a` is the
// pass's record (kernel parameters of k_fused_tile, or an entry of a
// device-side layer queue); chunks / rowoff are its descriptors.
template <typename R, int DMAX, typename A>
__device__ __forceinline__ void tile_pass(const A& a, const char* chunks, const uint64_t* rowoff, uint32_t tile_idx,
                                          unsigned char* smem_raw, int32_t* odig, uint64_t* sbase) {
    using T2 = typename Cplx<R>::T2;
    unsigned char* stage = smem_raw;
    uint64_t* srow = reinterpret_cast<uint64_t*>(smem_raw + a.stage);
    T2* tile = reinterpret_cast<T2*>(smem_raw + a.stage + fused_rows_bytes(a.rows));
    {
        // the row offsets and the first chunk arrive together (cp.async)
        // while thread 0 derives the tile's base and outside digits
        const uint32_t s0 = static_cast<uint32_t>(__cvta_generic_to_shared(srow));
        for (uint32_t r = threadIdx.x; r < a.rows; r += blockDim.x)
            asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(s0 + 8u * r), "l"(rowoff + r));
        const uint32_t d0 = static_cast<uint32_t>(__cvta_generic_to_shared(stage));
        if (a.nchunks > 0)
            for (uint32_t i = threadIdx.x; i < a.first_bytes / 16; i += blockDim.x)
                asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(d0 + 16u * i), "l"(chunks + 16u * i));
    }
    if (threadIdx.x == 0) {
        uint32_t rem = tile_idx;
        uint64_t base = 0;
        for (int i = 0; i < a.nfree; ++i) {
            const uint32_t q = a.free_div[i].div(rem);
            const uint32_t dig = rem - q * a.free_d[i];
            odig[a.free_w[i]] = (int32_t)dig;
            base += (uint64_t)dig * a.free_b[i];
            rem = q;
        }
        *sbase = base;
    }
    asm volatile("cp.async.wait_all;" ::: "memory");
    __syncthreads();
    T2* g = a.psi + *sbase;
    tile_load_async<R>(tile, g, srow, a);  // published by apply_chunks' first barrier
    apply_chunks<R, DMAX>(tile, chunks, a.nchunks, stage, odig, nullptr, true);
    __syncthreads();
    const uint64_t lim = (uint64_t)a.ntiles * a.T;  // bounds-checked build
    if (a.vec2) {
        for (uint32_t e = 2 * threadIdx.x; e < a.T; e += 2 * blockDim.x) {
            const uint32_t r = a.bLdiv.div(e);
            if (!in_bounds(*sbase + srow[r] + (e - r * a.bL) + 1, lim)) continue;
            *reinterpret_cast<float4*>(reinterpret_cast<float2*>(g) + srow[r] + (e - r * a.bL)) =
                reinterpret_cast<const float4*>(tile)[e >> 1];
        }
    } else {
        for (uint32_t e = threadIdx.x; e < a.T; e += blockDim.x) {
            const uint32_t r = a.bLdiv.div(e);
            if (!in_bounds(*sbase + srow[r] + (e - r * a.bL), lim)) continue;
            g[srow[r] + (e - r * a.bL)] = tile[e];
        }
    }
}

template <typename R, int DMAX>
__global__ void __launch_bounds__(256, 3) k_fused_tile(const __grid_constant__ FusedArgs<R> a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ int32_t odig[kMaxWires];
    __shared__ uint64_t sbase;
    tile_pass<R, DMAX>(a, a.chunks, a.rowoff, blockIdx.x, smem_raw, odig, &sbase);
}

// Tile passes of many circuits in one launch (batches): the device-side
// queue of one layer holds, for each circuit with a pass at that position,
// the pass's record, and prefix[e] = tiles of the entries before e.  CTA w
// applies tile w of the layer: its entry e is the last with prefix[e] <= w
// (binary search by one thread), staged in shared memory.  One CTA per
// tile, as k_fused_tile: the hardware scheduler balances tiles of unequal
// cost.  The queue is complete before the launch, so no CTA ever waits on
// another.
template <typename R, int DMAX>
__global__ void __launch_bounds__(256, 3) k_fused_layer(const LayerEntry<R>* entries, const uint64_t* prefix,
                                                         int32_t n, const char* base) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ int32_t odig[kMaxWires];
    __shared__ uint64_t sbase;
    __shared__ int32_t s_e;
    // the entry, staged in shared memory: read from global memory, its fields
    // would be reloaded after every store of the tile to global memory (the
    // compiler cannot rule out that the two alias)
    __shared__ __align__(16) LayerEntry<R> sE;
    const uint64_t w = blockIdx.x;
    if (threadIdx.x == 0) {
        int lo = 0, hi = n - 1;  // prefix[lo] <= w < prefix[n]
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (prefix[mid] <= w) lo = mid;
            else hi = mid - 1;
        }
        s_e = lo;
    }
    __syncthreads();
    const int e = s_e;
    {
        const uint4* src = reinterpret_cast<const uint4*>(entries + e);
        uint4* dst = reinterpret_cast<uint4*>(&sE);
        for (int i = threadIdx.x; i < (int)(sizeof(LayerEntry<R>) / 16); i += blockDim.x) dst[i] = src[i];
    }
    __syncthreads();
    tile_pass<R, DMAX>(sE, base + sE.chunks_off, reinterpret_cast<const uint64_t*>(base + sE.rows_off),
                       (uint32_t)(w - prefix[e]), smem_raw, odig, &sbase);
}

// Tile pass whose chunks hold tensor-core blocks (complex64): k_fused_tile
// plus tensor memory (256 columns), an MMA mbarrier and the 32 KB operand
// buffer.  At most two CTAs per SM (shared memory is padded to keep it so),
// which is what the 512 tensor-memory columns of an SM hold.  A timed-out
// MMA wait stops the tile (status QD_ERR_TIMEOUT, tile not written back).
constexpr size_t kTcTileMinSmem = 80 * 1024;  // > 228 KB / 3: at most two CTAs per SM

template <int DMAX>
__global__ void __launch_bounds__(256, 2) k_fused_tile_tc(const __grid_constant__ FusedArgs<float> a) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    unsigned char* stage = smem_raw;
    uint64_t* srow = reinterpret_cast<uint64_t*>(smem_raw + chunk_smem_max<float>());
    float2* tile = reinterpret_cast<float2*>(smem_raw + chunk_smem_max<float>() + fused_rows_bytes(a.rows));
    float* sB = reinterpret_cast<float*>(
        smem_raw + ((chunk_smem_max<float>() + fused_rows_bytes(a.rows) + 8 * (size_t)a.T + 127) & ~(size_t)127));
    __shared__ int32_t odig[kMaxWires];
    __shared__ uint64_t sbase;
    __shared__ __align__(8) uint64_t mbar;
    __shared__ uint32_t tmem_base;
    __shared__ float2 s_nin[256], s_nout[256];
    const int tid = threadIdx.x;
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&mbar)), "r"(1));
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if ((tid >> 5) == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base)),
                     "r"(256));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    for (uint32_t r = tid; r < a.rows; r += blockDim.x) srow[r] = a.rowoff[r];
    if (tid == 0) {
        uint32_t rem = blockIdx.x;
        uint64_t base = 0;
        for (int i = 0; i < a.nfree; ++i) {
            const uint32_t q = a.free_div[i].div(rem);
            const uint32_t dig = rem - q * a.free_d[i];
            odig[a.free_w[i]] = (int32_t)dig;
            base += (uint64_t)dig * a.free_b[i];
            rem = q;
        }
        sbase = base;
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    float2* g = a.psi + sbase;
    tile_load_async<float>(tile, g, srow, a);  // published by apply_chunks' first barrier
    TcTileCtx ctx{tmem_base, smem_u32(&mbar), 0u, sB, a.desc_base, s_nin, s_nout};
    const bool ok = apply_chunks<float, DMAX, true>(tile, a.chunks, a.nchunks, stage, odig, &ctx);
    __syncthreads();
    if (ok) {
        const uint64_t lim = (uint64_t)a.ntiles * a.T;  // bounds-checked build
        if (a.vec2) {
            for (uint32_t e = 2 * tid; e < a.T; e += 2 * blockDim.x) {
                const uint32_t r = a.bLdiv.div(e);
                if (!in_bounds(sbase + srow[r] + (e - r * a.bL) + 1, lim)) continue;
                *reinterpret_cast<float4*>(g + srow[r] + (e - r * a.bL)) = reinterpret_cast<const float4*>(tile)[e >> 1];
            }
        } else {
            for (uint32_t e = tid; e < a.T; e += blockDim.x) {
                const uint32_t r = a.bLdiv.div(e);
                if (!in_bounds(sbase + srow[r] + (e - r * a.bL), lim)) continue;
                g[srow[r] + (e - r * a.bL)] = tile[e];
            }
        }
    } else if (tid == 0) {
        atomicExch(a.status, QD_ERR_TIMEOUT);
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if ((tid >> 5) == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem_base), "r"(256));
}

size_t fused_tc_smem(uint32_t T, uint32_t rows) {
    const size_t s = ((chunk_smem_max<float>() + fused_rows_bytes(rows) + 8 * (size_t)T + 127) & ~(size_t)127) +
                     kTileTcOpBytes;
    return s < kTcTileMinSmem ? kTcTileMinSmem : s;
}

cudaError_t launch_fused_tc(const FusedArgs<float>& a, int dmax, cudaStream_t s) {
    static int attr_dev = -1;
    int dev = 0;
    cudaGetDevice(&dev);
    if (attr_dev != dev) {
        cudaError_t e = cudaFuncSetAttribute(k_fused_tile_tc<3>, cudaFuncAttributeMaxDynamicSharedMemorySize, 220 * 1024);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(k_fused_tile_tc<5>, cudaFuncAttributeMaxDynamicSharedMemorySize, 220 * 1024);
        if (e != cudaSuccess) return e;
        attr_dev = dev;
    }
    const size_t smem = fused_tc_smem(a.T, a.rows);
    if (smem > 220 * 1024) return cudaErrorInvalidValue;
    if (dmax <= 3)
        k_fused_tile_tc<3><<<(unsigned)a.ntiles, 256, smem, s>>>(a);
    else
        k_fused_tile_tc<5><<<(unsigned)a.ntiles, 256, smem, s>>>(a);
    count_launch();
    return cudaGetLastError();
}

template <typename R>
size_t fused_smem(const FusedArgs<R>& a) {
    return (size_t)a.stage + fused_rows_bytes(a.rows) + sizeof(typename Cplx<R>::T2) * (size_t)a.T;
}

// dmax: largest single-wire dimension among the pass's gates (selects the
// kernel instance, so qubit/qutrit passes do not pay for d = 5 registers).
template <typename R>
cudaError_t launch_fused(const FusedArgs<R>& a, int dmax, cudaStream_t s) {
    static int attr_dev = -1;
    int dev = 0;
    cudaGetDevice(&dev);
    if (attr_dev != dev) {
        cudaError_t e = cudaFuncSetAttribute(k_fused_tile<R, 3>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             220 * 1024);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(k_fused_tile<R, 5>, cudaFuncAttributeMaxDynamicSharedMemorySize, 220 * 1024);
        if (e != cudaSuccess) return e;
        attr_dev = dev;
    }
    if (dmax <= 3)
        k_fused_tile<R, 3><<<(unsigned)a.ntiles, 256, fused_smem<R>(a), s>>>(a);
    else
        k_fused_tile<R, 5><<<(unsigned)a.ntiles, 256, fused_smem<R>(a), s>>>(a);
    count_launch();
    return cudaGetLastError();
}

// One group of a layer of a batch's device-side queue: one CTA per tile.
template <typename R>
cudaError_t launch_fused_layer(const LayerEntry<R>* entries, const uint64_t* prefix, int32_t n, uint64_t total,
                               const char* base, int dmax, size_t smem, cudaStream_t s) {
    if (n <= 0 || total == 0) return cudaSuccess;
    if (total >= ((uint64_t)1 << 31)) return cudaErrorInvalidConfiguration;
    static int attr_dev = -1;
    int dev = 0;
    cudaGetDevice(&dev);
    if (attr_dev != dev) {
        cudaError_t e = cudaFuncSetAttribute(k_fused_layer<R, 3>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             220 * 1024);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(k_fused_layer<R, 5>, cudaFuncAttributeMaxDynamicSharedMemorySize, 220 * 1024);
        if (e != cudaSuccess) return e;
        attr_dev = dev;
    }
    if (dmax <= 3)
        k_fused_layer<R, 3><<<(unsigned)total, 256, smem, s>>>(entries, prefix, n, base);
    else
        k_fused_layer<R, 5><<<(unsigned)total, 256, smem, s>>>(entries, prefix, n, base);
    count_launch();
    return cudaGetLastError();
}

}  // namespace

QD_DEFINE_BOUNDS_TAKE(bounds_take_fusion)

namespace {

// Whole circuits of small states, one CTA per circuit: the state starts as
// |0...0> in shared memory, every chunk of the circuit is applied there,
// then the state is written to HBM once and its squared norm is reduced.
template <typename R, int DMAX>
__global__ void __launch_bounds__(256, 2) k_batch_small(const SmallTask* tasks, char* state_base,
                                                         const char* desc_base, double* norms) {
    using T2 = typename Cplx<R>::T2;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    unsigned char* stage = smem_raw;
    T2* tile = reinterpret_cast<T2*>(smem_raw + chunk_smem_max<R>());
    __shared__ double red_s[8], red_c[8];
    const SmallTask tk = tasks[blockIdx.x];
    for (uint32_t e = threadIdx.x; e < tk.D; e += blockDim.x) {
        T2 z;
        z.x = e == 0 ? (R)1 : (R)0;
        z.y = 0;
        tile[e] = z;
    }
    apply_chunks<R, DMAX>(tile, desc_base + tk.chunk_off, (int)tk.nchunks, stage, nullptr);
    __syncthreads();
    T2* psi = reinterpret_cast<T2*>(state_base + tk.psi_off);
    double s = 0.0, c = 0.0;  // Neumaier per thread, then a fixed-order tree
    for (uint32_t e = threadIdx.x; e < tk.D; e += blockDim.x) {
        const T2 v = tile[e];
        psi[e] = v;
        const double p = fma((double)v.x, (double)v.x, (double)v.y * (double)v.y);
        const double t = s + p;
        c += fabs(s) >= fabs(p) ? (s - t) + p : (p - t) + s;
        s = t;
    }
    for (int o = 16; o > 0; o >>= 1) {
        const double s2 = __shfl_down_sync(0xffffffffu, s, o);
        const double c2 = __shfl_down_sync(0xffffffffu, c, o);
        const double t = s + s2, bb = t - s;
        c = c + c2 + ((s - (t - bb)) + (s2 - bb));
        s = t;
    }
    if ((threadIdx.x & 31) == 0) {
        red_s[threadIdx.x >> 5] = s;
        red_c[threadIdx.x >> 5] = c;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double S = 0.0, C = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
            const double t = S + red_s[w], bb = t - S;
            C += red_c[w] + ((S - (t - bb)) + (red_s[w] - bb));
            S = t;
        }
        norms[tk.norm_index] = S + C;
    }
}

}  // namespace

template <typename R>
cudaError_t launch_batch_small(const SmallTask* tasks, int ntasks, int dmax, uint32_t max_d, char* state_base,
                               const char* desc_base, double* norms, cudaStream_t s) {
    if (ntasks <= 0) return cudaSuccess;
    static int attr_dev = -1;
    int dev = 0;
    cudaGetDevice(&dev);
    if (attr_dev != dev) {
        cudaError_t e = cudaFuncSetAttribute(k_batch_small<R, 3>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             220 * 1024);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(k_batch_small<R, 5>, cudaFuncAttributeMaxDynamicSharedMemorySize, 220 * 1024);
        if (e != cudaSuccess) return e;
        attr_dev = dev;
    }
    const size_t smem = chunk_smem_max<R>() + sizeof(typename Cplx<R>::T2) * (size_t)max_d;
    if (dmax <= 3)
        k_batch_small<R, 3><<<ntasks, 256, smem, s>>>(tasks, state_base, desc_base, norms);
    else
        k_batch_small<R, 5><<<ntasks, 256, smem, s>>>(tasks, state_base, desc_base, norms);
    count_launch();
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Planner
// ---------------------------------------------------------------------------
struct PassPlan {
    bool tile;
    bool block = false;  // QD_FUSE_BLOCK: gates composed into one block over the whole state
    std::vector<int> gates;
    uint64_t smask;   // cached wires
    int64_t T;
};

// Largest tile that fits the shared memory of one CTA (tile + row table).
int64_t tile_limit(int32_t prec) { return prec == QD_C64 ? 16384 : 8192; }

FuseCfg fuse_cfg(const qd_fusion_opts* o, int32_t prec) {
    FuseCfg c;
    c.mode = o ? o->mode : QD_FUSE_OFF;
    c.tc_mode = o ? o->tc_mode : QD_TC_TF32X3;
    c.runs = prec == QD_C64;
    c.Tmax = (o && o->max_tile_amps > 0) ? o->max_tile_amps : (prec == QD_C64 ? 8192 : 4096);
    c.min_gates = (o && o->min_gates > 0) ? o->min_gates : 2;
    c.min_row = (o && o->min_row > 0) ? o->min_row : (prec == QD_C64 ? 16 : 8);
    if (c.mode == QD_FUSE_BLOCK) {
        c.block_dim = (o && o->block_dim > 0) ? o->block_dim : (prec == QD_C64 ? 64 : 8);
        if (c.block_dim > 64) c.block_dim = 64;
    } else {
        // blocks of 17..32 dimensions run on the tensor cores (complex64 tiles only)
        const int cap = (prec == QD_C64 && c.tc_mode != QD_TC_OFF) ? kMaxTcBlock : kMaxBlock;
        c.block_dim = (o && o->block_dim > 0) ? o->block_dim : kMaxBlock;
        if (c.block_dim > cap) c.block_dim = cap;
    }
    // rows per tile are bounded by the row table
    const int64_t need = (c.Tmax + kMaxRows - 1) / kMaxRows;
    if (c.min_row < need) c.min_row = need;
    return c;
}

qd_status load_gates(const Layout& L, int32_t prec, const qd_gate_desc* gates, int32_t n,
                            const double* matrices, std::vector<HGate>& out) {
    if (n < 0) return fail(QD_ERR_ARG, "negative gate count");
    if (n > 0 && (!gates || !matrices)) return fail(QD_ERR_ARG, "gates or matrices is NULL");
    out.resize((size_t)n);
    for (int i = 0; i < n; ++i) {
        const qd_gate_desc& g = gates[i];
        HGate& h = out[(size_t)i];
        if (g.n_wires < 1 || g.n_wires > QD_MAX_GATE_WIRES)
            return fail(QD_ERR_ARG, "gate %d: %d wires outside [1, %d]", i, g.n_wires, QD_MAX_GATE_WIRES);
        if (g.matrix_offset < 0) return fail(QD_ERR_ARG, "gate %d: negative matrix offset", i);
        h.k = g.n_wires;
        h.nc = g.n_ctrl;
        for (int m = 0; m < h.k; ++m) h.wires[m] = g.wires[m];
        if (h.nc < 0 || h.nc > QD_MAX_CONTROLS) return fail(QD_ERR_ARG, "gate %d: bad control count", i);
        for (int m = 0; m < h.nc; ++m) {
            h.cw[m] = g.ctrl_wires[m];
            h.cv[m] = g.ctrl_vals[m];
        }
        h.U = matrices + 2 * g.matrix_offset;
        qd_status rc = make_plan(L, prec, h.wires, h.k, h.U, h.cw, h.cv, h.nc, h.plan);
        if (rc != QD_OK) {
            std::string msg = qd_last_error();
            return fail(rc, "gate %d: %s", i, msg.c_str());
        }
        h.P = h.plan.P;
        h.diag = h.plan.family == 0 && h.plan.kind == kDiag;
        h.unitary = block_is_unitary(h.U, h.P, 1e-10);
        h.fusable = h.plan.family == 0 && h.plan.d <= kMaxFusedD && h.nc <= kMaxTileCtrl;
        h.tmask = 0;
        h.cmask = 0;
        for (int m = 0; m < h.k; ++m) h.tmask |= 1ull << h.wires[m];
        for (int m = 0; m < h.nc; ++m) h.cmask |= 1ull << h.cw[m];
    }
    return QD_OK;
}

// Greedy pass formation.  Scan the remaining gates in order; a gate joins the
// pass if it commutes with every gate deferred before it and its target
// wires fit the tile; otherwise it is deferred and blocks the wires it
// writes (targets of non-diagonal gates) and reads (controls, diagonal
// targets) for later gates.
static void plan_blocks(const Layout& L, const std::vector<HGate>& G, const FuseCfg& cfg,
                        std::vector<PassPlan>& passes);

static void plan_passes(const Layout& L, const std::vector<HGate>& G, const FuseCfg& cfg,
                        std::vector<PassPlan>& passes) {
    passes.clear();
    if (cfg.mode == QD_FUSE_BLOCK) {
        plan_blocks(L, G, cfg, passes);
        return;
    }
    const int n = (int)G.size();
    std::vector<int> rem(n);
    for (int i = 0; i < n; ++i) rem[i] = i;
    int L0 = 0;
    while (L0 < L.n && L.b[L0] < cfg.min_row) ++L0;
    const int64_t T0 = L.b[L0];
    // tile indices are 32-bit (grid size, digit arithmetic)
    const bool can_tile = cfg.mode == QD_FUSE_TILE && T0 <= cfg.Tmax && L.D / T0 < ((int64_t)1 << 31);
    uint64_t low = 0;
    for (int w = 0; w < L0; ++w) low |= 1ull << w;
    std::vector<char> taken(n, 0);
    // Gates a pass on wire set S would take: those whose targets lie in S
    // and that commute with every gate left behind before them (a gate left
    // behind blocks later gates that touch what it writes or reads).  Only
    // the first kPlanWindow remaining gates are examined when choosing S.
    auto scan = [&](uint64_t S, size_t window, std::vector<int>* out) {
        uint64_t BW = 0, BR = 0;
        int cnt = 0;
        const size_t m = rem.size() < window ? rem.size() : window;
        for (size_t j = 0; j < m; ++j) {
            const HGate& g = G[rem[j]];
            const uint64_t W = g.diag ? 0 : g.tmask;
            const uint64_t Rd = g.cmask | (g.diag ? g.tmask : 0);
            const bool blocked = (W & (BW | BR)) || (Rd & BW);
            if (!blocked && g.fusable && (g.tmask & ~S) == 0 && cnt < kMaxPassGates) {
                ++cnt;
                if (out) out->push_back(rem[j]);
                continue;
            }
            BW |= W;
            BR |= Rd;
        }
        return cnt;
    };
    while (!rem.empty()) {
        if (can_tile) {
            // S: the low wires and the first gate's targets, then, one at a
            // time, the wire that lets the pass take the most gates, while
            // one adds any (measured on the 500-gate benchmark circuit: 12
            // passes instead of 15 for the first-come choice of wires)
            uint64_t S = low;
            int64_t T = T0;
            const HGate& g0 = G[rem.front()];
            if (g0.fusable) {
                int64_t T2 = T;
                for (int w = 0; w < L.n; ++w)
                    if ((g0.tmask & ~S) >> w & 1) T2 *= L.dims[w];
                if (T2 <= cfg.Tmax) {
                    S |= g0.tmask;
                    T = T2;
                }
            }
            uint64_t cand = 0;  // targets of the gates in the window
            for (size_t j = 0; j < rem.size() && j < kPlanWindow; ++j) cand |= G[rem[j]].tmask;
            int cur = scan(S, kPlanWindow, nullptr);
            for (;;) {
                int best = cur, bw = -1;
                for (int w = 0; w < L.n; ++w) {
                    if (!((cand & ~S) >> w & 1) || T * L.dims[w] > cfg.Tmax) continue;
                    const int c = scan(S | (1ull << w), kPlanWindow, nullptr);
                    if (c > best) {
                        best = c;
                        bw = w;
                    }
                }
                if (bw < 0) break;
                S |= 1ull << bw;
                T *= L.dims[bw];
                cur = best;
            }
            std::vector<int> sched;
            scan(S, rem.size(), &sched);
            if ((int)sched.size() >= cfg.min_gates) {
                // fill the tile with the lowest remaining wires while it fits:
                // longer contiguous rows and fewer, fuller tiles
                for (int w = 0; w < L.n; ++w) {
                    if (S >> w & 1) continue;
                    if (T * L.dims[w] > cfg.Tmax) break;
                    S |= 1ull << w;
                    T *= L.dims[w];
                }
                PassPlan p;
                p.tile = true;
                p.gates = sched;
                p.smask = S;
                p.T = T;
                passes.push_back(p);
                for (int idx : sched) taken[idx] = 1;
                std::vector<int> rest;
                for (int idx : rem)
                    if (!taken[idx]) rest.push_back(idx);
                rem.swap(rest);
                continue;
            }
        }
        PassPlan p;
        p.tile = false;
        p.gates = {rem.front()};
        p.smask = 0;
        p.T = 0;
        passes.push_back(p);
        taken[rem.front()] = 1;
        rem.erase(rem.begin());
    }
}

// Local layout of a pass: wires of S in ascending order with their dims.
struct TileGeom {
    int ns;
    int sw[kMaxWires];       // global wire of local wire i
    int loc[kMaxWires];      // local index of global wire (or -1)
    Layout local;
    int L0;
    uint32_t bL, R;
    std::vector<uint64_t> rowoff;
    int nfree;
    int free_w[kMaxWires];
    uint32_t free_d[kMaxWires];
    uint64_t free_b[kMaxWires];
};

static void tile_geometry(const Layout& L, uint64_t S, int64_t min_row, TileGeom& g, bool with_rows = true) {
    g.ns = 0;
    g.nfree = 0;
    for (int w = 0; w < L.n; ++w) g.loc[w] = -1;
    int32_t ldims[kMaxWires];
    for (int w = 0; w < L.n; ++w) {
        if (S >> w & 1) {
            g.loc[w] = g.ns;
            g.sw[g.ns] = w;
            ldims[g.ns] = L.dims[w];
            ++g.ns;
        } else {
            g.free_w[g.nfree] = w;
            g.free_d[g.nfree] = (uint32_t)L.dims[w];
            g.free_b[g.nfree] = (uint64_t)L.b[w];
            ++g.nfree;
        }
    }
    make_layout(ldims, g.ns, g.local);
    // rows: the run of the lowest wires (at least min_row amplitudes, all in S)
    int L0 = 0;
    while (L0 < L.n && L.b[L0] < min_row) ++L0;
    while (L0 < L.n && (S >> L0 & 1)) ++L0;
    g.L0 = L0;
    g.bL = (uint32_t)L.b[L0];
    g.R = (uint32_t)(g.local.D / (int64_t)g.bL);
    if (!with_rows) {
        g.R = 0;
        return;
    }
    g.rowoff.assign(g.R, 0);
    // row r enumerates the digits of the high cached wires (local wires L0..ns-1)
    for (uint32_t r = 0; r < g.R; ++r) {
        uint64_t rem = r, off = 0;
        for (int i = L0; i < g.ns; ++i) {
            const int w = g.sw[i];
            off += (rem % (uint64_t)L.dims[w]) * (uint64_t)L.b[w];
            rem /= (uint64_t)L.dims[w];
        }
        g.rowoff[r] = off;
    }
}


// ---------------------------------------------------------------------------
// Blocks inside a pass: runs of gates on a few wires composed into one matrix.
// ---------------------------------------------------------------------------
struct BlockPlan {
    std::vector<int> gates;  // in application order
    uint64_t lw;             // local wires (bit i = local wire i)
    bool single;
    bool run = false;        // applied gate by gate in registers (kRun), not composed
};

// Shape id of a run over the local wires lw (ascending), or -1.
static int run_shape_of(const TileGeom& geo, uint64_t lw);

static int padded_dim(int P) {
    static const int sizes[] = {4, 6, 8, 9, 12, 16};
    for (int q : sizes)
        if (P <= q) return q;
    return P <= kMaxBlock ? kMaxBlock : kMaxTcBlock;
}

static uint64_t local_mask(const TileGeom& geo, uint64_t global) {
    uint64_t m = 0;
    for (int w = 0; w < 64; ++w)
        if ((global >> w & 1) && geo.loc[w] >= 0) m |= 1ull << geo.loc[w];
    return m;
}

static int64_t local_prod(const TileGeom& geo, uint64_t lw) {
    int64_t p = 1;
    for (int i = 0; i < geo.ns; ++i)
        if (lw >> i & 1) p *= geo.local.dims[i];
    return p;
}

// Cost of a gate or block inside a tile pass, in units of about 6 us per
// 26.9M complex64 amplitudes (measured marginal costs: a dense P x P block
// costs about P units, 8 to 16 dimensions; a single gate of any kind, or a
// diagonal or monomial block, about 2.5 units -- one shared-memory sweep).
static double sweep_cost(int kind, int64_t P) { return kind == kDense && P > 2 ? (double)P : 2.5; }

static void form_blocks(const TileGeom& geo, const std::vector<HGate>& G, const std::vector<int>& pg, int Pmax,
                        std::vector<BlockPlan>& out, bool one_pass_each = false, bool runs = false) {
    out.clear();
    // per gate (index into pg): local wire mask, and whether it can join a block
    const size_t n = pg.size();
    std::vector<uint64_t> lwm(n);
    std::vector<char> inside(n);
    for (size_t i = 0; i < n; ++i) {
        const HGate& h = G[pg[i]];
        lwm[i] = local_mask(geo, h.tmask | h.cmask);
        bool in = h.k == 1;
        for (int c = 0; c < h.nc && in; ++c) in = geo.loc[h.cw[c]] >= 0;
        inside[i] = in;
    }
    // product of the local dimensions of the wires in `add`, times p
    auto grow = [&](int64_t p, uint64_t add) {
        while (add) {
            const int w = __builtin_ctzll(add);
            add &= add - 1;
            p *= geo.local.dims[w];
        }
        return p;
    };
    std::vector<size_t> rem(n);
    for (size_t i = 0; i < n; ++i) rem[i] = i;
    std::vector<char> taken(n, 0);
    while (!rem.empty()) {
        const size_t i0 = rem[0];
        const HGate& g0 = G[pg[i0]];
        BlockPlan bp;
        bp.single = true;
        bp.gates = {pg[i0]};
        bp.lw = lwm[i0];
        std::vector<size_t> sel = {i0};
        const int64_t P0 = grow(1, bp.lw);
        if (Pmax >= 4 && inside[i0] && P0 <= Pmax) {
            uint64_t W = bp.lw, BW = 0, BR = 0;
            int64_t PW = P0;
            double cost_single = sweep_cost(g0.plan.kind, g0.plan.d);
            for (size_t j = 1; j < rem.size(); ++j) {
                const size_t ij = rem[j];
                const HGate& g = G[pg[ij]];
                const uint64_t Wg = g.diag ? 0 : g.tmask;
                const uint64_t Rg = g.cmask | (g.diag ? g.tmask : 0);
                const bool blocked = (Wg & (BW | BR)) || (Rg & BW);
                if (!blocked && inside[ij]) {
                    const uint64_t add = lwm[ij] & ~W;
                    const int64_t P2 = add ? grow(PW, add) : PW;
                    if (P2 <= Pmax) {
                        W |= add;
                        PW = P2;
                        sel.push_back(ij);
                        cost_single += sweep_cost(g.plan.kind, g.plan.d);
                        continue;
                    }
                }
                BW |= Wg;
                BR |= Rg;
            }
            bool all_diag = true;
            for (size_t ij : sel) all_diag = all_diag && G[pg[ij]].diag;
            const double cost_block = sweep_cost(all_diag ? kDiag : kDense, PW);
            // a run: one sweep plus each gate's own arithmetic (d units for a
            // d x d gate, times the share of classes its controls admit)
            double cost_run = 1e300;
            if (runs && !one_pass_each && sel.size() <= (size_t)kMaxRunGates && run_shape_of(geo, W) >= 0) {
                cost_run = 2.5;
                for (size_t ij : sel) {
                    const HGate& g = G[pg[ij]];
                    double share = 1.0;
                    for (int c = 0; c < g.nc; ++c) share /= geo.local.dims[geo.loc[g.cw[c]]];
                    cost_run += g.plan.d * share;
                }
            }
            const double best = cost_run < cost_block ? cost_run : cost_block;
            // one_pass_each: every block or gate costs one pass over the state
            if (sel.size() > 1 && (one_pass_each || best <= cost_single)) {
                bp.single = false;
                bp.run = cost_run < cost_block;
                bp.gates.clear();
                for (size_t ij : sel) bp.gates.push_back(pg[ij]);
                bp.lw = W;
            } else {
                sel.resize(1);
            }
        }
        out.push_back(bp);
        for (size_t ij : sel) taken[ij] = 1;
        std::vector<size_t> rest;
        rest.reserve(rem.size());
        for (size_t ij : rem)
            if (!taken[ij]) rest.push_back(ij);
        rem.swap(rest);
    }
}

// Compose a block in binary64: M = G_k ... G_1 on the P-dimensional space of
// the block's wires (local wires ascending, first least significant).  Each
// gate acts on every column of M as on a state: classes of d entries spaced
// by the target's stride, controls checked on the class's digits.
static void compose_block(const TileGeom& geo, const std::vector<HGate>& G, const BlockPlan& bp,
                          std::vector<double>& M, int& P, std::vector<int>& wl) {
    wl.clear();
    for (int i = 0; i < geo.ns; ++i)
        if (bp.lw >> i & 1) wl.push_back(i);
    std::vector<int> wd(wl.size()), ws(wl.size());
    P = 1;
    for (size_t i = 0; i < wl.size(); ++i) {
        wd[i] = geo.local.dims[wl[i]];
        ws[i] = P;
        P *= wd[i];
    }
    auto pos = [&](int local) {
        for (size_t i = 0; i < wl.size(); ++i)
            if (wl[i] == local) return (int)i;
        return -1;
    };
    M.assign((size_t)2 * P * P, 0.0);
    for (int i = 0; i < P; ++i) M[2 * ((size_t)i * P + i)] = 1.0;
    std::vector<double> col(2 * (size_t)P * P);  // the d rows of one class (d <= P)
    for (int idx : bp.gates) {
        const HGate& h = G[idx];
        const int pt = pos(geo.loc[h.wires[0]]);
        const int d = wd[pt], st = ws[pt];
        std::vector<int> cp, cv;
        for (int c = 0; c < h.nc; ++c) {
            cp.push_back(pos(geo.loc[h.cw[c]]));
            cv.push_back(h.cv[c]);
        }
        // M <- U_g M: the gate acts on M's rows.  For each class (target
        // digit 0, controls met) its d rows are transformed together across
        // all P columns (contiguous inner loop).
        const bool diagonal = h.diag;
        for (int base = 0; base < P; ++base) {
            if ((base / st) % d != 0) continue;  // class representatives: target digit 0
            bool ok = true;
            for (size_t c = 0; c < cp.size(); ++c)
                if ((base / ws[cp[c]]) % wd[cp[c]] != cv[c]) ok = false;
            if (!ok) continue;
            if (diagonal) {
                for (int k = 0; k < d; ++k) {
                    const double ur = h.U[2 * (k * d + k)], ui = h.U[2 * (k * d + k) + 1];
                    if (ur == 1.0 && ui == 0.0) continue;
                    double* row = &M[2 * (size_t)(base + k * st) * P];
                    for (int j = 0; j < P; ++j) {
                        const double xr = row[2 * j], xi = row[2 * j + 1];
                        row[2 * j] = ur * xr - ui * xi;
                        row[2 * j + 1] = ur * xi + ui * xr;
                    }
                }
                continue;
            }
            for (int k = 0; k < d; ++k)
                std::memcpy(&col[2 * (size_t)k * P], &M[2 * (size_t)(base + k * st) * P], sizeof(double) * 2 * P);
            for (int r = 0; r < d; ++r) {
                double* out = &M[2 * (size_t)(base + r * st) * P];
                for (int j = 0; j < P; ++j) {
                    double re = 0.0, im = 0.0;
                    for (int k = 0; k < d; ++k) {
                        const double ur = h.U[2 * (r * d + k)], ui = h.U[2 * (r * d + k) + 1];
                        const double xr = col[2 * ((size_t)k * P + j)], xi = col[2 * ((size_t)k * P + j) + 1];
                        re += ur * xr - ui * xi;
                        im += ur * xi + ui * xr;
                    }
                    out[2 * j] = re;
                    out[2 * j + 1] = im;
                }
            }
        }
    }
}

template <typename R>
static void fill_single(const TileGeom& geo, const HGate& h, FGate& f, std::vector<typename Cplx<R>::T2>& pool) {
    std::memset(static_cast<void*>(&f), 0, sizeof f);
    const Plan& p = h.plan;
    f.single = 1;
    f.P = (uint8_t)p.d;
    f.PP = (uint8_t)p.d;
    f.kind = (uint8_t)p.kind;
    f.lmask = (uint16_t)p.lmask;
    f.smask = (uint16_t)p.smask;
    f.pure = p.pure ? 1 : 0;
    f.u_off = (uint32_t)pool.size();
    for (int i = 0; i < p.d * p.d; ++i) {
        typename Cplx<R>::T2 v;
        v.x = (R)h.U[2 * i];
        v.y = (R)h.U[2 * i + 1];
        pool.push_back(v);
    }
    const int t = geo.loc[h.wires[0]];
    f.lst = (uint32_t)geo.local.b[t];
    f.step = f.lst * (uint32_t)p.d;
    int32_t ins_w[kMaxLocalIns];
    int64_t ins_v[kMaxLocalIns];
    int m = 0;
    ins_w[m] = t;
    ins_v[m] = 0;
    ++m;
    f.n_out = 0;
    for (int c = 0; c < h.nc; ++c) {
        const int lc = geo.loc[h.cw[c]];
        if (lc >= 0) {
            ins_w[m] = lc;
            ins_v[m] = h.cv[c];
            ++m;
        } else {
            f.out_w[f.n_out] = (uint8_t)h.cw[c];
            f.out_v[f.n_out] = (uint8_t)h.cv[c];
            ++f.n_out;
        }
    }
    IndexMap im;
    uint64_t classes;
    build_map(geo.local, ins_w, ins_v, m, im, classes);
    f.map.m = im.m;
    f.map.fixed = (uint32_t)im.fixed;
    for (int i = 0; i < im.m; ++i) f.map.seg[i].init((uint32_t)im.seg[i].d);
    for (int i = 0; i <= im.m; ++i) f.map.off[i] = (uint32_t)im.off[i];
    f.nclasses = (uint32_t)classes;
}

// B operand of a tensor-core tile block: the real embedding of the P x P
// complex matrix M (binary64, row-major interleaved; P <= 32, zero-padded)
// as 64 rows (outputs: real parts 0..31, imaginary parts 32..63) by 64
// columns (inputs, same order), split into TF32 hi (rounded to nearest) and
// lo = value - hi, each 64 x 64 floats in the K-major no-swizzle layout.
static void tile_tc_pack(const std::vector<double>& M, int P, float* out) {
    std::memset(out, 0, kTileTcOpBytes);
    unsigned char* hi = reinterpret_cast<unsigned char*>(out);
    unsigned char* lo = hi + kTileTcOpBytes / 2;
    auto put = [&](int n, int k, double v) {
        const float f = (float)v;
        uint32_t bits;
        std::memcpy(&bits, &f, 4);
        bits = tf32_rne_bits(bits);
        float h;
        std::memcpy(&h, &bits, 4);
        const float l = (float)(v - (double)h);
        const uint32_t o = kmajor_off((uint32_t)n, (uint32_t)k, 64);
        std::memcpy(hi + o, &h, 4);
        std::memcpy(lo + o, &l, 4);
    };
    for (int r = 0; r < P; ++r)
        for (int c = 0; c < P; ++c) {
            const double re = M[2 * ((size_t)r * P + c)], im = M[2 * ((size_t)r * P + c) + 1];
            put(r, c, re);
            put(r, 32 + c, -im);
            put(32 + r, c, im);
            put(32 + r, 32 + c, re);
        }
}

template <typename R>
static void fill_block(const TileGeom& geo, const std::vector<HGate>& G, const BlockPlan& bp, FGate& f,
                       std::vector<typename Cplx<R>::T2>& pool, Program* prog = nullptr) {
    std::memset(static_cast<void*>(&f), 0, sizeof f);
    std::vector<double> M;
    std::vector<int> wl;
    int P = 0;
    compose_block(geo, G, bp, M, P, wl);
    const int PP = padded_dim(P);
    const bool tc = P > kMaxBlock;  // 17..32 dimensions: a tensor-core block (complex64 tiles)
    if (tc) {
        f.single = 0;
        f.P = (uint8_t)P;
        f.PP = (uint8_t)PP;
        f.kind = kTcBlock;
        bool unitary = true;
        for (int idx : bp.gates) unitary = unitary && G[idx].unitary;
        f.unitary = unitary ? 1 : 0;
        if (prog) {
            std::vector<float> B(kTileTcOpBytes / sizeof(float));
            tile_tc_pack(M, P, B.data());
            f.op_off = (uint32_t)prog->put(B.data(), kTileTcOpBytes);
        }
    }
    auto re = [&](int r, int c) { return M[2 * ((size_t)r * P + c)]; };
    auto im = [&](int r, int c) { return M[2 * ((size_t)r * P + c) + 1]; };
    auto nz = [&](int r, int c) { return re(r, c) != 0.0 || im(r, c) != 0.0; };
    auto one = [&](int r, int c) { return re(r, c) == 1.0 && im(r, c) == 0.0; };
    bool diag = !tc, mono = !tc;
    int src[kMaxBlock];
    bool used[kMaxBlock] = {false};
    for (int r = 0; r < P && !tc; ++r) {
        int cnt = 0;
        for (int c = 0; c < P; ++c)
            if (nz(r, c)) {
                ++cnt;
                src[r] = c;
                if (c != r) diag = false;
            }
        if (cnt != 1 || used[src[r]]) mono = false;
        else used[src[r]] = true;
    }
    if (!tc) {
    f.single = 0;
    f.P = (uint8_t)P;
    f.PP = (uint8_t)PP;
    f.lmask = f.smask = 0;
    f.pure = 0;
    if (diag) {
        f.kind = kDiag;
        for (int r = 0; r < P; ++r)
            if (!one(r, r)) f.lmask |= (uint16_t)(1u << r);
        f.smask = f.lmask;
    } else if (mono) {
        f.kind = kPerm;
        f.pure = 1;
        for (int r = 0; r < P; ++r) {
            if (!one(r, src[r])) f.pure = 0;
            if (src[r] != r || !one(r, src[r])) {
                f.smask |= (uint16_t)(1u << r);
                f.lmask |= (uint16_t)(1u << src[r]);
            }
        }
    } else {
        f.kind = kDense;
        f.lmask = f.smask = (uint16_t)((1u << P) - 1u);
    }
    if (pool.size() % 2) pool.push_back(typename Cplx<R>::T2{});  // 16-byte aligned rows for paired loads
    f.u_off = (uint32_t)pool.size();
    for (int r = 0; r < PP; ++r)
        for (int c = 0; c < PP; ++c) {
            typename Cplx<R>::T2 v;
            v.x = (r < P && c < P) ? (R)re(r, c) : (R)0;
            v.y = (r < P && c < P) ? (R)im(r, c) : (R)0;
            pool.push_back(v);
        }
    }  // !tc
    for (int r = 0; r < P; ++r) {
        uint32_t o = 0;
        int rem = r;
        for (int lw : wl) {
            const int d = geo.local.dims[lw];
            o += (uint32_t)(rem % d) * (uint32_t)geo.local.b[lw];
            rem /= d;
        }
        f.off[r] = (uint16_t)o;
    }
    int32_t ins_w[kMaxLocalIns];
    int64_t ins_v[kMaxLocalIns];
    int m = 0;
    for (int lw : wl) {
        ins_w[m] = lw;
        ins_v[m] = 0;
        ++m;
    }
    IndexMap imap;
    uint64_t classes;
    build_map(geo.local, ins_w, ins_v, m, imap, classes);
    f.map.m = imap.m;
    f.map.fixed = (uint32_t)imap.fixed;
    for (int i = 0; i < imap.m; ++i) f.map.seg[i].init((uint32_t)imap.seg[i].d);
    for (int i = 0; i <= imap.m; ++i) f.map.off[i] = (uint32_t)imap.off[i];
    f.nclasses = (uint32_t)classes;
    f.n_out = 0;
}

static int run_shape_of(const TileGeom& geo, uint64_t lw) {
    int d[4] = {1, 1, 1, 1}, n = 0;
    for (int i = 0; i < geo.ns; ++i)
        if (lw >> i & 1) {
            if (n == 4) return -1;
            d[n++] = geo.local.dims[i];
        }
    for (int id = 0; id < kRunShapes; ++id) {
        bool eq = true;
        for (int j = 0; j < 4; ++j) eq = eq && run_shape_dims(id, j) == d[j];
        if (eq) return id;
    }
    return -1;
}

// A run (kRun): the block's gates in order, each as its d x d matrix, target
// position and member mask, applied in registers by run_block.
template <typename R>
static void fill_run(const TileGeom& geo, const std::vector<HGate>& G, const BlockPlan& bp, FGate& f,
                     std::vector<typename Cplx<R>::T2>& pool) {
    std::memset(static_cast<void*>(&f), 0, sizeof f);
    std::vector<int> wl;
    for (int i = 0; i < geo.ns; ++i)
        if (bp.lw >> i & 1) wl.push_back(i);
    const int shape = run_shape_of(geo, bp.lw);
    int dm[4], st[4], P = 1;
    for (int j = 0; j < 4; ++j) {
        dm[j] = run_shape_dims(shape, j);
        st[j] = P;
        P *= dm[j];
    }
    auto pos = [&](int global_wire) {
        const int lw = geo.loc[global_wire];
        for (size_t j = 0; j < wl.size(); ++j)
            if (wl[j] == lw) return (int)j;
        return -1;
    };
    f.single = 0;
    f.kind = kRun;
    f.P = (uint8_t)P;
    f.PP = (uint8_t)P;
    f.lmask = f.smask = (uint16_t)((1u << P) - 1u);
    f.shape = (uint8_t)shape;
    f.nsub = (uint8_t)bp.gates.size();
    bool unitary = true;
    for (size_t s = 0; s < bp.gates.size(); ++s) {
        const HGate& h = G[bp.gates[s]];
        unitary = unitary && h.unitary;
        f.sub_pos[s] = (uint8_t)pos(h.wires[0]);
        uint32_t mask = 0;
        for (int m = 0; m < P; ++m) {
            bool ok = true;
            for (int c = 0; c < h.nc; ++c) {
                const int j = pos(h.cw[c]);
                ok = ok && (m / st[j]) % dm[j] == h.cv[c];
            }
            if (ok) mask |= 1u << m;
        }
        f.sub_mask[s] = (uint16_t)mask;
        f.sub_u[s] = (uint16_t)pool.size();
        const int d = h.plan.d;
        for (int i = 0; i < d * d; ++i) {
            typename Cplx<R>::T2 v;
            v.x = (R)h.U[2 * i];
            v.y = (R)h.U[2 * i + 1];
            pool.push_back(v);
        }
    }
    f.unitary = unitary ? 1 : 0;
    for (int r = 0; r < P; ++r) {
        uint32_t o = 0;
        for (size_t j = 0; j < wl.size(); ++j) o += (uint32_t)((r / st[j]) % dm[j]) * (uint32_t)geo.local.b[wl[j]];
        f.off[r] = (uint16_t)o;
    }
    int32_t ins_w[kMaxLocalIns];
    int64_t ins_v[kMaxLocalIns];
    int m = 0;
    for (int lw : wl) {
        ins_w[m] = lw;
        ins_v[m] = 0;
        ++m;
    }
    IndexMap imap;
    uint64_t classes;
    build_map(geo.local, ins_w, ins_v, m, imap, classes);
    f.map.m = imap.m;
    f.map.fixed = (uint32_t)imap.fixed;
    for (int i = 0; i < imap.m; ++i) f.map.seg[i].init((uint32_t)imap.seg[i].d);
    for (int i = 0; i <= imap.m; ++i) f.map.off[i] = (uint32_t)imap.off[i];
    f.nclasses = (uint32_t)classes;
}

// Chunks of a list of blocks, contiguous, appended to prog.desc (256-aligned
// start).  Returns the first chunk's offset; *nchunks the count; *dmax the
// largest single-wire dimension (kernel instance).
template <typename R>
static size_t emit_chunks(const TileGeom& geo, const std::vector<HGate>& G, const std::vector<BlockPlan>& blocks,
                          Program& prog, uint32_t* nchunks, int* dmax, bool* has_tc = nullptr,
                          uint32_t* max_bytes = nullptr, uint32_t* first_bytes = nullptr) {
    using T2 = typename Cplx<R>::T2;
    std::vector<char> buf;
    uint32_t n = 0, mb = 0;
    int dm = 2;
    size_t i = 0;
    while (i < blocks.size()) {
        std::vector<FGate> fg;
        std::vector<T2> pool;
        while (i < blocks.size() && fg.size() < (size_t)kMaxChunkGates) {
            const BlockPlan& bp = blocks[i];
            const int64_t Pb = bp.single ? 0 : local_prod(geo, bp.lw);
            size_t need = bp.single ? (size_t)G[bp.gates[0]].plan.d * G[bp.gates[0]].plan.d
                                    : (Pb > kMaxBlock ? 0 : (size_t)padded_dim((int)Pb) * padded_dim((int)Pb));
            if (bp.run) {
                need = 0;
                for (int idx : bp.gates) need += (size_t)G[idx].plan.d * G[idx].plan.d;
            }
            if (pool.size() + need + 1 > (size_t)kPoolEntries && !fg.empty()) break;
            FGate f;
            if (bp.single) {
                fill_single<R>(geo, G[bp.gates[0]], f, pool);
                dm = G[bp.gates[0]].plan.d > dm ? G[bp.gates[0]].plan.d : dm;
            } else if (bp.run) {
                fill_run<R>(geo, G, bp, f, pool);
            } else {
                fill_block<R>(geo, G, bp, f, pool, &prog);
                if (f.kind == kTcBlock && has_tc) *has_tc = true;
            }
            fg.push_back(f);
            ++i;
        }
        ChunkHdr h{};
        h.ngates = (uint32_t)fg.size();
        h.npool = (uint32_t)pool.size();
        h.bytes = (uint32_t)((chunk_bytes<R>(h.ngates, h.npool) + 15) & ~(size_t)15);
        mb = h.bytes > mb ? h.bytes : mb;
        if (n == 0 && first_bytes) *first_bytes = h.bytes;
        const size_t o = buf.size();
        buf.resize(o + h.bytes, 0);
        std::memcpy(buf.data() + o, &h, sizeof h);
        std::memcpy(buf.data() + o + sizeof h, fg.data(), sizeof(FGate) * fg.size());
        std::memcpy(buf.data() + o + sizeof h + sizeof(FGate) * fg.size(), pool.data(), sizeof(T2) * pool.size());
        ++n;
    }
    *nchunks = n;
    if (dmax) *dmax = dm;
    if (max_bytes) *max_bytes = mb;
    return prog.put(buf.data(), buf.size());
}

// QD_FUSE_BLOCK: blocks over the whole state, one pass each.
// Whole-state blocks (QD_FUSE_BLOCK), each one pass over the state.  A block
// starts from the wires of the first remaining gate and takes every later
// gate on its wires that commutes with the gates left behind before it; then,
// one gate's wires at a time, the block adds the wires that let it take the
// most gates (ties: the smaller block), while it stays within Pmax
// dimensions and the addition takes more gates.  Its wires are then those of
// the gates it took.  (Adding wires in gate order instead: 25 blocks for the
// 200 gates of the 18-qubit + 8-qutrit workload at Pmax = 64, this 20.)
static void form_whole_blocks(const TileGeom& geo, const std::vector<HGate>& G, int Pmax,
                              std::vector<BlockPlan>& out) {
    out.clear();
    const size_t n = G.size();
    std::vector<uint64_t> lwm(n);
    std::vector<char> inside(n);
    for (size_t i = 0; i < n; ++i) {
        const HGate& h = G[i];
        lwm[i] = local_mask(geo, h.tmask | h.cmask);
        bool in = h.k == 1;
        for (int c = 0; c < h.nc && in; ++c) in = geo.loc[h.cw[c]] >= 0;
        inside[i] = in;
    }
    auto prod_of = [&](uint64_t m) {
        int64_t p = 1;
        while (m) {
            p *= geo.local.dims[__builtin_ctzll(m)];
            m &= m - 1;
        }
        return p;
    };
    std::vector<int> rem(n);
    for (size_t i = 0; i < n; ++i) rem[i] = (int)i;
    // the gates a block on wires S takes from the first kPlanWindow remaining
    auto scan = [&](uint64_t S, std::vector<int>* sel) {
        uint64_t BW = 0, BR = 0;
        int cnt = 0;
        const size_t m = rem.size() < kPlanWindow ? rem.size() : kPlanWindow;
        for (size_t j = 0; j < m; ++j) {
            const int gi = rem[j];
            const HGate& g = G[gi];
            const uint64_t Wg = g.diag ? 0 : g.tmask;
            const uint64_t Rg = g.cmask | (g.diag ? g.tmask : 0);
            const bool blocked = (Wg & (BW | BR)) || (Rg & BW);
            if (!blocked && inside[gi] && (lwm[gi] & ~S) == 0) {
                ++cnt;
                if (sel) sel->push_back(gi);
                continue;
            }
            BW |= Wg;
            BR |= Rg;
        }
        return cnt;
    };
    std::vector<char> taken(n, 0);
    std::vector<uint64_t> tried;
    while (!rem.empty()) {
        const int g0 = rem[0];
        BlockPlan bp;
        bp.single = true;
        bp.gates = {g0};
        bp.lw = lwm[g0];
        if (Pmax >= 4 && inside[g0] && prod_of(lwm[g0]) <= Pmax) {
            uint64_t S = lwm[g0];
            int cur = scan(S, nullptr);
            for (;;) {
                uint64_t bestS = 0;
                int bestN = cur;
                int64_t bestP = 0;
                tried.clear();
                const size_t m = rem.size() < kPlanWindow ? rem.size() : kPlanWindow;
                for (size_t j = 0; j < m; ++j) {
                    const int gi = rem[j];
                    if (!inside[gi]) continue;
                    const uint64_t S2 = S | lwm[gi];
                    if (S2 == S) continue;
                    bool seen = false;
                    for (uint64_t t : tried) seen = seen || t == S2;
                    if (seen) continue;
                    tried.push_back(S2);
                    const int64_t P2 = prod_of(S2);
                    if (P2 > Pmax) continue;
                    const int c2 = scan(S2, nullptr);
                    if (c2 > bestN || (c2 == bestN && bestS != 0 && P2 < bestP)) {
                        bestS = S2;
                        bestN = c2;
                        bestP = P2;
                    }
                }
                if (bestS == 0) break;  // no addition takes more gates
                S = bestS;
                cur = bestN;
            }
            std::vector<int> sel;
            scan(S, &sel);
            if (sel.size() > 1) {
                bp.single = false;
                bp.gates = sel;
                bp.lw = 0;
                for (int gi : sel) bp.lw |= lwm[gi];
            }
        }
        out.push_back(bp);
        for (int gi : bp.gates) taken[gi] = 1;
        std::vector<int> rest;
        rest.reserve(rem.size());
        for (int gi : rem)
            if (!taken[gi]) rest.push_back(gi);
        rem.swap(rest);
    }
}

static void plan_blocks(const Layout& L, const std::vector<HGate>& G, const FuseCfg& cfg,
                        std::vector<PassPlan>& passes) {
    TileGeom geo;
    tile_geometry(L, (L.n >= 64) ? ~0ull : ((1ull << L.n) - 1), 1, geo, false);
    std::vector<BlockPlan> blocks;
    form_whole_blocks(geo, G, cfg.block_dim, blocks);
    for (const BlockPlan& bp : blocks) {
        PassPlan p;
        p.tile = false;
        p.block = !bp.single;
        p.gates = bp.gates;
        p.smask = bp.lw;  // local wires == global wires here
        p.T = 0;
        passes.push_back(p);
    }
}

// The single gate equivalent to a QD_FUSE_BLOCK pass: its wires (ascending)
// and its composed matrix.
static qd_status block_gate_of(const Layout& L, int32_t prec, const std::vector<HGate>& G, const PassPlan& p,
                               std::vector<int>& wl, std::vector<double>& M, Plan& q) {
    TileGeom geo;
    tile_geometry(L, (L.n >= 64) ? ~0ull : ((1ull << L.n) - 1), 1, geo, false);
    BlockPlan bp;
    bp.gates = p.gates;
    bp.lw = p.smask;
    bp.single = false;
    int P = 0;
    compose_block(geo, G, bp, M, P, wl);
    std::vector<int32_t> w32(wl.begin(), wl.end());
    return make_plan(L, prec, w32.data(), (int32_t)w32.size(), M.data(), nullptr, nullptr, 0, q);
}

// ---------------------------------------------------------------------------
// Programs: the launches of a circuit with their descriptors.  Building a
// program makes no CUDA call; running it uploads the descriptors once and
// issues the launches, so many programs can share one upload and be issued
// on several streams or inside a CUDA graph capture.
// ---------------------------------------------------------------------------
qd_status Arena::upload(const void* bytes, size_t n, cudaStream_t s) {
    if (n == 0) return QD_OK;
    if (n > cap) {
        QD_CUDA(cudaStreamSynchronize(s), "descriptor arena resize");
        if (ev_live) cudaEventSynchronize(ev);
        if (dev) cudaFree(dev);
        if (host) cudaFreeHost(host);
        dev = host = nullptr;
        cap = 0;
        const size_t want = n + n / 2;
        cudaError_t e = cudaMalloc(&dev, want);
        if (e != cudaSuccess) return fail(QD_ERR_OOM, "descriptor arena: %s", cudaGetErrorString(e));
        e = cudaMallocHost(&host, want);
        if (e != cudaSuccess) return fail(QD_ERR_OOM, "pinned descriptor arena: %s", cudaGetErrorString(e));
        cap = want;
        if (!ev_live) {
            QD_CUDA(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming), "cudaEventCreate");
            ev_live = true;
        }
    } else if (ev_live) {
        QD_CUDA(cudaEventSynchronize(ev), "descriptor staging wait");
    }
    std::memcpy(host, bytes, n);
    QD_CUDA(cudaMemcpyAsync(dev, host, n, cudaMemcpyHostToDevice, s), "descriptor upload");
    count_upload(n);
    QD_CUDA(cudaEventRecord(ev, s), "descriptor event");
    return QD_OK;
}

void Arena::release() {
    if (ev_live) {
        cudaEventSynchronize(ev);
        cudaEventDestroy(ev);
    }
    if (dev) cudaFree(dev);
    if (host) cudaFreeHost(host);
    dev = host = nullptr;
    cap = 0;
    ev_live = false;
}

template <typename R, int DT>
static Op gate1_op(void* psi, const Plan& p, const double* U) {
    using T2 = typename Cplx<R>::T2;
    Gate1Args<R, DT> a;
    std::memset(static_cast<void*>(&a), 0, sizeof a);
    a.psi = reinterpret_cast<T2*>(psi);
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
    if (sizeof(R) == 4 && p.vec == 2)
        return [a](cudaStream_t s, const char*) { return launch_gate1<R, DT, (sizeof(R) == 4 ? 2 : 1)>(a, s); };
    return [a](cudaStream_t s, const char*) { return launch_gate1<R, DT, 1>(a, s); };
}

// The op of one gate for the per-gate kernels (no fusion).
template <typename R>
static Op gate_op(void* psi, const Plan& p, const double* U, Program& prog, int tc_mode, bool unitary,
                  const Layout& L, const int32_t* wires, int nwires, int ncontrols) {
    using T2 = typename Cplx<R>::T2;
    if (p.family == 0) {
        switch (p.d) {
            case 2: return gate1_op<R, 2>(psi, p, U);
            case 3: return gate1_op<R, 3>(psi, p, U);
            case 4: return gate1_op<R, 4>(psi, p, U);
            case 5: return gate1_op<R, 5>(psi, p, U);
            case 6: return gate1_op<R, 6>(psi, p, U);
            case 7: return gate1_op<R, 7>(psi, p, U);
            default: return gate1_op<R, 8>(psi, p, U);
        }
    }
    const int P = p.P;
    if (sizeof(R) == 4 && P >= kRingMinP && tc_mode == QD_TC_BF16X3 && ncontrols == 0) {
        // BF16x3 through the ring of tiles, where the block suits it
        std::vector<unsigned char> bops;
        std::shared_ptr<const BlockRing> ring = block_ring_prepare(L, reinterpret_cast<float2*>(psi), wires, nwires, P,
                                                                   U, unitary, bops);
        if (ring) {
            const size_t boff = prog.put(bops.data(), bops.size());
            return [ring, boff](cudaStream_t s, const char* base) { return launch_block_ring(*ring, base + boff, s); };
        }
    }
    if (sizeof(R) == 4 && P >= kTcMinP && tc_mode != QD_TC_OFF) {
        // complex64 block of 17..64 dimensions: tensor cores
        std::vector<float> A(block_tc_operand_bytes() / sizeof(float));
        block_tc_pack(U, P, tc_mode, A.data());
        const size_t aoff = prog.put(A.data(), block_tc_operand_bytes());
        const uint64_t classes = p.classes;
        const IndexMap map = p.map;
        std::vector<uint64_t> off(p.off, p.off + P);
        float2* dpsi = reinterpret_cast<float2*>(psi);
        const bool renorm = unitary;
        const uint64_t D = p.D;
        return [dpsi, aoff, tc_mode, renorm, classes, map, P, off, D](cudaStream_t s, const char* base) {
            return launch_block_tc(dpsi, D, base + aoff, tc_mode, renorm, classes, map, P, off.data(), s);
        };
    }
    std::vector<T2> m((size_t)P * P);
    for (int i = 0; i < P * P; ++i) {
        m[i].x = (R)U[2 * i];
        m[i].y = (R)U[2 * i + 1];
    }
    const size_t uoff = prog.put(m.data(), sizeof(T2) * m.size());
    GateTileArgs<R> a;
    std::memset(static_cast<void*>(&a), 0, sizeof a);
    a.psi = reinterpret_cast<T2*>(psi);
    a.D = p.D - g_bounds_shrink;
    a.n_classes = p.classes;
    a.map = p.map;
    a.P = P;
    a.Q = 64;
    for (int r = 0; r < P; ++r) a.off[r] = p.off[r];
    const int smem = (int)gate_tile_smem<R>(P, a.Q);
    return [a, uoff, smem](cudaStream_t s, const char* base) {
        GateTileArgs<R> b = a;
        b.U = reinterpret_cast<const T2*>(base + uoff);
        return launch_gate_tile<R>(b, s, smem);
    };
}


// Ops of a whole circuit on the state at psi (layout L): optional reset to
// |0...0>, then the planned passes in order.
// Ops of passes[begin, end) (composition, chunk records, launch closures).
template <typename R>
static void build_passes(const Layout& L, void* psi, const std::vector<HGate>& G, const FuseCfg& cfg,
                         const std::vector<PassPlan>& passes, size_t begin, size_t end, Program& prog) {
    using T2 = typename Cplx<R>::T2;
    for (size_t pi = begin; pi < end; ++pi) {
        const PassPlan& p = passes[pi];
        if (p.block) {
            std::vector<int> wl;
            std::vector<double> M;
            Plan q;
            if (block_gate_of(L, sizeof(R) == 4 ? QD_C64 : QD_C128, G, p, wl, M, q) != QD_OK) continue;
            if (q.family == 0 && q.smask == 0) continue;  // identity
            bool unitary = true;
            for (int idx : p.gates) unitary = unitary && G[idx].unitary;
            std::vector<int32_t> w32(wl.begin(), wl.end());
            prog.ops.push_back(gate_op<R>(psi, q, M.data(), prog, cfg.tc_mode, unitary, L, w32.data(),
                                          (int)w32.size(), 0));
            continue;
        }
        if (!p.tile) {
            const HGate& h = G[p.gates[0]];
            if (h.plan.family == 0 && h.plan.smask == 0) continue;  // identity
            if (h.plan.classes == 0) continue;
            prog.ops.push_back(gate_op<R>(psi, h.plan, h.U, prog, cfg.tc_mode, h.unitary, L, h.wires, h.k, h.nc));
            continue;
        }
        TileGeom geo;
        tile_geometry(L, p.smask, cfg.min_row, geo);
        std::vector<BlockPlan> blocks;
        form_blocks(geo, G, p.gates, cfg.block_dim, blocks, false, cfg.runs && sizeof(R) == 4);
        uint32_t nchunks = 0;
        int dmax = 2;
        bool has_tc = false;
        uint32_t stage_bytes = 0, first_bytes = 0;
        const size_t offC = emit_chunks<R>(geo, G, blocks, prog, &nchunks, &dmax, &has_tc, &stage_bytes, &first_bytes);
        const size_t offR = prog.put(geo.rowoff.data(), sizeof(uint64_t) * geo.R);
        FusedArgs<R> a;
        std::memset(static_cast<void*>(&a), 0, sizeof a);
        a.psi = reinterpret_cast<T2*>(psi);
        a.nchunks = (int32_t)nchunks;
        a.T = (uint32_t)p.T;
        a.bL = geo.bL;
        a.rows = geo.R;
        a.vec2 = (sizeof(R) == 4 && geo.bL % 2 == 0) ? 1 : 0;
        a.bLdiv.init(geo.bL);
        a.ntiles = (uint64_t)(L.D / p.T);
        a.nfree = geo.nfree;
        for (int i = 0; i < geo.nfree; ++i) {
            a.free_w[i] = geo.free_w[i];
            a.free_d[i] = geo.free_d[i];
            a.free_div[i].init(geo.free_d[i]);
            a.free_b[i] = geo.free_b[i];
        }
        a.status = tc_status_ptr();
        a.stage = stage_bytes;
        a.first_bytes = first_bytes;
        prog.ops.push_back([a, offC, offR, dmax, has_tc](cudaStream_t s, const char* base) {
            FusedArgs<R> b = a;
            b.chunks = base + offC;
            b.rowoff = reinterpret_cast<const uint64_t*>(base + offR);
            b.desc_base = base;
            if constexpr (sizeof(R) == 4) {
                if (has_tc) {
                    if (!b.status) return cudaErrorInvalidSymbol;
                    return launch_fused_tc(b, dmax, s);
                }
            }
            return launch_fused<R>(b, dmax, s);
        });
    }
}

// The passes of one circuit as entries of a batch's layer queue (entry k
// goes to layer k), when every pass is a tile pass on CUDA cores with at
// most kLayerMaxFree wires outside its tile; false otherwise (the circuit
// then runs as its own program).  smem[k]: the dynamic shared memory of
// entry k; dmax[k]: its largest single-wire dimension.
template <typename R>
static bool build_layer_entries(const Layout& L, void* psi, const std::vector<HGate>& G, const FuseCfg& cfg,
                                const std::vector<PassPlan>& passes, Program& prog,
                                std::vector<LayerEntry<R>>& out, std::vector<int>& dmax_out,
                                std::vector<size_t>& smem) {
    using T2 = typename Cplx<R>::T2;
    out.clear();
    dmax_out.clear();
    smem.clear();
    for (const PassPlan& p : passes)
        if (!p.tile || p.block) return false;
    for (const PassPlan& p : passes) {
        TileGeom geo;
        tile_geometry(L, p.smask, cfg.min_row, geo);
        if (geo.nfree > kLayerMaxFree) return false;
        std::vector<BlockPlan> blocks;
        form_blocks(geo, G, p.gates, cfg.block_dim, blocks, false, cfg.runs && sizeof(R) == 4);
        uint32_t nchunks = 0, stage_bytes = 0, first_bytes = 0;
        int dmax = 2;
        bool has_tc = false;
        const size_t offC = emit_chunks<R>(geo, G, blocks, prog, &nchunks, &dmax, &has_tc, &stage_bytes, &first_bytes);
        if (has_tc) return false;
        const size_t offR = prog.put(geo.rowoff.data(), sizeof(uint64_t) * geo.R);
        LayerEntry<R> e;
        std::memset(static_cast<void*>(&e), 0, sizeof e);
        e.psi = reinterpret_cast<T2*>(psi);
        e.chunks_off = offC;
        e.rows_off = offR;
        e.nchunks = (int32_t)nchunks;
        e.T = (uint32_t)p.T;
        e.bL = geo.bL;
        e.rows = geo.R;
        e.vec2 = (sizeof(R) == 4 && geo.bL % 2 == 0) ? 1 : 0;
        e.bLdiv.init(geo.bL);
        e.ntiles = (uint64_t)(L.D / p.T);
        e.nfree = geo.nfree;
        for (int i = 0; i < geo.nfree; ++i) {
            e.free_w[i] = geo.free_w[i];
            e.free_d[i] = geo.free_d[i];
            e.free_div[i].init(geo.free_d[i]);
            e.free_b[i] = geo.free_b[i];
        }
        e.stage = stage_bytes;
        e.first_bytes = first_bytes;
        out.push_back(e);
        dmax_out.push_back(dmax);
        smem.push_back((size_t)stage_bytes + fused_rows_bytes(geo.R) + sizeof(T2) * (size_t)p.T);
    }
    return true;
}

template <typename R>
void build_program(const Layout& L, void* psi, const std::vector<HGate>& G, const FuseCfg& cfg,
                          bool reset_first, Program& prog) {
    if (reset_first) {
        const int64_t D = L.D;
        prog.ops.push_back([psi, D](cudaStream_t s, const char*) { return launch_set_basis<R>(psi, D, 0, s); });
    }
    std::vector<PassPlan> passes;
    plan_passes(L, G, cfg, passes);
    build_passes<R>(L, psi, G, cfg, passes, 0, passes.size(), prog);
}

qd_status issue(const Program& prog, const char* base, cudaStream_t s) {
    for (const Op& op : prog.ops) {
        NvtxRange r("pass");
        cudaError_t e = op(s, base);
        if (e != cudaSuccess) return cuda_fail(e, "circuit kernel launch");
    }
    return QD_OK;
}

qd_status check_cfg(const FuseCfg& cfg, int32_t prec) {
    if (cfg.mode != QD_FUSE_OFF && cfg.mode != QD_FUSE_TILE && cfg.mode != QD_FUSE_BLOCK)
        return fail(QD_ERR_ARG, "unknown fusion mode");
    if (cfg.tc_mode != QD_TC_TF32X3 && cfg.tc_mode != QD_TC_BF16X3 && cfg.tc_mode != QD_TC_OFF)
        return fail(QD_ERR_ARG, "unknown tc_mode %d", cfg.tc_mode);
    if (cfg.mode == QD_FUSE_TILE && cfg.Tmax > tile_limit(prec))
        return fail(QD_ERR_UNSUPPORTED, "tile of %lld amplitudes exceeds shared memory (limit %lld)",
                    (long long)cfg.Tmax, (long long)tile_limit(prec));
    return QD_OK;
}

bool small_eligible(const Layout& L, const std::vector<HGate>& G, int64_t small_max, int* dmax) {
    if (L.D > small_max || G.empty()) return false;
    int dm = 2;
    for (const HGate& h : G) {
        if (!h.fusable) return false;
        dm = h.plan.d > dm ? h.plan.d : dm;
    }
    if (dmax) *dmax = dm;
    return true;
}

template <typename R>
size_t put_small_chunks(const Layout& L, const std::vector<HGate>& G, const FuseCfg& cfg, Program& prog,
                        uint32_t* nchunks) {
    TileGeom geo;
    tile_geometry(L, (L.n >= 64) ? ~0ull : ((1ull << L.n) - 1), 1, geo, false);
    std::vector<int> all(G.size());
    for (size_t i = 0; i < G.size(); ++i) all[i] = (int)i;
    std::vector<BlockPlan> blocks;
    // one-CTA circuits apply chunks without tensor cores: blocks of at most 16 dimensions
    form_blocks(geo, G, all, cfg.block_dim < kMaxBlock ? cfg.block_dim : kMaxBlock, blocks, false,
                cfg.runs && sizeof(R) == 4);
    return emit_chunks<R>(geo, G, blocks, prog, nchunks, nullptr);
}

template size_t put_small_chunks<float>(const Layout&, const std::vector<HGate>&, const FuseCfg&, Program&,
                                        uint32_t*);
template size_t put_small_chunks<double>(const Layout&, const std::vector<HGate>&, const FuseCfg&, Program&,
                                         uint32_t*);

// Arithmetic of one gate or block over the whole state (real flops): 8 P per
// amplitude of each visited class when dense, 6 per changed amplitude when
// diagonal or a phased permutation, nothing for a pure permutation.
static double unit_flops(int kind, bool pure, int P, int changed_rows, double classes) {
    if (kind == kDense) return 8.0 * P * P * classes;
    if (kind == kPerm && pure) return 0.0;
    return 6.0 * changed_rows * classes;
}

static double pass_arith(const Layout& L, const std::vector<HGate>& G, const FuseCfg& cfg, const PassPlan& p) {
    auto popc = [](uint32_t m) { int c = 0; while (m) { c += m & 1u; m >>= 1; } return c; };
    if (p.block) {
        std::vector<int> wl;
        std::vector<double> M;
        Plan q;
        if (block_gate_of(L, QD_C128, G, p, wl, M, q) != QD_OK) return 0.0;
        if (q.family == 1) return 8.0 * q.P * q.P * (double)q.classes;
        return unit_flops(q.kind, q.pure, q.d, popc(q.smask), (double)q.classes);
    }
    if (!p.tile) {
        const Plan& q = G[p.gates[0]].plan;
        if (q.family == 1) return 8.0 * q.P * q.P * (double)q.classes;
        return unit_flops(q.kind, q.pure, q.d, popc(q.smask), (double)q.classes);
    }
    TileGeom geo;
    tile_geometry(L, p.smask, cfg.min_row, geo);
    std::vector<BlockPlan> blocks;
    form_blocks(geo, G, p.gates, cfg.block_dim, blocks, false, cfg.runs);
    const double tiles = (double)(L.D / p.T);
    double f = 0.0;
    std::vector<typename Cplx<double>::T2> pool;
    for (const BlockPlan& bp : blocks) {
        FGate fg;
        if (bp.run) {  // each gate's d x d product on the groups its controls admit
            fill_run<double>(geo, G, bp, fg, pool);
            for (int s = 0; s < fg.nsub; ++s) {
                int pm = 0;
                for (uint32_t m = fg.sub_mask[s]; m; m &= m - 1) ++pm;
                f += tiles * (double)fg.nclasses * 8.0 * run_shape_dims(fg.shape, fg.sub_pos[s]) * pm;
            }
            continue;
        }
        if (bp.single) fill_single<double>(geo, G[bp.gates[0]], fg, pool);
        else fill_block<double>(geo, G, bp, fg, pool);
        if (fg.kind == kTcBlock) f += tiles * 8.0 * fg.P * fg.P * (double)fg.nclasses;  // dense block
        else f += tiles * unit_flops(fg.kind, fg.pure != 0, fg.P, popc(fg.smask), (double)fg.nclasses);
    }
    return f;
}

template void build_program<float>(const Layout&, void*, const std::vector<HGate>&, const FuseCfg&, bool,
                                   Program&);
template void build_program<double>(const Layout&, void*, const std::vector<HGate>&, const FuseCfg&, bool,
                                    Program&);
template cudaError_t launch_batch_small<float>(const SmallTask*, int, int, uint32_t, char*, const char*, double*,
                                               cudaStream_t);
template cudaError_t launch_batch_small<double>(const SmallTask*, int, int, uint32_t, char*, const char*, double*,
                                                cudaStream_t);

}  // namespace qd

using namespace qd;

// ---------------------------------------------------------------------------
// Batches of independent circuits.
// ---------------------------------------------------------------------------
struct qd_batch {
    int32_t prec;
    cudaStream_t main;     // the caller's stream
    cudaStream_t work;     // private stream the run is issued (or captured) on
    cudaEvent_t in_ev, out_ev;
    bool work_live;
    std::vector<cudaStream_t> aux;
    std::vector<cudaEvent_t> aux_ev;
    cudaEvent_t fork_ev;
    bool fork_live;
    char* states;          // all states of the last run
    size_t states_cap;
    std::vector<uint64_t> psi_off;
    std::vector<int64_t> D;
    double* norms;         // device, one per circuit
    double* host_norms;    // pinned
    size_t norms_cap;
    double* partials;      // reduction scratch, one block per aux stream
    size_t partials_stride;
    double* lpartials;     // reduction scratch of the batched norms (layer path)
    size_t lpartials_cap;  // in doubles
    Arena arena;
    cudaGraph_t graph;
    cudaGraphExec_t graph_exec;
    bool graph_live;
};

static void batch_free(qd_batch* b) {
    if (!b) return;
    cudaStreamSynchronize(b->main);
    if (b->work_live) {
        cudaStreamSynchronize(b->work);
        cudaStreamDestroy(b->work);
        cudaEventDestroy(b->in_ev);
        cudaEventDestroy(b->out_ev);
    }
    for (size_t i = 0; i < b->aux.size(); ++i) {
        cudaStreamDestroy(b->aux[i]);
        cudaEventDestroy(b->aux_ev[i]);
    }
    if (b->fork_live) cudaEventDestroy(b->fork_ev);
    if (b->graph_live) {
        cudaGraphExecDestroy(b->graph_exec);
        cudaGraphDestroy(b->graph);
    }
    if (b->states) cudaFree(b->states);
    if (b->norms) cudaFree(b->norms);
    if (b->host_norms) cudaFreeHost(b->host_norms);
    if (b->partials) cudaFree(b->partials);
    if (b->lpartials) cudaFree(b->lpartials);
    b->arena.release();
    delete b;
}

template <typename R>
static qd_status batch_run_impl(qd_batch* b, const qd_circuit* circuits, int32_t n, const qd_batch_opts* opts) {
    using T2 = typename Cplx<R>::T2;
    const size_t ab = sizeof(T2);
    qd_fusion_opts fo{};
    if (opts) fo = opts->fusion;
    FuseCfg cfg = fuse_cfg(opts ? &fo : nullptr, b->prec);
    if (!opts) cfg.mode = QD_FUSE_TILE;
    qd_status rc = check_cfg(cfg, b->prec);
    if (rc != QD_OK) return rc;
    const int64_t small_max = (opts && opts->small_max_amps > 0) ? opts->small_max_amps : (b->prec == QD_C64 ? 8192 : 4096);
    if (small_max > tile_limit(b->prec)) return fail(QD_ERR_UNSUPPORTED, "small-circuit tile above shared memory");
    int nstreams = (opts && opts->n_streams > 0) ? opts->n_streams : 8;
    if (nstreams > 64) nstreams = 64;
    const bool use_graph = opts && opts->use_graph;
    // 0: circuits whose passes are all tile passes go through the layer queue
    // (one launch per pass position for all of them); 1: one program per circuit
    const int path = opts ? opts->path : 0;
    if (path != 0 && path != 1) return fail(QD_ERR_ARG, "unknown batch path %d", path);

    // 1. validate every circuit and lay out the states
    std::vector<Layout> Ls((size_t)n);
    std::vector<std::vector<HGate>> Gs((size_t)n);
    b->psi_off.assign((size_t)n, 0);
    b->D.assign((size_t)n, 0);
    size_t total = 0;
    for (int i = 0; i < n; ++i) {
        const qd_circuit& c = circuits[i];
        rc = make_layout(c.dims, c.n_wires, Ls[i]);
        if (rc == QD_OK) rc = load_gates(Ls[i], b->prec, c.gates, c.n_gates, c.matrices, Gs[i]);
        if (rc != QD_OK) {
            std::string msg = qd_last_error();
            return fail(rc, "circuit %d: %s", i, msg.c_str());
        }
        b->psi_off[i] = total;
        b->D[i] = Ls[i].D;
        total += ((size_t)Ls[i].D * ab + 255) & ~(size_t)255;
    }
    // 2. device buffers (grown when needed)
    QD_CUDA(cudaStreamSynchronize(b->main), "batch sync");
    if (b->graph_live) {
        cudaGraphExecDestroy(b->graph_exec);
        cudaGraphDestroy(b->graph);
        b->graph_live = false;
    }
    if (total > b->states_cap) {
        if (b->states) cudaFree(b->states);
        b->states = nullptr;
        b->states_cap = 0;
        cudaError_t e = cudaMalloc(&b->states, total);
        if (e != cudaSuccess) return fail(QD_ERR_OOM, "batch states (%zu bytes): %s", total, cudaGetErrorString(e));
        b->states_cap = total;
    }
    if ((size_t)n > b->norms_cap) {
        if (b->norms) cudaFree(b->norms);
        if (b->host_norms) cudaFreeHost(b->host_norms);
        b->norms = nullptr;
        b->host_norms = nullptr;
        b->norms_cap = 0;
        const size_t cap = (size_t)n + 16;
        cudaError_t e = cudaMalloc(&b->norms, sizeof(double) * cap);
        if (e == cudaSuccess) e = cudaMallocHost(&b->host_norms, sizeof(double) * cap);
        if (e != cudaSuccess) return fail(QD_ERR_OOM, "batch norms: %s", cudaGetErrorString(e));
        b->norms_cap = cap;
    }
    while ((int)b->aux.size() < nstreams) {
        cudaStream_t s;
        cudaEvent_t e;
        QD_CUDA(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking), "batch stream");
        QD_CUDA(cudaEventCreateWithFlags(&e, cudaEventDisableTiming), "batch event");
        b->aux.push_back(s);
        b->aux_ev.push_back(e);
    }
    if (!b->partials) {
        b->partials_stride = 2 * 1024;
        cudaError_t e = cudaMalloc(&b->partials, sizeof(double) * b->partials_stride * 64);
        if (e != cudaSuccess) return fail(QD_ERR_OOM, "batch reduction scratch: %s", cudaGetErrorString(e));
    }
    // 3. programs: small circuits whole in one CTA; the rest through the planner
    Program prog;
    std::vector<SmallTask> small3, small5;
    uint32_t maxd3 = 1, maxd5 = 1;
    std::vector<Program> big;
    std::vector<int> big_idx;
    std::vector<int> layered;  // circuits on the layer path, and per such circuit its passes' entries
    std::vector<std::vector<LayerEntry<R>>> c_ents;
    std::vector<std::vector<int>> c_dmax;
    std::vector<std::vector<size_t>> c_smem;
    FuseCfg lcfg = cfg;
    lcfg.min_gates = 1;  // a pass of one gate stays a tile pass
    const bool try_layers = path == 0 && cfg.mode == QD_FUSE_TILE;
    for (int i = 0; i < n; ++i) {
        const Layout& L = Ls[i];
        bool fits = L.D <= small_max && (int)Gs[i].size() > 0;
        int dmax = 2;
        for (const HGate& h : Gs[i]) {
            if (!h.fusable) fits = false;
            dmax = h.plan.d > dmax ? h.plan.d : dmax;
        }
        if (fits) {
            SmallTask t{};
            t.psi_off = b->psi_off[i];
            t.D = (uint32_t)L.D;
            t.norm_index = (uint32_t)i;
            t.chunk_off = put_small_chunks<R>(L, Gs[i], cfg, prog, &t.nchunks);
            if (dmax <= 3) {
                small3.push_back(t);
                maxd3 = t.D > maxd3 ? t.D : maxd3;
            } else {
                small5.push_back(t);
                maxd5 = t.D > maxd5 ? t.D : maxd5;
            }
        } else {
            Program pg;
            pg.desc.swap(prog.desc);  // share one descriptor buffer: offsets stay global
            if (try_layers) {
                std::vector<PassPlan> passes;
                plan_passes(L, Gs[i], lcfg, passes);
                std::vector<LayerEntry<R>> ents;
                std::vector<int> dms;
                std::vector<size_t> sms;
                const size_t mark = pg.desc.size();
                if (build_layer_entries<R>(L, b->states + b->psi_off[i], Gs[i], lcfg, passes, pg, ents, dms, sms)) {
                    prog.desc.swap(pg.desc);
                    c_ents.push_back(std::move(ents));
                    c_dmax.push_back(std::move(dms));
                    c_smem.push_back(std::move(sms));
                    layered.push_back(i);
                    continue;
                }
                pg.desc.resize(mark);  // drop the descriptors of the attempt
            }
            build_program<R>(L, b->states + b->psi_off[i], Gs[i], cfg, true, pg);
            prog.desc.swap(pg.desc);
            big.push_back(std::move(pg));
            big_idx.push_back(i);
        }
    }
    // The layer queue: layer k holds pass k of every layered circuit, split
    // by shared memory per CTA (so that a launch's CTAs reside at the
    // occupancy of its own passes) and by the largest wire dimension (the
    // kernel instance); each launch has the prefix of its entries' tile
    // counts.  (Measured: grouping the circuits so that each group's states
    // fit in L2 and running a group's layers back to back was slower, 1.27 s
    // against 0.65 s for the 8192-circuit workload: many small launches.)
    // Per layered circuit a norm / reset record with the prefix of its
    // reduction blocks and of its reset chunks.
    struct LaunchGroup {
        size_t offE, offP;
        int32_t n;
        uint64_t total;
        int dmax;
        size_t smem;
    };
    std::vector<LaunchGroup> groups;
    for (size_t j0 = 0; j0 < layered.size();) {
        const size_t j1 = layered.size();
        size_t nl = 0;
        for (size_t j = j0; j < j1; ++j) nl = std::max(nl, c_ents[j].size());
        for (size_t k = 0; k < nl; ++k) {
            const size_t bounds[6] = {72 * 1024, 110 * 1024, (size_t)1 << 40, 72 * 1024, 110 * 1024, (size_t)1 << 40};
            size_t lo = 0;
            for (int bi = 0; bi < 6; ++bi) {
                const size_t hi = bounds[bi];
                const bool want5 = bi >= 3;  // first the passes of wires up to dimension 3, then up to 5
                if (bi == 3) lo = 0;
                std::vector<LayerEntry<R>> ge;
                std::vector<uint64_t> pre(1, 0);
                int dm = 2;
                size_t sm = 0;
                for (size_t j = j0; j < j1; ++j) {
                    if (k >= c_ents[j].size()) continue;
                    const size_t x = c_smem[j][k];
                    if (x <= lo || x > hi || (c_dmax[j][k] > 3) != want5) continue;
                    ge.push_back(c_ents[j][k]);
                    pre.push_back(pre.back() + c_ents[j][k].ntiles);
                    dm = std::max(dm, c_dmax[j][k]);
                    sm = std::max(sm, x);
                }
                lo = hi;
                if (ge.empty()) continue;
                LaunchGroup g;
                g.offE = prog.put(ge.data(), sizeof(LayerEntry<R>) * ge.size());
                g.offP = prog.put(pre.data(), sizeof(uint64_t) * pre.size());
                g.n = (int32_t)ge.size();
                g.total = pre.back();
                g.dmax = dm;
                g.smem = sm;
                groups.push_back(g);
            }
        }
        j0 = j1;
    }
    size_t offN = 0, offNB = 0, offNC = 0;
    uint64_t nblocks_total = 0, nchunks_total = 0;
    if (!layered.empty()) {
        std::vector<NormEntry> ne(layered.size());
        std::vector<uint64_t> pb(layered.size() + 1, 0), pc(layered.size() + 1, 0);
        for (size_t j = 0; j < layered.size(); ++j) {
            const int i = layered[j];
            NormEntry& e = ne[j];
            std::memset(&e, 0, sizeof e);
            e.psi = b->states + b->psi_off[i];
            e.D = b->D[i];
            e.nb = (uint32_t)reduce_blocks(b->D[i]);
            e.a16 = 1;  // states are 256-byte aligned
            e.part_off = pb[j];
            e.out_index = (uint32_t)i;
            pb[j + 1] = pb[j] + e.nb;
            pc[j + 1] = pc[j] + (uint64_t)((b->D[i] + kBasisChunkAmps - 1) / kBasisChunkAmps);
        }
        nblocks_total = pb.back();
        nchunks_total = pc.back();
        offN = prog.put(ne.data(), sizeof(NormEntry) * ne.size());
        offNB = prog.put(pb.data(), sizeof(uint64_t) * pb.size());
        offNC = prog.put(pc.data(), sizeof(uint64_t) * pc.size());
        if (2 * nblocks_total > b->lpartials_cap) {
            if (b->lpartials) cudaFree(b->lpartials);
            b->lpartials = nullptr;
            b->lpartials_cap = 0;
            cudaError_t e = cudaMalloc(&b->lpartials, sizeof(double) * 2 * nblocks_total);
            if (e != cudaSuccess) return fail(QD_ERR_OOM, "batch norm scratch: %s", cudaGetErrorString(e));
            b->lpartials_cap = 2 * nblocks_total;
        }
    }
    const size_t off3 = small3.empty() ? 0 : prog.put(small3.data(), sizeof(SmallTask) * small3.size());
    const size_t off5 = small5.empty() ? 0 : prog.put(small5.data(), sizeof(SmallTask) * small5.size());
    rc = b->arena.upload(prog.desc.data(), prog.desc.size(), b->main);
    if (rc != QD_OK) return rc;
    const char* base = static_cast<const char*>(b->arena.dev);

    // 4. issue on the private work stream: small circuits first, the others
    //    round-robin on the auxiliary streams, joined back at the end.  The
    //    work stream follows the caller's stream and the caller's stream
    //    follows it; with use_graph the work stream is captured and the
    //    graph is launched on the caller's stream instead.
    if (!b->work_live) {
        QD_CUDA(cudaStreamCreateWithFlags(&b->work, cudaStreamNonBlocking), "batch work stream");
        QD_CUDA(cudaEventCreateWithFlags(&b->in_ev, cudaEventDisableTiming), "batch event");
        QD_CUDA(cudaEventCreateWithFlags(&b->out_ev, cudaEventDisableTiming), "batch event");
        b->work_live = true;
    }
    if (!b->fork_live) {
        QD_CUDA(cudaEventCreateWithFlags(&b->fork_ev, cudaEventDisableTiming), "fork event");
        b->fork_live = true;
    }
    // the descriptor upload was issued on the caller's stream
    QD_CUDA(cudaEventRecord(b->in_ev, b->main), "batch order");
    QD_CUDA(cudaStreamWaitEvent(b->work, b->in_ev, 0), "batch order");
    if (use_graph) {
        QD_CUDA(cudaStreamSynchronize(b->work), "batch pre-capture sync");
        QD_CUDA(cudaStreamBeginCapture(b->work, cudaStreamCaptureModeRelaxed), "graph capture");
    }
    cudaStream_t ws = b->work;
    QD_CUDA(cudaEventRecord(b->fork_ev, ws), "fork record");
    for (int k = 0; k < nstreams; ++k) QD_CUDA(cudaStreamWaitEvent(b->aux[k], b->fork_ev, 0), "fork wait");
    cudaError_t e = launch_batch_small<R>(reinterpret_cast<const SmallTask*>(base + off3), (int)small3.size(), 3,
                                          maxd3, b->states, base, b->norms, ws);
    if (e == cudaSuccess)
        e = launch_batch_small<R>(reinterpret_cast<const SmallTask*>(base + off5), (int)small5.size(), 5, maxd5,
                                  b->states, base, b->norms, ws);
    if (e == cudaSuccess && !layered.empty()) {
        const NormEntry* ne = reinterpret_cast<const NormEntry*>(base + offN);
        e = launch_basis_batch<R>(ne, reinterpret_cast<const uint64_t*>(base + offNC), (int32_t)layered.size(),
                                  nchunks_total, ws);
        for (size_t k = 0; k < groups.size() && e == cudaSuccess; ++k) {
            NvtxRange r("batch layer group");
            const LaunchGroup& g = groups[k];
            e = launch_fused_layer<R>(reinterpret_cast<const LayerEntry<R>*>(base + g.offE),
                                      reinterpret_cast<const uint64_t*>(base + g.offP), g.n, g.total, base, g.dmax,
                                      g.smem, ws);
        }
        if (e == cudaSuccess)
            e = launch_norm_batch<R>(ne, reinterpret_cast<const uint64_t*>(base + offNB), (int32_t)layered.size(),
                                     nblocks_total, b->lpartials, b->norms, ws);
    }
    if (e != cudaSuccess) {
        if (use_graph) {
            cudaGraph_t g;
            if (cudaStreamEndCapture(ws, &g) == cudaSuccess && g) cudaGraphDestroy(g);
        }
        return cuda_fail(e, "small-circuit batch kernel");
    }
    for (size_t j = 0; j < big.size(); ++j) {
        const int k = (int)(j % (size_t)nstreams);
        const int i = big_idx[j];
        rc = issue(big[j], base, b->aux[k]);
        if (rc == QD_OK) {
            const int nb = reduce_blocks(b->D[i]);
            e = launch_norm<R>(b->states + b->psi_off[i], b->D[i], b->partials + b->partials_stride * k, nb,
                               b->norms + i, b->aux[k]);
            if (e != cudaSuccess) rc = cuda_fail(e, "batch norm");
        }
        if (rc != QD_OK) {
            if (use_graph) {
                cudaGraph_t g;
                if (cudaStreamEndCapture(ws, &g) == cudaSuccess && g) cudaGraphDestroy(g);
            }
            return rc;
        }
    }
    for (int k = 0; k < nstreams; ++k) {
        QD_CUDA(cudaEventRecord(b->aux_ev[k], b->aux[k]), "join record");
        QD_CUDA(cudaStreamWaitEvent(ws, b->aux_ev[k], 0), "join wait");
    }
    if (use_graph) {
        QD_CUDA(cudaStreamEndCapture(ws, &b->graph), "graph end capture");
        QD_CUDA(cudaGraphInstantiate(&b->graph_exec, b->graph, 0), "graph instantiate");
        b->graph_live = true;
        QD_CUDA(cudaGraphLaunch(b->graph_exec, b->main), "graph launch");
    } else {
        QD_CUDA(cudaEventRecord(b->out_ev, ws), "batch order");
        QD_CUDA(cudaStreamWaitEvent(b->main, b->out_ev, 0), "batch order");
    }
    return QD_OK;
}

extern "C" {

qd_status qd_apply_circuit(qd_state* st, const qd_gate_desc* gates, int32_t n_gates, const double* matrices,
                           const qd_fusion_opts* opts) {
    NvtxRange nvtx_("qd_apply_circuit");
    if (!st) return fail(QD_ERR_ARG, "state is NULL");
    qd_status rc = flush_pending(st);
    if (rc == QD_OK) rc = materialize(st);
    if (rc != QD_OK) return rc;
    return run_circuit(st, gates, n_gates, matrices, opts);
}

}  // extern "C"

// The last circuit of qd_apply_circuit on a state.  Its key holds
// everything the built program depends on besides the state itself (fusion
// settings, every gate's wires, controls and matrix), compared byte for
// byte.  A key seen for the second time in a row is built whole -- plan,
// composed blocks, descriptors -- and its descriptors stay on the device;
// from then on the same circuit only launches.
struct qd::CircuitCache {
    std::vector<char> key;
    bool seen = false, built = false;
    // the last whole-state block plan and its structure key (settings,
    // every gate's wires, controls and diagonal flag; no matrix values):
    // the plan depends on nothing else
    std::vector<char> skey;
    std::vector<PassPlan> splan;
    Program prog;
    void* dev = nullptr;   // descriptors of prog
    void* host = nullptr;  // pinned copy they were uploaded from
    size_t cap = 0;
    cudaEvent_t done{};    // after the last launch of prog
    bool ev_live = false;
};

void qd::circuit_cache_free(CircuitCache* c) {
    if (!c) return;
    if (c->ev_live) {
        cudaEventSynchronize(c->done);
        cudaEventDestroy(c->done);
    }
    if (c->dev) cudaFree(c->dev);
    if (c->host) cudaFreeHost(c->host);
    delete c;
}

static void circuit_key(const FuseCfg& cfg, const std::vector<HGate>& G, std::vector<char>& key) {
    key.clear();
    auto put = [&](const void* p, size_t n) {
        const char* c = static_cast<const char*>(p);
        key.insert(key.end(), c, c + n);
    };
    put(&cfg, sizeof cfg);
    const size_t n = G.size();
    put(&n, sizeof n);
    for (const HGate& h : G) {
        put(&h.k, sizeof h.k);
        put(&h.nc, sizeof h.nc);
        put(h.wires, sizeof(int) * (size_t)h.k);
        put(h.cw, sizeof(int) * (size_t)h.nc);
        put(h.cv, sizeof(int) * (size_t)h.nc);
        put(h.U, sizeof(double) * 2 * (size_t)h.P * (size_t)h.P);
    }
}

// The pass plan of G; QD_FUSE_BLOCK plans are kept per structure, so a
// circuit that differs from the last one only in its matrices is not
// planned again.
static void plan_cached(const qd_state* st, CircuitCache& c, const std::vector<HGate>& G, const FuseCfg& cfg,
                        std::vector<PassPlan>& passes) {
    if (cfg.mode != QD_FUSE_BLOCK) {
        plan_passes(st->L, G, cfg, passes);
        return;
    }
    std::vector<char> key;
    auto put = [&](const void* p, size_t n) {
        const char* b = static_cast<const char*>(p);
        key.insert(key.end(), b, b + n);
    };
    put(&cfg, sizeof cfg);
    const size_t n = G.size();
    put(&n, sizeof n);
    for (const HGate& h : G) {
        put(&h.k, sizeof h.k);
        put(&h.nc, sizeof h.nc);
        put(h.wires, sizeof(int) * (size_t)h.k);
        put(h.cw, sizeof(int) * (size_t)h.nc);
        put(h.cv, sizeof(int) * (size_t)h.nc);
        const char d = h.diag ? 1 : 0;
        put(&d, 1);
    }
    if (!c.skey.empty() && key == c.skey) {
        passes = c.splan;
        return;
    }
    plan_passes(st->L, G, cfg, passes);
    c.skey.swap(key);
    c.splan = passes;
}

// Build the whole circuit as one program, upload its descriptors to the
// cache's own device buffer (after the previous program's launches have
// finished with it) and mark it built.
static qd_status cache_build(qd_state* st, CircuitCache& c, const std::vector<HGate>& G, const FuseCfg& cfg) {
    Program prog;
    std::vector<PassPlan> passes;
    plan_cached(st, c, G, cfg, passes);
    if (st->prec == QD_C64)
        build_passes<float>(st->L, st->psi, G, cfg, passes, 0, passes.size(), prog);
    else
        build_passes<double>(st->L, st->psi, G, cfg, passes, 0, passes.size(), prog);
    if (c.ev_live) QD_CUDA(cudaEventSynchronize(c.done), "circuit cache reuse");
    const size_t n = prog.desc.size() > 0 ? prog.desc.size() : 16;
    if (n > c.cap) {
        if (c.dev) cudaFree(c.dev);
        if (c.host) cudaFreeHost(c.host);
        c.dev = c.host = nullptr;
        c.cap = 0;
        cudaError_t e = cudaMalloc(&c.dev, n);
        if (e == cudaSuccess) e = cudaMallocHost(&c.host, n);
        if (e != cudaSuccess) return fail(QD_ERR_OOM, "circuit cache (%zu bytes): %s", n, cudaGetErrorString(e));
        c.cap = n;
    }
    if (!prog.desc.empty()) {
        std::memcpy(c.host, prog.desc.data(), prog.desc.size());
        QD_CUDA(cudaMemcpyAsync(c.dev, c.host, prog.desc.size(), cudaMemcpyHostToDevice, st->stream),
                "circuit cache upload");
        count_upload(prog.desc.size());
    }
    if (!c.ev_live) {
        QD_CUDA(cudaEventCreateWithFlags(&c.done, cudaEventDisableTiming), "circuit cache event");
        c.ev_live = true;
    }
    c.prog = std::move(prog);
    c.built = true;
    return QD_OK;
}

qd_status qd::run_circuit(qd_state* st, const qd_gate_desc* gates, int32_t n_gates, const double* matrices,
                          const qd_fusion_opts* opts) {
    try {
        if (!st) return fail(QD_ERR_ARG, "state is NULL");
        std::vector<HGate> G;
        qd_status rc = load_gates(st->L, st->prec, gates, n_gates, matrices, G);
        if (rc != QD_OK) return rc;
        const FuseCfg cfg = fuse_cfg(opts, st->prec);
        rc = check_cfg(cfg, st->prec);
        if (rc != QD_OK) return rc;
        if (!st->ccache) st->ccache = new CircuitCache;
        CircuitCache& cc = *st->ccache;
        std::vector<char> key;
        circuit_key(cfg, G, key);
        if (cc.seen && key == cc.key) {
            if (!cc.built) {
                rc = cache_build(st, cc, G, cfg);
                if (rc != QD_OK) return rc;
            }
            rc = issue(cc.prog, static_cast<const char*>(cc.dev), st->stream);
            if (rc != QD_OK) return rc;
            QD_CUDA(cudaEventRecord(cc.done, st->stream), "circuit cache event");
            return QD_OK;
        }
        cc.key.swap(key);
        cc.seen = true;
        cc.built = false;
        // Build, upload and launch the passes in segments of 1, 2, 4, ...
        // passes: the host composes the next segment while the GPU runs the
        // previous one.  Two descriptor arenas alternate, so an upload only
        // waits for the copy two segments back.
        std::vector<PassPlan> passes;
        plan_cached(st, cc, G, cfg, passes);
        if (!st->arena) st->arena = new Arena[2];
        size_t i = 0;
        for (int seg = 0; i < passes.size(); ++seg) {
            const size_t n = std::min(passes.size() - i, (size_t)1 << (seg < 16 ? seg : 16));
            Program prog;
            if (st->prec == QD_C64)
                build_passes<float>(st->L, st->psi, G, cfg, passes, i, i + n, prog);
            else
                build_passes<double>(st->L, st->psi, G, cfg, passes, i, i + n, prog);
            i += n;
            if (prog.ops.empty()) continue;
            Arena& ar = st->arena[seg & 1];
            rc = ar.upload(prog.desc.data(), prog.desc.size(), st->stream);
            if (rc != QD_OK) return rc;
            rc = issue(prog, static_cast<const char*>(ar.dev), st->stream);
            if (rc != QD_OK) return rc;
        }
        return QD_OK;
    } catch (...) {
        return fail(QD_ERR_OOM, "host exception in qd_apply_circuit");
    }
}

extern "C" {

qd_status qd_plan_circuit(const int32_t* dims, int32_t n, int32_t prec, const qd_gate_desc* gates, int32_t n_gates,
                          const double* matrices, const qd_fusion_opts* opts, int32_t* exec_order, int32_t* pass_of,
                          int64_t* pass_tile_amps, double* pass_flops, int32_t* n_passes) {
    try {
        if (!exec_order || !pass_of || !n_passes) return fail(QD_ERR_ARG, "output array is NULL");
        Layout L;
        qd_status rc = make_layout(dims, n, L);
        if (rc != QD_OK) return rc;
        std::vector<HGate> G;
        rc = load_gates(L, prec, gates, n_gates, matrices, G);
        if (rc != QD_OK) return rc;
        const FuseCfg cfg = fuse_cfg(opts, prec);
        std::vector<PassPlan> passes;
        plan_passes(L, G, cfg, passes);
        int pos = 0;
        for (size_t p = 0; p < passes.size(); ++p) {
            for (int idx : passes[p].gates) {
                exec_order[pos] = idx;
                pass_of[pos] = (int32_t)p;
                ++pos;
            }
            if (pass_tile_amps) pass_tile_amps[p] = passes[p].tile ? passes[p].T : 0;
            if (pass_flops) pass_flops[p] = pass_arith(L, G, cfg, passes[p]);
        }
        *n_passes = (int32_t)passes.size();
        return QD_OK;
    } catch (...) {
        return fail(QD_ERR_OOM, "host exception in qd_plan_circuit");
    }
}

qd_status qd_batch_create(int32_t prec, void* stream, qd_batch** out) {
    if (!out) return fail(QD_ERR_ARG, "out is NULL");
    if (prec != QD_C64 && prec != QD_C128) return fail(QD_ERR_ARG, "unknown precision %d", prec);
    qd_batch* b = new (std::nothrow) qd_batch();
    if (!b) return fail(QD_ERR_OOM, "host allocation failed");
    b->prec = prec;
    b->main = reinterpret_cast<cudaStream_t>(stream);
    b->work_live = false;
    b->fork_live = false;
    b->states = nullptr;
    b->states_cap = 0;
    b->norms = nullptr;
    b->host_norms = nullptr;
    b->norms_cap = 0;
    b->partials = nullptr;
    b->partials_stride = 0;
    b->graph_live = false;
    *out = b;
    return QD_OK;
}

qd_status qd_batch_run(qd_batch* b, const qd_circuit* circuits, int32_t n, const qd_batch_opts* opts) {
    NvtxRange nvtx_("qd_batch_run");
    try {
        if (!b) return fail(QD_ERR_ARG, "batch is NULL");
        if (n < 0 || (n > 0 && !circuits)) return fail(QD_ERR_ARG, "bad circuit list");
        return b->prec == QD_C64 ? batch_run_impl<float>(b, circuits, n, opts)
                                 : batch_run_impl<double>(b, circuits, n, opts);
    } catch (...) {
        return fail(QD_ERR_OOM, "host exception in qd_batch_run");
    }
}

qd_status qd_batch_relaunch(qd_batch* b) {
    if (!b) return fail(QD_ERR_ARG, "batch is NULL");
    if (!b->graph_live) return fail(QD_ERR_ARG, "the last qd_batch_run was not captured in a graph");
    QD_CUDA(cudaGraphLaunch(b->graph_exec, b->main), "graph launch");
    return QD_OK;
}

qd_status qd_batch_state(qd_batch* b, int32_t i, void** dev_ptr, int64_t* num_amplitudes) {
    if (!b || !dev_ptr) return fail(QD_ERR_ARG, "batch or out is NULL");
    if (i < 0 || (size_t)i >= b->D.size()) return fail(QD_ERR_ARG, "circuit index %d out of range", i);
    *dev_ptr = b->states + b->psi_off[i];
    if (num_amplitudes) *num_amplitudes = b->D[i];
    return QD_OK;
}

qd_status qd_batch_get_amplitudes(qd_batch* b, int32_t i, double* host) {
    if (!b || !host) return fail(QD_ERR_ARG, "batch or out is NULL");
    if (i < 0 || (size_t)i >= b->D.size()) return fail(QD_ERR_ARG, "circuit index %d out of range", i);
    const size_t D = (size_t)b->D[i];
    const char* src = b->states + b->psi_off[i];
    if (b->prec == QD_C128) {
        QD_CUDA(cudaMemcpyAsync(host, src, D * 16, cudaMemcpyDeviceToHost, b->main), "batch download");
        QD_CUDA(cudaStreamSynchronize(b->main), "batch download sync");
    } else {
        // binary32 pairs into the upper half of the caller's buffer, widened front to back
        float* raw = reinterpret_cast<float*>(reinterpret_cast<char*>(host) + D * 8);
        QD_CUDA(cudaMemcpyAsync(raw, src, D * 8, cudaMemcpyDeviceToHost, b->main), "batch download");
        QD_CUDA(cudaStreamSynchronize(b->main), "batch download sync");
        for (size_t e = 0; e < 2 * D; ++e) host[e] = (double)raw[e];
    }
    return QD_OK;
}

qd_status qd_batch_norms(qd_batch* b, double* host_out) {
    if (!b || !host_out) return fail(QD_ERR_ARG, "batch or out is NULL");
    const size_t n = b->D.size();
    if (n == 0) return QD_OK;
    QD_CUDA(cudaMemcpyAsync(b->host_norms, b->norms, sizeof(double) * n, cudaMemcpyDeviceToHost, b->main),
            "norm copy");
    QD_CUDA(cudaStreamSynchronize(b->main), "norm sync");
    std::memcpy(host_out, b->host_norms, sizeof(double) * n);
    return QD_OK;
}

qd_status qd_batch_synchronize(qd_batch* b) {
    if (!b) return fail(QD_ERR_ARG, "batch is NULL");
    QD_CUDA(cudaStreamSynchronize(b->main), "batch synchronize");
    return QD_OK;
}

qd_status qd_batch_destroy(qd_batch* b) {
    batch_free(b);
    return QD_OK;
}

}  // extern "C"
