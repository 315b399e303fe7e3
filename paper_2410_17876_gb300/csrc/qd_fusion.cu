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
#include <string>
#include <vector>

#include "qd_internal.cuh"
#include "qd_runtime.h"

namespace qd {

// ---------------------------------------------------------------------------
// 32-bit division by invariant integers (same method as FastDiv, N = 32).
// ---------------------------------------------------------------------------
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

constexpr int kMaxFusedD = 5;      // single-wire gates up to this dimension join fused passes
constexpr int kMaxTileCtrl = 7;    // controls of a fused gate (inside or outside the tile)
constexpr int kMaxLocalIns = 1 + kMaxTileCtrl;
constexpr int kMaxPassGates = 64;  // gates per fused pass (their descriptors live in shared memory)
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

// One gate of a pass.  Built on the host, copied to shared memory by every CTA.
template <typename R>
struct __align__(16) FGate {
    using T2 = typename Cplx<R>::T2;
    T2 U[kMaxFusedD * kMaxFusedD];
    LocalMap map;
    uint32_t nclasses;  // classes in a tile
    uint32_t lst;       // local stride of the target
    uint32_t step;      // lst * d (class base step when the target is the only inserted wire)
    uint32_t pad_;
    uint8_t d, kind, lmask, smask, pure, n_out, pad2_[2];
    uint8_t perm[8];
    uint8_t out_w[kMaxTileCtrl + 1];  // controls outside S: global wire, value
    uint8_t out_v[kMaxTileCtrl + 1];
};

template <typename R>
struct FusedArgs {
    using T2 = typename Cplx<R>::T2;
    T2* psi;
    const FGate<R>* gates;
    int32_t ngates;
    uint32_t T;      // tile amplitudes
    uint32_t bL;     // contiguous run (row) length
    uint32_t rows;   // rows per tile
    int32_t vec2;    // complex64 with even rows: 16-byte accesses
    FastDiv32 bLdiv;
    uint64_t ntiles;
    int32_t nfree;   // wires outside S, ascending
    int32_t free_w[kMaxWires];
    uint32_t free_d[kMaxWires];
    uint64_t free_b[kMaxWires];
    const uint64_t* rowoff;  // device, rows entries: offset of each row from the tile base
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

// Small fixed-size arrays passed by value, so that they stay in registers.
template <typename T, int N>
struct Arr {
    T v[N];
};

// y = G x for one class held in registers (dense, diagonal or permutation).
template <typename T2, int DT>
__device__ __forceinline__ Arr<T2, DT> class_math(const Arr<T2, DT> x, int kind, bool pure, const Arr<int, DT> perm,
                                                  const Arr<T2, DT * DT> u) {
    Arr<T2, DT> y;
    if (kind == kDense) {
#pragma unroll
        for (int r = 0; r < DT; ++r) {
            T2 acc = fcmul(u.v[r * DT], x.v[0]);
#pragma unroll
            for (int k = 1; k < DT; ++k) fcmac(acc, u.v[r * DT + k], x.v[k]);
            y.v[r] = acc;
        }
    } else if (kind == kDiag) {
#pragma unroll
        for (int r = 0; r < DT; ++r) y.v[r] = fcmul(u.v[r * DT + r], x.v[r]);
    } else {
#pragma unroll
        for (int r = 0; r < DT; ++r) {
            T2 v = x.v[0], w = u.v[r * DT];
#pragma unroll
            for (int k = 1; k < DT; ++k)
                if (perm.v[r] == k) {
                    v = x.v[k];
                    w = u.v[r * DT + k];
                }
            y.v[r] = pure ? v : fcmul(w, v);
        }
    }
    return y;
}

// Apply one single-wire gate of dimension DT to the tile in shared memory.
// Matrix, permutation and masks are loop invariants read once per gate from
// the shared-memory descriptor.  With no control inside the tile (m == 1) a
// class index c = hi * lst + lo has base hi * lst * d + lo (one division);
// complex64 with an even local stride processes two adjacent classes with
// 16-byte accesses.
template <typename R, int DT>
__device__ __forceinline__ void tile_gate(typename Cplx<R>::T2* tile, const FGate<R>& G) {
    using T2 = typename Cplx<R>::T2;
    const int kind = G.kind;
    const uint32_t lmask = G.lmask, smask = G.smask, lst = G.lst, nc = G.nclasses;
    const bool pure = G.pure != 0;
    Arr<int, DT> perm;
#pragma unroll
    for (int r = 0; r < DT; ++r) perm.v[r] = G.perm[r];
    Arr<T2, DT * DT> u;
#pragma unroll
    for (int i = 0; i < DT * DT; ++i) u.v[i] = G.U[i];
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
                    const Arr<T2, DT> y0 = class_math<T2, DT>(x0, kind, pure, perm, u);
                    const Arr<T2, DT> y1 = class_math<T2, DT>(x1, kind, pure, perm, u);
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
                    const Arr<T2, DT> y = class_math<T2, DT>(x, kind, pure, perm, u);
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
            const Arr<T2, DT> y = class_math<T2, DT>(x, kind, pure, perm, u);
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
            const Arr<T2, DT> y = class_math<T2, DT>(x, kind, pure, perm, u);
#pragma unroll
            for (int r = 0; r < DT; ++r)
                if (smask >> r & 1u) tile[b + r * lst] = y.v[r];
        }
    }
}

// Shared memory of a CTA: [pass descriptors][row offsets][tile], each 16-byte aligned.
template <typename R>
__host__ __device__ inline size_t fused_desc_bytes(int ngates) {
    return sizeof(FGate<R>) * (size_t)ngates;
}
__host__ __device__ inline size_t fused_rows_bytes(uint32_t rows) { return ((size_t)rows * 8 + 15) & ~(size_t)15; }

template <typename R, int DMAX>
__global__ void __launch_bounds__(256, 2) k_fused_tile(const __grid_constant__ FusedArgs<R> a) {
    using T2 = typename Cplx<R>::T2;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    FGate<R>* sg = reinterpret_cast<FGate<R>*>(smem_raw);
    uint64_t* srow = reinterpret_cast<uint64_t*>(smem_raw + fused_desc_bytes<R>(a.ngates));
    T2* tile = reinterpret_cast<T2*>(smem_raw + fused_desc_bytes<R>(a.ngates) + fused_rows_bytes(a.rows));
    __shared__ int32_t odig[kMaxWires];
    __shared__ uint64_t sbase;
    {
        const uint4* src = reinterpret_cast<const uint4*>(a.gates);
        uint4* dst = reinterpret_cast<uint4*>(sg);
        const uint32_t n16 = (uint32_t)(fused_desc_bytes<R>(a.ngates) / 16);
        for (uint32_t i = threadIdx.x; i < n16; i += blockDim.x) dst[i] = src[i];
    }
    for (uint32_t r = threadIdx.x; r < a.rows; r += blockDim.x) srow[r] = a.rowoff[r];
    if (threadIdx.x == 0) {
        uint64_t rem = blockIdx.x, base = 0;
        for (int i = 0; i < a.nfree; ++i) {
            const uint64_t q = rem / a.free_d[i];
            const uint32_t dig = (uint32_t)(rem - q * a.free_d[i]);
            odig[a.free_w[i]] = (int32_t)dig;
            base += (uint64_t)dig * a.free_b[i];
            rem = q;
        }
        sbase = base;
    }
    __syncthreads();
    T2* g = a.psi + sbase;
    if (a.vec2) {
        for (uint32_t e = 2 * threadIdx.x; e < a.T; e += 2 * blockDim.x) {
            const uint32_t r = a.bLdiv.div(e);
            reinterpret_cast<float4*>(tile)[e >> 1] =
                *reinterpret_cast<const float4*>(reinterpret_cast<const float2*>(g) + srow[r] + (e - r * a.bL));
        }
    } else {
        for (uint32_t e = threadIdx.x; e < a.T; e += blockDim.x) {
            const uint32_t r = a.bLdiv.div(e);
            tile[e] = g[srow[r] + (e - r * a.bL)];
        }
    }
    __syncthreads();
    for (int gi = 0; gi < a.ngates; ++gi) {
        const FGate<R>& G = sg[gi];
        bool ok = true;
        for (int c = 0; c < G.n_out; ++c) ok = ok && (odig[G.out_w[c]] == (int32_t)G.out_v[c]);
        if (!ok) continue;  // uniform across the CTA
        if (G.d == 2) tile_gate<R, 2>(tile, G);
        else if (DMAX == 3 || G.d == 3) tile_gate<R, 3>(tile, G);
        else if (G.d == 4) tile_gate<R, (DMAX > 3 ? 4 : 3)>(tile, G);
        else tile_gate<R, DMAX>(tile, G);
        __syncthreads();
    }
    if (a.vec2) {
        for (uint32_t e = 2 * threadIdx.x; e < a.T; e += 2 * blockDim.x) {
            const uint32_t r = a.bLdiv.div(e);
            *reinterpret_cast<float4*>(reinterpret_cast<float2*>(g) + srow[r] + (e - r * a.bL)) =
                reinterpret_cast<const float4*>(tile)[e >> 1];
        }
    } else {
        for (uint32_t e = threadIdx.x; e < a.T; e += blockDim.x) {
            const uint32_t r = a.bLdiv.div(e);
            g[srow[r] + (e - r * a.bL)] = tile[e];
        }
    }
}

template <typename R>
size_t fused_smem(const FusedArgs<R>& a) {
    return fused_desc_bytes<R>(a.ngates) + fused_rows_bytes(a.rows) + sizeof(typename Cplx<R>::T2) * (size_t)a.T;
}

// dmax: largest wire dimension among the pass's gates (selects the kernel
// instance, so passes of qubits and qutrits do not pay for d = 5 registers).
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

}  // namespace

// ---------------------------------------------------------------------------
// Planner
// ---------------------------------------------------------------------------
struct HGate {
    int k, nc, P;
    int wires[QD_MAX_GATE_WIRES];
    int cw[QD_MAX_CONTROLS], cv[QD_MAX_CONTROLS];
    const double* U;
    Plan plan;
    bool diag, fusable;
    uint64_t tmask, cmask;
};

struct PassPlan {
    bool tile;
    std::vector<int> gates;
    uint64_t smask;   // cached wires
    int64_t T;
};

struct FuseCfg {
    int mode;
    int64_t Tmax;
    int min_gates;
    int64_t min_row;
};

// Largest tile that fits the shared memory of one CTA (tile + row table).
static int64_t tile_limit(int32_t prec) { return prec == QD_C64 ? 16384 : 8192; }

static FuseCfg fuse_cfg(const qd_fusion_opts* o, int32_t prec) {
    FuseCfg c;
    c.mode = o ? o->mode : QD_FUSE_OFF;
    c.Tmax = (o && o->max_tile_amps > 0) ? o->max_tile_amps : (prec == QD_C64 ? 8192 : 4096);
    c.min_gates = (o && o->min_gates > 0) ? o->min_gates : 2;
    c.min_row = (o && o->min_row > 0) ? o->min_row : (prec == QD_C64 ? 16 : 8);
    // rows per tile are bounded by the row table
    const int64_t need = (c.Tmax + kMaxRows - 1) / kMaxRows;
    if (c.min_row < need) c.min_row = need;
    return c;
}

static qd_status load_gates(const Layout& L, int32_t prec, const qd_gate_desc* gates, int32_t n,
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
static void plan_passes(const Layout& L, const std::vector<HGate>& G, const FuseCfg& cfg,
                        std::vector<PassPlan>& passes) {
    passes.clear();
    const int n = (int)G.size();
    std::vector<int> rem(n);
    for (int i = 0; i < n; ++i) rem[i] = i;
    int L0 = 0;
    while (L0 < L.n && L.b[L0] < cfg.min_row) ++L0;
    const int64_t T0 = L.b[L0];
    const bool can_tile = cfg.mode == QD_FUSE_TILE && T0 <= cfg.Tmax;
    uint64_t low = 0;
    for (int w = 0; w < L0; ++w) low |= 1ull << w;
    std::vector<char> taken(n, 0);
    while (!rem.empty()) {
        if (can_tile) {
            uint64_t S = low, BW = 0, BR = 0;
            int64_t T = T0;
            std::vector<int> sched;
            for (int idx : rem) {
                const HGate& g = G[idx];
                const uint64_t W = g.diag ? 0 : g.tmask;
                const uint64_t Rd = g.cmask | (g.diag ? g.tmask : 0);
                const bool blocked = (W & (BW | BR)) || (Rd & BW);
                bool ok = !blocked && g.fusable && (int)sched.size() < kMaxPassGates;
                if (ok) {
                    const uint64_t need = g.tmask & ~S;
                    int64_t T2 = T;
                    for (int w = 0; w < L.n; ++w)
                        if (need >> w & 1) T2 *= L.dims[w];
                    if (T2 <= cfg.Tmax) {
                        S |= need;
                        T = T2;
                        sched.push_back(idx);
                        continue;
                    }
                }
                BW |= W;
                BR |= Rd;
            }
            if ((int)sched.size() >= cfg.min_gates) {
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

static void tile_geometry(const Layout& L, uint64_t S, int64_t min_row, TileGeom& g) {
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
    int L0 = 0;
    while (L0 < L.n && L.b[L0] < min_row) ++L0;
    g.L0 = L0;
    g.bL = (uint32_t)L.b[L0];
    g.R = (uint32_t)(g.local.D / (int64_t)g.bL);
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


template <typename R>
static void build_fgate(const TileGeom& geo, const HGate& h, FGate<R>& f) {
    std::memset(static_cast<void*>(&f), 0, sizeof f);
    const Plan& p = h.plan;
    f.d = (uint8_t)p.d;
    f.kind = (uint8_t)p.kind;
    f.lmask = (uint8_t)p.lmask;
    f.smask = (uint8_t)p.smask;
    f.pure = p.pure ? 1 : 0;
    for (int r = 0; r < 8; ++r) f.perm[r] = (uint8_t)(r < kMaxSmallD ? p.perm[r] : 0);
    for (int i = 0; i < p.d * p.d; ++i) {
        f.U[i].x = (R)h.U[2 * i];
        f.U[i].y = (R)h.U[2 * i + 1];
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

template <typename R>
static qd_status run_circuit_impl(qd_state* st, std::vector<HGate>& G, const FuseCfg& cfg) {
    std::vector<PassPlan> passes;
    plan_passes(st->L, G, cfg, passes);
    // descriptors of all tile passes of this call, uploaded once
    size_t bytes = 0;
    for (const PassPlan& p : passes)
        if (p.tile) {
            bytes += sizeof(FGate<R>) * p.gates.size();
            bytes = (bytes + 255) & ~(size_t)255;
            bytes += sizeof(uint64_t) * kMaxRows;
            bytes = (bytes + 255) & ~(size_t)255;
        }
    if (bytes > 0) {
        if (bytes > st->fuse_bytes) {
            QD_CUDA(cudaStreamSynchronize(st->stream), "fusion arena resize");
            if (st->fuse_dev) cudaFree(st->fuse_dev);
            if (st->fuse_host) cudaFreeHost(st->fuse_host);
            st->fuse_dev = st->fuse_host = nullptr;
            st->fuse_bytes = 0;
            size_t cap = bytes + bytes / 2;
            cudaError_t e = cudaMalloc(&st->fuse_dev, cap);
            if (e != cudaSuccess) return fail(QD_ERR_OOM, "fusion arena: %s", cudaGetErrorString(e));
            e = cudaMallocHost(&st->fuse_host, cap);
            if (e != cudaSuccess) return fail(QD_ERR_OOM, "pinned fusion arena: %s", cudaGetErrorString(e));
            st->fuse_bytes = cap;
            if (!st->fuse_ev_live) {
                QD_CUDA(cudaEventCreateWithFlags(&st->fuse_ev, cudaEventDisableTiming), "cudaEventCreate");
                st->fuse_ev_live = true;
            }
        } else if (st->fuse_ev_live) {
            QD_CUDA(cudaEventSynchronize(st->fuse_ev), "fusion staging wait");
        }
    }
    // fill the staging buffer
    struct Launch {
        FusedArgs<R> a;
        int dmax;
    };
    std::vector<Launch> launches;
    size_t off = 0;
    char* hb = static_cast<char*>(st->fuse_host);
    char* db = static_cast<char*>(st->fuse_dev);
    for (const PassPlan& p : passes) {
        if (!p.tile) continue;
        TileGeom geo;
        tile_geometry(st->L, p.smask, cfg.min_row, geo);
        FGate<R>* hg = reinterpret_cast<FGate<R>*>(hb + off);
        const FGate<R>* dg = reinterpret_cast<const FGate<R>*>(db + off);
        for (size_t i = 0; i < p.gates.size(); ++i) build_fgate<R>(geo, G[p.gates[i]], hg[i]);
        off += sizeof(FGate<R>) * p.gates.size();
        off = (off + 255) & ~(size_t)255;
        uint64_t* hr = reinterpret_cast<uint64_t*>(hb + off);
        const uint64_t* dr = reinterpret_cast<const uint64_t*>(db + off);
        std::memcpy(hr, geo.rowoff.data(), sizeof(uint64_t) * geo.R);
        off += sizeof(uint64_t) * kMaxRows;
        off = (off + 255) & ~(size_t)255;
        Launch L;
        std::memset(static_cast<void*>(&L.a), 0, sizeof L.a);
        L.a.psi = reinterpret_cast<typename Cplx<R>::T2*>(st->psi);
        L.a.gates = dg;
        L.a.ngates = (int32_t)p.gates.size();
        L.a.T = (uint32_t)p.T;
        L.a.bL = geo.bL;
        L.a.rows = geo.R;
        L.a.vec2 = (sizeof(R) == 4 && geo.bL % 2 == 0) ? 1 : 0;
        L.a.bLdiv.init(geo.bL);
        L.a.ntiles = (uint64_t)(st->L.D / p.T);
        L.a.nfree = geo.nfree;
        for (int i = 0; i < geo.nfree; ++i) {
            L.a.free_w[i] = geo.free_w[i];
            L.a.free_d[i] = geo.free_d[i];
            L.a.free_b[i] = geo.free_b[i];
        }
        L.a.rowoff = dr;
        L.dmax = 2;
        for (int idx : p.gates) L.dmax = G[idx].plan.d > L.dmax ? G[idx].plan.d : L.dmax;
        launches.push_back(L);
    }
    if (bytes > 0) {
        QD_CUDA(cudaMemcpyAsync(st->fuse_dev, st->fuse_host, off, cudaMemcpyHostToDevice, st->stream),
                "fusion descriptor upload");
        QD_CUDA(cudaEventRecord(st->fuse_ev, st->stream), "fusion event");
    }
    size_t li = 0;
    for (const PassPlan& p : passes) {
        if (p.tile) {
            const Launch& ln = launches[li++];
            cudaError_t e = launch_fused<R>(ln.a, ln.dmax, st->stream);
            if (e != cudaSuccess) return cuda_fail(e, "fused tile kernel");
        } else {
            const HGate& h = G[p.gates[0]];
            qd_status rc = apply_any(st, h.wires, h.k, h.U, h.cw, h.cv, h.nc);
            if (rc != QD_OK) return rc;
        }
    }
    return QD_OK;
}

}  // namespace qd

using namespace qd;

extern "C" {

qd_status qd_apply_circuit(qd_state* st, const qd_gate_desc* gates, int32_t n_gates, const double* matrices,
                           const qd_fusion_opts* opts) {
    try {
        if (!st) return fail(QD_ERR_ARG, "state is NULL");
        std::vector<HGate> G;
        qd_status rc = load_gates(st->L, st->prec, gates, n_gates, matrices, G);
        if (rc != QD_OK) return rc;
        const FuseCfg cfg = fuse_cfg(opts, st->prec);
        if (cfg.mode != QD_FUSE_OFF && cfg.mode != QD_FUSE_TILE) return fail(QD_ERR_ARG, "unknown fusion mode");
        if (cfg.Tmax > tile_limit(st->prec))
            return fail(QD_ERR_UNSUPPORTED, "tile of %lld amplitudes exceeds shared memory (limit %lld)",
                        (long long)cfg.Tmax, (long long)tile_limit(st->prec));
        return st->prec == QD_C64 ? run_circuit_impl<float>(st, G, cfg) : run_circuit_impl<double>(st, G, cfg);
    } catch (...) {
        return fail(QD_ERR_OOM, "host exception in qd_apply_circuit");
    }
}

qd_status qd_plan_circuit(const int32_t* dims, int32_t n, int32_t prec, const qd_gate_desc* gates, int32_t n_gates,
                          const double* matrices, const qd_fusion_opts* opts, int32_t* exec_order, int32_t* pass_of,
                          int64_t* pass_tile_amps, int32_t* n_passes) {
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
        }
        *n_passes = (int32_t)passes.size();
        return QD_OK;
    } catch (...) {
        return fail(QD_ERR_OOM, "host exception in qd_plan_circuit");
    }
}

}  // extern "C"
