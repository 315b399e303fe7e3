// Per-gate and readout kernels for sm_103a.
//
// Gate kernels implement the "grouping and transformation" step of the
// paper's block method (section "Example Circuit"): every equivalence class
// of amplitudes that differ only in the digits of the gate's wires (section
// "Superposition gates") is gathered, multiplied by the gate matrix and
// scattered back in place.  Classes are independent, so one thread (or one
// tile column) owns one class and no synchronisation between classes is
// needed -- the parallelism "across blocks as well as the repetitions of
// the blocks" that the paper leaves as future scope.
#include <algorithm>

#include "qd_internal.cuh"

namespace qd {

namespace {

template <typename T2> __device__ __forceinline__ T2 cmul(const T2& u, const T2& x) {
    T2 r;
    r.x = u.x * x.x - u.y * x.y;
    r.y = u.x * x.y + u.y * x.x;
    return r;
}

template <typename T2> __device__ __forceinline__ void cmac(T2& acc, const T2& u, const T2& x) {
    acc.x = fma(u.x, x.x, acc.x);
    acc.x = fma(-u.y, x.y, acc.x);
    acc.y = fma(u.x, x.y, acc.y);
    acc.y = fma(u.y, x.x, acc.y);
}

// VEC consecutive amplitudes starting at p (16-byte aligned when VEC = 2).
template <int VEC> struct Ld;
template <> struct Ld<1> {
    template <typename T2> __device__ __forceinline__ static void load(const T2* p, T2* x) { x[0] = *p; }
    template <typename T2> __device__ __forceinline__ static void store(T2* p, const T2* x) { *p = x[0]; }
};
template <> struct Ld<2> {  // complex64 only: one 16-byte access
    __device__ __forceinline__ static void load(const float2* p, float2* x) {
        const float4 t = *reinterpret_cast<const float4*>(p);
        x[0] = make_float2(t.x, t.y);
        x[1] = make_float2(t.z, t.w);
    }
    __device__ __forceinline__ static void store(float2* p, const float2* x) {
        *reinterpret_cast<float4*>(p) = make_float4(x[0].x, x[0].y, x[1].x, x[1].y);
    }
};

// The update of VEC consecutive classes whose first member is psi[j].
template <typename R, int DT, int VEC>
__device__ __forceinline__ void gate1_class(const Gate1Args<R, DT>& a, uint64_t j) {
    using T2 = typename Cplx<R>::T2;
    if (!in_bounds(j + (uint64_t)(DT - 1) * a.bt + (VEC - 1), a.D)) return;  // the class's last member
    T2* base = a.psi + j;
    T2 x[DT][VEC];
#pragma unroll
    for (int k = 0; k < DT; ++k)
        if (a.lmask >> k & 1u) Ld<VEC>::load(base + (uint64_t)k * a.bt, x[k]);
    T2 y[DT][VEC];
    if (a.kind == kDense) {
#pragma unroll
        for (int r = 0; r < DT; ++r)
#pragma unroll
            for (int v = 0; v < VEC; ++v) {
                T2 acc = cmul(a.U[r * DT], x[0][v]);
#pragma unroll
                for (int k = 1; k < DT; ++k) cmac(acc, a.U[r * DT + k], x[k][v]);
                y[r][v] = acc;
            }
    } else if (a.kind == kDiag) {
#pragma unroll
        for (int r = 0; r < DT; ++r)
#pragma unroll
            for (int v = 0; v < VEC; ++v) y[r][v] = cmul(a.U[r * DT + r], x[r][v]);
    } else {  // kPerm: y_r = U[r, perm_r] * x_{perm_r}
#pragma unroll
        for (int r = 0; r < DT; ++r) {
            const int src = a.perm[r];
#pragma unroll
            for (int v = 0; v < VEC; ++v) {
                T2 s = x[0][v];
#pragma unroll
                for (int k = 1; k < DT; ++k)
                    if (src == k) s = x[k][v];
                y[r][v] = a.pure_perm ? s : cmul(a.U[r * DT + src], s);
            }
        }
    }
#pragma unroll
    for (int r = 0; r < DT; ++r)
        if (a.smask >> r & 1u) Ld<VEC>::store(base + (uint64_t)r * a.bt, y[r]);
}

// One thread = VEC consecutive classes of a single-wire gate of dimension DT.
// Members of a class sit bt apart; consecutive threads own consecutive
// classes, so each row access of a warp is one contiguous run whenever the
// enumeration's run (the smallest inserted stride) is at least 32*VEC.
// Control digits are inserted into the enumeration: only matching classes
// are visited.
template <typename R, int DT, int VEC>
__global__ void __launch_bounds__(256) k_gate1(const __grid_constant__ Gate1Args<R, DT> a) {
    const uint64_t e = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= a.n_elems) return;
    gate1_class<R, DT, VEC>(a, a.map.map(e * VEC));
}

// The paper's formulation of a controlled gate, kept for comparison: every
// class of the target wire is visited and its control digits
// floor(j / b_c) mod d_c are tested against the control values one by one
// (section "Controlled and Multi-Controlled Gates": a check per index and
// control, O(D M)); matching classes get the same update as in k_gate1.
template <typename R, int DT>
__global__ void __launch_bounds__(256) k_gate1_scan(const __grid_constant__ Gate1Args<R, DT> a,
                                                    const __grid_constant__ ScanControls c) {
    const uint64_t e = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= a.n_elems) return;
    const uint64_t j = a.map.map(e);
    for (int m = 0; m < c.m; ++m) {
        const uint64_t q = c.stride[m].div(j);
        if (q - c.dim[m].div(q) * c.dim[m].d != c.val[m]) return;
    }
    gate1_class<R, DT, 1>(a, j);
}

// Shared-memory tile kernel for any gate with P <= 64 (multi-wire gates and
// single wires of dimension > 8).  A CTA owns Q consecutive classes: it
// stages the P x P matrix and the P x Q member tile in shared memory, then
// each thread computes output rows of one class, y_r = sum_c U[r,c] x_c,
// with warp-uniform rows (broadcast matrix reads) and lane-consecutive
// classes (conflict-free tile reads).
template <typename R>
__global__ void __launch_bounds__(256) k_gate_tile(const __grid_constant__ GateTileArgs<R> a) {
    using T2 = typename Cplx<R>::T2;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T2* sU = reinterpret_cast<T2*>(smem_raw);
    const int P = a.P, Q = a.Q;
    T2* sX = sU + P * P;
    for (int i = threadIdx.x; i < P * P; i += blockDim.x) sU[i] = a.U[i];
    const int q = threadIdx.x % Q;
    const int rg = threadIdx.x / Q;
    const int nrg = blockDim.x / Q;
    const uint64_t g = (uint64_t)blockIdx.x * Q + q;
    const bool valid = g < a.n_classes;
    const uint64_t j = valid ? a.map.map(g) : 0;
    for (int r = rg; r < P; r += nrg) {
        T2 v;
        v.x = 0;
        v.y = 0;
        if (valid && in_bounds(j + a.off[r], a.D)) v = a.psi[j + a.off[r]];
        sX[r * Q + q] = v;
    }
    __syncthreads();
    if (!valid) return;
    constexpr int RB = 4;
    for (int r0 = rg; r0 < P; r0 += RB * nrg) {
        T2 acc[RB];
#pragma unroll
        for (int i = 0; i < RB; ++i) { acc[i].x = 0; acc[i].y = 0; }
        for (int c = 0; c < P; ++c) {
            const T2 xv = sX[c * Q + q];
#pragma unroll
            for (int i = 0; i < RB; ++i) {
                const int r = r0 + i * nrg;
                if (r < P) cmac(acc[i], sU[r * P + c], xv);
            }
        }
#pragma unroll
        for (int i = 0; i < RB; ++i) {
            const int r = r0 + i * nrg;
            if (r < P && in_bounds(j + a.off[r], a.D)) a.psi[j + a.off[r]] = acc[i];
        }
    }
}

// Zero n words of the state (grid-stride); the reset's fill runs on the SMs
// rather than as a runtime memset, which may be served by a copy engine and
// then queue behind another stream's host copies.
template <typename W>
__global__ void k_zero_words(W* p, int64_t n) {
    W z;
    __builtin_memset(&z, 0, sizeof z);
    const int64_t step = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += step) p[i] = z;
}

template <typename R>
__global__ void k_set_basis(typename Cplx<R>::T2* psi, int64_t index) {
    typename Cplx<R>::T2 one;
    one.x = 1;
    one.y = 0;
    psi[index] = one;
}

// ---------------------------------------------------------------------------
// Readouts: binary64, compensated, fixed reduction order.
// ---------------------------------------------------------------------------
struct CSum {  // value s with running compensation c (Neumaier 1974)
    double s, c;
};

__device__ __forceinline__ void csum_add(CSum& a, double x) {
    const double t = a.s + x;
    if (fabs(a.s) >= fabs(x))
        a.c += (a.s - t) + x;
    else
        a.c += (x - t) + a.s;
    a.s = t;
}

// Merge two compensated sums: the error of s1 + s2 (Knuth's TwoSum) joins the compensations.
__device__ __forceinline__ CSum csum_merge(const CSum& a, const CSum& b) {
    const double s = a.s + b.s;
    const double bb = s - a.s;
    const double err = (a.s - (s - bb)) + (b.s - bb);
    CSum r;
    r.s = s;
    r.c = a.c + b.c + err;
    return r;
}

// Deterministic block reduction (fixed tree for a fixed blockDim = 256).
__device__ CSum block_reduce(CSum v) {
    __shared__ double ss[8], sc[8];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        CSum w;
        w.s = __shfl_down_sync(0xffffffffu, v.s, o);
        w.c = __shfl_down_sync(0xffffffffu, v.c, o);
        v = csum_merge(v, w);
    }
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) { ss[wid] = v.s; sc[wid] = v.c; }
    __syncthreads();
    if (wid == 0) {
        v.s = lane < (int)(blockDim.x >> 5) ? ss[lane] : 0.0;
        v.c = lane < (int)(blockDim.x >> 5) ? sc[lane] : 0.0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            CSum w;
            w.s = __shfl_down_sync(0xffffffffu, v.s, o);
            w.c = __shfl_down_sync(0xffffffffu, v.c, o);
            v = csum_merge(v, w);
        }
    }
    return v;
}

template <typename T2> __device__ __forceinline__ double prob(const T2& v) {
    const double re = (double)v.x, im = (double)v.y;
    return fma(re, re, im * im);
}

// Partial sum of block `blk` of `nblk` over psi[0, D): grid-stride from
// blk * blockDim, then the fixed block tree; (s, c) written to out[0..1].
template <typename R>
__device__ __forceinline__ void norm_partial_body(const typename Cplx<R>::T2* psi, int64_t D, uint32_t blk,
                                                  uint32_t nblk, double* out) {
    CSum acc{0.0, 0.0};
    const int64_t stride = (int64_t)nblk * blockDim.x;
    for (int64_t i = (int64_t)blk * blockDim.x + threadIdx.x; i < D; i += stride)
        csum_add(acc, prob(psi[i]));
    acc = block_reduce(acc);
    if (threadIdx.x == 0) {
        out[0] = acc.s;
        out[1] = acc.c;
    }
}

template <typename R>
__global__ void __launch_bounds__(256) k_norm_partial(const typename Cplx<R>::T2* psi, int64_t D,
                                                       double* partials) {
    norm_partial_body<R>(psi, D, blockIdx.x, gridDim.x, partials + 2 * blockIdx.x);
}

// Complex64 norm with little binary64 work (binary64 is slow on this part):
// |a|^2 = x^2 + y^2 is exactly p1 + e1 + p2 + e2 with p = x*x and e =
// fma(x, x, -p) (TwoProduct); runs of 16 amplitudes are summed in binary32
// with Neumaier compensation, the exact product errors going into the
// compensation, and each run's (s, c) is added to the binary64 compensated
// sum.  The binary32 run sum errs by at most about 16 u^2 sum|x| (u = 2^-24),
// below 1e-14 relative.  Two amplitudes per step: one 16-byte load when psi
// is 16-byte aligned (A16), else two 8-byte loads -- the same arithmetic in
// the same order either way, so both alignments give the same bits.
__device__ __forceinline__ void fsum_add(float& s, float& c, float x) {
    const float t = s + x;
    if (fabsf(s) >= fabsf(x))
        c += (s - t) + x;
    else
        c += (x - t) + s;
    s = t;
}
__device__ __forceinline__ void fsum_prob(float& s, float& c, float x, float y) {
    const float p1 = x * x, p2 = y * y;
    c += fmaf(x, x, -p1) + fmaf(y, y, -p2);
    fsum_add(s, c, p1);
    fsum_add(s, c, p2);
}

template <bool A16>
__device__ __forceinline__ void norm_partial_c64_body(const float2* psi, int64_t D, uint32_t blk, uint32_t nblk,
                                                      double* out) {
    CSum acc{0.0, 0.0};
    const int64_t pairs = D >> 1;
    const int64_t stride = (int64_t)nblk * blockDim.x;
    int64_t i = (int64_t)blk * blockDim.x + threadIdx.x;
    while (i < pairs) {
        float s = 0.f, c = 0.f;
#pragma unroll 8
        for (int k = 0; k < 8 && i < pairs; ++k, i += stride) {
            float4 v;
            if constexpr (A16) {
                v = reinterpret_cast<const float4*>(psi)[i];
            } else {
                const float2 a = psi[2 * i], b = psi[2 * i + 1];
                v = make_float4(a.x, a.y, b.x, b.y);
            }
            fsum_prob(s, c, v.x, v.y);
            fsum_prob(s, c, v.z, v.w);
        }
        csum_add(acc, (double)s);
        acc.c += (double)c;
    }
    if ((D & 1) && blk == 0 && threadIdx.x == 0) {
        const float2 v = psi[D - 1];
        float s = 0.f, c = 0.f;
        fsum_prob(s, c, v.x, v.y);
        csum_add(acc, (double)s);
        acc.c += (double)c;
    }
    acc = block_reduce(acc);
    if (threadIdx.x == 0) {
        out[0] = acc.s;
        out[1] = acc.c;
    }
}

template <bool A16>
__global__ void __launch_bounds__(256) k_norm_partial_c64(const float2* psi, int64_t D, double* partials) {
    norm_partial_c64_body<A16>(psi, D, blockIdx.x, gridDim.x, partials + 2 * blockIdx.x);
}

// Sum of nb (s, c) pairs at p, in a fixed order, into *out.
__device__ __forceinline__ void reduce_final_body(const double* p, int nb, double* out) {
    CSum acc{0.0, 0.0};
    for (int i = threadIdx.x; i < nb; i += blockDim.x) {
        CSum w{p[2 * i], p[2 * i + 1]};
        acc = csum_merge(acc, w);
    }
    acc = block_reduce(acc);
    if (threadIdx.x == 0) *out = acc.s + acc.c;
}

// Reduce rows of partials: out[row] = sum over nb (s, c) pairs of row `blockIdx.x`.
__global__ void __launch_bounds__(256) k_reduce_final(const double* partials, int nb, double* out) {
    reduce_final_body(partials + (size_t)blockIdx.x * 2 * nb, nb, out + blockIdx.x);
}

// Norms of many states in two launches, each state's arithmetic exactly that
// of its own launch_norm: block w of the first launch is block w - prefix[e]
// of entry e's nb blocks (the last e with prefix[e] <= w).
__device__ __forceinline__ int find_entry(const uint64_t* prefix, int n, uint64_t w) {
    int lo = 0, hi = n - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (prefix[mid] <= w) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

template <typename R>
__global__ void __launch_bounds__(256) k_norm_partial_batch(const NormEntry* entries, const uint64_t* prefix,
                                                             int32_t n, double* partials) {
    __shared__ int s_e;
    if (threadIdx.x == 0) s_e = find_entry(prefix, n, blockIdx.x);
    __syncthreads();
    const NormEntry& E = entries[s_e];
    const uint32_t blk = (uint32_t)(blockIdx.x - prefix[s_e]);
    double* out = partials + 2 * (E.part_off + blk);
    if constexpr (sizeof(R) == 4) {
        if (E.a16)
            norm_partial_c64_body<true>(static_cast<const float2*>(E.psi), E.D, blk, E.nb, out);
        else
            norm_partial_c64_body<false>(static_cast<const float2*>(E.psi), E.D, blk, E.nb, out);
    } else {
        norm_partial_body<R>(static_cast<const typename Cplx<R>::T2*>(E.psi), E.D, blk, E.nb, out);
    }
}

__global__ void __launch_bounds__(256) k_reduce_final_batch(const NormEntry* entries, double* partials,
                                                            double* norms) {
    const NormEntry& E = entries[blockIdx.x];
    reduce_final_body(partials + 2 * E.part_off, (int)E.nb, norms + E.out_index);
}

template <typename R>
__global__ void __launch_bounds__(256) k_probs(const typename Cplx<R>::T2* psi, int64_t D, double* out) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < D; i += stride)
        out[i] = prob(psi[i]);
}

// Marginal of one wire: blockIdx.y = digit x; the digit is inserted into the
// enumeration of the other wires, so each block row visits D / d amplitudes.
template <typename R>
__global__ void __launch_bounds__(256) k_marginal_partial(const typename Cplx<R>::T2* psi,
                                                           const __grid_constant__ IndexMap map,
                                                           uint64_t n_per_digit, uint64_t stride_w,
                                                           double* partials) {
    CSum acc{0.0, 0.0};
    const uint64_t shift = (uint64_t)blockIdx.y * stride_w;
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n_per_digit; i += stride)
        csum_add(acc, prob(psi[map.map(i) + shift]));
    acc = block_reduce(acc);
    if (threadIdx.x == 0) {
        double* p = partials + (size_t)blockIdx.y * 2 * gridDim.x;
        p[2 * blockIdx.x] = acc.s;
        p[2 * blockIdx.x + 1] = acc.c;
    }
}

template <typename R>
__global__ void __launch_bounds__(256) k_widen(const typename Cplx<R>::T2* psi, int64_t D, double* out) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < D; i += stride) {
        out[2 * i] = (double)psi[i].x;
        out[2 * i + 1] = (double)psi[i].y;
    }
}

template <typename R>
__global__ void __launch_bounds__(256) k_narrow(const double* in, int64_t D, typename Cplx<R>::T2* psi) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < D; i += stride) {
        psi[i].x = (R)in[2 * i];
        psi[i].y = (R)in[2 * i + 1];
    }
}

// Wire move (the data movement of the wire-swap exchange between shards of a
// partitioned state): thread -> element e of the moved order
// (y, h, l) = digits of e over (d, hi, lo), l fastest; the natural index is
// (h d + y) lo + l.  Consecutive threads touch consecutive l in both
// layouts, so accesses coalesce in runs of lo.
template <typename R>
__global__ void __launch_bounds__(256) k_wire_move(const typename Cplx<R>::T2* __restrict__ src,
                                                  typename Cplx<R>::T2* __restrict__ dst, uint64_t D,
                                                  FastDiv lo_div, FastDiv hi_div, uint64_t d, bool to_top) {
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t e = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; e < D; e += stride) {
        uint64_t q, l, y, h;
        lo_div.divmod(e, q, l);
        hi_div.divmod(q, y, h);
        const uint64_t nat = (h * d + y) * lo_div.d + l;
        if (to_top)
            dst[e] = src[nat];
        else
            dst[nat] = src[e];
    }
}

int grid_for(int64_t n, int per_block = 256, int cap = 152 * 16) {
    int64_t g = (n + per_block - 1) / per_block;
    if (g < 1) g = 1;
    if (g > cap) g = cap;
    return (int)g;
}

}  // namespace

int reduce_blocks(int64_t D) { return grid_for(D, 256 * 4, 1024); }

QD_DEFINE_BOUNDS_TAKE(bounds_take_kernels)
uint64_t g_bounds_shrink = 0;

template <typename R, int DT, int VEC>
cudaError_t launch_gate1(const Gate1Args<R, DT>& a, cudaStream_t s) {
    if (a.n_elems == 0) return cudaSuccess;
    const uint64_t blocks = (a.n_elems + 255) / 256;
    k_gate1<R, DT, VEC><<<(unsigned)blocks, 256, 0, s>>>(a);
    count_launch();
    return cudaGetLastError();
}

template <typename R>
size_t gate_tile_smem(int P, int Q) {
    return sizeof(typename Cplx<R>::T2) * (size_t)(P * P + P * Q);
}

template <typename R>
cudaError_t launch_gate_tile(const GateTileArgs<R>& a, cudaStream_t s, int smem_bytes) {
    if (a.n_classes == 0) return cudaSuccess;
    static bool attr_set = false;  // per template instance
    if (!attr_set) {
        cudaError_t e = cudaFuncSetAttribute(k_gate_tile<R>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)gate_tile_smem<R>(kMaxGateDim, 64));
        if (e != cudaSuccess) return e;
        attr_set = true;
    }
    const uint64_t blocks = (a.n_classes + a.Q - 1) / a.Q;
    k_gate_tile<R><<<(unsigned)blocks, 256, smem_bytes, s>>>(a);
    count_launch();
    return cudaGetLastError();
}

template <typename R, int DT>
cudaError_t launch_gate1_scan(const Gate1Args<R, DT>& a, const ScanControls& c, cudaStream_t s) {
    if (a.n_elems == 0) return cudaSuccess;
    const uint64_t blocks = (a.n_elems + 255) / 256;
    k_gate1_scan<R, DT><<<(unsigned)blocks, 256, 0, s>>>(a, c);
    count_launch();
    return cudaGetLastError();
}

template <typename R>
cudaError_t launch_set_basis(void* psi, int64_t D, int64_t index, cudaStream_t s) {
    // |index>: every amplitude zeroed (16-byte stores where the buffer allows,
    // the state's size is a multiple of 8 bytes), then the one set to 1.
    const int64_t bytes = D * (int64_t)sizeof(typename Cplx<R>::T2);
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) !=
                                                   cudaSuccess || sms <= 0)
        sms = 152;
    auto grid = [sms](int64_t n) { return (unsigned)std::min<int64_t>((n + 255) / 256, (int64_t)sms * 8); };
    if (reinterpret_cast<uintptr_t>(psi) % 16 == 0) {
        const int64_t n16 = bytes / 16;
        if (n16 > 0) {
            k_zero_words<ulonglong2><<<grid(n16), 256, 0, s>>>(reinterpret_cast<ulonglong2*>(psi), n16);
            count_launch();
        }
        if (bytes % 16 != 0) {
            k_zero_words<unsigned long long><<<1, 32, 0, s>>>(
                reinterpret_cast<unsigned long long*>(psi) + 2 * n16, 1);
            count_launch();
        }
    } else {
        k_zero_words<unsigned long long><<<grid(bytes / 8), 256, 0, s>>>(
            reinterpret_cast<unsigned long long*>(psi), bytes / 8);
        count_launch();
    }
    k_set_basis<R><<<1, 1, 0, s>>>(reinterpret_cast<typename Cplx<R>::T2*>(psi), index);
    count_launch();
    return cudaGetLastError();
}

template <typename R>
cudaError_t launch_norm(const void* psi, int64_t D, double* partials, int nblocks, double* dev_out,
                        cudaStream_t s) {
    if (sizeof(R) == 4 && reinterpret_cast<uintptr_t>(psi) % 16 == 0)
        k_norm_partial_c64<true><<<nblocks, 256, 0, s>>>(reinterpret_cast<const float2*>(psi), D, partials);
    else if (sizeof(R) == 4)
        k_norm_partial_c64<false><<<nblocks, 256, 0, s>>>(reinterpret_cast<const float2*>(psi), D, partials);
    else
        k_norm_partial<R><<<nblocks, 256, 0, s>>>(reinterpret_cast<const typename Cplx<R>::T2*>(psi), D,
                                                  partials);
    k_reduce_final<<<1, 256, 0, s>>>(partials, nblocks, dev_out);
    count_launch(2);
    return cudaGetLastError();
}

// |0...0> for many states: unit w of the launch zeroes chunk w - prefix[e]
// (kBasisChunk amplitudes) of entry e's state; the unit that zeroed chunk 0
// then sets amplitude 0 to 1.
constexpr int64_t kBasisChunk = kBasisChunkAmps;

template <typename R>
__global__ void __launch_bounds__(256) k_basis_batch(const NormEntry* entries, const uint64_t* prefix, int32_t n) {
    using T2 = typename Cplx<R>::T2;
    __shared__ int s_e;
    if (threadIdx.x == 0) s_e = find_entry(prefix, n, blockIdx.x);
    __syncthreads();
    const NormEntry& E = entries[s_e];
    const int64_t c = (int64_t)(blockIdx.x - prefix[s_e]);
    const int64_t lo = c * kBasisChunk, hi = lo + kBasisChunk < E.D ? lo + kBasisChunk : E.D;
    T2* psi = static_cast<T2*>(const_cast<void*>(E.psi));
    T2 z;
    z.x = 0;
    z.y = 0;
    for (int64_t i = lo + threadIdx.x; i < hi; i += blockDim.x) psi[i] = z;
    __syncthreads();
    if (c == 0 && threadIdx.x == 0) psi[0].x = (R)1;
}

template <typename R>
cudaError_t launch_basis_batch(const NormEntry* entries, const uint64_t* chunk_prefix, int32_t n,
                               uint64_t total_chunks, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    k_basis_batch<R><<<(unsigned)total_chunks, 256, 0, s>>>(entries, chunk_prefix, n);
    count_launch();
    return cudaGetLastError();
}

template <typename R>
cudaError_t launch_norm_batch(const NormEntry* entries, const uint64_t* block_prefix, int32_t n,
                              uint64_t total_blocks, double* partials, double* norms, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    k_norm_partial_batch<R><<<(unsigned)total_blocks, 256, 0, s>>>(entries, block_prefix, n, partials);
    k_reduce_final_batch<<<(unsigned)n, 256, 0, s>>>(entries, partials, norms);
    count_launch(2);
    return cudaGetLastError();
}

template <typename R>
cudaError_t launch_probs(const void* psi, int64_t D, double* out, cudaStream_t s) {
    k_probs<R><<<grid_for(D), 256, 0, s>>>(reinterpret_cast<const typename Cplx<R>::T2*>(psi), D, out);
    count_launch();
    return cudaGetLastError();
}

template <typename R>
cudaError_t launch_marginal(const void* psi, const IndexMap& map, uint64_t n_per_digit, uint64_t stride,
                            int d, double* partials, int nblocks, double* dev_out, cudaStream_t s) {
    dim3 grid(nblocks, d);
    k_marginal_partial<R><<<grid, 256, 0, s>>>(reinterpret_cast<const typename Cplx<R>::T2*>(psi), map,
                                               n_per_digit, stride, partials);
    k_reduce_final<<<d, 256, 0, s>>>(partials, nblocks, dev_out);
    count_launch(2);
    return cudaGetLastError();
}

template <typename R>
cudaError_t launch_widen(const void* psi, int64_t D, double* out, cudaStream_t s) {
    k_widen<R><<<grid_for(D), 256, 0, s>>>(reinterpret_cast<const typename Cplx<R>::T2*>(psi), D, out);
    count_launch();
    return cudaGetLastError();
}

template <typename R>
cudaError_t launch_narrow(const double* in, int64_t D, void* psi, cudaStream_t s) {
    k_narrow<R><<<grid_for(D), 256, 0, s>>>(in, D, reinterpret_cast<typename Cplx<R>::T2*>(psi));
    count_launch();
    return cudaGetLastError();
}

template <typename R>
cudaError_t launch_wire_move(const void* src, void* dst, int64_t lo, int64_t d, int64_t hi, bool to_top,
                             cudaStream_t s) {
    const uint64_t D = (uint64_t)lo * (uint64_t)d * (uint64_t)hi;
    if (D == 0) return cudaSuccess;
    using T2 = typename Cplx<R>::T2;
    k_wire_move<R><<<grid_for((int64_t)D), 256, 0, s>>>(reinterpret_cast<const T2*>(src), reinterpret_cast<T2*>(dst),
                                                        D, FastDiv((uint64_t)lo), FastDiv((uint64_t)hi), (uint64_t)d,
                                                        to_top);
    count_launch();
    return cudaGetLastError();
}

// Explicit instantiations.
#define QD_INST_GATE1(R, DT, VEC) \
    template cudaError_t launch_gate1<R, DT, VEC>(const Gate1Args<R, DT>&, cudaStream_t);
#define QD_INST_SCAN(R, DT) \
    template cudaError_t launch_gate1_scan<R, DT>(const Gate1Args<R, DT>&, const ScanControls&, cudaStream_t);
#define QD_INST_GATE1_ALL(DT)       \
    QD_INST_GATE1(float, DT, 1)     \
    QD_INST_GATE1(float, DT, 2)     \
    QD_INST_GATE1(double, DT, 1)    \
    QD_INST_SCAN(float, DT)         \
    QD_INST_SCAN(double, DT)
QD_INST_GATE1_ALL(2)
QD_INST_GATE1_ALL(3)
QD_INST_GATE1_ALL(4)
QD_INST_GATE1_ALL(5)
QD_INST_GATE1_ALL(6)
QD_INST_GATE1_ALL(7)
QD_INST_GATE1_ALL(8)

#define QD_INST_R(R)                                                                                    \
    template cudaError_t launch_gate_tile<R>(const GateTileArgs<R>&, cudaStream_t, int);                \
    template size_t gate_tile_smem<R>(int, int);                                                        \
    template cudaError_t launch_set_basis<R>(void*, int64_t, int64_t, cudaStream_t);                    \
    template cudaError_t launch_norm<R>(const void*, int64_t, double*, int, double*, cudaStream_t);     \
    template cudaError_t launch_norm_batch<R>(const NormEntry*, const uint64_t*, int32_t, uint64_t, double*,   \
                                              double*, cudaStream_t);                                         \
    template cudaError_t launch_basis_batch<R>(const NormEntry*, const uint64_t*, int32_t, uint64_t,          \
                                               cudaStream_t);                                                 \
    template cudaError_t launch_probs<R>(const void*, int64_t, double*, cudaStream_t);                  \
    template cudaError_t launch_marginal<R>(const void*, const IndexMap&, uint64_t, uint64_t, int,      \
                                            double*, int, double*, cudaStream_t);                       \
    template cudaError_t launch_widen<R>(const void*, int64_t, double*, cudaStream_t);                  \
    template cudaError_t launch_narrow<R>(const double*, int64_t, void*, cudaStream_t);                 \
    template cudaError_t launch_wire_move<R>(const void*, void*, int64_t, int64_t, int64_t, bool, cudaStream_t);
QD_INST_R(float)
QD_INST_R(double)

}  // namespace qd
