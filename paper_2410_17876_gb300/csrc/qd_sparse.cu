// Sparse states: only the non-zero amplitudes are stored (the paper's
// sparse variant: a unitary is applied by inspecting the indices of the
// non-zero amplitudes, end of section "Example Circuit"; GHZ circuits of
// section "Experimental Analysis").
//
// A basis state is held as a packed-digit key: wire w owns bits
// [pos_w, pos_w + bits_w) of a 128-bit word, bits_w = ceil(log2 d_w), so a
// digit is read and replaced with a shift and a mask; the key <-> mixed-radix
// index map is a bijection, applied only at readout.  128 key bits cover
// e.g. 127 qubits, 64 qutrits or ququads, 42 ququints (the paper's C++ keys
// are 64-bit integer indices, limiting it to 62 qubits / 39 qutrits / 31
// ququads / 27 ququints).
//
// A whole circuit runs in one launch of one CTA, the entries in shared
// memory (supports of up to QD_SPARSE_MAX_NNZ amplitudes, complex128):
//   - a diagonal or monomial gate (one non-zero per column) maps each key to
//     one key: applied in place;
//   - a dense gate groups the stored keys by class (key with the target
//     digit cleared) in a shared-memory hash table: a slot is claimed by a
//     CAS with the index of the first entry of its class, so the class key
//     is re-derived from that (unchanged) entry, never written concurrently;
//     each member stores its amplitude at its digit; then one thread per
//     class computes y_r = sum_x U[r, x] a_x over the present members in
//     ascending x (a fixed order) and appends the non-zero outputs;
//   - entries whose control digits are not all met are copied unchanged;
//     they cannot collide with outputs (those meet the controls).
// Exact zeros are dropped.  More than QD_SPARSE_MAX_NNZ entries after a gate stops
// the circuit with QD_ERR_UNSUPPORTED (the state is left as it was before
// the call).
//
// Larger supports (after qd_sparse_reserve) run gate by gate on the whole
// GPU with the same steps: the entries in global memory, diagonal and
// monomial gates in place, dense gates through a global hash table of
// classes (clear, insert with the same first-entry CAS, emit one class per
// thread, then fix the count).  The state is snapshotted first, so an
// overflow of the reserved capacity also leaves it as before the call.
#include <algorithm>
#include <cstdint>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "qd_internal.cuh"
#include "qd_runtime.h"
#include "qudit.h"

namespace qd {
namespace {

using u128 = unsigned __int128;
constexpr int kSparseMaxD = 8;
constexpr int kSparseThreads = 512;
constexpr int kSparseSlots = 2 * QD_SPARSE_MAX_NNZ;  // hash slots (power of two)

struct SparseGate {
    int32_t pos, bits, d, kind;  // target: bit position, width, dimension; kDense / kDiag / kPerm
    int32_t nc, pad[3];
    int32_t cpos[QD_MAX_CONTROLS], cbits[QD_MAX_CONTROLS], cval[QD_MAX_CONTROLS];
    int32_t rowof[kSparseMaxD];  // monomial: the row receiving member x
    double2 U[kSparseMaxD * kSparseMaxD];
};

__device__ __forceinline__ int digit_of(u128 k, int pos, int bits) {
    return (int)((k >> pos) & (((u128)1 << bits) - 1));
}
__device__ __forceinline__ u128 with_digit(u128 k, int pos, int bits, int v) {
    const u128 m = (((u128)1 << bits) - 1) << pos;
    return (k & ~m) | ((u128)(unsigned)v << pos);
}
__device__ __forceinline__ bool controls_met(const SparseGate& g, u128 k) {
    for (int c = 0; c < g.nc; ++c)
        if (digit_of(k, g.cpos[c], g.cbits[c]) != g.cval[c]) return false;
    return true;
}
__device__ __forceinline__ uint32_t slot_hash(u128 k) {
    uint64_t z = (uint64_t)k ^ ((uint64_t)(k >> 64) + 0x9E3779B97F4A7C15ull);
    z ^= z >> 33;
    z *= 0xff51afd7ed558ccdull;
    z ^= z >> 33;
    z *= 0xc4ceb9fe1a85ec53ull;
    z ^= z >> 33;
    return (uint32_t)z;
}
__device__ __forceinline__ double2 zmul(double2 u, double2 x) {
    return make_double2(fma(u.x, x.x, -u.y * x.y), fma(u.x, x.y, u.y * x.x));
}

// Shared memory: keys and amplitudes (two buffers), hash slots, members.
struct SparseSmem {
    u128 key[2][QD_SPARSE_MAX_NNZ];
    double2 amp[2][QD_SPARSE_MAX_NNZ];
    int32_t slot[kSparseSlots];
    uint32_t mask[kSparseSlots];
    double2 member[kSparseSlots][kSparseMaxD];
};

__global__ void __launch_bounds__(kSparseThreads, 1)
    k_sparse_circuit(const SparseGate* gates, int ngates, u128* keys, double2* amps, int32_t* nnz,
                     int32_t* status) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    SparseSmem& S = *reinterpret_cast<SparseSmem*>(smem_raw);
    __shared__ int n_out, overflow;
    const int tid = threadIdx.x;
    int n = *nnz;
    for (int i = tid; i < n; i += kSparseThreads) {
        S.key[0][i] = keys[i];
        S.amp[0][i] = amps[i];
    }
    if (tid == 0) overflow = 0;
    int cur = 0;
    __syncthreads();
    for (int gi = 0; gi < ngates; ++gi) {
        const SparseGate& g = gates[gi];
        if (g.kind != kDense) {
            // one output key per input key: in place
            for (int i = tid; i < n; i += kSparseThreads) {
                const u128 k = S.key[cur][i];
                if (!controls_met(g, k)) continue;
                const int x = digit_of(k, g.pos, g.bits);
                const int r = g.kind == kDiag ? x : g.rowof[x];
                S.key[cur][i] = with_digit(k, g.pos, g.bits, r);
                S.amp[cur][i] = zmul(g.U[r * g.d + x], S.amp[cur][i]);
            }
            __syncthreads();
            continue;
        }
        int H = 64;
        while (H < 2 * n && H < kSparseSlots) H <<= 1;
        for (int s = tid; s < H; s += kSparseThreads) {
            S.slot[s] = 0;
            S.mask[s] = 0;
        }
        if (tid == 0) n_out = 0;
        __syncthreads();
        const int nxt = cur ^ 1;
        for (int i = tid; i < n; i += kSparseThreads) {
            const u128 k = S.key[cur][i];
            if (!controls_met(g, k)) {
                const int o = atomicAdd(&n_out, 1);
                if (o < QD_SPARSE_MAX_NNZ) {
                    S.key[nxt][o] = k;
                    S.amp[nxt][o] = S.amp[cur][i];
                }
                continue;
            }
            const int x = digit_of(k, g.pos, g.bits);
            const u128 ck = with_digit(k, g.pos, g.bits, 0);
            uint32_t h = slot_hash(ck) & (uint32_t)(H - 1);
            for (int probe = 0; probe < H; ++probe) {  // at most H probes: H > n classes
                const int old = atomicCAS(&S.slot[h], 0, i + 1);
                if (old == 0) break;
                if (with_digit(S.key[cur][old - 1], g.pos, g.bits, 0) == ck) break;
                h = (h + 1) & (uint32_t)(H - 1);
            }
            S.member[h][x] = S.amp[cur][i];
            atomicOr(&S.mask[h], 1u << x);
        }
        __syncthreads();
        for (int s = tid; s < H; s += kSparseThreads) {
            const int first = S.slot[s];
            if (first == 0) continue;
            const u128 ck = with_digit(S.key[cur][first - 1], g.pos, g.bits, 0);
            const uint32_t m = S.mask[s];
            for (int r = 0; r < g.d; ++r) {
                double2 y = make_double2(0.0, 0.0);
                for (int x = 0; x < g.d; ++x)
                    if (m >> x & 1u) {
                        const double2 t = zmul(g.U[r * g.d + x], S.member[s][x]);
                        y.x += t.x;
                        y.y += t.y;
                    }
                if (y.x == 0.0 && y.y == 0.0) continue;
                const int o = atomicAdd(&n_out, 1);
                if (o < QD_SPARSE_MAX_NNZ) {
                    S.key[nxt][o] = with_digit(ck, g.pos, g.bits, r);
                    S.amp[nxt][o] = y;
                }
            }
        }
        __syncthreads();
        if (n_out > QD_SPARSE_MAX_NNZ) {
            if (tid == 0) overflow = 1;
            break;
        }
        n = n_out;
        cur = nxt;
        __syncthreads();
    }
    __syncthreads();
    if (overflow) {
        if (tid == 0) *status = QD_ERR_UNSUPPORTED;
        return;  // keys / amps / nnz keep the state before the call
    }
    for (int i = tid; i < n; i += kSparseThreads) {
        keys[i] = S.key[cur][i];
        amps[i] = S.amp[cur][i];
    }
    if (tid == 0) {
        *nnz = n;
        *status = 0;
    }
}

// ---- grid tier: one gate at a time over the whole GPU ----
// cnt[0] = entries, cnt[1] = entries emitted by the current gate, cnt[2] =
// overflow flag (sticky until the call ends).
constexpr int kGridThreads = 256;

__global__ void __launch_bounds__(kGridThreads) kg_inplace(const SparseGate* gp, u128* keys, double2* amps,
                                                           const int32_t* cnt) {
    const SparseGate& g = *gp;
    const int n = cnt[0];
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const u128 k = keys[i];
        if (!controls_met(g, k)) continue;
        const int x = digit_of(k, g.pos, g.bits);
        const int r = g.kind == kDiag ? x : g.rowof[x];
        keys[i] = with_digit(k, g.pos, g.bits, r);
        amps[i] = zmul(g.U[r * g.d + x], amps[i]);
    }
}

__global__ void __launch_bounds__(kGridThreads) kg_clear(int32_t* slot, uint32_t* mask, int64_t H, int32_t* cnt) {
    for (int64_t h = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; h < H; h += (int64_t)gridDim.x * blockDim.x) {
        slot[h] = 0;
        mask[h] = 0;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) cnt[1] = 0;
}

__global__ void __launch_bounds__(kGridThreads)
    kg_insert(const SparseGate* gp, const u128* keys, const double2* amps, int32_t* cnt, u128* okeys,
              double2* oamps, int32_t* slot, uint32_t* mask, double2* member, int64_t H, int64_t cap) {
    const SparseGate& g = *gp;
    const int n = cnt[0];
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const u128 k = keys[i];
        if (!controls_met(g, k)) {
            const int o = atomicAdd(&cnt[1], 1);
            if (o < cap) {
                okeys[o] = k;
                oamps[o] = amps[i];
            }
            continue;
        }
        const int x = digit_of(k, g.pos, g.bits);
        const u128 ck = with_digit(k, g.pos, g.bits, 0);
        uint64_t h = slot_hash(ck) & (uint64_t)(H - 1);
        for (int64_t probe = 0; probe < H; ++probe) {  // at most H probes: H > n classes
            const int old = atomicCAS(&slot[h], 0, i + 1);
            if (old == 0) break;
            if (with_digit(keys[old - 1], g.pos, g.bits, 0) == ck) break;
            h = (h + 1) & (uint64_t)(H - 1);
        }
        member[h * kSparseMaxD + x] = amps[i];
        atomicOr(&mask[h], 1u << x);
    }
}

__global__ void __launch_bounds__(kGridThreads)
    kg_emit(const SparseGate* gp, const u128* keys, int32_t* cnt, u128* okeys, double2* oamps, const int32_t* slot,
            const uint32_t* mask, const double2* member, int64_t H, int64_t cap) {
    const SparseGate& g = *gp;
    for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < H; s += (int64_t)gridDim.x * blockDim.x) {
        const int first = slot[s];
        if (first == 0) continue;
        const u128 ck = with_digit(keys[first - 1], g.pos, g.bits, 0);
        const uint32_t m = mask[s];
        for (int r = 0; r < g.d; ++r) {
            double2 y = make_double2(0.0, 0.0);
            for (int x = 0; x < g.d; ++x)
                if (m >> x & 1u) {
                    const double2 t = zmul(g.U[r * g.d + x], member[s * kSparseMaxD + x]);
                    y.x += t.x;
                    y.y += t.y;
                }
            if (y.x == 0.0 && y.y == 0.0) continue;
            const int o = atomicAdd(&cnt[1], 1);
            if (o < cap) {
                okeys[o] = with_digit(ck, g.pos, g.bits, r);
                oamps[o] = y;
            }
        }
    }
}

__global__ void kg_finish(int32_t* cnt, int64_t cap) {
    if (cnt[1] > cap) {
        cnt[2] = 1;
        cnt[0] = (int32_t)cap;
    } else {
        cnt[0] = cnt[1];
    }
}

}  // namespace
}  // namespace qd

using qd::u128;

struct qd_sparse {
    int32_t n;
    int32_t dims[QD_SPARSE_MAX_WIRES];
    int32_t pos[QD_SPARSE_MAX_WIRES], bits[QD_SPARSE_MAX_WIRES];
    u128 stride[QD_SPARSE_MAX_WIRES];  // mixed-radix strides (D < 2^128)
    cudaStream_t stream;
    u128* keys;        // device, QD_SPARSE_MAX_NNZ
    double2* amps;     // device
    int32_t* dev_i;    // device: nnz, status
    qd::SparseGate* gates;  // device, grown on demand
    size_t gates_cap;
    int32_t nnz_host;
    // grid tier (qd_sparse_reserve): capacity, entries (two buffers and a
    // snapshot), hash table of H slots, counters; grid = the state lives in
    // gk[cur] / ga[cur] instead of keys / amps
    int64_t cap, H;
    u128* gk[3];
    double2* ga[3];
    int32_t* gslot;
    uint32_t* gmask;
    double2* gmember;
    int32_t* gcnt;
    int cur;
    bool grid;
};

namespace {

qd_status sparse_fail_cuda(cudaError_t e, const char* what) { return qd::cuda_fail(e, what); }

void grid_free(qd_sparse* s) {
    for (int b = 0; b < 3; ++b) {
        if (s->gk[b]) cudaFree(s->gk[b]);
        if (s->ga[b]) cudaFree(s->ga[b]);
        s->gk[b] = nullptr;
        s->ga[b] = nullptr;
    }
    if (s->gslot) cudaFree(s->gslot);
    if (s->gmask) cudaFree(s->gmask);
    if (s->gmember) cudaFree(s->gmember);
    if (s->gcnt) cudaFree(s->gcnt);
    s->gslot = nullptr;
    s->gmask = nullptr;
    s->gmember = nullptr;
    s->gcnt = nullptr;
    s->cap = 0;
    s->H = 0;
}

void sparse_free(qd_sparse* s) {
    if (!s) return;
    if (s->keys) cudaFree(s->keys);
    if (s->amps) cudaFree(s->amps);
    if (s->dev_i) cudaFree(s->dev_i);
    if (s->gates) cudaFree(s->gates);
    grid_free(s);
    delete s;
}

unsigned grid_blocks(int64_t work) {
    const int64_t b = (work + qd::kGridThreads - 1) / qd::kGridThreads;
    return (unsigned)(b < 1 ? 1 : (b > 152 * 16 ? 152 * 16 : b));
}

// The entries move between the one-CTA buffers (keys / amps) and the grid
// tier's current buffer; n entries, on the state's stream.
cudaError_t to_grid(qd_sparse* s) {
    const int32_t n = s->nnz_host;
    cudaError_t e = cudaSuccess;
    if (n > 0) e = cudaMemcpyAsync(s->gk[0], s->keys, sizeof(u128) * n, cudaMemcpyDeviceToDevice, s->stream);
    if (e == cudaSuccess && n > 0)
        e = cudaMemcpyAsync(s->ga[0], s->amps, sizeof(double2) * n, cudaMemcpyDeviceToDevice, s->stream);
    const int32_t c[3] = {n, 0, 0};
    if (e == cudaSuccess) e = cudaMemcpyAsync(s->gcnt, c, sizeof c, cudaMemcpyHostToDevice, s->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
    if (e == cudaSuccess) {
        s->cur = 0;
        s->grid = true;
    }
    return e;
}

cudaError_t from_grid(qd_sparse* s) {  // only when the support fits the one-CTA buffers
    const int32_t n = s->nnz_host;
    cudaError_t e = cudaSuccess;
    if (n > 0)
        e = cudaMemcpyAsync(s->keys, s->gk[s->cur], sizeof(u128) * n, cudaMemcpyDeviceToDevice, s->stream);
    if (e == cudaSuccess && n > 0)
        e = cudaMemcpyAsync(s->amps, s->ga[s->cur], sizeof(double2) * n, cudaMemcpyDeviceToDevice, s->stream);
    const int32_t c[2] = {n, 0};
    if (e == cudaSuccess) e = cudaMemcpyAsync(s->dev_i, c, sizeof c, cudaMemcpyHostToDevice, s->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
    if (e == cudaSuccess) s->grid = false;
    return e;
}

// All gates of a call on the grid tier (gates already on the device).
qd_status grid_run(qd_sparse* s, int n_gates, const std::vector<qd::SparseGate>& hg) {
    const int32_t n0 = s->nnz_host;
    const unsigned be = grid_blocks(s->cap), bh = grid_blocks(s->H);
    // snapshot (buffer 2) so that an overflow leaves the state as before the call
    if (n0 > 0) {
        QD_CUDA(cudaMemcpyAsync(s->gk[2], s->gk[s->cur], sizeof(u128) * n0, cudaMemcpyDeviceToDevice, s->stream),
                "sparse snapshot");
        QD_CUDA(cudaMemcpyAsync(s->ga[2], s->ga[s->cur], sizeof(double2) * n0, cudaMemcpyDeviceToDevice, s->stream),
                "sparse snapshot");
    }
    const int32_t c0[3] = {n0, 0, 0};
    QD_CUDA(cudaMemcpyAsync(s->gcnt, c0, sizeof c0, cudaMemcpyHostToDevice, s->stream), "sparse counters");
    int cur = s->cur;
    for (int gi = 0; gi < n_gates; ++gi) {
        const qd::SparseGate* g = s->gates + gi;
        if (hg[(size_t)gi].kind != qd::kDense) {
            qd::kg_inplace<<<be, qd::kGridThreads, 0, s->stream>>>(g, s->gk[cur], s->ga[cur], s->gcnt);
            qd::count_launch();
            continue;
        }
        const int nxt = cur ^ 1;
        qd::kg_clear<<<bh, qd::kGridThreads, 0, s->stream>>>(s->gslot, s->gmask, s->H, s->gcnt);
        qd::kg_insert<<<be, qd::kGridThreads, 0, s->stream>>>(g, s->gk[cur], s->ga[cur], s->gcnt, s->gk[nxt],
                                                                s->ga[nxt], s->gslot, s->gmask, s->gmember, s->H,
                                                                s->cap);
        qd::kg_emit<<<bh, qd::kGridThreads, 0, s->stream>>>(g, s->gk[cur], s->gcnt, s->gk[nxt], s->ga[nxt], s->gslot,
                                                              s->gmask, s->gmember, s->H, s->cap);
        qd::kg_finish<<<1, 1, 0, s->stream>>>(s->gcnt, s->cap);
        for (int k = 0; k < 4; ++k) qd::count_launch();
        cur = nxt;
    }
    QD_CUDA(cudaGetLastError(), "sparse grid launch");
    int32_t h[3];
    QD_CUDA(cudaMemcpyAsync(h, s->gcnt, sizeof h, cudaMemcpyDeviceToHost, s->stream), "sparse counters");
    QD_CUDA(cudaStreamSynchronize(s->stream), "sparse grid sync");
    if (h[2] != 0) {  // restore the snapshot
        if (n0 > 0) {
            QD_CUDA(cudaMemcpyAsync(s->gk[s->cur], s->gk[2], sizeof(u128) * n0, cudaMemcpyDeviceToDevice, s->stream),
                    "sparse restore");
            QD_CUDA(cudaMemcpyAsync(s->ga[s->cur], s->ga[2], sizeof(double2) * n0, cudaMemcpyDeviceToDevice, s->stream),
                    "sparse restore");
        }
        const int32_t c[3] = {n0, 0, 0};
        QD_CUDA(cudaMemcpyAsync(s->gcnt, c, sizeof c, cudaMemcpyHostToDevice, s->stream), "sparse restore");
        QD_CUDA(cudaStreamSynchronize(s->stream), "sparse restore");
        return qd::fail(QD_ERR_UNSUPPORTED, "sparse circuit: more than %lld non-zero amplitudes after a gate "
                                            "(state unchanged)", (long long)s->cap);
    }
    s->cur = cur;
    s->nnz_host = h[0];
    return QD_OK;
}

}  // namespace

extern "C" {

qd_status qd_sparse_create(const int32_t* dims, int32_t n, void* stream, qd_sparse** out) {
    try {
        if (!out || !dims) return qd::fail(QD_ERR_ARG, "dims or out is NULL");
        if (n < 1 || n > QD_SPARSE_MAX_WIRES)
            return qd::fail(QD_ERR_ARG, "%d wires outside [1, %d]", n, QD_SPARSE_MAX_WIRES);
        qd_sparse* s = new (std::nothrow) qd_sparse();
        if (!s) return qd::fail(QD_ERR_OOM, "host allocation failed");
        s->n = n;
        int pos = 0;
        u128 D = 1;
        for (int w = 0; w < n; ++w) {
            const int d = dims[w];
            if (d < 2 || d > qd::kSparseMaxD) {
                delete s;
                return qd::fail(QD_ERR_ARG, "wire %d: dimension %d outside [2, %d] for sparse states", w, d,
                                qd::kSparseMaxD);
            }
            int b = 0;
            while ((1 << b) < d) ++b;
            s->dims[w] = d;
            s->pos[w] = pos;
            s->bits[w] = b;
            s->stride[w] = D;
            pos += b;
            if (pos > 128 || D > (~(u128)0) / (u128)d) {
                delete s;
                return qd::fail(QD_ERR_ARG, "the basis does not fit 128-bit keys and indices");
            }
            D *= (u128)d;
        }
        s->stream = reinterpret_cast<cudaStream_t>(stream);
        cudaError_t e = cudaMalloc(&s->keys, sizeof(u128) * QD_SPARSE_MAX_NNZ);
        if (e == cudaSuccess) e = cudaMalloc(&s->amps, sizeof(double2) * QD_SPARSE_MAX_NNZ);
        if (e == cudaSuccess) e = cudaMalloc(&s->dev_i, 2 * sizeof(int32_t));
        if (e != cudaSuccess) {
            sparse_free(s);
            return qd::fail(QD_ERR_OOM, "sparse state: %s", cudaGetErrorString(e));
        }
        const u128 k0 = 0;
        const double2 a0 = make_double2(1.0, 0.0);
        const int32_t init[2] = {1, 0};
        e = cudaMemcpyAsync(s->keys, &k0, sizeof k0, cudaMemcpyHostToDevice, s->stream);
        if (e == cudaSuccess) e = cudaMemcpyAsync(s->amps, &a0, sizeof a0, cudaMemcpyHostToDevice, s->stream);
        if (e == cudaSuccess) e = cudaMemcpyAsync(s->dev_i, init, sizeof init, cudaMemcpyHostToDevice, s->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
        if (e != cudaSuccess) {
            sparse_free(s);
            return sparse_fail_cuda(e, "sparse state init");
        }
        s->nnz_host = 1;
        *out = s;
        return QD_OK;
    } catch (...) {
        return qd::fail(QD_ERR_OOM, "host exception in qd_sparse_create");
    }
}

qd_status qd_sparse_destroy(qd_sparse* s) {
    sparse_free(s);
    return QD_OK;
}

qd_status qd_sparse_run(qd_sparse* s, const qd_gate_desc* gates, int32_t n_gates, const double* matrices) {
    try {
        if (!s) return qd::fail(QD_ERR_ARG, "sparse state is NULL");
        if (n_gates < 0 || (n_gates > 0 && (!gates || !matrices))) return qd::fail(QD_ERR_ARG, "bad gate list");
        if (n_gates == 0) return QD_OK;
        std::vector<qd::SparseGate> hg((size_t)n_gates);
        for (int i = 0; i < n_gates; ++i) {
            const qd_gate_desc& g = gates[i];
            qd::SparseGate& q = hg[(size_t)i];
            std::memset(&q, 0, sizeof q);
            if (g.n_wires != 1) return qd::fail(QD_ERR_UNSUPPORTED, "gate %d: sparse states take single-wire gates", i);
            const int t = g.wires[0];
            if (t < 0 || t >= s->n) return qd::fail(QD_ERR_ARG, "gate %d: target %d out of range", i, t);
            if (g.n_ctrl < 0 || g.n_ctrl > QD_MAX_CONTROLS) return qd::fail(QD_ERR_ARG, "gate %d: bad control count", i);
            if (g.matrix_offset < 0) return qd::fail(QD_ERR_ARG, "gate %d: negative matrix offset", i);
            const int d = s->dims[t];
            q.pos = s->pos[t];
            q.bits = s->bits[t];
            q.d = d;
            q.nc = g.n_ctrl;
            for (int c = 0; c < g.n_ctrl; ++c) {
                const int w = g.ctrl_wires[c], v = g.ctrl_vals[c];
                if (w < 0 || w >= s->n || w == t) return qd::fail(QD_ERR_ARG, "gate %d: bad control wire %d", i, w);
                for (int c2 = 0; c2 < c; ++c2)
                    if (g.ctrl_wires[c2] == w) return qd::fail(QD_ERR_ARG, "gate %d: duplicate control %d", i, w);
                if (v < 0 || v >= s->dims[w]) return qd::fail(QD_ERR_ARG, "gate %d: control value %d out of range", i, v);
                q.cpos[c] = s->pos[w];
                q.cbits[c] = s->bits[w];
                q.cval[c] = v;
            }
            const double* U = matrices + 2 * g.matrix_offset;
            bool diag = true, mono = true;
            for (int x = 0; x < d; ++x) {  // columns
                int cnt = 0;
                for (int r = 0; r < d; ++r) {
                    const double re = U[2 * (r * d + x)], im = U[2 * (r * d + x) + 1];
                    q.U[r * d + x] = make_double2(re, im);
                    if (re != 0.0 || im != 0.0) {
                        ++cnt;
                        q.rowof[x] = r;
                        if (r != x) diag = false;
                    }
                }
                if (cnt != 1) mono = false;
            }
            if (mono) {  // one non-zero per column: a bijection when rows are distinct
                bool seen[qd::kSparseMaxD] = {false};
                for (int x = 0; x < d && mono; ++x) {
                    if (seen[q.rowof[x]]) mono = false;
                    seen[q.rowof[x]] = true;
                }
            }
            q.kind = diag && mono ? qd::kDiag : (mono ? qd::kPerm : qd::kDense);
        }
        const size_t bytes = sizeof(qd::SparseGate) * hg.size();
        if (hg.size() > s->gates_cap) {
            QD_CUDA(cudaStreamSynchronize(s->stream), "sparse gate buffer resize");
            if (s->gates) cudaFree(s->gates);
            s->gates = nullptr;
            s->gates_cap = 0;
            cudaError_t e = cudaMalloc(&s->gates, bytes);
            if (e != cudaSuccess) return qd::fail(QD_ERR_OOM, "sparse gate buffer: %s", cudaGetErrorString(e));
            s->gates_cap = hg.size();
        }
        QD_CUDA(cudaMemcpyAsync(s->gates, hg.data(), bytes, cudaMemcpyHostToDevice, s->stream), "sparse gates upload");
        if (s->grid) {  // the support is beyond the one-CTA buffers
            const qd_status rc = grid_run(s, n_gates, hg);
            if (rc == QD_OK && s->nnz_host <= QD_SPARSE_MAX_NNZ) QD_CUDA(from_grid(s), "sparse tier change");
            return rc;
        }
        static int attr_dev = -1;
        int dev = 0;
        cudaGetDevice(&dev);
        if (attr_dev != dev) {
            QD_CUDA(cudaFuncSetAttribute(qd::k_sparse_circuit, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)sizeof(qd::SparseSmem)),
                    "sparse kernel attribute");
            attr_dev = dev;
        }
        qd::k_sparse_circuit<<<1, qd::kSparseThreads, sizeof(qd::SparseSmem), s->stream>>>(
            s->gates, n_gates, s->keys, s->amps, s->dev_i, s->dev_i + 1);
        qd::count_launch();
        QD_CUDA(cudaGetLastError(), "sparse kernel launch");
        int32_t h[2];
        QD_CUDA(cudaMemcpyAsync(h, s->dev_i, sizeof h, cudaMemcpyDeviceToHost, s->stream), "sparse status");
        QD_CUDA(cudaStreamSynchronize(s->stream), "sparse sync");
        if (h[1] != 0) {
            if (s->cap <= QD_SPARSE_MAX_NNZ)
                return qd::fail(QD_ERR_UNSUPPORTED, "sparse circuit: more than %d non-zero amplitudes after a gate "
                                                    "(state unchanged; qd_sparse_reserve allows more)",
                                QD_SPARSE_MAX_NNZ);
            // the one-CTA launch left the state as it was: run the call on the grid tier
            QD_CUDA(to_grid(s), "sparse tier change");
            const qd_status rc = grid_run(s, n_gates, hg);
            if (rc == QD_OK && s->nnz_host <= QD_SPARSE_MAX_NNZ) QD_CUDA(from_grid(s), "sparse tier change");
            if (rc != QD_OK && s->nnz_host <= QD_SPARSE_MAX_NNZ) (void)from_grid(s);
            return rc;
        }
        s->nnz_host = h[0];
        return QD_OK;
    } catch (...) {
        return qd::fail(QD_ERR_OOM, "host exception in qd_sparse_run");
    }
}

qd_status qd_sparse_reserve(qd_sparse* s, int64_t max_nnz) {
    try {
        if (!s) return qd::fail(QD_ERR_ARG, "sparse state is NULL");
        if (max_nnz <= QD_SPARSE_MAX_NNZ || max_nnz > QD_SPARSE_MAX_RESERVE)
            return qd::fail(QD_ERR_ARG, "capacity %lld outside (%d, %d]", (long long)max_nnz, QD_SPARSE_MAX_NNZ,
                            QD_SPARSE_MAX_RESERVE);
        if (max_nnz <= s->cap) return QD_OK;
        qd_sparse t{};  // the new buffers
        t.cap = max_nnz;
        t.H = 1024;
        while (t.H < 2 * max_nnz) t.H <<= 1;
        cudaError_t e = cudaSuccess;
        for (int b = 0; b < 3 && e == cudaSuccess; ++b) {
            e = cudaMalloc(&t.gk[b], sizeof(u128) * (size_t)t.cap);
            if (e == cudaSuccess) e = cudaMalloc(&t.ga[b], sizeof(double2) * (size_t)t.cap);
        }
        if (e == cudaSuccess) e = cudaMalloc(&t.gslot, sizeof(int32_t) * (size_t)t.H);
        if (e == cudaSuccess) e = cudaMalloc(&t.gmask, sizeof(uint32_t) * (size_t)t.H);
        if (e == cudaSuccess) e = cudaMalloc(&t.gmember, sizeof(double2) * qd::kSparseMaxD * (size_t)t.H);
        if (e == cudaSuccess) e = cudaMalloc(&t.gcnt, 4 * sizeof(int32_t));
        if (e == cudaSuccess && s->grid && s->nnz_host > 0) {  // move the current entries over
            e = cudaMemcpyAsync(t.gk[0], s->gk[s->cur], sizeof(u128) * s->nnz_host, cudaMemcpyDeviceToDevice, s->stream);
            if (e == cudaSuccess)
                e = cudaMemcpyAsync(t.ga[0], s->ga[s->cur], sizeof(double2) * s->nnz_host, cudaMemcpyDeviceToDevice,
                                    s->stream);
        }
        const int32_t c[4] = {s->nnz_host, 0, 0, 0};
        if (e == cudaSuccess) e = cudaMemcpyAsync(t.gcnt, c, sizeof c, cudaMemcpyHostToDevice, s->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
        if (e != cudaSuccess) {
            grid_free(&t);
            return qd::fail(QD_ERR_OOM, "sparse capacity %lld: %s", (long long)max_nnz, cudaGetErrorString(e));
        }
        grid_free(s);
        for (int b = 0; b < 3; ++b) {
            s->gk[b] = t.gk[b];
            s->ga[b] = t.ga[b];
        }
        s->gslot = t.gslot;
        s->gmask = t.gmask;
        s->gmember = t.gmember;
        s->gcnt = t.gcnt;
        s->cap = t.cap;
        s->H = t.H;
        s->cur = 0;
        return QD_OK;
    } catch (...) {
        return qd::fail(QD_ERR_OOM, "host exception in qd_sparse_reserve");
    }
}

qd_status qd_sparse_nnz(const qd_sparse* s, int64_t* nnz) {
    if (!s || !nnz) return qd::fail(QD_ERR_ARG, "state or out is NULL");
    *nnz = s->nnz_host;
    return QD_OK;
}

qd_status qd_sparse_get(qd_sparse* s, uint64_t* index_lo, uint64_t* index_hi, double* amps_interleaved,
                        int64_t max, int64_t* n_out) {
    try {
        if (!s || !index_lo || !index_hi || !amps_interleaved || !n_out)
            return qd::fail(QD_ERR_ARG, "a pointer is NULL");
        const int n = s->nnz_host;
        if (max < n) return qd::fail(QD_ERR_ARG, "room for %lld entries, %d stored", (long long)max, n);
        std::vector<u128> k((size_t)n);
        std::vector<double2> a((size_t)n);
        const u128* dk = s->grid ? s->gk[s->cur] : s->keys;
        const double2* da = s->grid ? s->ga[s->cur] : s->amps;
        if (n > 0) {
            QD_CUDA(cudaMemcpyAsync(k.data(), dk, sizeof(u128) * n, cudaMemcpyDeviceToHost, s->stream), "sparse keys");
            QD_CUDA(cudaMemcpyAsync(a.data(), da, sizeof(double2) * n, cudaMemcpyDeviceToHost, s->stream), "sparse amps");
        }
        QD_CUDA(cudaStreamSynchronize(s->stream), "sparse readout");
        std::vector<std::pair<u128, double2>> e((size_t)n);
        for (int i = 0; i < n; ++i) {
            u128 idx = 0;  // packed digits -> mixed-radix index
            for (int w = 0; w < s->n; ++w) {
                const u128 dg = (k[i] >> s->pos[w]) & (((u128)1 << s->bits[w]) - 1);
                idx += dg * s->stride[w];
            }
            e[(size_t)i] = {idx, a[(size_t)i]};
        }
        std::sort(e.begin(), e.end(), [](const auto& x, const auto& y) { return x.first < y.first; });
        for (int i = 0; i < n; ++i) {
            index_lo[i] = (uint64_t)e[(size_t)i].first;
            index_hi[i] = (uint64_t)(e[(size_t)i].first >> 64);
            amps_interleaved[2 * i] = e[(size_t)i].second.x;
            amps_interleaved[2 * i + 1] = e[(size_t)i].second.y;
        }
        *n_out = n;
        return QD_OK;
    } catch (...) {
        return qd::fail(QD_ERR_OOM, "host exception in qd_sparse_get");
    }
}

}  // extern "C"
