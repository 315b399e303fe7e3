// Composed blocks of up to 64 dimensions on the 5th-generation tensor cores
// (tcgen05, sm_103a), complex64 states.
//
// A block is a P x P complex matrix M (P <= 64) on a wire set W; its classes
// are the P amplitudes that differ only in the digits of W (the paper's
// equivalence classes, section "Superposition gates", generalised to several
// wires).  For N classes at once the block is one dense contraction
//     [Re Y; Im Y] (128 x N) = [[Re M, -Im M], [Im M, Re M]] (128 x 128) . [Re X; Im X] (128 x N),
// run as tcgen05.mma kind::tf32 with FP32 accumulation in tensor memory.
// TF32 keeps 11 significand bits, so both operands are split, a = a_hi + a_lo
// (a_hi = a with its low 13 bits cleared, a_lo = a - a_hi exactly), and three
// products are accumulated: A_hi X_hi + A_hi X_lo + A_lo X_hi (the dropped
// A_lo X_lo term is below 2^-21 relative).
//
// One persistent CTA per SM keeps A_hi and A_lo in tensor memory (loaded
// once with tcgen05.st: lane = output row, column = K) next to two FP32
// accumulators, and runs a two-stage pipeline over chunks of 64 classes:
//   - the 256 threads split the next chunk's members (prefetched into
//     registers) into that stage's B operand in shared memory (K-major, no
//     swizzle, 16-byte stores); one thread issues its 3 x 16 MMAs (M = 128,
//     N = 64, K = 8, A from tensor memory) into that stage's accumulator and
//     commits them to the stage's mbarrier;
//   - meanwhile the chunk after it is loaded into registers, and the current
//     chunk's accumulator is waited for (bounded), read with tcgen05.ld,
//     staged in shared memory and written out with warps running along the
//     classes (coalesced).
// Every wait is bounded: on timeout the kernel records the error in a status
// word, stops issuing work, releases its tensor memory and returns.
#include <cstdint>

#include "qd_internal.cuh"
#include "qudit.h"

namespace qd {

namespace {

constexpr int kTcN = 64;              // classes per chunk (MMA N)
constexpr int kTcK = 128;             // real K (64 members x re/im)
constexpr int kTcM = 128;             // real M (64 outputs x re/im)
constexpr uint32_t kABytes = kTcM * kTcK * 4;   // one of A_hi / A_lo
constexpr uint32_t kBBytes = kTcN * kTcK * 4;   // one of B_hi / B_lo
constexpr uint32_t kStageBytes = 2 * kBBytes;   // B_hi | B_lo of one pipeline stage
constexpr uint32_t kTmemCols = 512;             // A_hi [0,128) A_lo [128,256) D0 [256,320) D1 [320,384)
constexpr int kYStride = 68;          // floats per staged accumulator row (bank-conflict-free float4 stores)
constexpr uint32_t kSpinLimit = 1u << 26;

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// Shared-memory matrix descriptor: no swizzle, K-major canonical layout.
// Core matrices of 8 rows x 16 bytes (128 contiguous bytes); lbo = bytes
// between core matrices adjacent along K, sbo = along M/N.
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr >> 4) & 0x3FFFu);
    d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
    d |= (uint64_t)1 << 46;  // descriptor version
    return d;                // base offset 0, relative LBO, layout type 0 (no swizzle)
}

// Instruction descriptor: D = F32, A = B = TF32, both K-major, M = 128, N = kTcN.
__host__ __device__ constexpr uint32_t tc_idesc() {
    return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(kTcN >> 3) << 17) | ((uint32_t)(kTcM >> 4) << 24);
}

// Byte offset of element (row, k) in a K-major no-swizzle operand with `rows` rows.
__host__ __device__ __forceinline__ uint32_t kmajor_off(uint32_t row, uint32_t k, uint32_t rows) {
    return (k >> 2) * (rows / 8) * 128 + (row >> 3) * 128 + (row & 7) * 16 + (k & 3) * 4;
}

__device__ __forceinline__ float tf32_hi(float x) { return __uint_as_float(__float_as_uint(x) & 0xFFFFE000u); }

__device__ __forceinline__ void mma_tf32(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                         uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}"
        :
        : "r"(tmem_d), "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate));
}

__device__ __forceinline__ void mma_tf32_ta(uint32_t tmem_d, uint32_t tmem_a, uint64_t bdesc, uint32_t idesc,
                                            uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::tf32 [%0], [%1], %2, %3, p;\n\t}"
        :
        : "r"(tmem_d), "r"(tmem_a), "l"(bdesc), "r"(idesc), "r"(accumulate));
}

__device__ __forceinline__ void tmem_st32(uint32_t taddr, const float* v) {
    asm volatile(
        "tcgen05.st.sync.aligned.32x32b.x32.b32 [%0], "
        "{%1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, %16, "
        "%17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31, %32};"
        :
        : "r"(taddr), "r"(__float_as_uint(v[0])), "r"(__float_as_uint(v[1])), "r"(__float_as_uint(v[2])),
          "r"(__float_as_uint(v[3])), "r"(__float_as_uint(v[4])), "r"(__float_as_uint(v[5])),
          "r"(__float_as_uint(v[6])), "r"(__float_as_uint(v[7])), "r"(__float_as_uint(v[8])),
          "r"(__float_as_uint(v[9])), "r"(__float_as_uint(v[10])), "r"(__float_as_uint(v[11])),
          "r"(__float_as_uint(v[12])), "r"(__float_as_uint(v[13])), "r"(__float_as_uint(v[14])),
          "r"(__float_as_uint(v[15])), "r"(__float_as_uint(v[16])), "r"(__float_as_uint(v[17])),
          "r"(__float_as_uint(v[18])), "r"(__float_as_uint(v[19])), "r"(__float_as_uint(v[20])),
          "r"(__float_as_uint(v[21])), "r"(__float_as_uint(v[22])), "r"(__float_as_uint(v[23])),
          "r"(__float_as_uint(v[24])), "r"(__float_as_uint(v[25])), "r"(__float_as_uint(v[26])),
          "r"(__float_as_uint(v[27])), "r"(__float_as_uint(v[28])), "r"(__float_as_uint(v[29])),
          "r"(__float_as_uint(v[30])), "r"(__float_as_uint(v[31])));
}

__device__ __forceinline__ bool mbar_wait(uint32_t mbar, uint32_t phase) {
    for (uint32_t it = 0; it < kSpinLimit; ++it) {
        uint32_t done;
        asm volatile(
            "{\n\t.reg .pred P;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 P, [%1], %2;\n\t"
            "selp.b32 %0, 1, 0, P;\n\t}"
            : "=r"(done)
            : "r"(mbar), "r"(phase));
        if (done) return true;
    }
    return false;
}

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float* v) {
    uint32_t r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
        "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
        "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

struct TcArgs {
    float2* psi;
    const float* a_hilo;  // A_hi then A_lo, each 128 x 128 row-major (row = output, column = K)
    uint64_t n_classes;
    IndexMap map;
    int32_t P;
    uint64_t off[64];
    int32_t* status;      // set to QD_ERR_TIMEOUT-like code on a bounded-wait timeout
};

__global__ void __launch_bounds__(256, 1) k_block_tc(const __grid_constant__ TcArgs a) {
    extern __shared__ __align__(1024) unsigned char smem[];
    unsigned char* sB = smem;                                   // two stages of B_hi | B_lo
    float* Y = reinterpret_cast<float*>(smem + 2 * kStageBytes);  // staged accumulator, [128][kYStride]
    __shared__ __align__(8) uint64_t mbar[2];
    __shared__ uint32_t tmem_base;
    __shared__ int abort_flag;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

    if (tid == 0) {
        abort_flag = 0;
        asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&mbar[0])), "r"(1));
        asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&mbar[1])), "r"(1));
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base)),
                     "r"(kTmemCols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tm = tmem_base;
    // A_hi, A_lo -> tensor memory: warp w (< 4) writes lanes 32 w .. 32 w + 31
    if (warp < 4) {
        const uint32_t row = 32u * (uint32_t)warp + (uint32_t)lane;
#pragma unroll 1
        for (int h = 0; h < 2; ++h)
#pragma unroll 1
            for (int c = 0; c < 4; ++c) {
                float v[32];
                const float4* src = reinterpret_cast<const float4*>(a.a_hilo + (size_t)h * kTcM * kTcK +
                                                                    (size_t)row * kTcK + 32 * c);
#pragma unroll
                for (int i = 0; i < 8; ++i) {
                    const float4 t = src[i];
                    v[4 * i] = t.x;
                    v[4 * i + 1] = t.y;
                    v[4 * i + 2] = t.z;
                    v[4 * i + 3] = t.w;
                }
                tmem_st32(tm + ((32u * (uint32_t)warp) << 16) + (uint32_t)(h * 128 + 32 * c), v);
            }
        asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");

    const uint32_t idesc = tc_idesc();
    const uint32_t sB_u = smem_u32(sB);
    uint32_t phase0 = 0u, phase1 = 0u;
    const uint64_t n_chunks = (a.n_classes + kTcN - 1) / kTcN;

    // thread -> class n = tid % 64 of each chunk, member quads q = tid / 64 + 4 j (j < 4)
    const int n = tid & (kTcN - 1);
    const int q0 = tid >> 6;
    float2 pre[16];  // the members of the next chunk to stage
    uint64_t pre_base = 0;
    bool pre_valid = false;
    auto prefetch = [&](uint64_t chunk) {
        const uint64_t g = chunk * kTcN + (uint64_t)n;
        pre_valid = chunk < n_chunks && g < a.n_classes;
        pre_base = pre_valid ? a.map.map(g) : 0;
#pragma unroll
        for (int j = 0; j < 4; ++j)
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const int r = 4 * (q0 + 4 * j) + i;
                pre[4 * j + i] = (pre_valid && r < a.P) ? a.psi[pre_base + a.off[r]] : make_float2(0.f, 0.f);
            }
    };
    auto stage_b = [&](int st) {
        unsigned char* b = sB + st * kStageBytes;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int q = q0 + 4 * j;
            float4 rh, rl, ih, il;
            rh.x = tf32_hi(pre[4 * j].x); rh.y = tf32_hi(pre[4 * j + 1].x);
            rh.z = tf32_hi(pre[4 * j + 2].x); rh.w = tf32_hi(pre[4 * j + 3].x);
            ih.x = tf32_hi(pre[4 * j].y); ih.y = tf32_hi(pre[4 * j + 1].y);
            ih.z = tf32_hi(pre[4 * j + 2].y); ih.w = tf32_hi(pre[4 * j + 3].y);
            rl.x = pre[4 * j].x - rh.x; rl.y = pre[4 * j + 1].x - rh.y;
            rl.z = pre[4 * j + 2].x - rh.z; rl.w = pre[4 * j + 3].x - rh.w;
            il.x = pre[4 * j].y - ih.x; il.y = pre[4 * j + 1].y - ih.y;
            il.z = pre[4 * j + 2].y - ih.z; il.w = pre[4 * j + 3].y - ih.w;
            // K index: real parts at 4q..4q+3, imaginary parts at 64 + 4q..
            *reinterpret_cast<float4*>(b + kmajor_off(n, 4 * q, kTcN)) = rh;
            *reinterpret_cast<float4*>(b + kmajor_off(n, 64 + 4 * q, kTcN)) = ih;
            *reinterpret_cast<float4*>(b + kBBytes + kmajor_off(n, 4 * q, kTcN)) = rl;
            *reinterpret_cast<float4*>(b + kBBytes + kmajor_off(n, 64 + 4 * q, kTcN)) = il;
        }
    };
    // one thread: 3 products x 16 k-steps into accumulator st, committed to mbar[st]
    auto issue_mma = [&](int st) {
        const uint32_t lboB = (kTcN / 8) * 128;
        const uint64_t bd0 = smem_desc(sB_u + (uint32_t)st * kStageBytes, lboB, 128);
        constexpr uint64_t kStepB = 2 * (kTcN / 8) * 128 / 16;  // descriptor address field: 16-byte units
        const uint32_t d = tm + 256u + (uint32_t)st * kTcN;
#pragma unroll
        for (int term = 0; term < 3; ++term) {
            const uint32_t a0 = tm + (term == 2 ? 128u : 0u);                       // A_lo for the third product
            const uint64_t b0 = bd0 + (term == 1 ? (uint64_t)(kBBytes >> 4) : 0);  // B_lo for the second
#pragma unroll
            for (int ks = 0; ks < kTcK / 8; ++ks)
                mma_tf32_ta(d, a0 + 8u * (uint32_t)ks, b0 + (uint64_t)ks * kStepB, idesc, (term | ks) != 0 ? 1u : 0u);
        }
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                         smem_u32(&mbar[st]))
                     : "memory");
    };
    auto publish_b = [&]() {
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncthreads();
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    };

    uint64_t chunk = blockIdx.x;
    prefetch(chunk);
    bool cur_valid = pre_valid;
    uint64_t cur_base = pre_base;
    int st = 0;
    stage_b(0);
    publish_b();
    if (chunk < n_chunks && tid == 0) issue_mma(0);
    prefetch(chunk + gridDim.x);

    for (; chunk < n_chunks; chunk += gridDim.x) {
        const uint64_t next = chunk + gridDim.x;
        const bool nxt_valid = pre_valid;
        const uint64_t nxt_base = pre_base;
        // stage the next chunk and start its MMAs; they run during this chunk's epilogue
        if (next < n_chunks) {
            stage_b(st ^ 1);
            publish_b();
            if (tid == 0) issue_mma(st ^ 1);
            prefetch(next + gridDim.x);
        }
        // wait for this chunk's accumulator (bounded); on timeout also wait
        // (bounded) for the other stage before the tensor memory is released
        uint32_t& ph = st ? phase1 : phase0;
        if (!mbar_wait(smem_u32(&mbar[st]), ph)) {
            if (lane == 0) atomicExch(&abort_flag, 1);
            mbar_wait(smem_u32(&mbar[st]), ph);
            if (next < n_chunks) mbar_wait(smem_u32(&mbar[st ^ 1]), st ? phase0 : phase1);
        }
        ph ^= 1u;
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        __syncthreads();
        if (abort_flag) break;
        // TMEM -> registers -> shared: warp w reads lanes 32 (w % 4) .. +31,
        // warps 0-3 columns 0..31 of the accumulator, warps 4-7 columns 32..63
        {
            const uint32_t row = 32u * (uint32_t)(warp & 3) + (uint32_t)lane;
            const uint32_t col = (uint32_t)(warp >> 2) * 32u;
            float v[32];
            tmem_ld32(tm + ((32u * (uint32_t)(warp & 3)) << 16) + 256u + (uint32_t)st * kTcN + col, v);
#pragma unroll
            for (int i = 0; i < 32; i += 4)
                *reinterpret_cast<float4*>(Y + row * kYStride + col + i) = make_float4(v[i], v[i + 1], v[i + 2], v[i + 3]);
        }
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncthreads();
        // outputs: y_r = (Y[r][n], Y[64 + r][n]), lanes along the classes
        if (cur_valid) {
#pragma unroll 4
            for (int r = q0; r < a.P; r += 4)
                a.psi[cur_base + a.off[r]] = make_float2(Y[r * kYStride + n], Y[(64 + r) * kYStride + n]);
        }
        cur_valid = nxt_valid;
        cur_base = nxt_base;
        st ^= 1;
        // Y is rewritten only after the next iteration's publish_b barrier
    }
    __syncthreads();
    if (abort_flag && tid == 0) atomicExch(a.status, QD_ERR_TIMEOUT);
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tm), "r"(kTmemCols));
}

// Status word of the tensor-core kernels: 0, or an error code set by a
// kernel whose bounded wait gave up.  Read and cleared by tc_status_take().
__device__ int32_t g_tc_status;

}  // namespace

size_t block_tc_operand_bytes() { return 2 * (size_t)kABytes; }

int32_t* tc_status_ptr() {
    static int32_t* ptr[64] = {nullptr};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return nullptr;
    if (!ptr[dev]) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_tc_status) != cudaSuccess) return nullptr;
        ptr[dev] = static_cast<int32_t*>(p);
    }
    return ptr[dev];
}

int32_t tc_status_take(cudaStream_t s) {
    int32_t* p = tc_status_ptr();
    if (!p) return 0;
    int32_t h = 0;
    if (cudaMemcpyAsync(&h, p, sizeof h, cudaMemcpyDeviceToHost, s) != cudaSuccess) return 0;
    if (cudaStreamSynchronize(s) != cudaSuccess) return 0;
    if (h != 0) {
        const int32_t z = 0;
        cudaMemcpyAsync(p, &z, sizeof z, cudaMemcpyHostToDevice, s);
        cudaStreamSynchronize(s);
    }
    return h;
}

// A_hi | A_lo (each 128 x 128 row-major, row = output, column = K) from a
// P x P complex binary64 matrix (row-major interleaved), padded with zeros.
void block_tc_pack(const double* U, int P, float* out) {
    for (int i = 0; i < 2 * kTcM * kTcK; ++i) out[i] = 0.f;
    float* hi = out;
    float* lo = out + kTcM * kTcK;
    auto put = [&](int m, int k, double v) {
        const float f = (float)v;
        uint32_t bits;
        __builtin_memcpy(&bits, &f, 4);
        bits &= 0xFFFFE000u;
        float h;
        __builtin_memcpy(&h, &bits, 4);
        hi[m * kTcK + k] = h;
        lo[m * kTcK + k] = (float)(v - (double)h);
    };
    for (int r = 0; r < P; ++r)
        for (int c = 0; c < P; ++c) {
            const double re = U[2 * (r * P + c)], im = U[2 * (r * P + c) + 1];
            put(r, c, re);
            put(r, 64 + c, -im);
            put(64 + r, c, im);
            put(64 + r, 64 + c, re);
        }
}

cudaError_t launch_block_tc(float2* psi, const float* a_hilo, uint64_t n_classes, const IndexMap& map, int P,
                            const uint64_t* off, cudaStream_t s) {
    if (n_classes == 0) return cudaSuccess;
    static int sm_count = 0;
    if (sm_count == 0) {
        int dv = 0;
        cudaGetDevice(&dv);
        cudaDeviceGetAttribute(&sm_count, cudaDevAttrMultiProcessorCount, dv);
        if (sm_count <= 0) sm_count = 148;
    }
    int32_t* status = tc_status_ptr();
    if (!status) return cudaErrorInvalidSymbol;
    static int attr_dev = -1;
    int dev = 0;
    cudaGetDevice(&dev);
    const size_t smem = 2 * (size_t)kStageBytes + sizeof(float) * kTcM * kYStride;
    if (attr_dev != dev) {
        cudaError_t e = cudaFuncSetAttribute(k_block_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        attr_dev = dev;
    }
    TcArgs a;
    a.psi = psi;
    a.a_hilo = a_hilo;
    a.n_classes = n_classes;
    a.map = map;
    a.P = P;
    for (int r = 0; r < 64; ++r) a.off[r] = r < P ? off[r] : 0;
    a.status = status;
    const uint64_t chunks = (n_classes + kTcN - 1) / kTcN;
    const unsigned grid = (unsigned)(chunks < (uint64_t)sm_count ? chunks : (uint64_t)sm_count);
    k_block_tc<<<grid, 256, smem, s>>>(a);
    count_launch();
    return cudaGetLastError();
}

}  // namespace qd
