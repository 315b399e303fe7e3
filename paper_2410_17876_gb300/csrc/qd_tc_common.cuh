// Device helpers shared by the tcgen05 kernels (sm_103a): shared-memory
// matrix descriptors, instruction descriptors, operand layouts, the TF32 and
// BF16 splits, MMA issue, tensor-memory loads and stores, bounded mbarrier
// waits.  Included by the translation units that run tensor-core passes.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstdint>

namespace qd {
namespace {

constexpr int kTcN = 64;   // MMA N: classes per chunk (block kernel) or outputs (tile kernel)
constexpr int kTcK = 128;  // real K of a 64-dimensional block (64 members x re/im)
constexpr int kTcM = 128;  // MMA M
constexpr uint32_t kSpinLimit = 1u << 26;  // bounded mbarrier polls (default)

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

// Instruction descriptor: D = F32, A = B = TF32 (format 2) or BF16 (format 1),
// both K-major, M = 128, N = kTcN.
__host__ __device__ constexpr uint32_t tc_idesc(uint32_t fmt) {
    return (1u << 4) | (fmt << 7) | (fmt << 10) | ((uint32_t)(kTcN >> 3) << 17) | ((uint32_t)(kTcM >> 4) << 24);
}

// The same with an explicit N (a multiple of 16, 16 <= N <= 256).
__host__ __device__ constexpr uint32_t tc_idesc_n(uint32_t fmt, uint32_t n) {
    return (1u << 4) | (fmt << 7) | (fmt << 10) | ((n >> 3) << 17) | ((uint32_t)(kTcM >> 4) << 24);
}

// Byte offset of element (row, k) in a K-major no-swizzle operand with `rows`
// rows: 4-byte elements (4 per core-matrix row) ...
__host__ __device__ __forceinline__ uint32_t kmajor_off(uint32_t row, uint32_t k, uint32_t rows) {
    return (k >> 2) * (rows / 8) * 128 + (row >> 3) * 128 + (row & 7) * 16 + (k & 3) * 4;
}
// ... and 2-byte elements (8 per core-matrix row).
__host__ __device__ __forceinline__ uint32_t kmajor_off_h(uint32_t row, uint32_t k, uint32_t rows) {
    return (k >> 3) * (rows / 8) * 128 + (row >> 3) * 128 + (row & 7) * 16 + (k & 7) * 2;
}

// x rounded to nearest (ties to even) at TF32 precision (10 explicit
// significand bits).  Rounding, not truncation: the tensor core drops the
// low 13 bits of its TF32 inputs, so with a truncated hi part every lo part
// would have the sign of its value and each block would shrink the state by
// about 2^-22; with hi rounded, lo has either sign and the error is unbiased.
__host__ __device__ __forceinline__ uint32_t tf32_rne_bits(uint32_t u) {
    u += 0x0FFFu + ((u >> 13) & 1u);
    return u & 0xFFFFE000u;
}
__device__ __forceinline__ float tf32_hi(float x) { return __uint_as_float(tf32_rne_bits(__float_as_uint(x))); }

// Squared 2-norm of a class's members for the norm restoration of unitary
// blocks, accumulated without loss: each x^2 is split exactly into p + e
// (p = x*x, e = fma(x, x, -p), the TwoProduct of Dekker / Ogita-Rump-Oishi)
// and added to a binary32 Neumaier sum (s, c) whose compensation also
// collects the e's; the parts of a class are then combined by NormFF.
struct NormAcc {
    float s = 0.f, c = 0.f;
    __device__ __forceinline__ void add_sq(float x) {
        const float p = x * x;
        c += fmaf(x, x, -p);
        const float t = s + p;
        c += fabsf(s) >= fabsf(p) ? (s - t) + p : (p - t) + s;
        s = t;
    }
};

// A squared norm held as an unevaluated sum hi + lo of binary32 values
// (double-binary32): the partial sums (s, c) of the threads of a class are
// added with Knuth's TwoSum, so the total keeps about twice the binary32
// significand -- as accurate as binary64 for these sums, without the
// binary64 pipe (1/64 of the FP32 rate on this part).
struct NormFF {
    float hi = 0.f, lo = 0.f;
    __device__ __forceinline__ void add(float s, float c) {
        const float t = hi + s;
        const float bb = t - hi;
        lo += ((hi - (t - bb)) + (s - bb)) + c;
        hi = t;
    }
};

// Restoration factor c = sqrt(ni / no) - 1 of a class with squared norms ni
// (input) and no (output).  The difference ni - no carries the whole
// information and is formed from the double-binary32 sums without loss
// (ni.hi - no.hi is exact when the two are within a factor 2); delta =
// (ni - no) / no is then needed to binary32 precision only, and
// sqrt(1 + delta) - 1 = delta / 2 - delta^2 / 8 + O(delta^3) (|delta| is
// about 1e-6 for the tensor cores' accumulation bias).
__device__ __forceinline__ float norm_fix(const NormFF& ni, const NormFF& no) {
    if (!(ni.hi > 0.f) || !(no.hi > 0.f)) return 0.f;
    const float delta = ((ni.hi - no.hi) + (ni.lo - no.lo)) / no.hi;
    if (fabsf(delta) > 1e-2f) return sqrtf(1.f + delta) - 1.f;
    return delta * fmaf(-0.125f, delta, 0.5f);
}

__device__ __forceinline__ void mma_bf16(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                         uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}"
        :
        : "r"(tmem_d), "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate));
}

// bf16 hi / lo parts of two floats, packed in one 32-bit word each (x0 in
// the low half): hi = bf16(x) and lo = bf16(x - hi), both rounded to
// nearest even, two values per conversion instruction.
__device__ __forceinline__ void bf16_split2(float x0, float x1, uint32_t& hi, uint32_t& lo) {
    const __nv_bfloat162 h = __floats2bfloat162_rn(x0, x1);
    const float2 hf = __bfloat1622float2(h);
    const __nv_bfloat162 l = __floats2bfloat162_rn(x0 - hf.x, x1 - hf.y);
    hi = *reinterpret_cast<const uint32_t*>(&h);
    lo = *reinterpret_cast<const uint32_t*>(&l);
}

// ... and of four floats (element k in the low half, k + 1 in the high half).
__device__ __forceinline__ void bf16_split4(float x0, float x1, float x2, float x3, uint2& hi, uint2& lo) {
    bf16_split2(x0, x1, hi.x, lo.x);
    bf16_split2(x2, x3, hi.y, lo.y);
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

// BF16 MMA with the A operand in tensor memory (lane = row of A, 32-bit
// column = two consecutive K elements, the lower K index in the low half).
__device__ __forceinline__ void mma_bf16_ta(uint32_t tmem_d, uint32_t tmem_a, uint64_t bdesc, uint32_t idesc,
                                            uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], [%1], %2, %3, p;\n\t}"
        :
        : "r"(tmem_d), "r"(tmem_a), "l"(bdesc), "r"(idesc), "r"(accumulate));
}

__device__ __forceinline__ void tmem_st4u(uint32_t taddr, uint32_t v0, uint32_t v1, uint32_t v2, uint32_t v3) {
    asm volatile("tcgen05.st.sync.aligned.32x32b.x4.b32 [%0], {%1, %2, %3, %4};" ::"r"(taddr), "r"(v0), "r"(v1),
                 "r"(v2), "r"(v3));
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

__device__ __forceinline__ bool mbar_wait(uint32_t mbar, uint32_t phase, uint32_t limit = kSpinLimit) {
    for (uint32_t it = 0; it < limit; ++it) {
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

// Bounded wait whose polls suspend the thread (up to hint_ns per poll) until
// the phase completes, instead of spinning on the issue slots.
__device__ __forceinline__ bool mbar_wait_sleep(uint32_t mbar, uint32_t phase, uint32_t limit,
                                                uint32_t hint_ns = 1000) {
    for (uint32_t it = 0; it < limit; ++it) {
        uint32_t done;
        asm volatile(
            "{\n\t.reg .pred P;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 P, [%1], %2, %3;\n\t"
            "selp.b32 %0, 1, 0, P;\n\t}"
            : "=r"(done)
            : "r"(mbar), "r"(phase), "r"(hint_ns));
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

__device__ __forceinline__ void tmem_st16(uint32_t taddr, const float* v) {
    asm volatile(
        "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], "
        "{%1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, %16};"
        :
        : "r"(taddr), "r"(__float_as_uint(v[0])), "r"(__float_as_uint(v[1])), "r"(__float_as_uint(v[2])),
          "r"(__float_as_uint(v[3])), "r"(__float_as_uint(v[4])), "r"(__float_as_uint(v[5])),
          "r"(__float_as_uint(v[6])), "r"(__float_as_uint(v[7])), "r"(__float_as_uint(v[8])),
          "r"(__float_as_uint(v[9])), "r"(__float_as_uint(v[10])), "r"(__float_as_uint(v[11])),
          "r"(__float_as_uint(v[12])), "r"(__float_as_uint(v[13])), "r"(__float_as_uint(v[14])),
          "r"(__float_as_uint(v[15])));
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float* v) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
        "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

}  // namespace
}  // namespace qd
