// qd_norm_noalloc: the squared norm of caller-owned device amplitudes with
// no allocation at all (see its declaration in include/qudit.h).
//
// Who needs this: code that must not call cudaMalloc -- for example a
// framework whose caching allocator owns all device memory and forbids side
// allocations, or a latency-critical loop that cannot afford the
// device-wide synchronisation an allocation can trigger.  qd_norm needs a qd_state, and creating one allocates a
// reduction workspace; this entry point instead keeps that workspace in a
// fixed file-scope device array.
//
// The array holds one compensated partial sum (two doubles) per thread block
// of the first reduction pass.  The pass launches at most
// QD_NORM_NOALLOC_BLOCKS blocks (a grid-stride loop covers any state size),
// so 16 KiB per device suffice; every device that loads the library keeps
// these 16 KiB until the process exits.
#include <mutex>

#include "qd_internal.cuh"
#include "qudit.h"

namespace qd {
void set_last_error(const char* msg);
}

namespace {

static __device__ __align__(256) double g_norm_scratch[2 * QD_NORM_NOALLOC_BLOCKS];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
double* g_scratch[kMaxDevices] = {nullptr};

// Device address of the scratch array on the current device.  The name
// g_norm_scratch in host code is only a host-side stand-in, so the address
// is looked up once per device, with that device current.
qd_status scratch_for_current_device(double** out) {
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) {
        qd::set_last_error(cudaGetErrorString(e));
        return QD_ERR_CUDA;
    }
    if (dev < 0 || dev >= kMaxDevices) {
        qd::set_last_error("qd_norm_noalloc: device ordinal outside the supported range");
        return QD_ERR_UNSUPPORTED;
    }
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_scratch[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_norm_scratch);
        if (e != cudaSuccess || !p) {
            qd::set_last_error("qd_norm_noalloc: cudaGetSymbolAddress of the static scratch failed");
            return QD_ERR_CUDA;
        }
        g_scratch[dev] = static_cast<double*>(p);
    }
    *out = g_scratch[dev];
    return QD_OK;
}

}  // namespace

extern "C" qd_status qd_norm_noalloc(const void* dev_amps, int64_t num_amplitudes, int32_t prec, void* stream,
                                     double* dev_out) {
    if (!dev_amps || !dev_out) {
        qd::set_last_error("qd_norm_noalloc: dev_amps or dev_out is NULL");
        return QD_ERR_ARG;
    }
    if (prec != QD_C64 && prec != QD_C128) {
        qd::set_last_error("qd_norm_noalloc: unknown precision");
        return QD_ERR_ARG;
    }
    const uintptr_t align = prec == QD_C64 ? 8 : 16;
    if (reinterpret_cast<uintptr_t>(dev_amps) % align != 0 || reinterpret_cast<uintptr_t>(dev_out) % 8 != 0) {
        qd::set_last_error("qd_norm_noalloc: misaligned dev_amps or dev_out");
        return QD_ERR_ARG;
    }
    if (num_amplitudes < 1 || num_amplitudes > QD_NORM_NOALLOC_MAX_AMPLITUDES) {
        qd::set_last_error("qd_norm_noalloc: number of amplitudes outside [1, QD_NORM_NOALLOC_MAX_AMPLITUDES]");
        return QD_ERR_ARG;
    }
    // reduce_blocks never returns more than 1024 blocks, which is what the
    // array holds; checked here so that a change there cannot overrun it
    const int nb = qd::reduce_blocks(num_amplitudes);
    if (nb > QD_NORM_NOALLOC_BLOCKS) {
        qd::set_last_error("qd_norm_noalloc: internal error: more partial sums than the static scratch holds");
        return QD_ERR_CUDA;
    }
    double* scratch = nullptr;
    qd_status rc = scratch_for_current_device(&scratch);
    if (rc != QD_OK) return rc;
    // Every partial that the final pass reads is written by this call's first
    // pass, so nothing left in the array by an earlier call is ever used.
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    cudaError_t e = prec == QD_C64 ? qd::launch_norm<float>(dev_amps, num_amplitudes, scratch, nb, dev_out, s)
                                   : qd::launch_norm<double>(dev_amps, num_amplitudes, scratch, nb, dev_out, s);
    if (e != cudaSuccess) {
        qd::set_last_error(cudaGetErrorString(e));
        return QD_ERR_CUDA;
    }
    return QD_OK;
}
