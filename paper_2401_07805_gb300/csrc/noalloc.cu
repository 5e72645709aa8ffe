// Allocation-free Jacobi diagonal.
//
// evap_jacobi_diagonal allocates its FP32 accumulator (and a cached double copy) with cudaMalloc on first use.
// Some callers cannot do that at the moment they need the diagonal: code whose device memory is owned by another
// allocator (a framework's memory pool that must see every byte), or code that must not let the library
// synchronize the device, which cudaMalloc and cudaFree may do.  evap_jacobi_diagonal_noalloc computes the same
// diagonal with the accumulator in a fixed array that is part of the loaded library image instead.
//
// The array below is a file-scope __device__ array: every GPU on which the library's kernels are loaded holds its
// EVAP_NOALLOC_DIAG_MAX floats (16 MiB) until the process exits.  In host code its name is only a host-side
// stand-in for the device symbol, so its device address is looked up once per device with cudaGetSymbolAddress
// (on the first call made with that device current) and passed to the kernels.
#include <mutex>

#include "evap_internal.cuh"

namespace {

constexpr int64_t kNoallocDiagMax = (int64_t)1 << 22;  // entries of the accumulator: 3 N_u must not exceed this
constexpr int kMaxDevices = 64;

__device__ __align__(256) float g_noalloc_diag[kNoallocDiagMax];

float* g_noalloc_ptr[kMaxDevices] = {};
std::mutex g_noalloc_mu;

}  // namespace

extern "C" int evap_jacobi_diagonal_noalloc(evap_handle h, double* diag, void* stream) {
    if (!h || !diag) {
        evap::set_error("evap_jacobi_diagonal_noalloc: null argument");
        return EVAP_EINVAL;
    }
    const int64_t n = 3 * h->m.Nu;
    if (n > kNoallocDiagMax) {
        evap::set_error("evap_jacobi_diagonal_noalloc: 3 N_u = " + std::to_string(n) +
                        " exceeds the static accumulator of " + std::to_string(kNoallocDiagMax) +
                        " entries; use evap_jacobi_diagonal");
        return EVAP_EINVAL;
    }
    if (!h->has_fields) {
        evap::set_error("evap_jacobi_diagonal_noalloc: call evap_set_fields first");
        return EVAP_ENOFIELDS;
    }
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return evap::cuda_fail("evap_jacobi_diagonal_noalloc: cudaGetDevice", e);
    if (dev != h->device || dev < 0 || dev >= kMaxDevices) {
        evap::set_error("evap_jacobi_diagonal_noalloc: the handle's device must be the current device");
        return EVAP_EINVAL;
    }
    float* acc = nullptr;
    {
        std::lock_guard<std::mutex> lock(g_noalloc_mu);
        if (!g_noalloc_ptr[dev]) {
            void* p = nullptr;
            e = cudaGetSymbolAddress(&p, g_noalloc_diag);
            if (e != cudaSuccess) return evap::cuda_fail("evap_jacobi_diagonal_noalloc: cudaGetSymbolAddress", e);
            g_noalloc_ptr[dev] = (float*)p;
        }
        acc = g_noalloc_ptr[dev];
    }
    return evap::launch_diagonal_into(h, acc, diag, (cudaStream_t)stream);
}
