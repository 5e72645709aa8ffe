// Arithmetic-rate probe: the FP64 or FP32 FMA throughput this GPU sustains at its current clocks, the denominator of
// the roofline fractions of the ALU-bound kernels.  Each thread runs 8 independent FMA chains (enough to cover the
// pipe latency) over a grid of 152 SMs x 8 blocks x 256 threads; the chains' results are summed into one word so
// the compiler keeps every FMA.
#include "evap_internal.cuh"

namespace evap {

template <typename T>
__global__ void __launch_bounds__(256) k_fma_probe(int iters, T a, T b, T* out) {
    T c[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) c[k] = T(threadIdx.x + k) * T(1e-3);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int k = 0; k < 8; ++k) c[k] = fma(c[k], a, b);
    }
    T s = 0;
#pragma unroll
    for (int k = 0; k < 8; ++k) s += c[k];
    if (s == T(12345.678)) out[0] = s;  // practically never taken; keeps the chains alive
}

}  // namespace evap

using namespace evap;

extern "C" int evap_fma_probe(int prec, double* tflops, void* stream) {
    if (!tflops || (prec != 32 && prec != 64)) {
        set_error("evap_fma_probe: prec must be 32 or 64 and tflops not NULL");
        return EVAP_EINVAL;
    }
    cudaStream_t s = (cudaStream_t)stream;
    const int blocks = 152 * 8, threads = 256;
    // about 50 ms of work at the nominal rates (FP64 1.25 TFLOP/s, FP32 80 TFLOP/s)
    const int iters = prec == 64 ? 4000 : 250000;
    void* out = nullptr;
    EVAP_CUDA(cudaMalloc(&out, sizeof(double)));
    cudaEvent_t e0, e1;
    EVAP_CUDA(cudaEventCreate(&e0));
    EVAP_CUDA(cudaEventCreate(&e1));
    float ms = 0.f;
    for (int rep = 0; rep < 2; ++rep) {  // the first launch warms up (clocks, module load)
        EVAP_CUDA(cudaEventRecord(e0, s));
        if (prec == 64)
            k_fma_probe<double><<<blocks, threads, 0, s>>>(iters, 0.999999, 1e-7, (double*)out);
        else
            k_fma_probe<float><<<blocks, threads, 0, s>>>(iters, 0.9999f, 1e-4f, (float*)out);
        EVAP_CHECK_LAUNCH("fma_probe");
        EVAP_CUDA(cudaEventRecord(e1, s));
        EVAP_CUDA(cudaEventSynchronize(e1));
        EVAP_CUDA(cudaEventElapsedTime(&ms, e0, e1));
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(out);
    const double flop = 2.0 * 8.0 * (double)iters * (double)blocks * threads;
    *tflops = flop / (ms * 1e-3) / 1e12;
    return EVAP_OK;
}
