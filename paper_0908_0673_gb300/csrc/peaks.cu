// Measured arithmetic peaks for the roofline denominators: FP32 and FP64
// fused multiply-add throughput of this device, timed with CUDA events.
// (Memory bandwidth and tensor-core peaks come from separate measurements.)
#include "bem_internal.cuh"

namespace bem {

constexpr int PK_CHAINS = 8, PK_ITERS = 4096, PK_T = 256;

template <class R>
__global__ void __launch_bounds__(PK_T) k_fma_peak(R seed, R *out) {
    R a[PK_CHAINS];
#pragma unroll
    for (int c = 0; c < PK_CHAINS; c++) a[c] = seed + (R)(threadIdx.x + c);
    const R b = (R)0.999999, d = (R)1e-7;
    for (int i = 0; i < PK_ITERS; i++)
#pragma unroll
        for (int c = 0; c < PK_CHAINS; c++) a[c] = a[c] * b + d;
    R s = (R)0;
#pragma unroll
    for (int c = 0; c < PK_CHAINS; c++) s += a[c];
    if (s == (R)-1) out[0] = s;   // never true; keeps the chains alive
}

}  // namespace bem

using namespace bem;

extern "C" int bem_measure_peak(int kind, double *tflops, void *cuda_stream) {
    if (!tflops || (kind != 0 && kind != 1)) { set_error("bem_measure_peak: bad argument"); return BEM_EINVAL; }
    cudaStream_t s = (cudaStream_t)cuda_stream;
    int dev = 0, sms = 0;
    BEM_CUDA(cudaGetDevice(&dev));
    BEM_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    double *out = nullptr;
    BEM_CUDA(cudaMalloc(&out, sizeof(double)));
    cudaEvent_t e0, e1;
    BEM_CUDA(cudaEventCreate(&e0));
    BEM_CUDA(cudaEventCreate(&e1));
    const int blocks = sms * 8;
    float best = 1e30f;
    for (int rep = 0; rep < 5; rep++) {
        cudaEventRecord(e0, s);
        if (kind == 0) (k_fma_peak<float><<<blocks, PK_T, 0, s>>>(1.0f, (float *)out), ::bem::count_launch());
        else (k_fma_peak<double><<<blocks, PK_T, 0, s>>>(1.0, out), ::bem::count_launch());
        cudaEventRecord(e1, s);
        cudaEventSynchronize(e1);
        float t = 0.f;
        cudaEventElapsedTime(&t, e0, e1);
        if (rep > 0 && t < best) best = t;
    }
    cudaError_t e = cudaGetLastError();
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(out);
    if (e != cudaSuccess) return cuda_fail(e, "k_fma_peak", __FILE__, __LINE__);
    const double flops = 2.0 * (double)blocks * PK_T * PK_CHAINS * PK_ITERS;
    *tflops = flops / (best * 1e-3) / 1e12;
    return BEM_OK;
}
