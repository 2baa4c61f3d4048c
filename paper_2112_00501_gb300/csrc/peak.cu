// Arithmetic-rate probe (no paper counterpart): the FP32 and FP64 fused
// multiply-add rates this GPU sustains, measured rather than derived from unit
// counts, so that the roofline of the arithmetic-bound kernels (the SAP
// smoother in FP32, the operator in FP64) divides by a rate taken on the same
// device, at the same clocks, in the same run.
//
// Every thread runs NCH independent FMA chains (enough independent work to
// cover the pipe latency at full occupancy); the grid puts eight 256-thread
// blocks on every SM; the rate is 2 flop x FMAs / event time of the fastest
// of a few launches.
#include "mgc_host.h"

namespace mgc {

static __device__ float g_peak_sink[256];

template <typename T, int NCH>
__global__ void __launch_bounds__(256) k_fma_rate(int iters, T a0, T m, T c)
{
    T a[NCH];
#pragma unroll
    for (int k = 0; k < NCH; ++k) a[k] = a0 + T(k) + T(1e-3) * T(threadIdx.x);
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int u = 0; u < 16; ++u)
#pragma unroll
            for (int k = 0; k < NCH; ++k) a[k] = fma(a[k], m, c);
    }
    T s = T(0);
#pragma unroll
    for (int k = 0; k < NCH; ++k) s += a[k];
    // never true for the arguments the host passes; keeps the chains alive
    if (s == T(-1.2345e30)) g_peak_sink[threadIdx.x] = (float)s;
}

template <typename T>
static int fma_rate(int iters, double *flops, cudaStream_t s)
{
    constexpr int NCH = 8;
    int dev = 0, sms = 0;
    MGC_CUDA(cudaGetDevice(&dev));
    MGC_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const int blocks = sms * 8;
    cudaEvent_t e0, e1;
    MGC_CUDA(cudaEventCreate(&e0));
    MGC_CUDA(cudaEventCreate(&e1));
    const T a0 = T(1), m = T(0.999999), c = T(1e-7);
    k_fma_rate<T, NCH><<<blocks, 256, 0, s>>>(iters / 8 + 1, a0, m, c);  // warm-up
    float best = 0.f;
    int st = MGC_OK;
    for (int rep = 0; rep < 5 && st == MGC_OK; ++rep) {
        cudaEventRecord(e0, s);
        k_fma_rate<T, NCH><<<blocks, 256, 0, s>>>(iters, a0, m, c);
        cudaEventRecord(e1, s);
        const cudaError_t e = cudaEventSynchronize(e1);
        if (e != cudaSuccess) {
            st = cuda_fail(e, "cudaEventSynchronize", __FILE__, __LINE__);
            break;
        }
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (rep == 0 || ms < best) best = ms;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (st != MGC_OK) return st;
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "k_fma_rate", __FILE__, __LINE__);
    count(6, 0.0);
    *flops = 2.0 * (double)blocks * 256.0 * (double)iters * 16.0 * NCH / (best * 1e-3);
    return MGC_OK;
}

int fma_peak(int prec, double *flops, cudaStream_t s)
{
    if (prec == 32) return fma_rate<float>(8192, flops, s);
    if (prec == 64) return fma_rate<double>(128, flops, s);
    return fail(MGC_ERR_INVALID_ARG, "mgc_fma_peak: prec must be 32 or 64");
}

}  // namespace mgc
