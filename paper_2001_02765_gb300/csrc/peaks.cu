// Calibration of the arithmetic pipes the roofline fractions divide by (not in
// the paper): sustained FP32 and FP64 fused multiply-add throughput and the
// FP32 special-function (base-2 logarithm) throughput of the current device,
// measured with CUDA events on a grid of 8 CTAs x 256 threads per SM, every
// thread running independent dependency chains so that issue, not latency,
// limits the rate.
#include "common.cuh"

#include <math.h>

namespace {

constexpr int PEAK_THREADS = 256;
constexpr int PEAK_CTAS_PER_SM = 8;
constexpr int PEAK_UNROLL = 16;

template <typename T, int CHAINS>
__global__ void __launch_bounds__(PEAK_THREADS) k_fma_peak(T *out, int iters, T a, T b)
{
    T x[CHAINS];
#pragma unroll
    for (int i = 0; i < CHAINS; ++i) x[i] = (T)(threadIdx.x & 31) * (T)1e-3 + (T)i;
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int k = 0; k < PEAK_UNROLL; ++k) {
#pragma unroll
            for (int i = 0; i < CHAINS; ++i) x[i] = fma(x[i], a, b);
        }
    }
    T s = 0;
#pragma unroll
    for (int i = 0; i < CHAINS; ++i) s += x[i];
    // never true for the arguments used; keeps the chains live
    if (s == (T)-1.0) out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

template <int CHAINS>
__global__ void __launch_bounds__(PEAK_THREADS) k_lg2_peak(float *out, int iters)
{
    float x[CHAINS];
#pragma unroll
    for (int i = 0; i < CHAINS; ++i) x[i] = 2.0f + (float)(threadIdx.x & 31) * 1e-3f + (float)i;
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int k = 0; k < PEAK_UNROLL; ++k) {
#pragma unroll
            // log2 of a value in [2, 16) stays in [1, 4): add 2 to stay in range
            for (int i = 0; i < CHAINS; ++i) x[i] = __log2f(x[i]) + 2.0f;
        }
    }
    float s = 0;
#pragma unroll
    for (int i = 0; i < CHAINS; ++i) s += x[i];
    if (s == -1.0f) out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

template <typename F>
sg_status time_best(F launch, int reps, float *best_ms)
{
    cudaEvent_t e0, e1;
    SG_CUDA_TRY(cudaEventCreate(&e0));
    SG_CUDA_TRY(cudaEventCreate(&e1));
    launch();  // warm-up
    cudaError_t err = cudaGetLastError();
    float best = 1e30f;
    for (int r = 0; r < reps && err == cudaSuccess; ++r) {
        cudaEventRecord(e0, 0);
        launch();
        cudaEventRecord(e1, 0);
        err = cudaEventSynchronize(e1);
        float ms = 0;
        if (err == cudaSuccess) err = cudaEventElapsedTime(&ms, e0, e1);
        if (ms < best) best = ms;
    }
    if (err == cudaSuccess) err = cudaGetLastError();
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    SG_CUDA_TRY(err);
    *best_ms = best;
    return SG_OK;
}

}  // namespace

extern "C" sg_status sg_alu_peak(int kind, double *ops_per_s)
{
    if (!ops_per_s || kind < 0 || kind > 2) {
        sg_set_last_error_message("sg_alu_peak: kind must be 0, 1 or 2 and ops_per_s non-NULL");
        return SG_EINVAL;
    }
    int dev = 0, nsm = 0;
    SG_CUDA_TRY(cudaGetDevice(&dev));
    SG_CUDA_TRY(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    const int grid = nsm * PEAK_CTAS_PER_SM;
    const double threads = (double)grid * PEAK_THREADS;
    void *out = nullptr;
    SG_CUDA_TRY(cudaMalloc(&out, (size_t)grid * PEAK_THREADS * sizeof(double)));
    float ms = 0;
    double ops = 0;
    sg_status s = SG_OK;
    if (kind == SG_PEAK_FP64_FMA) {
        constexpr int C = 8;
        const int iters = 64;
        s = time_best([&] { k_fma_peak<double, C><<<grid, PEAK_THREADS>>>((double *)out, iters, 0.999999, 1e-7); },
                      5, &ms);
        ops = 2.0 * C * PEAK_UNROLL * (double)iters * threads;
    } else if (kind == SG_PEAK_FP32_FMA) {
        constexpr int C = 8;
        const int iters = 2048;
        s = time_best([&] { k_fma_peak<float, C><<<grid, PEAK_THREADS>>>((float *)out, iters, 0.9999f, 1e-5f); }, 5,
                      &ms);
        ops = 2.0 * C * PEAK_UNROLL * (double)iters * threads;
    } else {
        constexpr int C = 8;
        const int iters = 256;
        s = time_best([&] { k_lg2_peak<C><<<grid, PEAK_THREADS>>>((float *)out, iters); }, 5, &ms);
        ops = (double)C * PEAK_UNROLL * (double)iters * threads;
    }
    cudaFree(out);
    if (s != SG_OK) return s;
    *ops_per_s = ops / (ms * 1e-3);
    return SG_OK;
}
