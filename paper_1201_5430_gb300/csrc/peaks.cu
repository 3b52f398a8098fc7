// Throughput probes of the pipes the kernels of this library are bound by, so that
// the roofline fractions divide by rates measured on the running GPU at its
// current clocks (no clock is set or locked here):
//   FP32 FMA (scalar fmaf and packed FP32x2 __ffma2_rn: the near-field pair loop
//   uses the packed form), the SFU (rsqrt.approx, one MUFU operation each), and the
//   tensor pipe (tcgen05.mma TF32 and BF16, tc_gemm.cu).
// Every probe runs register- or shared-memory-resident loops with no global
// traffic; work per launch is counted exactly from the loop trip counts.
#include <cuda_runtime.h>

#include <algorithm>
#include <vector>

#include "lhv_internal.cuh"

namespace lhv {

double tc_peak_launch(int iters, int bf16, int* err, cudaStream_t s);  // tc_gemm.cu

namespace {

constexpr int PK_THREADS = 256;
constexpr int PK_CHAINS = 8;   // independent dependency chains per thread
constexpr int PK_UNROLL = 16;  // operations per chain per loop trip

// a <- a m + c in PK_CHAINS chains; 2 flops per lane per fma
__global__ void __launch_bounds__(PK_THREADS) k_peak_ffma(int iters, float m, float c, float* sink) {
    float a[PK_CHAINS];
#pragma unroll
    for (int k = 0; k < PK_CHAINS; ++k) a[k] = 1.0f + 1e-3f * (float)(threadIdx.x + k);
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int u = 0; u < PK_UNROLL; ++u)
#pragma unroll
            for (int k = 0; k < PK_CHAINS; ++k) a[k] = fmaf(a[k], m, c);
    }
    float s = 0.0f;
#pragma unroll
    for (int k = 0; k < PK_CHAINS; ++k) s += a[k];
    if (s == -1.0f) sink[threadIdx.x] = s;  // never taken for the arguments used; keeps the chains live
}

// the same with packed FP32x2 operands: 4 flops per lane per instruction
__global__ void __launch_bounds__(PK_THREADS) k_peak_ffma2(int iters, float m, float c, float* sink) {
    float2 a[PK_CHAINS];
    const float2 m2 = make_float2(m, m), c2 = make_float2(c, c);
#pragma unroll
    for (int k = 0; k < PK_CHAINS; ++k) a[k] = make_float2(1.0f + 1e-3f * (float)(threadIdx.x + k), 1.5f);
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int u = 0; u < PK_UNROLL; ++u)
#pragma unroll
            for (int k = 0; k < PK_CHAINS; ++k) a[k] = __ffma2_rn(a[k], m2, c2);
    }
    float s = 0.0f;
#pragma unroll
    for (int k = 0; k < PK_CHAINS; ++k) s += a[k].x + a[k].y;
    if (s == -1.0f) sink[threadIdx.x] = s;
}

// a <- rsqrt(a): one MUFU operation per step (the chains settle at 1 and stay finite)
__global__ void __launch_bounds__(PK_THREADS) k_peak_mufu(int iters, float* sink) {
    float a[PK_CHAINS];
#pragma unroll
    for (int k = 0; k < PK_CHAINS; ++k) a[k] = 2.0f + 1e-3f * (float)(threadIdx.x + k);
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int u = 0; u < PK_UNROLL; ++u)
#pragma unroll
            for (int k = 0; k < PK_CHAINS; ++k) asm volatile("rsqrt.approx.ftz.f32 %0, %0;" : "+f"(a[k]));
    }
    float s = 0.0f;
#pragma unroll
    for (int k = 0; k < PK_CHAINS; ++k) s += a[k];
    if (s == -1.0f) sink[threadIdx.x] = s;
}

}  // namespace
}  // namespace lhv

extern "C" int lhv_peak_probe(int what, int iters, int reps, void* cuda_stream, double* rate_out, double* ms_out) {
    using namespace lhv;
    if (!rate_out || iters < 1 || reps < 1 || what < LHV_PEAK_FFMA || what > LHV_PEAK_BF16_MMA) return LHV_EINVAL;
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    if (cudaPeekAtLastError() != cudaSuccess) return LHV_ECUDA;
    int dev = 0, sms = 152;
    if (cudaGetDevice(&dev) != cudaSuccess) return LHV_ECUDA;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    float* sink = nullptr;
    if (cudaMalloc(&sink, PK_THREADS * sizeof(float) + 64) != cudaSuccess) {
        cudaGetLastError();
        return LHV_ENOMEM;
    }
    int* err = reinterpret_cast<int*>(reinterpret_cast<char*>(sink) + PK_THREADS * sizeof(float));
    cudaMemsetAsync(err, 0, sizeof(int), s);
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    int per_sm = 1;
    const void* kern = what == LHV_PEAK_FFMA ? (const void*)k_peak_ffma
                       : what == LHV_PEAK_FFMA2 ? (const void*)k_peak_ffma2 : (const void*)k_peak_mufu;
    if (what <= LHV_PEAK_MUFU) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, PK_THREADS, 0);
    const int grid = sms * std::max(per_sm, 1);
    const double ops_per_thread = (double)iters * PK_UNROLL * PK_CHAINS;
    double work = 0.0;
    auto launch = [&]() {
        switch (what) {
            case LHV_PEAK_FFMA:
                k_peak_ffma<<<grid, PK_THREADS, 0, s>>>(iters, 0.999999f, 1e-7f, sink);
                work = 2.0 * ops_per_thread * grid * PK_THREADS;
                break;
            case LHV_PEAK_FFMA2:
                k_peak_ffma2<<<grid, PK_THREADS, 0, s>>>(iters, 0.999999f, 1e-7f, sink);
                work = 4.0 * ops_per_thread * grid * PK_THREADS;
                break;
            case LHV_PEAK_MUFU:
                k_peak_mufu<<<grid, PK_THREADS, 0, s>>>(iters, sink);
                work = ops_per_thread * grid * PK_THREADS;
                break;
            default:
                work = tc_peak_launch(iters, what == LHV_PEAK_BF16_MMA ? 1 : 0, err, s);
                break;
        }
    };
    launch();  // warm-up
    std::vector<float> ms(reps);
    for (int r = 0; r < reps; ++r) {
        cudaEventRecord(e0, s);
        launch();
        cudaEventRecord(e1, s);
        cudaEventSynchronize(e1);
        cudaEventElapsedTime(&ms[r], e0, e1);
    }
    int herr = 0;
    const cudaError_t ce = cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, s);
    const cudaError_t se = cudaStreamSynchronize(s);
    const cudaError_t le = cudaGetLastError();
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(sink);
    if (ce != cudaSuccess || se != cudaSuccess || le != cudaSuccess) return LHV_ECUDA;
    if (herr) return LHV_ETIMEOUT;
    std::sort(ms.begin(), ms.end());
    const double med = ms[reps / 2];
    *rate_out = med > 0.0 ? work / (med * 1e-3) : 0.0;
    if (ms_out) *ms_out = med;
    return LHV_OK;
}
