// Measured arithmetic ceilings of the device, the denominators of the force
// kernel's roofline next to the nominal FP32 peak (SMs x 128 lanes x 2 x
// clock): register-only loops of independent FP32 FMA chains, scalar and
// FP32x2, and of the MUFU reciprocal square root the force kernel uses.
// Also the FP64 throughput and dependent-operation latencies that shape the
// hard part's Hermite kernel.
#include "p3t_internal.cuh"

namespace {

constexpr int PB = 256;   // threads per block
constexpr int CH = 16;    // independent chains per thread

__device__ __forceinline__ float rsqrt_ftz(float x)
{
    float r;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

// MODE 0: CH scalar FMAs per iteration; 1: CH/2 FP32x2 FMAs (CH FMAs);
// 2: CH reciprocal square roots.  One store per thread keeps the chains live.
template <int MODE>
__global__ void __launch_bounds__(PB) k_peak(float *out, int iters, float b, float c)
{
    float a[CH];
#pragma unroll
    for (int i = 0; i < CH; ++i) a[i] = 1.0f + 1e-3f * (threadIdx.x + i);
    for (int it = 0; it < iters; ++it) {
        if (MODE == 0) {
#pragma unroll
            for (int i = 0; i < CH; ++i) a[i] = fmaf(a[i], b, c);
        } else if (MODE == 1) {
#pragma unroll
            for (int i = 0; i < CH; i += 2) {
                const float2 v = __ffma2_rn(make_float2(a[i], a[i + 1]),
                                            make_float2(b, b), make_float2(c, c));
                a[i] = v.x;
                a[i + 1] = v.y;
            }
        } else {
#pragma unroll
            for (int i = 0; i < CH; ++i) a[i] = rsqrt_ftz(a[i]);
        }
    }
    float s = 0.0f;
#pragma unroll
    for (int i = 0; i < CH; ++i) s += a[i];
    out[blockIdx.x * PB + threadIdx.x] = s;
}

template <int MODE>
int time_loop(float *out, int blocks, int iters, cudaStream_t s,
              cudaEvent_t e0, cudaEvent_t e1, double *per_second)
{
    k_peak<MODE><<<blocks, PB, 0, s>>>(out, iters / 8 + 1, 1.0000001f, 1e-7f);
    P3T_CUDA_TRY(cudaEventRecord(e0, s));
    k_peak<MODE><<<blocks, PB, 0, s>>>(out, iters, 1.0000001f, 1e-7f);
    P3T_CUDA_TRY(cudaEventRecord(e1, s));
    P3T_CUDA_TRY(cudaEventSynchronize(e1));
    float ms = 0.0f;
    P3T_CUDA_TRY(cudaEventElapsedTime(&ms, e0, e1));
    const double ops = (double)blocks * PB * iters * CH;
    *per_second = ops / (ms * 1e-3);
    p3t_count_launches(2);
    return P3T_OK;
}

// FP64: MODE 0 independent DFMA chains on every SM (throughput); the
// latency kernel runs one warp through dependent operations: 0 add, 1
// division, 2 square root, timed with the SM clock.
__global__ void __launch_bounds__(PB) k_dfma(double *out, int iters, double b, double c)
{
    double a[CH];
#pragma unroll
    for (int i = 0; i < CH; ++i) a[i] = 1.0 + 1e-3 * (threadIdx.x + i);
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int i = 0; i < CH; ++i) a[i] = __fma_rn(a[i], b, c);
    }
    double s = 0.0;
#pragma unroll
    for (int i = 0; i < CH; ++i) s += a[i];
    out[blockIdx.x * PB + threadIdx.x] = s;
}

template <int OP>
__global__ void k_dlat(double *out, long long *cycles, int iters, double b)
{
    double x = 1.5 + 1e-9 * threadIdx.x;
    const long long t0 = clock64();
    for (int it = 0; it < iters; ++it) {
        if (OP == 0) x = __dadd_rn(x, b);
        if (OP == 1) x = __ddiv_rn(b, x);
        if (OP == 2) x = __dsqrt_rn(x);
    }
    const long long t1 = clock64();
    out[threadIdx.x] = x;
    if (threadIdx.x == 0) *cycles = t1 - t0;
}

template <int OP>
int time_latency(double *out, long long *cyc, double b, cudaStream_t s,
                 double *per_op)
{
    constexpr int iters = 4096;
    k_dlat<OP><<<1, 32, 0, s>>>(out, cyc, iters / 8, b);
    k_dlat<OP><<<1, 32, 0, s>>>(out, cyc, iters, b);
    long long h = 0;
    P3T_CUDA_TRY(cudaMemcpyAsync(&h, cyc, sizeof(h), cudaMemcpyDeviceToHost, s));
    P3T_CUDA_TRY(cudaStreamSynchronize(s));
    *per_op = (double)h / iters;
    p3t_count_launches(2);
    return P3T_OK;
}

}  // namespace

// FP64 figures that set the hard part's design: DFMA/s over all SMs, and the
// latency in SM cycles of one dependent add, division and square root.
extern "C" int p3t_fp64_peaks(double *dfma_ops, double *add_cycles,
                              double *div_cycles, double *sqrt_cycles)
{
    int dev = 0, sms = 0;
    P3T_CUDA_TRY(cudaGetDevice(&dev));
    P3T_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const int blocks = sms * 4;
    cudaStream_t s = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    double *out = nullptr;
    long long *cyc = nullptr;
    int rc = P3T_OK;
    double tp = 0.0, la = 0.0, ld = 0.0, ls = 0.0;
    if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess ||
        cudaMalloc((void **)&out, sizeof(double) * (size_t)blocks * PB) != cudaSuccess ||
        cudaMalloc((void **)&cyc, sizeof(long long)) != cudaSuccess)
        rc = P3T_ERR_CUDA;
    // about 10 ms at the B300's ~0.6 T DFMA/s
    const int iters = 1024;
    if (rc == P3T_OK) {
        k_dfma<<<blocks, PB, 0, s>>>(out, iters / 8, 1.0000001, 1e-7);
        if (cudaEventRecord(e0, s) != cudaSuccess) rc = P3T_ERR_CUDA;
        k_dfma<<<blocks, PB, 0, s>>>(out, iters, 1.0000001, 1e-7);
        p3t_count_launches(2);
        float ms = 0.0f;
        if (rc == P3T_OK && (cudaEventRecord(e1, s) != cudaSuccess ||
                             cudaEventSynchronize(e1) != cudaSuccess ||
                             cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess))
            rc = P3T_ERR_CUDA;
        if (rc == P3T_OK) tp = (double)blocks * PB * iters * CH / (ms * 1e-3);
    }
    if (rc == P3T_OK) rc = time_latency<0>(out, cyc, 1e-12, s, &la);
    if (rc == P3T_OK) rc = time_latency<1>(out, cyc, 1.0, s, &ld);
    if (rc == P3T_OK) rc = time_latency<2>(out, cyc, 0.0, s, &ls);
    if (out) cudaFree(out);
    if (cyc) cudaFree(cyc);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (s) cudaStreamDestroy(s);
    if (rc != P3T_OK) return rc;
    if (dfma_ops) *dfma_ops = tp;
    if (add_cycles) *add_cycles = la;
    if (div_cycles) *div_cycles = ld;
    if (sqrt_cycles) *sqrt_cycles = ls;
    return P3T_OK;
}

extern "C" int p3t_alu_peaks(double *fma_flops, double *fma2_flops,
                             double *rsqrt_ops)
{
    int dev = 0, sms = 0;
    P3T_CUDA_TRY(cudaGetDevice(&dev));
    P3T_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const int blocks = sms * 8;  // 2048 threads per SM
    cudaStream_t s = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    float *out = nullptr;
    int rc = P3T_OK;
    double fma = 0.0, fma2 = 0.0, rsq = 0.0;
    if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess ||
        cudaMalloc((void **)&out, sizeof(float) * (size_t)blocks * PB) != cudaSuccess)
        rc = P3T_ERR_CUDA;
    // about 10 ms per loop at the B300's rates (36 T FMA/s, 4.5 T rsqrt/s)
    if (rc == P3T_OK) rc = time_loop<0>(out, blocks, 65536, s, e0, e1, &fma);
    if (rc == P3T_OK) rc = time_loop<1>(out, blocks, 65536, s, e0, e1, &fma2);
    if (rc == P3T_OK) rc = time_loop<2>(out, blocks, 8192, s, e0, e1, &rsq);
    if (out) cudaFree(out);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (s) cudaStreamDestroy(s);
    if (rc != P3T_OK) return rc;
    if (fma_flops) *fma_flops = 2.0 * fma;
    if (fma2_flops) *fma2_flops = 2.0 * fma2;
    if (rsqrt_ops) *rsqrt_ops = rsq;
    return P3T_OK;
}
