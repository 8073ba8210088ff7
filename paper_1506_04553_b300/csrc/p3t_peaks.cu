// Measured arithmetic ceilings of the device, the denominators of the force
// kernel's roofline next to the nominal FP32 peak (SMs x 128 lanes x 2 x
// clock): register-only loops of independent FP32 FMA chains, scalar and
// FP32x2, and of the MUFU reciprocal square root the force kernel uses.
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

}  // namespace

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
