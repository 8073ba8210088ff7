// Elementwise FP64 updates (kick, drift), energy reductions and the scan that
// turns per-particle neighbour counts into CSR offsets.
#include <cstring>
#include <mutex>

#include <climits>

#include "p3t_internal.cuh"

namespace {

constexpr int TB = 256;

// Velocity kick of Eq. 11 / Sect. 2.2: v <- v + dt * a (FP64, no FMA).
__global__ void __launch_bounds__(TB)
k_kick(long long n3, double *__restrict__ v, const float *__restrict__ a,
       double dt)
{
    for (long long i = blockIdx.x * (long long)TB + threadIdx.x; i < n3;
         i += (long long)gridDim.x * TB)
        v[i] = __dadd_rn(v[i], __dmul_rn(dt, (double)a[i]));
}

// Drift of Sect. 2.2 step 5: x <- x + dt * v (FP64, no FMA).
__global__ void __launch_bounds__(TB)
k_drift(long long n3, double *__restrict__ x, const double *__restrict__ v,
        double dt)
{
    for (long long i = blockIdx.x * (long long)TB + threadIdx.x; i < n3;
         i += (long long)gridDim.x * TB)
        x[i] = __dadd_rn(x[i], __dmul_rn(dt, v[i]));
}

__device__ __forceinline__ double block_sum(double v)
{
    __shared__ double ws[TB / 32];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (lane == 0) ws[w] = v;
    __syncthreads();
    double s = 0.0;
    if (threadIdx.x == 0)
        for (int q = 0; q < TB / 32; ++q) s += ws[q];
    __syncthreads();
    return s;
}

// Per-block partial sums of 1/2 m |v|^2 and 1/2 m phi.  The index is 64-bit:
// a thread's last increment may pass n by up to one grid stride.
__global__ void __launch_bounds__(TB)
k_energy_part(long long n, const double *__restrict__ m,
              const double *__restrict__ v, const double *__restrict__ phi,
              double *__restrict__ part)
{
    double ek = 0.0, ep = 0.0;
    const long long stride = (long long)gridDim.x * TB;
    for (long long i = (long long)blockIdx.x * TB + threadIdx.x; i < n; i += stride) {
        double vx = v[i], vy = v[n + i], vz = v[2 * n + i];
        ek += 0.5 * m[i] * (vx * vx + vy * vy + vz * vz);
        if (phi) ep += 0.5 * m[i] * phi[i];
    }
    double a = block_sum(ek);
    double b = block_sum(ep);
    if (threadIdx.x == 0) {
        part[2 * blockIdx.x] = a;
        part[2 * blockIdx.x + 1] = b;
    }
}

__global__ void k_energy_final(int nblk, const double *__restrict__ part,
                               double *__restrict__ out)
{
    if (threadIdx.x != 0) return;
    double a = 0.0, b = 0.0;
    for (int q = 0; q < nblk; ++q) {
        a += part[2 * q];
        b += part[2 * q + 1];
    }
    out[0] = a;
    out[1] = b;
}

// ---- exclusive scan int -> int64 (three phases) ----
constexpr int SC_T = 256;
constexpr int SC_ITEMS = 16;
constexpr int SC_TILE = SC_T * SC_ITEMS;

__device__ __forceinline__ long long block_excl_scan_ll(long long v,
                                                        long long *total)
{
    __shared__ long long ws[SC_T / 32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    long long inc = warp_incl_scan_ll(v);
    if (lane == 31) ws[w] = inc;
    __syncthreads();
    if (w == 0) {
        long long x = lane < SC_T / 32 ? ws[lane] : 0;
        long long xi = warp_incl_scan_ll(x);
        __syncwarp();
        if (lane < SC_T / 32) ws[lane] = xi - x;
        if (lane == 31) *total = xi;
    }
    __syncthreads();
    long long r = inc - v + ws[w];
    __syncthreads();
    return r;
}

__global__ void __launch_bounds__(SC_T)
k_scan_reduce(int n, const int *__restrict__ in, long long *__restrict__ part)
{
    __shared__ long long tot;
    long long s = 0;
    const int base = blockIdx.x * SC_TILE;
    for (int q = 0; q < SC_ITEMS; ++q) {
        int i = base + q * SC_T + threadIdx.x;
        if (i < n) s += in[i];
    }
    block_excl_scan_ll(s, &tot);
    if (threadIdx.x == 0) part[blockIdx.x] = tot;
}

__global__ void __launch_bounds__(SC_T)
k_scan_partials(int nb, long long *__restrict__ part)
{
    __shared__ long long tot;
    long long carry = 0;
    for (int b = 0; b < nb; b += SC_T) {
        int i = b + threadIdx.x;
        long long v = i < nb ? part[i] : 0;
        long long ex = block_excl_scan_ll(v, &tot);
        if (i < nb) part[i] = ex + carry;
        carry += tot;
        __syncthreads();
    }
    if (threadIdx.x == 0) part[nb] = carry;
}

__global__ void __launch_bounds__(SC_T)
k_scan_apply(int n, const int *__restrict__ in,
             const long long *__restrict__ part, long long *__restrict__ out,
             int nb)
{
    __shared__ long long tot;
    // thread t owns the SC_ITEMS consecutive items [base + t*ITEMS, ...)
    const int base = blockIdx.x * SC_TILE + threadIdx.x * SC_ITEMS;
    int v[SC_ITEMS];
    long long s = 0;
#pragma unroll
    for (int q = 0; q < SC_ITEMS; ++q) {
        int i = base + q;
        v[q] = i < n ? in[i] : 0;
        s += v[q];
    }
    long long ex = block_excl_scan_ll(s, &tot) + part[blockIdx.x];
#pragma unroll
    for (int q = 0; q < SC_ITEMS; ++q) {
        int i = base + q;
        if (i < n) out[i] = ex;
        ex += v[q];
    }
    if (blockIdx.x == nb - 1 && threadIdx.x == 0) out[n] = part[nb];
}

}  // namespace

int p3t_scan_ll(p3t_ctx *c, const int *in, long long *out, int n,
                cudaStream_t s)
{
    if (n == 0) {
        P3T_CUDA_TRY(cudaMemsetAsync(out, 0, sizeof(long long), s));
        return P3T_OK;
    }
    int nb = (n + SC_TILE - 1) / SC_TILE;
    if (nb + 1 > c->cap_scan) return P3T_ERR_STATE;
    k_scan_reduce<<<nb, SC_T, 0, s>>>(n, in, c->scan_part);
    k_scan_partials<<<1, SC_T, 0, s>>>(nb, c->scan_part);
    k_scan_apply<<<nb, SC_T, 0, s>>>(n, in, c->scan_part, out, nb);
    p3t_count_launches(3);
    P3T_CUDA_TRY(cudaGetLastError());
    return P3T_OK;
}

int64_t p3t_scan_blocks(int64_t n) { return (n + SC_TILE - 1) / SC_TILE; }

static int grid_for(long long n3)
{
    long long b = (n3 + TB - 1) / TB;
    if (b > 148 * 16) b = 148 * 16;
    if (b < 1) b = 1;
    return (int)b;
}

extern "C" int p3t_kick(int64_t n, double *vel, const float *acc, double dt,
                        void *stream)
{
    if (n < 0 || (n > 0 && (!vel || !acc))) return P3T_ERR_INVALID;
    if (n == 0) return P3T_OK;
    long long n3 = 3 * (long long)n;
    k_kick<<<grid_for(n3), TB, 0, (cudaStream_t)stream>>>(n3, vel, acc, dt);
    p3t_count_launches(1);
    P3T_CUDA_TRY(cudaGetLastError());
    return P3T_OK;
}

extern "C" int p3t_drift(int64_t n, double *pos, const double *vel, double dt,
                         void *stream)
{
    if (n < 0 || (n > 0 && (!pos || !vel))) return P3T_ERR_INVALID;
    if (n == 0) return P3T_OK;
    long long n3 = 3 * (long long)n;
    k_drift<<<grid_for(n3), TB, 0, (cudaStream_t)stream>>>(n3, pos, vel, dt);
    p3t_count_launches(1);
    P3T_CUDA_TRY(cudaGetLastError());
    return P3T_OK;
}

int p3t_energy_launch(p3t_ctx *c, long long n, const double *mass,
                      const double *vel, const double *pot, double *out,
                      cudaStream_t s)
{
    long long nb = (n + TB - 1) / TB;
    if (nb > c->sms * 4LL) nb = c->sms * 4LL;
    if (nb < 1) nb = 1;
    k_energy_part<<<(int)nb, TB, 0, s>>>(n, mass, vel, pot, c->red_part);
    k_energy_final<<<1, 32, 0, s>>>((int)nb, c->red_part, out);
    p3t_count_launches(2);
    P3T_CUDA_TRY(cudaGetLastError());
    return P3T_OK;
}

// ---- relative difference of two force fields (the autotuner's accuracy
// check) ----
// e_i = |a_i - r_i| / max(|r_i|, 1e-3 rms |r|): its maximum and a histogram
// of log10 e over [1e-12, 1e4) in 1/128 decade bins, from which the host
// reads the median (to 2 %).
constexpr int ERR_BINS = 2048;

__global__ void __launch_bounds__(TB)
k_err_sumsq(long long n, const float *__restrict__ r, double *__restrict__ part)
{
    double q = 0.0;
    const long long stride = (long long)gridDim.x * TB;
    for (long long i = (long long)blockIdx.x * TB + threadIdx.x; i < n; i += stride) {
        const double x = r[i], y = r[n + i], z = r[2 * n + i];
        q += x * x + y * y + z * z;
    }
    q = block_sum(q);
    if (threadIdx.x == 0) part[blockIdx.x] = q;
}

__global__ void __launch_bounds__(TB)
k_err_hist(long long n, const float *__restrict__ a, const float *__restrict__ r,
           const double *__restrict__ part, int nb,
           unsigned long long *__restrict__ hist, unsigned long long *__restrict__ emax)
{
    __shared__ double floor_s;
    if (threadIdx.x == 0) {
        double q = 0.0;
        for (int b = 0; b < nb; ++b) q += part[b];
        floor_s = 1e-3 * sqrt(q / (double)n);
    }
    __syncthreads();
    const double fl = floor_s;
    double mx = 0.0;
    const long long stride = (long long)gridDim.x * TB;
    for (long long i = (long long)blockIdx.x * TB + threadIdx.x; i < n; i += stride) {
        const double rx = r[i], ry = r[n + i], rz = r[2 * n + i];
        const double dx = (double)a[i] - rx, dy = (double)a[n + i] - ry,
                     dz = (double)a[2 * n + i] - rz;
        const double den = fmax(sqrt(rx * rx + ry * ry + rz * rz), fl);
        const double e = den > 0.0 ? sqrt(dx * dx + dy * dy + dz * dz) / den : 0.0;
        mx = fmax(mx, e);
        int b = e > 0.0 ? (int)floor((log10(e) + 12.0) * 128.0) : 0;
        b = b < 0 ? 0 : (b >= ERR_BINS ? ERR_BINS - 1 : b);
        atomicAdd(hist + b, 1ull);
    }
    // a non-negative double orders like its bit pattern
    atomicMax(emax, (unsigned long long)__double_as_longlong(mx));
}

// Median and maximum of e over n particles; scratch: device double[4 x SMs]
// + ERR_BINS + 1 unsigned long long (allocated by the caller).  Synchronises.
int p3t_force_err(p3t_ctx *c, long long n, const float *a, const float *r,
                  void *scratch, double *median, double *emax, cudaStream_t s)
{
    double *part = (double *)scratch;
    const int nb = c->sms * 4;
    unsigned long long *hist = (unsigned long long *)(part + nb);
    P3T_CUDA_TRY(cudaMemsetAsync(hist, 0, (ERR_BINS + 1) * sizeof(unsigned long long), s));
    k_err_sumsq<<<nb, TB, 0, s>>>(n, r, part);
    k_err_hist<<<nb, TB, 0, s>>>(n, a, r, part, nb, hist, hist + ERR_BINS);
    p3t_count_launches(2);
    P3T_CUDA_TRY(cudaGetLastError());
    unsigned long long h[ERR_BINS + 1];
    P3T_CUDA_TRY(cudaMemcpyAsync(h, hist, sizeof(h), cudaMemcpyDeviceToHost, s));
    P3T_CUDA_TRY(cudaStreamSynchronize(s));
    unsigned long long cum = 0;
    int b = 0;
    for (; b < ERR_BINS - 1; ++b) {
        cum += h[b];
        if (2 * cum >= (unsigned long long)n) break;
    }
    *median = pow(10.0, (b + 0.5) / 128.0 - 12.0);
    double m;
    memcpy(&m, &h[ERR_BINS], sizeof m);
    *emax = m;
    return P3T_OK;
}

size_t p3t_force_err_scratch(const p3t_ctx *c)
{
    return sizeof(double) * 4 * c->sms + sizeof(unsigned long long) * (ERR_BINS + 1);
}

// ---- energy sums without allocation -------------------------------------
// Block partials live in this file-scope device array instead of memory from
// cudaMalloc.  Host code must not pass the symbol itself to a kernel (on the
// host it names a host-side shadow, not device memory): the device address is
// looked up once per device with cudaGetSymbolAddress while that device is
// current, and that address is what the kernels receive.
static __device__ __align__(256) double
    g_energy_scratch[2 * P3T_ENERGY_NOALLOC_MAX_PARTIALS];

// The largest index k_energy_part forms is below n + (blocks x TB), with at
// most P3T_ENERGY_NOALLOC_MAX_PARTIALS blocks; it must fit its index type.
static_assert(P3T_ENERGY_NOALLOC_MAX_N
                  <= LLONG_MAX - (long long)P3T_ENERGY_NOALLOC_MAX_PARTIALS * TB,
              "k_energy_part's index can overflow");

namespace {
constexpr int kMaxDevices = 64;
std::mutex g_scratch_mutex;
double *g_scratch_ptr[kMaxDevices];
}  // namespace

static int energy_scratch(double **out)
{
    int dev = 0;
    P3T_CUDA_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDevices) return P3T_ERR_CUDA;
    std::lock_guard<std::mutex> lock(g_scratch_mutex);
    if (!g_scratch_ptr[dev]) {
        double *ptr = nullptr;
        P3T_CUDA_TRY(cudaGetSymbolAddress((void **)&ptr, g_energy_scratch));
        g_scratch_ptr[dev] = ptr;
    }
    *out = g_scratch_ptr[dev];
    return P3T_OK;
}

extern "C" int p3t_energy_noalloc(int64_t n, const double *mass,
                                  const double *vel, const double *pot,
                                  double *out, void *stream)
{
    if (n < 0 || !out || (n > 0 && (!mass || !vel))) return P3T_ERR_INVALID;
    if (n > P3T_ENERGY_NOALLOC_MAX_N) return P3T_ERR_CAPACITY;
    cudaStream_t s = (cudaStream_t)stream;
    double *scratch = nullptr;
    int rc = energy_scratch(&scratch);
    if (rc != P3T_OK) return rc;
    int dev = 0, sms = 0;
    P3T_CUDA_TRY(cudaGetDevice(&dev));
    P3T_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    long long nb = (n + TB - 1) / TB;
    if (nb > 4LL * sms) nb = 4LL * sms;
    if (nb < 1) nb = 1;
    if (nb > P3T_ENERGY_NOALLOC_MAX_PARTIALS) return P3T_ERR_CAPACITY;
    k_energy_part<<<(int)nb, TB, 0, s>>>((long long)n, mass, vel, pot, scratch);
    k_energy_final<<<1, 32, 0, s>>>((int)nb, scratch, out);
    p3t_count_launches(2);
    P3T_CUDA_TRY(cudaGetLastError());
    return P3T_OK;
}
