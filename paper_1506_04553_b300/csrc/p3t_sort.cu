// Stable LSD radix sort of (63-bit Morton key, original index) pairs.
//
// Eight passes of 8-bit digits.  Each pass is three kernels:
//   rs_hist    per-tile digit histogram (tile = 2048 keys), digit-major
//              counts[d][tile]
//   rs_scan    one block per digit: exclusive scan of counts[d][*] over the
//              tiles, digit total
//   rs_scatter per tile: stable rank of every key among the keys of the same
//              digit (warp match + per-warp digit counters); the tile is
//              reordered by digit in shared memory and each digit's run is
//              written to base[d] + tile_offset[d][tile] + rank with
//              consecutive threads on consecutive positions
// Stability: a tile is split into 8 warp segments of 256 keys; inside a
// segment keys are handled in 8 rounds of 32 consecutive keys; the rank of a
// key counts equal digits in earlier segments, earlier rounds and lower lanes,
// i.e. exactly the equal-digit keys that precede it in memory.
// Traffic per pass and key: read 8 B (hist) + read 12 B + write 12 B.
#include "p3t_internal.cuh"

namespace {

constexpr int RS_THREADS = 256;
constexpr int RS_WARPS = RS_THREADS / 32;
constexpr int RS_ROUNDS = 8;                       // per warp segment
constexpr int RS_SEG = 32 * RS_ROUNDS;             // 256 keys per warp
constexpr int RS_TILE = RS_WARPS * RS_SEG;         // 2048 keys per block

// Digit of element i: a byte of its key, or (CL) a byte of the cluster of
// its original index.
template <bool CL>
__device__ __forceinline__ int rs_digit(u64 key, int val,
                                        const int *__restrict__ pclus,
                                        int shift)
{
    return CL ? ((pclus[val] >> shift) & 255) : (int)((key >> shift) & 255u);
}

template <bool CL>
__global__ void __launch_bounds__(RS_THREADS)
rs_hist(int n, const u64 *__restrict__ keys, const int *__restrict__ vals,
        const int *__restrict__ pclus, int shift, int ntiles,
        int *__restrict__ counts)
{
    __shared__ int hist[256];
    hist[threadIdx.x] = 0;
    __syncthreads();
    const int base = blockIdx.x * RS_TILE;
#pragma unroll
    for (int k = 0; k < RS_TILE / RS_THREADS; ++k) {
        int i = base + k * RS_THREADS + threadIdx.x;
        if (i < n)
            atomicAdd(&hist[rs_digit<CL>(CL ? 0ull : keys[i], CL ? vals[i] : 0,
                                         pclus, shift)], 1);
    }
    __syncthreads();
    counts[threadIdx.x * ntiles + blockIdx.x] = hist[threadIdx.x];
}

// Block-wide exclusive scan of one int per thread (256 threads).
__device__ __forceinline__ int block_excl_scan256(int v, int *total)
{
    __shared__ int wsum[RS_WARPS];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    int inc = warp_incl_scan(v);
    if (lane == 31) wsum[w] = inc;
    __syncthreads();
    if (w == 0) {
        int x = lane < RS_WARPS ? wsum[lane] : 0;
        int xi = warp_incl_scan(x);
        __syncwarp();
        if (lane < RS_WARPS) wsum[lane] = xi - x;
        if (lane == 31) *total = xi;
    }
    __syncthreads();
    int r = inc - v + wsum[w];
    __syncthreads();
    return r;
}

__global__ void __launch_bounds__(RS_THREADS)
rs_scan(int ntiles, int *__restrict__ counts, int *__restrict__ totals)
{
    __shared__ int tot;
    int *row = counts + (long long)blockIdx.x * ntiles;
    int carry = 0;
    for (int b = 0; b < ntiles; b += RS_THREADS) {
        int i = b + threadIdx.x;
        int v = i < ntiles ? row[i] : 0;
        int ex = block_excl_scan256(v, &tot);
        if (i < ntiles) row[i] = ex + carry;
        carry += tot;
        __syncthreads();
    }
    if (threadIdx.x == 0) totals[blockIdx.x] = carry;
}

template <bool CL>
__global__ void __launch_bounds__(RS_THREADS)
rs_scatter(int n, const u64 *__restrict__ kin, const int *__restrict__ vin,
           u64 *__restrict__ kout, int *__restrict__ vout,
           const int *__restrict__ pclus, int shift, int ntiles,
           const int *__restrict__ counts, const int *__restrict__ totals)
{
    __shared__ int tile_off[256];
    __shared__ int tile_start[256];  // first position of each digit in the tile
    __shared__ int whist[RS_WARPS][256];
    __shared__ u64 sk[RS_TILE];
    __shared__ int sv[RS_TILE];
    __shared__ int tot;
    const int t = threadIdx.x, lane = t & 31, w = t >> 5;
    // digit base = exclusive scan of the digit totals
    int dbase = block_excl_scan256(totals[t], &tot);
    tile_off[t] = dbase + counts[t * ntiles + blockIdx.x];
#pragma unroll
    for (int q = 0; q < RS_WARPS; ++q) whist[q][t] = 0;
    __syncthreads();

    const int seg = blockIdx.x * RS_TILE + w * RS_SEG;
    const unsigned lt = lanemask_lt();
    u64 k[RS_ROUNDS];
    int v[RS_ROUNDS], rank[RS_ROUNDS], dig[RS_ROUNDS];
#pragma unroll
    for (int r = 0; r < RS_ROUNDS; ++r) {
        int i = seg + r * 32 + lane;
        bool ok = i < n;
        k[r] = ok ? kin[i] : 0ull;
        v[r] = ok ? vin[i] : 0;
        int d = ok ? rs_digit<CL>(k[r], v[r], pclus, shift) : 256;
        unsigned peers = __match_any_sync(0xffffffffu, d);
        int leader = __ffs(peers) - 1;
        int prior = ok ? whist[w][d] : 0;
        __syncwarp();
        if (ok && lane == leader) whist[w][d] = prior + __popc(peers);
        __syncwarp();
        rank[r] = prior + __popc(peers & lt);
        dig[r] = d;
    }
    __syncthreads();
    // exclusive prefix over warps for digit t, then over digits
    int run = 0;
#pragma unroll
    for (int q = 0; q < RS_WARPS; ++q) {
        int c = whist[q][t];
        whist[q][t] = run;
        run += c;
    }
    const int start = block_excl_scan256(run, &tot);
    tile_start[t] = start;
    __syncthreads();
    // reorder the tile by digit (stable) in shared memory
#pragma unroll
    for (int r = 0; r < RS_ROUNDS; ++r) {
        int d = dig[r];
        if (d < 256) {
            int lp = tile_start[d] + whist[w][d] + rank[r];
            sk[lp] = k[r];
            sv[lp] = v[r];
        }
    }
    __syncthreads();
    // runs of equal digits to consecutive global positions
    const int cnt = min(RS_TILE, n - blockIdx.x * RS_TILE);
    for (int j = t; j < cnt; j += RS_THREADS) {
        const u64 kk = sk[j];
        const int vv = sv[j];
        const int d = rs_digit<CL>(kk, vv, pclus, shift);
        const int pos = tile_off[d] + (j - tile_start[d]);
        kout[pos] = kk;
        vout[pos] = vv;
    }
}

}  // namespace

// Sorts ctx->key_a / idx_a (n entries) in place (result in key_a / idx_a;
// key_b / idx_b are the ping-pong buffers).
int p3t_sort_keys(p3t_ctx *c, int n, cudaStream_t s)
{
    if (n <= 1) return P3T_OK;
    int ntiles = (n + RS_TILE - 1) / RS_TILE;
    if (ntiles > c->cap_tiles) return P3T_ERR_STATE;
    u64 *ka = c->key_a, *kb = c->key_b;
    int *va = c->idx_a, *vb = c->idx_b;
    for (int pass = 0; pass < 8; ++pass) {
        int shift = 8 * pass;
        rs_hist<false><<<ntiles, RS_THREADS, 0, s>>>(n, ka, va, nullptr, shift,
                                                      ntiles, c->rs_counts);
        rs_scan<<<256, RS_THREADS, 0, s>>>(ntiles, c->rs_counts, c->rs_totals);
        rs_scatter<false><<<ntiles, RS_THREADS, 0, s>>>(
            n, ka, va, kb, vb, nullptr, shift, ntiles, c->rs_counts,
            c->rs_totals);
        u64 *tk = ka; ka = kb; kb = tk;
        int *tv = va; va = vb; vb = tv;
    }
    p3t_count_launches(24);
    // 8 passes: the result is back in the _a buffers
    P3T_CUDA_TRY(cudaGetLastError());
    return P3T_OK;
}

int64_t p3t_sort_tiles(int64_t n) { return (n + RS_TILE - 1) / RS_TILE; }

// Stable passes on the cluster id (most significant), after the key passes:
// the result is ordered by (cluster, key, original index).
int p3t_sort_cluster_passes(p3t_ctx *c, int n, cudaStream_t s)
{
    int ntiles = (n + RS_TILE - 1) / RS_TILE;
    if (ntiles > c->cap_tiles) return P3T_ERR_STATE;
    int passes = 0;
    for (long long v = (long long)c->nclus - 1; v > 0; v >>= 8) ++passes;
    u64 *ka = c->key_a, *kb = c->key_b;
    int *va = c->idx_a, *vb = c->idx_b;
    for (int pass = 0; pass < passes; ++pass) {
        int shift = 8 * pass;
        rs_hist<true><<<ntiles, RS_THREADS, 0, s>>>(n, ka, va, c->pclus, shift,
                                                     ntiles, c->rs_counts);
        rs_scan<<<256, RS_THREADS, 0, s>>>(ntiles, c->rs_counts, c->rs_totals);
        rs_scatter<true><<<ntiles, RS_THREADS, 0, s>>>(
            n, ka, va, kb, vb, c->pclus, shift, ntiles, c->rs_counts,
            c->rs_totals);
        u64 *tk = ka; ka = kb; kb = tk;
        int *tv = va; va = vb; vb = tv;
    }
    p3t_count_launches(3 * passes);
    if (ka != c->key_a) {
        P3T_CUDA_TRY(cudaMemcpyAsync(c->key_a, ka, (size_t)n * sizeof(u64),
                                     cudaMemcpyDeviceToDevice, s));
        P3T_CUDA_TRY(cudaMemcpyAsync(c->idx_a, va, (size_t)n * sizeof(int),
                                     cudaMemcpyDeviceToDevice, s));
    }
    P3T_CUDA_TRY(cudaGetLastError());
    return P3T_OK;
}
