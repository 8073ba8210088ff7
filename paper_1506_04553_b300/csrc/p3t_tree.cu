// Tree construction (Sect. 2.2: Barnes-Hut tree up to the quadrupole moment).
//
//   bbox      root cube: componentwise min, largest extent, side =
//             extent * (1 + 2^-20) (1 when all particles coincide); input
//             validation (finite coordinates, finite positive masses)
//   keys      21-bit quantisation per axis, floor((x - lo) / side * 2^21)
//             with one FP64 rounding per operation, interleaved x-highest
//             into a 63-bit Morton key
//   (sort)    p3t_sort.cu
//   gather    Morton-ordered FP64 copies and the FP32 hi/lo split
//   split     level by level: a cell of level L < 21 holding more than n_leaf
//             particles gets its non-empty octants (found by binary search
//             on the sorted keys) as children, contiguous and in Morton order
//   moments   bottom-up in one launch (each internal cell by the last of
//             its children to finish): M, centre of mass, traceless
//             quadrupole Q_ab = sum m (3 d_a d_b - |d|^2 delta_ab) about the
//             centre of mass, member box; leaves from their particles,
//             internal cells from their children (parallel-axis shift) in
//             FP64; then the FP32 walk and force records
//   groups    chunks of n_group consecutive particles (Morton order) inside
//             containers: cells of at most 16 n_group particles whose parent
//             holds more (leaves of any size whose parent holds more)
#include <math.h>

#include "p3t_internal.cuh"

namespace {

constexpr int TB = 256;

// containers hold at most this many times n_group particles
#ifndef P3T_CONTAINER_FACTOR
#define P3T_CONTAINER_FACTOR 16
#endif

// ---------------------------------------------------------------- bbox ----
// Minima and maxima run on order-preserving integer images of the
// coordinates (ord64), so the reductions occupy the integer pipe, not the
// FP64 unit; finiteness is read from the exponent field.
// images of +inf and -inf: the neutral elements of min and max
constexpr long long ORD_HI = 0x7ff0000000000000LL;
constexpr long long ORD_LO = (long long)0x800fffffffffffffULL;

// Block-wide min of mn[3] and max of mx[3]; the result in thread 0.
__device__ __forceinline__ void block_minmax3(long long *mn, long long *mx)
{
#pragma unroll
    for (int a = 0; a < 3; ++a)
        for (int o = 16; o > 0; o >>= 1) {
            mn[a] = min(mn[a], __shfl_xor_sync(0xffffffffu, mn[a], o));
            mx[a] = max(mx[a], __shfl_xor_sync(0xffffffffu, mx[a], o));
        }
    __shared__ long long smn[3][TB / 32], smx[3][TB / 32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (lane == 0)
        for (int a = 0; a < 3; ++a) {
            smn[a][w] = mn[a];
            smx[a][w] = mx[a];
        }
    __syncthreads();
    if (threadIdx.x == 0)
        for (int a = 0; a < 3; ++a)
            for (int q = 1; q < TB / 32; ++q) {
                mn[a] = min(mn[a], smn[a][q]);
                mx[a] = max(mx[a], smx[a][q]);
            }
}

// Particles [b, e) with stride: box images and validity (finite
// coordinates, finite positive masses).
__device__ __forceinline__ bool scan_box(int b, int e, int stride, int n,
                                         const double *__restrict__ pos,
                                         const double *__restrict__ mass,
                                         long long *mn, long long *mx)
{
    bool bad = false;
    for (int i = b; i < e; i += stride) {
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            const double v = pos[(size_t)a * n + i];
            bad |= !finite64(v);
            const long long o = ord64(v);
            mn[a] = min(mn[a], o);
            mx[a] = max(mx[a], o);
        }
        const double m = mass[i];
        bad |= !(m > 0.0) || !finite64(m);
    }
    return bad;
}

__global__ void __launch_bounds__(TB)
k_bbox_partial(int n, const double *__restrict__ pos,
               const double *__restrict__ mass, double *__restrict__ part,
               P3TDevState *st)
{
    long long mn[3] = {ORD_HI, ORD_HI, ORD_HI}, mx[3] = {ORD_LO, ORD_LO, ORD_LO};
    const bool bad = scan_box(blockIdx.x * TB + threadIdx.x, n, gridDim.x * TB, n,
                              pos, mass, mn, mx);
    if (__syncthreads_or(bad) && threadIdx.x == 0) p3t_raise(st, P3T_ERR_INVALID);
    block_minmax3(mn, mx);
    if (threadIdx.x == 0)
        for (int a = 0; a < 3; ++a) {
            part[blockIdx.x * 6 + a] = unord64(mn[a]);
            part[blockIdx.x * 6 + 3 + a] = unord64(mx[a]);
        }
}

// Root cube from the box: side = largest extent (1 + 2^-20), 1 if zero.
__device__ __forceinline__ void root_cube(const long long *mn, const long long *mx,
                                          double *lo, double *size)
{
    double ext = 0.0;
    for (int a = 0; a < 3; ++a) {
        const double u = unord64(mn[a]), v = unord64(mx[a]);
        const double e = __dsub_rn(v, u);
        if (e > ext) ext = e;
        lo[a] = u;
    }
    *size = (ext == 0.0) ? 1.0 : __dmul_rn(ext, 1.0 + 0x1p-20);
}

__global__ void __launch_bounds__(TB)
k_bbox_final(int nblk, const double *__restrict__ part, P3TDevState *st,
             double *__restrict__ clus_box)
{
    long long mn[3] = {ORD_HI, ORD_HI, ORD_HI}, mx[3] = {ORD_LO, ORD_LO, ORD_LO};
    for (int b = threadIdx.x; b < nblk; b += TB)
        for (int a = 0; a < 3; ++a) {
            mn[a] = min(mn[a], ord64(part[6 * b + a]));
            mx[a] = max(mx[a], ord64(part[6 * b + 3 + a]));
        }
    block_minmax3(mn, mx);
    if (threadIdx.x != 0) return;
    double lo[3], size;
    root_cube(mn, mx, lo, &size);
    for (int a = 0; a < 3; ++a) {
        st->lo[a] = lo[a];
        clus_box[a] = lo[a];
    }
    st->size = size;
    clus_box[3] = size;
    clus_box[4] = __dmul_rn(__drcp_rn(size), 2097152.0);
}

// One block per cluster of an ensemble: root cube of [off[k], off[k+1])
// (same rule as for a single cluster) and input validation.
__global__ void __launch_bounds__(TB)
k_bbox_seg(const long long *__restrict__ off, int n,
           const double *__restrict__ pos, const double *__restrict__ mass,
           double *__restrict__ clus_box, P3TDevState *st)
{
    const int k = blockIdx.x;
    const int b = (int)off[k], e = (int)off[k + 1];
    long long mn[3] = {ORD_HI, ORD_HI, ORD_HI}, mx[3] = {ORD_LO, ORD_LO, ORD_LO};
    const bool bad = scan_box(b + threadIdx.x, e, TB, n, pos, mass, mn, mx);
    if (__syncthreads_or(bad) && threadIdx.x == 0) p3t_raise(st, P3T_ERR_INVALID);
    block_minmax3(mn, mx);
    if (threadIdx.x != 0) return;
    double lo[3], size;
    root_cube(mn, mx, lo, &size);
    for (int a = 0; a < 3; ++a) clus_box[8 * k + a] = lo[a];
    clus_box[8 * k + 3] = size;
    clus_box[8 * k + 4] = __dmul_rn(__drcp_rn(size), 2097152.0);
}

// Cluster of every particle (original index) of an ensemble.
__global__ void __launch_bounds__(TB)
k_cluster_ids(int n, int nc, const long long *__restrict__ off,
              int *__restrict__ pclus)
{
    int i = blockIdx.x * TB + threadIdx.x;
    if (i >= n) return;
    int lo = 0, hi = nc;  // off[lo] <= i < off[hi]
    while (hi - lo > 1) {
        int mid = (lo + hi) >> 1;
        if (off[mid] <= i)
            lo = mid;
        else
            hi = mid;
    }
    pclus[i] = lo;
}

// ---------------------------------------------------------------- keys ----
// floor(((x - lo) / size) 2^21), each operation rounded once, clamped to
// [0, 2^21 - 1].  The quotient is formed as v = t s21 with s21 = (1/size)
// 2^21 (an exact scaling of the rounded reciprocal): v differs from the
// rounded, scaled quotient by less than 2^-30, so their floors agree unless
// v lies within 2^-28 of an integer; there (rarely) the division itself
// decides.  The floor and the distance to the nearest integer are read from
// the bits of v with integer operations (0 <= v < 2^21 + 1), which keeps the
// FP64 unit to one subtraction and one multiplication per coordinate.
__device__ __forceinline__ u64 quantise(double x, double lo, double size,
                                        double s21)
{
    const double t = __dsub_rn(x, lo);  // >= 0: lo is the minimum
    const double v = __dmul_rn(t, s21);
    const long long b = __double_as_longlong(v);
    const int e = (int)((b >> 52) & 0x7ff) - 1023;
    long long q;
    bool near;
    if (b <= 0) {  // +0 or -0
        q = 0;
        near = true;
    } else if (e < 0) {  // (0, 1)
        q = 0;
        near = v < 0x1p-28 || v > 1.0 - 0x1p-28;
    } else if (e >= 21) {  // the exact quotient is below 2^21 and v below 2^21 + 1
        q = 2097151;
        near = false;
    } else {
        const int sh = 52 - e;  // fraction bits: 32 .. 52
        const long long m = (b & ((1LL << 52) - 1)) | (1LL << 52);
        q = m >> sh;
        const long long fb = m & ((1LL << sh) - 1), lim = 1LL << (sh - 28);
        near = fb < lim || fb > (1LL << sh) - lim;
    }
    if (near) q = __double2ll_rd(__dmul_rn(__ddiv_rn(t, size), 2097152.0));
    q = q < 0 ? 0 : q;
    q = q > 2097151 ? 2097151 : q;
    return (u64)q;
}

// Spreads the low 21 bits of v so that bit b lands on bit 3b.
__device__ __forceinline__ u64 spread3(u64 v)
{
    v &= 0x1fffffull;
    v = (v | (v << 32)) & 0x1f00000000ffffull;
    v = (v | (v << 16)) & 0x1f0000ff0000ffull;
    v = (v | (v << 8)) & 0x100f00f00f00f00full;
    v = (v | (v << 4)) & 0x10c30c30c30c30c3ull;
    v = (v | (v << 2)) & 0x1249249249249249ull;
    return v;
}

__global__ void __launch_bounds__(TB)
k_keys(int n, const double *__restrict__ pos, int nc,
       const int *__restrict__ pclus, const double *__restrict__ clus_box,
       u64 *__restrict__ key, int *__restrict__ idx)
{
    int i = blockIdx.x * TB + threadIdx.x;
    if (i >= n) return;
    const double *bx = clus_box + 8 * (nc > 1 ? pclus[i] : 0);
    const double size = bx[3], s21 = bx[4];
    u64 qx = quantise(pos[i], bx[0], size, s21);
    u64 qy = quantise(pos[(size_t)n + i], bx[1], size, s21);
    u64 qz = quantise(pos[2 * (size_t)n + i], bx[2], size, s21);
    key[i] = (spread3(qx) << 2) | (spread3(qy) << 1) | spread3(qz);
    idx[i] = i;
}

// -------------------------------------------------------------- gather ----
__global__ void __launch_bounds__(TB)
k_gather(int n, const int *__restrict__ sidx, const double *__restrict__ pos,
         const double *__restrict__ mass, int *__restrict__ order,
         double *__restrict__ xs, double *__restrict__ ms,
         float4 *__restrict__ phi, float4 *__restrict__ plo)
{
    int k = blockIdx.x * TB + threadIdx.x;
    if (k >= n) return;
    int i = sidx[k];
    order[k] = i;
    double x = pos[i], y = pos[(size_t)n + i], z = pos[2 * (size_t)n + i];
    double m = mass[i];
    xs[k] = x;
    xs[(size_t)n + k] = y;
    xs[2 * (size_t)n + k] = z;
    ms[k] = m;
    float xh = __double2float_rn(x), yh = __double2float_rn(y),
          zh = __double2float_rn(z);
    phi[k] = make_float4(xh, yh, zh, __double2float_rn(m));
    plo[k] = make_float4(__double2float_rn(x - (double)xh),
                         __double2float_rn(y - (double)yh),
                         __double2float_rn(z - (double)zh), 0.0f);
}

// --------------------------------------------------------------- split ----
// One root per cluster: cells 0 .. nc-1 are the roots, in cluster order
// (the sort keeps clusters contiguous and in order).
__global__ void k_tree_init(int nc, const long long *__restrict__ off,
                            int4 *node, int *parent, int *cpend, P3TDevState *st)
{
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < nc;
         k += gridDim.x * blockDim.x) {
        node[k] = make_int4((int)off[k], (int)(off[k + 1] - off[k]), -1, 0);
        parent[k] = -1;
        cpend[k] = 0;
    }
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    st->ncell = nc;
    st->ngroup = 0;
    st->max_level = 0;
    st->need_cells = 0;
    st->blocks_done = 0;
    st->max_stack = 0;
    st->level_start[0] = 0;
    for (int L = 1; L < P3T_MAX_LEVEL + 3; ++L) st->level_start[L] = nc;
    st->nleaf = 0;
    for (int b = 0; b < P3T_LEAF_BINS; ++b) st->leaf_bin[b] = st->leaf_fill[b] = 0;
    for (int b = 0; b < 256; ++b) st->gord_cnt[b] = st->gord_fill[b] = 0;
}

__device__ __forceinline__ int digit_at(u64 key, int L)
{
    return (int)((key >> (3 * (P3T_MAX_LEVEL - L))) & 7u);
}

// All seven child boundaries of the cell [lo, hi) at once: b[d] (d = 1..7)
// is the first position with digit_at >= d.  The seven 32-ary searches run
// side by side, each round issuing the probes of all of them before any is
// examined, so a round costs one memory latency (4 rounds for 2^20 keys).
__device__ __forceinline__ void warp_lower_digits7(const u64 *__restrict__ key,
                                                   int lo0, int hi0, int L,
                                                   int lane, int *b)
{
    int lo[8], hi[8];
#pragma unroll
    for (int d = 1; d < 8; ++d) {
        lo[d] = lo0;
        hi[d] = hi0;
    }
    for (int round = 0; round < 8; ++round) {  // 32^8 > 2^31: always enough
        bool more = false;
#pragma unroll
        for (int d = 1; d < 8; ++d) more |= hi[d] - lo[d] > 32;
        if (!more) break;
        int dg[8];
#pragma unroll
        for (int d = 1; d < 8; ++d) {
            const int step = (hi[d] - lo[d] + 31) / 32;
            const int p = lo[d] + lane * step;
            dg[d] = (hi[d] - lo[d] > 32 && p < hi[d]) ? digit_at(key[p], L) : 8;
        }
#pragma unroll
        for (int d = 1; d < 8; ++d) {
            if (hi[d] - lo[d] <= 32) continue;  // warp-uniform
            const int step = (hi[d] - lo[d] + 31) / 32;
            const int p = lo[d] + lane * step;
            const unsigned m = __ballot_sync(0xffffffffu, p < hi[d] && dg[d] >= d);
            const int f = m ? __ffs(m) - 1 : 32;
            const int lastv = (hi[d] - 1 - lo[d]) / step;
            const int nlo = f == 0 ? lo[d] : lo[d] + min(f - 1, lastv) * step + 1;
            const int nhi = f == 32 ? hi[d] : min(hi[d], lo[d] + f * step);
            lo[d] = nlo;
            hi[d] = nhi;
        }
    }
    int dg[8];
#pragma unroll
    for (int d = 1; d < 8; ++d) {
        const int p = lo[d] + lane;
        dg[d] = p < hi[d] ? digit_at(key[p], L) : 8;
    }
#pragma unroll
    for (int d = 1; d < 8; ++d) {
        const int p = lo[d] + lane;
        const unsigned m = __ballot_sync(0xffffffffu, p < hi[d] && dg[d] >= d);
        b[d] = m ? lo[d] + __ffs(m) - 1 : hi[d];
    }
}

// Child boundaries of the cell [lo, hi) by one warp reading its keys in
// coalesced chunks of 32: the digit at level L never decreases inside a cell,
// so b[d] (first position with digit >= d) is the position where the digit
// steps over d.  Each boundary is found by exactly one lane and written to
// the warp's sb[0..8); b[d] = hi for digits above the last one present.
__device__ __forceinline__ void warp_scan_digits(const u64 *__restrict__ key,
                                                 int lo, int hi, int L,
                                                 int *sb, int lane)
{
    constexpr int K = 8;  // chunks loaded before any is examined
    if (lane < 9) sb[lane] = hi;
    __syncwarp();
    int prev_last = 0;  // digits below the first key's are empty
    for (int base = lo; base < hi; base += 32 * K) {
        int dg[K];
#pragma unroll
        for (int u = 0; u < K; ++u) {
            const int p = base + 32 * u + lane;
            dg[u] = p < hi ? digit_at(key[p], L) : 7;
        }
#pragma unroll
        for (int u = 0; u < K; ++u) {
            const int p = base + 32 * u + lane;
            int prev = __shfl_up_sync(0xffffffffu, dg[u], 1);
            if (lane == 0) prev = prev_last;
            if (p < hi)
                for (int d = prev + 1; d <= dg[u]; ++d) sb[d] = p;
            prev_last = __shfl_sync(0xffffffffu, dg[u], 31);
        }
    }
    __syncwarp();
}

// Children of one cell (boundaries b[0..8]) appended to the cell arrays;
// children at the deepest level are never split and join the leaf list.
__device__ __forceinline__ void emit_children(int c, int L, int cap,
                                              const int *b, int4 *node,
                                              int *parent, int *cpend,
                                              int *leaf_list, P3TDevState *st)
{
    int k = 0;
#pragma unroll
    for (int d = 0; d < 8; ++d) k += b[d + 1] > b[d];
    int base = atomicAdd(&st->ncell, k);
    if (base + k > cap) {
        p3t_raise(st, P3T_ERR_CAPACITY);
        atomicMax(&st->need_cells, base + k);
        return;
    }
    int j = 0;
#pragma unroll
    for (int d = 0; d < 8; ++d) {
        if (b[d + 1] > b[d]) {
            node[base + j] = make_int4(b[d], b[d + 1] - b[d], -1, (L + 1) << 8);
            parent[base + j] = c;
            cpend[base + j] = 0;
            if (L + 1 >= P3T_MAX_LEVEL) leaf_list[atomicAdd(&st->nleaf, 1)] = base + j;
            ++j;
        }
    }
    node[c].z = base;
    node[c].w = (L << 8) | k;
}

// Above BIG_CELL particles a cell's child boundaries come from 32-ary
// searches (at most 5 rounds of loads at 2^20), below from one coalesced
// scan (at most 2 rounds of 8 x 32 keys); 512 took the split levels of a
// 2^20 build from 0.267 to 0.255 ms against 2048 (same-box A/B).
constexpr int BIG_CELL = 512;
// Blocks per SM of a split level: as many as stay resident (58 registers
// at 256 threads), so that a level runs in one wave; 4 took the split
// levels of a 2^20 build from 0.256 to 0.244 ms against 8 (2: 0.262, 3:
// 0.246, 16: 0.272; same-box A/B).
constexpr int SPLIT_BLOCKS_PER_SM = 4;

// Level L in two passes over its cells: one thread per cell files the
// cells holding at most n_leaf particles in the leaf list (one aggregated
// append per warp); then one warp per cell to split finds the child
// boundaries.
__global__ void __launch_bounds__(TB)
k_tree_split(int L, int n_leaf, int cap, const u64 *__restrict__ key,
             int4 *__restrict__ node, int *__restrict__ parent,
             int *__restrict__ cpend, int *__restrict__ leaf_list,
             P3TDevState *st)
{
    __shared__ int sbuf[TB / 32][9];
    const int beg = st->level_start[L], end = st->level_start[L + 1];
    const bool stop = st->error != 0 || L >= P3T_MAX_LEVEL;
    if (beg == end && !stop) {  // empty level: the next one is empty too
        if (blockIdx.x == 0 && threadIdx.x == 0) st->level_start[L + 2] = end;
        return;
    }
    const unsigned full = 0xffffffffu, lt = lanemask_lt();
    const int lane = threadIdx.x & 31;
    const int wg = (blockIdx.x * TB + threadIdx.x) >> 5;
    const int nw = gridDim.x * (TB / 32);
    int *sb = sbuf[threadIdx.x >> 5];
    for (int base = beg + 32 * wg; base < end && !stop; base += 32 * nw) {
        const int cl = base + lane;
        const int cnt = cl < end ? node[cl].y : -1;
        const unsigned lm = __ballot_sync(full, cnt >= 0 && cnt <= n_leaf);
        int lb = 0;
        if (lane == 0 && lm) lb = atomicAdd(&st->nleaf, __popc(lm));
        lb = __shfl_sync(full, lb, 0);
        if ((lm >> lane) & 1u) leaf_list[lb + __popc(lm & lt)] = cl;
    }
    for (int c = beg + wg; c < end && !stop; c += nw) {
        const int4 nd = node[c];
        if (nd.y <= n_leaf) continue;
        int b[9];
        b[0] = nd.x;
        b[8] = nd.x + nd.y;
        if (nd.y > BIG_CELL) {
            warp_lower_digits7(key, b[0], b[8], L + 1, lane, b);
        } else {
            warp_scan_digits(key, b[0], b[8], L + 1, sb, lane);
#pragma unroll
            for (int d = 1; d < 8; ++d) b[d] = sb[d];
            __syncwarp();  // sb is rewritten by the next cell
        }
        if (lane == 0) emit_children(c, L, cap, b, node, parent, cpend, leaf_list, st);
    }
    // the last block to finish closes the next level's range
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        unsigned t = atomicAdd(&st->blocks_done, 1u);
        if (t == gridDim.x - 1) {
            int nc = atomicAdd(&st->ncell, 0);
            if (nc > cap) nc = cap;
            st->level_start[L + 2] = nc;
            if (nc > st->level_start[L + 1]) st->max_level = L + 1;
            st->blocks_done = 0;
            __threadfence();
        }
    }
}

// ------------------------------------------------------- leaf ordering ----
// The leaves, largest first (a counting sort by size): the leaf moments take
// one thread per leaf, and a warp of equal sizes runs no idle iterations.
__device__ __forceinline__ int leaf_bin(int count)
{
    return P3T_LEAF_BINS - 1 - (count < P3T_LEAF_BINS - 1 ? count : P3T_LEAF_BINS - 1);
}

__global__ void __launch_bounds__(TB)
k_leaf_hist(const int *__restrict__ leaf_list, const int4 *__restrict__ node,
            P3TDevState *st)
{
    __shared__ int h[P3T_LEAF_BINS];
    for (int b = threadIdx.x; b < P3T_LEAF_BINS; b += TB) h[b] = 0;
    __syncthreads();
    const int nl = st->error ? 0 : st->nleaf;
    for (int q = blockIdx.x * TB + threadIdx.x; q < nl; q += gridDim.x * TB)
        atomicAdd(&h[leaf_bin(node[leaf_list[q]].y)], 1);
    __syncthreads();
    for (int b = threadIdx.x; b < P3T_LEAF_BINS; b += TB)
        if (h[b]) atomicAdd(&st->leaf_bin[b], h[b]);
}

__global__ void __launch_bounds__(TB)
k_leaf_scatter(const int *__restrict__ leaf_list, const int4 *__restrict__ node,
               int *__restrict__ leaf_sorted, P3TDevState *st)
{
    __shared__ int start[P3T_LEAF_BINS], cnt[P3T_LEAF_BINS], base[P3T_LEAF_BINS];
    const int nl = st->error ? 0 : st->nleaf;
    if (threadIdx.x == 0) {
        int run = 0;
        for (int b = 0; b < P3T_LEAF_BINS; ++b) {
            start[b] = run;
            run += st->leaf_bin[b];
        }
    }
    for (int q0 = blockIdx.x * TB; q0 < nl; q0 += gridDim.x * TB) {
        for (int b = threadIdx.x; b < P3T_LEAF_BINS; b += TB) cnt[b] = 0;
        __syncthreads();
        const int q = q0 + threadIdx.x;
        const int c = q < nl ? leaf_list[q] : -1;
        const int b = c >= 0 ? leaf_bin(node[c].y) : 0;
        const int rk = c >= 0 ? atomicAdd(&cnt[b], 1) : 0;
        __syncthreads();
        for (int k = threadIdx.x; k < P3T_LEAF_BINS; k += TB)
            if (cnt[k]) base[k] = start[k] + atomicAdd(&st->leaf_fill[k], cnt[k]);
        __syncthreads();
        if (c >= 0) leaf_sorted[base[b] + rk] = c;
        __syncthreads();
    }
}

// ------------------------------------------------------------- moments ----
// Writes the FP32 records of cell c from its FP64 moments.
__device__ __forceinline__ void write_records(
    int c, int4 nd, double M, const double *com, const double *Q,
    const double *bmn, const double *bmx, float4 *wmin, float4 *wmax,
    float4 *cf0, float4 *cf1, float4 *cf2)
{
    // .w: an internal cell's first child and number of children; a leaf's
    // first particle and minus its particle count, so that a walk finds a
    // leaf's range without a second, dependent load
    const bool leaf = (nd.w & 255) == 0;
    wmin[c] = make_float4(__double2float_rd(bmn[0]), __double2float_rd(bmn[1]),
                          __double2float_rd(bmn[2]),
                          __int_as_float(leaf ? nd.x : nd.z));
    wmax[c] = make_float4(__double2float_ru(bmx[0]), __double2float_ru(bmx[1]),
                          __double2float_ru(bmx[2]),
                          __int_as_float(leaf ? -nd.y : (nd.w & 255)));
    float ch[3], cl[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        ch[a] = __double2float_rn(com[a]);
        cl[a] = __double2float_rn(com[a] - (double)ch[a]);
    }
    cf0[c] = make_float4(ch[0], ch[1], ch[2], __double2float_rn(M));
    cf1[c] = make_float4(cl[0], cl[1], cl[2], __double2float_rn(Q[0]));
    cf2[c] = make_float4(__double2float_rn(Q[1]), __double2float_rn(Q[3]),
                         __double2float_rn(Q[4]), __double2float_rn(Q[5]));
}

// Moments of cell c (node nd), written to the FP64 arrays and the FP32
// records: a leaf from its particles, an internal cell from its children
// (parallel-axis shift).  The children's records are read through L2
// (__ldcg): another SM may have written them during this launch.
__device__ __forceinline__ double ld(const double *p) { return __ldcg(p); }

__device__ void cell_moments(int c, int4 nd, const double *__restrict__ xs,
                             const double *__restrict__ ms, int n,
                             double *cM, double *ccom, double *cQ,
                             double *cbmin, double *cbmax,
                             float4 *__restrict__ wmin, float4 *__restrict__ wmax,
                             float4 *__restrict__ cf0, float4 *__restrict__ cf1,
                             float4 *__restrict__ cf2)
{
    // Q = 3 S - tr(S) I with S = sum m d d^T about the centre of mass (plus,
    // for an internal cell, the children's own Q)
    double M = 0.0, com[3] = {0, 0, 0}, Q[6] = {0, 0, 0, 0, 0, 0};
    double S[6] = {0, 0, 0, 0, 0, 0};
    long long omn[3] = {ORD_HI, ORD_HI, ORD_HI};  // box images (ord64)
    long long omx[3] = {ORD_LO, ORD_LO, ORD_LO};
    const int nch = nd.w & 255;
    if (nch == 0) {
        // leaf: from its particles, in chunks of LCH whose loads are all
        // issued before the sums that wait on them
        constexpr int LCH = 8;
        const int k0 = nd.x, k1 = nd.x + nd.y;
        for (int kb = k0; kb < k1; kb += LCH) {
            double pm[LCH], px[LCH], py[LCH], pz[LCH];
#pragma unroll
            for (int u = 0; u < LCH; ++u) {
                const int k = kb + u < k1 ? kb + u : k0;
                pm[u] = ms[k];
                px[u] = xs[k];
                py[u] = xs[(size_t)n + k];
                pz[u] = xs[2 * (size_t)n + k];
            }
#pragma unroll
            for (int u = 0; u < LCH; ++u) {
                if (kb + u >= k1) continue;
                M += pm[u];
                com[0] += pm[u] * px[u];
                com[1] += pm[u] * py[u];
                com[2] += pm[u] * pz[u];
                const long long ox = ord64(px[u]), oy = ord64(py[u]), oz = ord64(pz[u]);
                omn[0] = min(omn[0], ox);
                omn[1] = min(omn[1], oy);
                omn[2] = min(omn[2], oz);
                omx[0] = max(omx[0], ox);
                omx[1] = max(omx[1], oy);
                omx[2] = max(omx[2], oz);
            }
        }
        const double iM = 1.0 / M;
#pragma unroll
        for (int a = 0; a < 3; ++a) com[a] *= iM;
        for (int kb = k0; kb < k1; kb += LCH) {
            double pm[LCH], px[LCH], py[LCH], pz[LCH];
#pragma unroll
            for (int u = 0; u < LCH; ++u) {
                const int k = kb + u < k1 ? kb + u : k0;
                pm[u] = ms[k];
                px[u] = xs[k];
                py[u] = xs[(size_t)n + k];
                pz[u] = xs[2 * (size_t)n + k];
            }
#pragma unroll
            for (int u = 0; u < LCH; ++u) {
                if (kb + u >= k1) continue;
                const double m = pm[u];
                const double dx = px[u] - com[0];
                const double dy = py[u] - com[1];
                const double dz = pz[u] - com[2];
                const double mx = m * dx, my = m * dy, mz = m * dz;
                S[0] = fma(mx, dx, S[0]);
                S[1] = fma(my, dy, S[1]);
                S[2] = fma(mz, dz, S[2]);
                S[3] = fma(mx, dy, S[3]);
                S[4] = fma(mx, dz, S[4]);
                S[5] = fma(my, dz, S[5]);
            }
        }
    } else {
        // internal: combine the children (parallel-axis shift); the
        // (at most 8) children's records are loaded before the sums
        double cm[8], cx[8], cy[8], cz[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            const int ch = nd.z + (q < nch ? q : 0);
            cm[q] = ld(cM + ch);
            cx[q] = ld(ccom + 3 * ch + 0);
            cy[q] = ld(ccom + 3 * ch + 1);
            cz[q] = ld(ccom + 3 * ch + 2);
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                omn[a] = min(omn[a], ord64(ld(cbmin + 3 * ch + a)));  // repeats child 0: harmless
                omx[a] = max(omx[a], ord64(ld(cbmax + 3 * ch + a)));
            }
        }
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            if (q >= nch) continue;
            M += cm[q];
            com[0] += cm[q] * cx[q];
            com[1] += cm[q] * cy[q];
            com[2] += cm[q] * cz[q];
        }
        const double iM = 1.0 / M;
#pragma unroll
        for (int a = 0; a < 3; ++a) com[a] *= iM;
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            if (q >= nch) continue;
            const int ch = nd.z + q;
            const double m = cm[q];
            const double dx = cx[q] - com[0];
            const double dy = cy[q] - com[1];
            const double dz = cz[q] - com[2];
            const double mx = m * dx, my = m * dy, mz = m * dz;
            S[0] = fma(mx, dx, S[0]);
            S[1] = fma(my, dy, S[1]);
            S[2] = fma(mz, dz, S[2]);
            S[3] = fma(mx, dy, S[3]);
            S[4] = fma(mx, dz, S[4]);
            S[5] = fma(my, dz, S[5]);
            const double *qc = cQ + 6 * ch;
#pragma unroll
            for (int v = 0; v < 6; ++v) Q[v] += ld(qc + v);
        }
    }
    {
        const double tr = S[0] + S[1] + S[2];
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            Q[a] += fma(3.0, S[a], -tr);
            Q[3 + a] += 3.0 * S[3 + a];
        }
    }
    double bmn[3], bmx[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        bmn[a] = unord64(omn[a]);
        bmx[a] = unord64(omx[a]);
    }
    cM[c] = M;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        ccom[3 * c + a] = com[a];
        cbmin[3 * c + a] = bmn[a];
        cbmax[3 * c + a] = bmx[a];
    }
#pragma unroll
    for (int q = 0; q < 6; ++q) cQ[6 * c + q] = Q[q];
    write_records(c, nd, M, com, Q, bmn, bmx, wmin, wmax, cf0, cf1, cf2);
}

// All moments in one launch, bottom-up: one thread per leaf (largest
// first) computes the leaf, then climbs.  At each parent it counts itself
// in (after a fence that publishes its cell); the last child to arrive
// computes the parent from all its children, in child order, and climbs on;
// the others stop.  Every cell is computed once, by whichever thread comes
// last, with the same arithmetic: the result does not depend on the order.
// Threads per block of k_moments_up.  A block stays resident until its
// slowest thread has climbed, so small blocks let finished threads' slots
// take new leaves sooner: 64 took the moments of a 2^20 build from 0.308 to
// 0.280 ms against 256 (same-box A/B).
constexpr int MB = 64;

__global__ void __launch_bounds__(MB)
k_moments_up(const double *__restrict__ xs, const double *__restrict__ ms,
             int n, const int4 *__restrict__ node, const int *__restrict__ parent,
             const int *__restrict__ leaf_sorted, int *cpend, double *cM,
             double *ccom, double *cQ, double *cbmin, double *cbmax,
             float4 *__restrict__ wmin, float4 *__restrict__ wmax,
             float4 *__restrict__ cf0, float4 *__restrict__ cf1,
             float4 *__restrict__ cf2, const P3TDevState *st)
{
    if (st->error) return;
    const int nl = st->nleaf;
    for (int q = blockIdx.x * MB + threadIdx.x; q < nl; q += gridDim.x * MB) {
        int c = leaf_sorted[q];
        cell_moments(c, node[c], xs, ms, n, cM, ccom, cQ, cbmin, cbmax, wmin,
                     wmax, cf0, cf1, cf2);
        for (int up = 0; up <= P3T_MAX_LEVEL; ++up) {  // at most one per level
            const int p = parent[c];
            if (p < 0) break;
            const int4 np = node[p];
            __threadfence();  // this cell's records before the count
            if (atomicAdd(cpend + p, 1) != (np.w & 255) - 1) break;
            __threadfence();  // the siblings' records after it
            cell_moments(p, np, xs, ms, n, cM, ccom, cQ, cbmin, cbmax, wmin,
                         wmax, cf0, cf1, cf2);
            c = p;
        }
    }
}

// -------------------------------------------------------------- groups ----
__device__ __forceinline__ void emit_group(int first, int count,
                                           int2 *grange, int &slot)
{
    grange[slot++] = make_int2(first, count);
}

__device__ __forceinline__ int chunks(int count, int ng)
{
    return (count + ng - 1) / ng;
}

// One thread per cell.  A container is a cell holding at most 16 n_group
// particles whose parent holds more (or a leaf whose parent holds more, or
// the root if it qualifies); its particles are cut into consecutive chunks of
// n_group in Morton order, the last one partial.
__global__ void __launch_bounds__(TB)
k_groups(int ng, int gcap, const int4 *__restrict__ node,
         const int *__restrict__ parent, int2 *__restrict__ grange,
         P3TDevState *st)
{
    if (st->error) return;
    const int ncell = st->ncell;
    const int cap = P3T_CONTAINER_FACTOR * ng;
    for (int c = blockIdx.x * TB + threadIdx.x; c < ncell;
         c += gridDim.x * TB) {
        const int4 nd = node[c];
        const bool small = nd.y <= cap || (nd.w & 255) == 0;
        if (!small) continue;
        if (parent[c] >= 0 && node[parent[c]].y <= cap) continue;
        const int k = chunks(nd.y, ng);
        int slot = atomicAdd(&st->ngroup, k);
        if (slot + k > gcap) {
            p3t_raise(st, P3T_ERR_STATE);
            continue;
        }
        for (int q = 0; q < k; ++q)
            emit_group(nd.x + q * ng, min(ng, nd.y - q * ng), grange, slot);
    }
}

// Group boxes (FP32 outward), relative origin and neighbour screening radius.
// gmin.w = hs2: squared screening radius; any pair of the group with
// |x_i - x_j| < h has an FP32 group-relative r^2 below hs2.
constexpr int GB = 1024;  // k_group_box: one warp per group, 32 groups per block

__global__ void __launch_bounds__(GB)
k_group_box(const int2 *__restrict__ grange, const double *__restrict__ xs,
            int n, int nc, const int *__restrict__ order,
            const int *__restrict__ pclus, const ClusterConsts *__restrict__ cc,
            int *__restrict__ gclus, float4 *__restrict__ gmin,
            float4 *__restrict__ gmax, float4 *__restrict__ gctr,
            const P3TDevState *st)
{
    __shared__ long long sbox[GB / 32][6];
    if (st->error) return;
    const int G = st->ngroup;  // <= capacity (k_groups checks)
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    // each warp the box of one group (lanes over its particles, integer
    // images); then warp 0 finishes the block's 32 groups, one per lane, so
    // that the FP64 tail is one set of instructions for 32 groups
    for (int g0 = blockIdx.x * (GB / 32); g0 < G; g0 += gridDim.x * (GB / 32)) {
        if (g0 + w < G) {
            const int2 rw = grange[g0 + w];
            long long omn[3] = {ORD_HI, ORD_HI, ORD_HI}, omx[3] = {ORD_LO, ORD_LO, ORD_LO};
            for (int k = rw.x + lane; k < rw.x + rw.y; k += 32)
#pragma unroll
                for (int a = 0; a < 3; ++a) {
                    const long long o = ord64(xs[(size_t)a * n + k]);
                    omn[a] = min(omn[a], o);
                    omx[a] = max(omx[a], o);
                }
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                for (int o = 16; o > 0; o >>= 1) {
                    omn[a] = min(omn[a], __shfl_xor_sync(0xffffffffu, omn[a], o));
                    omx[a] = max(omx[a], __shfl_xor_sync(0xffffffffu, omx[a], o));
                }
                if (lane == 0) {
                    sbox[w][a] = omn[a];
                    sbox[w][3 + a] = omx[a];
                }
            }
        }
        __syncthreads();
        if (w == 0 && g0 + lane < G) {
            const int g = g0 + lane;
            const int2 r = grange[g];
            long long omn[3], omx[3];
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                omn[a] = sbox[lane][a];
                omx[a] = sbox[lane][3 + a];
            }
            const int cl = nc > 1 ? pclus[order[r.x]] : 0;
            gclus[g] = cl;
            const double h = cc[cl].h;
            double mn[3], mx[3];
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                mn[a] = unord64(omn[a]);
                mx[a] = unord64(omx[a]);
            }
            float c[3];
            double R2 = 0.0, cabs = 0.0;
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                c[a] = __double2float_rn(0.5 * (mn[a] + mx[a]));
                double e = fmax(fabs(mx[a] - (double)c[a]), fabs(mn[a] - (double)c[a]));
                R2 += e * e;
                cabs = fmax(cabs, fabs((double)c[a]));
            }
            double R = sqrt(R2);
            // screening margin: 2^-14 h (R + h) + 2^-30 h |c| (>> the FP32
            // rounding of group-relative coordinates and of r^2)
            double hs2 = h * h + 0x1p-14 * h * (R + h) + 0x1p-30 * h * cabs;
            gmin[g] = make_float4(__double2float_rd(mn[0]), __double2float_rd(mn[1]),
                                  __double2float_rd(mn[2]),
                                  __double2float_ru(hs2));
            // w: radius about the centre of a sphere holding the group
            gmax[g] = make_float4(__double2float_ru(mx[0]), __double2float_ru(mx[1]),
                                  __double2float_ru(mx[2]), __double2float_ru(R));
            gctr[g] = make_float4(c[0], c[1], c[2], 0.0f);
        }
        __syncthreads();  // sbox is rewritten by the next round
    }
}

// Evaluation order of the groups, most expensive first (longest processing
// time first shortens the tail of the dynamically scheduled group kernels).
// The work of a new group is estimated from the work per particle slot of
// the group that held its first particle at the last force evaluation of the
// same n (its lists depend on where it is), times the slots of the new group
// (two particles per lane above 32 particles); groups are bucketed by log2 of
// that estimate (8 buckets per octave) and written out bucket by bucket, the
// order inside a bucket being arbitrary.  Without a recorded evaluation the
// order is the identity.
constexpr int NBUCKET = 256;

__device__ __forceinline__ int order_bucket(int g, const int2 *grange,
                                            const int *order,
                                            const int *pgroup,
                                            const float *gcost, int cg)
{
    const int2 gr = grange[g];
    float sum = 0.0f;
#pragma unroll
    for (int q = 0; q < 3; ++q) {  // first, middle and last particle
        const int og = pgroup[order[gr.x + (q * (gr.y - 1)) / 2]];
        sum += (og >= 0 && og < cg) ? gcost[og] : 0.0f;
    }
    const float est = sum * (1.0f / 3.0f) * (gr.y > 32 ? 2.0f : 1.0f);
    int b = 0;
    if (est >= 1.0f) b = min(NBUCKET - 1, (int)(8.0f * __log2f(est)));
    return NBUCKET - 1 - b;  // descending work
}

// Counting sort of the groups by bucket: histogram over many blocks, then
// every block scatters its chunk of groups (positions reserved per bucket
// with one global atomic per bucket and block).
__global__ void __launch_bounds__(TB)
k_group_hist(int n, const int2 *__restrict__ grange, const int *__restrict__ order,
             const int *__restrict__ pgroup, const float *__restrict__ gcost,
             P3TDevState *st)
{
    __shared__ int h[NBUCKET];
    if (st->error) return;
    const int G = st->ngroup, cg = st->cost_groups;
    if (st->cost_n != n || cg <= 0) return;  // identity order
    for (int b = threadIdx.x; b < NBUCKET; b += TB) h[b] = 0;
    __syncthreads();
    for (int g = blockIdx.x * TB + threadIdx.x; g < G; g += gridDim.x * TB)
        atomicAdd(&h[order_bucket(g, grange, order, pgroup, gcost, cg)], 1);
    __syncthreads();
    for (int b = threadIdx.x; b < NBUCKET; b += TB)
        if (h[b]) atomicAdd(&st->gord_cnt[b], h[b]);
}

__global__ void __launch_bounds__(TB)
k_group_order(int n, const int2 *__restrict__ grange,
              const int *__restrict__ order, const int *__restrict__ pgroup,
              const float *__restrict__ gcost, int *__restrict__ gperm,
              P3TDevState *st)
{
    __shared__ int start[NBUCKET], cnt[NBUCKET], base[NBUCKET];
    if (st->error) return;
    const int G = st->ngroup;  // <= capacity (k_groups checks)
    const int cg = st->cost_groups;
    if (st->cost_n != n || cg <= 0) {
        for (int g = blockIdx.x * TB + threadIdx.x; g < G; g += gridDim.x * TB)
            gperm[g] = g;
        return;
    }
    if (threadIdx.x < 32) {  // exclusive scan of the 256 counts, 8 per lane
        const int lane = threadIdx.x;
        int v[NBUCKET / 32], sum = 0;
#pragma unroll
        for (int q = 0; q < NBUCKET / 32; ++q) {
            v[q] = st->gord_cnt[lane * (NBUCKET / 32) + q];
            sum += v[q];
        }
        int off = warp_incl_scan(sum) - sum;
#pragma unroll
        for (int q = 0; q < NBUCKET / 32; ++q) {
            start[lane * (NBUCKET / 32) + q] = off;
            off += v[q];
        }
    }
    for (int g0 = blockIdx.x * TB; g0 < G; g0 += gridDim.x * TB) {
        for (int b = threadIdx.x; b < NBUCKET; b += TB) cnt[b] = 0;
        __syncthreads();
        const int g = g0 + threadIdx.x;
        const int b = g < G ? order_bucket(g, grange, order, pgroup, gcost, cg) : 0;
        const int rk = g < G ? atomicAdd(&cnt[b], 1) : 0;
        __syncthreads();
        for (int k = threadIdx.x; k < NBUCKET; k += TB)
            if (cnt[k]) base[k] = start[k] + atomicAdd(&st->gord_fill[k], cnt[k]);
        __syncthreads();
        if (g < G) gperm[base[b] + rk] = g;
        __syncthreads();
    }
}

}  // namespace

// Bounding box, keys, sort, gather, level-wise split, moments, groups.
int p3t_build_levels(p3t_ctx *c, int n, cudaStream_t s, const double *pos,
                     const double *mass)
{
    const int grid_small = c->sms * 4;
    int nb = (n + TB - 1) / TB;
    int nbb = nb < grid_small ? nb : grid_small;
    if (nbb < 1) nbb = 1;
    const int nc = c->nclus;
    const long long *off = (const long long *)c->clus_off;
    // sub-phases timed when profiling is on (p3t_profile.build_*_ms)
    int slot = p3t_prof_open(c, P3T_PH_B_KEYS, s);
    if (nc == 1) {
        k_bbox_partial<<<nbb, TB, 0, s>>>(n, pos, mass, c->bbox_part, c->st);
        k_bbox_final<<<1, TB, 0, s>>>(nbb, c->bbox_part, c->st, c->clus_box);
    } else {
        k_bbox_seg<<<nc, TB, 0, s>>>(off, n, pos, mass, c->clus_box, c->st);
        k_cluster_ids<<<nb, TB, 0, s>>>(n, nc, off, c->pclus);
    }
    k_keys<<<nb, TB, 0, s>>>(n, pos, nc, c->pclus, c->clus_box, c->key_a,
                             c->idx_a);
    p3t_prof_close(c, slot, s);
    slot = p3t_prof_open(c, P3T_PH_B_SORT, s);
    int rc = p3t_sort_keys(c, n, s);
    if (rc) return rc;
    if (nc > 1) {
        rc = p3t_sort_cluster_passes(c, n, s);
        if (rc) return rc;
    }
    k_gather<<<nb, TB, 0, s>>>(n, c->idx_a, pos, mass, c->order, c->xs, c->ms,
                               c->phi, c->plo);
    p3t_prof_close(c, slot, s);
    slot = p3t_prof_open(c, P3T_PH_B_SPLIT, s);
    k_tree_init<<<(nc + 255) / 256, 256, 0, s>>>(nc, off, c->node, c->parent,
                                                 c->cpend, c->st);
    const int cap = (int)c->cap_cells;
    // one warp per cell: enough warps to fill every SM once
    for (int L = 0; L < P3T_MAX_LEVEL; ++L)
        k_tree_split<<<c->sms * SPLIT_BLOCKS_PER_SM, TB, 0, s>>>(L, c->p.n_leaf, cap, c->key_a,
                                                c->node, c->parent, c->cpend,
                                                c->leaf_list, c->st);
    k_leaf_hist<<<c->sms * 4, TB, 0, s>>>(c->leaf_list, c->node, c->st);
    k_leaf_scatter<<<c->sms * 4, TB, 0, s>>>(c->leaf_list, c->node,
                                              c->leaf_sorted, c->st);
    p3t_prof_close(c, slot, s);
    slot = p3t_prof_open(c, P3T_PH_B_MOMENTS, s);
    k_moments_up<<<c->sms * 8 * (TB / MB), MB, 0, s>>>(c->xs, c->ms, n, c->node, c->parent,
                                            c->leaf_sorted, c->cpend, c->cM,
                                            c->ccom, c->cQ, c->cbmin, c->cbmax,
                                            c->wmin, c->wmax, c->cf0, c->cf1,
                                            c->cf2, c->st);
    p3t_prof_close(c, slot, s);
    slot = p3t_prof_open(c, P3T_PH_B_GROUPS, s);
    k_groups<<<grid_small, TB, 0, s>>>(c->p.n_group, (int)c->cap_groups,
                                        c->node, c->parent, c->grange, c->st);
    k_group_box<<<c->sms * 2, GB, 0, s>>>(c->grange, c->xs, n, nc, c->order,
                                           c->pclus, c->cc, c->gclus, c->gmin,
                                           c->gmax, c->gctr, c->st);
    k_group_hist<<<grid_small, TB, 0, s>>>(n, c->grange, c->order, c->pgroup,
                                            c->gcost, c->st);
    k_group_order<<<grid_small, TB, 0, s>>>(n, c->grange, c->order, c->pgroup,
                                             c->gcost, c->gperm, c->st);
    p3t_prof_close(c, slot, s);
    // bbox 2, keys, gather, init, 21 splits, leaf order 2, moments, groups,
    // boxes, order 2
    p3t_count_launches(2 + 1 + 1 + 1 + P3T_MAX_LEVEL + 2 + 1 + 4);
    P3T_CUDA_TRY(cudaGetLastError());
    return P3T_OK;
}
