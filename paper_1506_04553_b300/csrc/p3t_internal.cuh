// Internal declarations shared by the translation units of libp3t.
// Device data layout (all in HBM, owned by the context):
//   particles, Morton order : key u64[n], order i32[n] (original index),
//                             xs f64[3][n], ms f64[n],
//                             phi float4[n] = (x_hi, y_hi, z_hi, m),
//                             plo float4[n] = (x_lo, y_lo, z_lo, 0)
//                             where x = x_hi + x_lo to ~2^-48 relative
//   cells                   : node int4[C] = (first, count, child, level<<8|nchild)
//                             FP64 moments M[C], com[C][3], Q[C][6], bmin/bmax[C][3]
//                             walk record wmin/wmax float4[C] (outward FP32 box,
//                             .w = child / nchild bit patterns)
//                             force record cf0/cf1/cf2 float4[C]
//   groups                  : grange int2[G] = (first, count),
//                             gmin/gmax/gctr float4[G], gperm i32[G]
//                             (evaluation order), gcost f32[G] and
//                             pgroup i32[n] (work per group and group per
//                             particle at the last force evaluation)
//   lists (CSR per group)   : pc i32, ppn i32, ppf i32 with int64 offsets
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/p3t.h"

#define P3T_MAX_LEVEL 21
#define P3T_WARP 32
// leaf sizes 0..64 and larger: bins of the size-ordered leaf list
#define P3T_LEAF_BINS 66
// neighbour rows up to this length are kept by the counting walk
#define P3T_NGB_SLOTS 8
// Hard step: components are ordered in 32 level buckets x 33 size classes;
// the bucket scratch holds four int arrays of that length and a counter.
#define P3T_HERM_BUCKETS (32 * 33)
#define P3T_HERM_BUCKET_LL (2 * P3T_HERM_BUCKETS + 8)

typedef unsigned long long u64;

// Device-side state of one context (one copy in device memory, mirrored to
// pinned host memory when a call synchronises).
struct P3TDevState {
    double lo[3];
    double size;
    int error;        // first P3T_ERR_* raised by a kernel (0 = none)
    int ncell;        // cells allocated
    int ngroup;       // groups allocated
    int max_level;    // deepest level holding a cell
    int need_cells;   // cells requested when the cell capacity overflowed
    unsigned int blocks_done;
    unsigned int work;  // dynamic work counter of the force walk
    unsigned int work_ngb;  // ... of the neighbour walk
    unsigned int work_vjp;  // ... of the backward walk
    int pad0;
    int level_start[P3T_MAX_LEVEL + 3];
    int novf;           // groups listed in ngb_ovf
    int gord_cnt[256];  // groups per work bucket (group order)
    int gord_fill[256]; // fill counters of the group order
    int leaf_bin[P3T_LEAF_BINS];   // leaves per size (sizes > 64 share the last)
    int leaf_fill[P3T_LEAF_BINS];  // fill counters of the size-ordered leaf list
    int nleaf;          // leaves listed by the split (leaf_list)
    long long tot[3];   // list totals: pc, ppn, ppf
    long long int_pc;   // particle-cell interactions
    long long int_pp;   // particle-particle interactions
    long long int_ppn;  // of which near-list interactions
    long long nnz;      // neighbour pairs
    long long cum_int[3];  // pc, pp, pp-near interactions since profile reset
    int max_stack;      // deepest walk stack seen (ranges)
    int cost_n;         // n of the force evaluation that wrote gcost/pgroup
    int cost_groups;    // number of groups of that evaluation
    int pad1;
    long long rec_n;    // source records written by a recording force walk
    long long herm[7];  // hard step: block steps (summed over components),
                        // particle steps, pair evaluations, steps capped at
                        // the finest level, components, largest component,
                        // most block steps of one component
};

// Phase timing with CUDA events (resolved lazily at p3t_get_profile).
enum { P3T_PH_BUILD = 0, P3T_PH_WALK, P3T_PH_FORCE, P3T_PH_NGB,
       P3T_PH_VJPWALK, P3T_PH_B_KEYS, P3T_PH_B_SORT, P3T_PH_B_SPLIT,
       P3T_PH_B_MOMENTS, P3T_PH_B_GROUPS, P3T_NPH };
struct P3TEvents {
    cudaEvent_t *ev;   // pairs: ev[2k] start, ev[2k+1] stop
    int *phase;
    int used, cap;
};

// Per-cluster constants of the force, neighbour and backward kernels (an
// ensemble holds independent clusters; a plain build is one cluster).
struct ClusterConsts {
    float eps2;    // softening squared
    float kA, kB;  // x = s * kA + kB = (s / r_cut - gamma) / (1 - gamma)
    float hg2;     // guard of the opening test, fl(max(h, r_cut))^2 (1 + 2^-10)
    double h;      // neighbour radius
    double h2;     // h * h (exact FP64 predicate)
    double r_out;  // r_cut
    double w_in;   // W = w_in * y below r_in (potential)
};

struct p3t_ctx {
    p3t_params p;
    int device;
    int sms;
    // capacities (elements)
    int64_t cap_n, cap_cells, cap_groups, cap_list[3], cap_scan;
    int64_t n;
    int built;         // a tree exists
    int lists_valid;   // inspection lists match the current tree
    int64_t list_tot[3];
    // device state
    P3TDevState *st;
    P3TDevState *hst;  // pinned host mirror
    // particles
    u64 *key_a, *key_b;
    int *idx_a, *idx_b;
    int *order;
    double *xs, *ms;
    float4 *phi, *plo;
    int *ngb_cnt;      // per original index
    int *ngb_slots;    // first P3T_NGB_SLOTS neighbours of each particle
    int *ngb_ovf;      // groups with a row longer than P3T_NGB_SLOTS
    // sort scratch
    int *rs_counts, *rs_totals;
    int64_t cap_tiles;
    double *bbox_part;
    // cells
    int4 *node;
    int *parent;
    int *leaf_list;             // leaves, as the split found them
    int *leaf_sorted;           // leaves, largest first
    int *cpend;                 // children whose moments are done (bottom-up pass)
    double *cM, *ccom, *cQ, *cbmin, *cbmax;
    float4 *wmin, *wmax, *cf0, *cf1, *cf2;
    // groups
    int2 *grange;
    float4 *gmin, *gmax, *gctr;
    int *gperm;        // [G] order in which the group kernels take the groups
    float *gcost;      // [G] work of each group at the last force evaluation
    int *pgroup;       // [n] group of each original index at that evaluation
    // lists
    long long *lcnt;   // [3][G] counts, then offsets [3][G+1]
    long long *loff;
    int *list[3];
    // generic scan scratch
    long long *scan_part;
    // backward pass: 10 adjoints per cell
    double *cadj;
    int64_t cap_cadj;
    // energy scratch
    double *red_part;
    // hard step (Hermite) scratch, per particle; hbucket is the fixed-size
    // scratch of the component ordering (P3T_HERM_BUCKET_LL long longs)
    int *hparent, *hcsize, *hcfill, *hmember, *hlev, *hroots, *hloc;
    long long *hcstart, *ht, *hbucket;
    double *ha, *hj, *hxp, *hvp;
    int64_t cap_herm;
    int herm_pad;            // dynamic shared memory of the Hermite kernel
    int force_warps;         // warps per block of the walk + force kernel (0: 4)
    int vjp_warps;           // warps per block of the backward kernel (0: 4)
    // bounds of the kernels' loops and waits (p3t_set_limits)
    long long lim_walk;      // walk iterations per group
    long long lim_uf;        // union-find rounds per edge
    long long lim_block;     // block steps per component
    int64_t lim_cells;       // cells a build may allocate (0: no bound)
    int64_t need_cells;      // cells the last build found it needed
    // clusters (one for a plain build)
    int nclus, cap_clus;
    int ensemble;            // layout fixed by p3t_set_ensemble or p3t_set_species
    // two species (p3t_set_species): the last n_bh particles are black holes
    int64_t n_bh;
    p3t_species sp;
    long long *sp_off;       // device [cap_n + 1]: star rows by the tree
    int *sp_idx;             // device [cap_sp_idx]
    int64_t cap_sp_idx;
    int *sp_inv;             // device [cap_n]: sorted position of each index
    int *sp_bh;              // device [32 + star blocks * n_bh]: black hole
                             // positions, per-block neighbour counts
    double *sp_part;         // device [star blocks * n_bh * 4]: force partials
    int64_t *clus_off_h;     // pinned host [nclus + 1]
    ClusterConsts *cc_h;     // pinned host [nclus]
    double *clus_par;        // host [3][nclus]: r_out, eps, h (ensemble)
    int64_t *clus_off;       // device [nclus + 1]
    ClusterConsts *cc;       // device [nclus]
    double *clus_box;        // device [nclus][8]: lo xyz, side, RN(1/side) 2^21, pad
    int *pclus;              // device [cap_n]: cluster of each original index
    int *gclus;              // device [cap_groups]: cluster of each group
    int cap_pclus;
    int no_sync;             // P3T_FLAG_NO_SYNC: build without host sync
    // profiling
    int prof_on;
    P3TEvents prof;
    double prof_ms[P3T_NPH];
    long long prof_calls[P3T_NPH];
};

// Kernel launch accounting (all contexts).
void p3t_count_launches(long long k);
// Profiling helpers: open returns a slot (or -1), close records the stop.
int p3t_prof_open(p3t_ctx *c, int phase, cudaStream_t s);
void p3t_prof_close(p3t_ctx *c, int slot, cudaStream_t s);

// ---- error helpers ----
#define P3T_CUDA_TRY(expr)                                              \
    do {                                                                \
        cudaError_t e__ = (expr);                                       \
        if (e__ != cudaSuccess) return P3T_ERR_CUDA;                    \
    } while (0)

__device__ __forceinline__ void p3t_raise(P3TDevState *st, int code)
{
    atomicCAS(&st->error, 0, code);
}

// ---- warp helpers ----
// Order-preserving map of a double to an int64 (its own inverse): for
// values that are not NaN, a < b iff ord64(a) < ord64(b), with -0 below +0.
// Minima and maxima of doubles then run on the integer pipe, bit for bit the
// values fmin / fmax return (up to the sign of a zero), without occupying
// the slow FP64 unit.
__device__ __forceinline__ long long ord64(double x)
{
    const long long b = __double_as_longlong(x);
    return b ^ ((b >> 63) & 0x7fffffffffffffffLL);
}
__device__ __forceinline__ double unord64(long long o)
{
    return __longlong_as_double(o ^ ((o >> 63) & 0x7fffffffffffffffLL));
}
__device__ __forceinline__ bool finite64(double x)
{
    return ((__double_as_longlong(x) >> 52) & 0x7ff) != 0x7ff;
}

__device__ __forceinline__ int warp_incl_scan(int v)
{
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int t = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += t;
    }
    return v;
}

__device__ __forceinline__ long long warp_incl_scan_ll(long long v)
{
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        long long t = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += t;
    }
    return v;
}

__device__ __forceinline__ unsigned lanemask_lt()
{
    return (1u << (threadIdx.x & 31)) - 1u;
}

// ---- opening test (identical in every walk) ----
// Squared gap between two FP32 boxes, one rounding per operation, no FMA.
__device__ __forceinline__ float box_d2(float4 gmn, float4 gmx, float4 cmn,
                                        float4 cmx)
{
    float gx = fmaxf(fmaxf(__fsub_rn(cmn.x, gmx.x), __fsub_rn(gmn.x, cmx.x)), 0.0f);
    float gy = fmaxf(fmaxf(__fsub_rn(cmn.y, gmx.y), __fsub_rn(gmn.y, cmx.y)), 0.0f);
    float gz = fmaxf(fmaxf(__fsub_rn(cmn.z, gmx.z), __fsub_rn(gmn.z, cmx.z)), 0.0f);
    float s = __fadd_rn(__fmul_rn(gx, gx), __fmul_rn(gy, gy));
    return __fadd_rn(s, __fmul_rn(gz, gz));
}

// Largest side of an FP32 box.
__device__ __forceinline__ float box_side(float4 cmn, float4 cmx)
{
    float lx = __fsub_rn(cmx.x, cmn.x);
    float ly = __fsub_rn(cmx.y, cmn.y);
    float lz = __fsub_rn(cmx.z, cmn.z);
    return fmaxf(fmaxf(lx, ly), lz);
}

// Cell c is accepted for a group iff l*l < theta2*d2 and d2 > hg2.
__device__ __forceinline__ bool mac_accept(float d2, float l, float theta2,
                                           float hg2)
{
    return __fmul_rn(l, l) < __fmul_rn(theta2, d2) && d2 > hg2;
}

// ---- kernel-launch helpers implemented in the .cu files ----
int p3t_sort_keys(p3t_ctx *c, int n, cudaStream_t s);          // p3t_sort.cu
int p3t_scan_ll(p3t_ctx *c, const int *in, long long *out, int n,
                cudaStream_t s);                                 // p3t_misc.cu
int p3t_hard_setup(p3t_ctx *c);                                 // p3t_hard.cu
int p3t_build_levels(p3t_ctx *c, int n, cudaStream_t s, const double *pos,
                     const double *mass);                       // p3t_tree.cu
int p3t_sort_cluster_passes(p3t_ctx *c, int n, cudaStream_t s); // p3t_sort.cu
void p3t_cluster_consts(const p3t_params *p, double r_out, double eps,
                        double h, ClusterConsts *out);          // p3t_api.cu
int p3t_run_walk(p3t_ctx *c, int fill, cudaStream_t s);        // p3t_walk.cu
int p3t_scan_lists(p3t_ctx *c, cudaStream_t s);                 // p3t_walk.cu
constexpr long long P3T_LIM_WALK = 1LL << 24;   // default p3t_limits
constexpr long long P3T_LIM_UF = 1LL << 20;
constexpr long long P3T_LIM_BLOCK = 1LL << 26;
int p3t_run_force(p3t_ctx *c, float *acc, double *pot, cudaStream_t s,
                  long long *rec = nullptr, long long rec_cap = 0);   // p3t_force.cu
int p3t_run_ngb_species(p3t_ctx *c, long long *offsets, int *idx, long long cap,
                        long long *needed, cudaStream_t s);
int p3t_run_ngb(p3t_ctx *c, int fill, const long long *row_off, int *idx,
                long long cap, cudaStream_t s);                  // p3t_ngb.cu
int p3t_run_vjp(p3t_ctx *c, const float *w, double *gpos, double *gmass,
                double *cadj, cudaStream_t s);                   // p3t_vjp.cu
int p3t_run_hard_step(p3t_ctx *c, int n, double *pos, double *vel,
                      const double *mass, const long long *off, const int *idx,
                      const p3t_hermite_params *hp, cudaStream_t s); // p3t_hard.cu
int p3t_force_err(p3t_ctx *c, long long n, const float *a, const float *r,
                  void *scratch, double *median, double *emax, cudaStream_t s);
size_t p3t_force_err_scratch(const p3t_ctx *c);               // p3t_misc.cu
int p3t_energy_launch(p3t_ctx *c, long long n, const double *mass,
                      const double *vel, const double *pot, double *out,
                      cudaStream_t s);                           // p3t_misc.cu
int64_t p3t_sort_tiles(int64_t n);                               // p3t_sort.cu
int64_t p3t_scan_blocks(int64_t n);                              // p3t_misc.cu
void p3t_mac_constants(const p3t_params *p, float *theta2, float *hg2);
