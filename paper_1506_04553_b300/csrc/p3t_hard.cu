// Hard part of the P3T step (Sect. 2.1 and 2.2): the hard force F_hard over
// the neighbour lists with its jerk, and the fourth-order Hermite integrator
// with block timesteps (Makino & Aarseth 1992) for the particles that have
// neighbours; isolated particles drift.
//
// The hard force of particle i sums over its neighbour row (CSR, ascending
// j): with q = x_i - x_j, u = v_i - v_j, s^2 = |q|^2 + eps^2 (Eq. 2) and the
// pair weight 1 - K(s) (Eq. 7, K of Eq. 12-15),
//   a_i  = -sum G m_j (1-K) q / s^3
//   da_i = -sum G m_j [ (1-K) (u - 3 (q.u) q / s^2) / s^3
//                       - (dK/ds) ((q.u) / s) q / s^3 ].
// All of it is FP64 with one rounding per operation (explicit __d*_rn and
// __fma_rn intrinsics: products that feed a sum are fused, as written, and
// nothing else is contracted), in a fixed order, so the results do not
// depend on the compiler's choices.  Divisions and square roots are costly
// in FP64 (about 600 cycles of latency each on B300, ten times an add) and
// few: 1/s per pair; 1/h is the exact scaling 2^k / dt_max; the timestep
// criteria are tested in squares; constants
// (1/r_cut, 1/(1 - gamma), alpha G / r_cut^2, 1/6, 1/24, 1/120, 1/dt_max)
// are formed once.
//
// Integration.  Neighbour rows are symmetric (the neighbour predicate is),
// and a particle never comes within r_cut of one outside its row during
// dt_soft (h is chosen so), so the connected components of the neighbour
// graph evolve independently for dt_soft.  The block-step schedule
// restricted to one component is exactly the global one, so each component
// runs its own: components are labelled by a lock-free union-find (label =
// smallest index of the component), counted, scanned and filled into a
// member list, then bucketed by depth and size.  Components of up to 32
// particles are packed into warps, one particle per lane with its state in
// registers (all slots of a warp step in lock-step, each at its own t_n);
// larger ones take a warp each, lanes over the members.  No synchronisation
// reaches beyond a warp.
//
// Time is counted in integer ticks of dt_max 2^-kmax, dt_max = dt_soft 2^-p.
// A particle at level k steps dt_max 2^-k and its time is a multiple of its
// step.  First step: Eq. 20 with eta_s = eta / 10; later steps:
// Eq. 18 with a_0 = alpha G m_i / r_cut^2, a^(2), a^(3) from the
// Hermite interpolation of the step just taken and |a^(1)| |a^(3)| as the
// first term of the denominator (the dimensionally consistent reading); the step may at most double
// and is halved until the current time is a multiple of it.  Each block step
// predicts every member to the next time t_n (the least t_i + dt_i),
// evaluates a and da at t_n for the members due then from the predicted
// values, and corrects them:
//   a2 = (-6 (a0 - a1) - h (4 j0 + 2 j1)) / h^2
//   a3 = (12 (a0 - a1) + 6 h (j0 + j1)) / h^3
//   x = xp + a2 h^4 / 24 + a3 h^5 / 120,  v = vp + a2 h^3 / 6 + a3 h^4 / 24.
#include <float.h>
#include <math.h>

#include "p3t_internal.cuh"

namespace {

constexpr int HB = 256;

__device__ __forceinline__ double dadd(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ double dsub(double a, double b) { return __dsub_rn(a, b); }
__device__ __forceinline__ double dmul(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ double ddiv(double a, double b) { return __ddiv_rn(a, b); }
__device__ __forceinline__ double dsqrt(double a) { return __dsqrt_rn(a); }

// x 2^n: the exponent field moved when x and the result are normal (exact,
// so equal to ldexp), ldexp otherwise.
__device__ __forceinline__ double scale2(double x, int n)
{
    const long long b = __double_as_longlong(x);
    const int e = (int)((b >> 52) & 0x7ff);
    if (e > 0 && e < 0x7ff && e + n > 0 && e + n < 0x7ff)
        return __longlong_as_double(b + ((long long)n << 52));
    return ldexp(x, n);
}

// a b + c with one rounding; products that feed a sum are fused, in the
// order written, here and in the reference alike
__device__ __forceinline__ double dfma(double a, double b, double c) { return __fma_rn(a, b, c); }

__device__ __forceinline__ double dot3(double ax, double ay, double az,
                                       double bx, double by, double bz)
{
    return dfma(ax, bx, dfma(ay, by, dmul(az, bz)));
}

// Eq. 12 in Horner form: K = x^4 (35 + x (-84 + x (70 - 20 x)))
__device__ __forceinline__ double K_of_x(double x)
{
    if (x < 0.0) return 0.0;
    if (x >= 1.0) return 1.0;
    const double x2 = dmul(x, x), x4 = dmul(x2, x2);
    return dmul(x4, dfma(dfma(dfma(-20.0, x, 70.0), x, -84.0), x, 35.0));
}

// dK/dx of Eq. 12: 140 x^3 (1 - x)^3 = x^3 (140 + x (-420 + x (420 - 140 x)))
__device__ __forceinline__ double dK_of_x(double x)
{
    if (x <= 0.0 || x >= 1.0) return 0.0;
    const double x3 = dmul(dmul(x, x), x);
    return dmul(x3, dfma(dfma(dfma(-140.0, x, 420.0), x, -420.0), x, 140.0));
}

// Softening and cut-off of one pair type.  Types (Sect. 3.2.2): 0 star-
// star, 1 black hole-star, 2 black hole-black hole; the black holes are the
// particles from nfs on, so the type of (i, j) is [i >= nfs] + [j >= nfs].
// r_cut = infinity (the black hole pair, not split): 1 / r_cut = 0, hence
// x = -gamma / (1 - gamma) < 0 and K = 0.
struct PairPar {
    double eps2;
    double irc;     // 1 / r_cut
    double iomgrc;  // 1 / ((1 - gamma) r_cut)
};

// Constants of the hard part, formed once on the host in this order.
struct HardPar {
    double G, gamma;
    double iomg;    // 1 / (1 - gamma)
    PairPar pt[3];
    int nfs;        // particles [nfs, n) are black holes (INT_MAX: none)
};

PairPar pair_par(double eps, double r_cut, double gamma)
{
    PairPar q;
    q.eps2 = eps * eps;
    q.irc = isinf(r_cut) ? 0.0 : 1.0 / r_cut;
    q.iomgrc = isinf(r_cut) ? 0.0 : 1.0 / ((1.0 - gamma) * r_cut);
    return q;
}

HardPar hard_par(double G, double eps, double r_cut, double gamma)
{
    HardPar P;
    P.G = G;
    P.gamma = gamma;
    P.iomg = 1.0 / (1.0 - gamma);
    P.pt[0] = pair_par(eps, r_cut, gamma);
    P.pt[1] = P.pt[0];
    P.pt[2] = P.pt[0];
    P.nfs = INT_MAX;
    return P;
}

// The constants of pair type t, by selects (no indexed access to the
// parameter block).
__device__ __forceinline__ PairPar pair_of(const HardPar &P, int t)
{
    PairPar q;
    q.eps2 = t == 0 ? P.pt[0].eps2 : (t == 1 ? P.pt[1].eps2 : P.pt[2].eps2);
    q.irc = t == 0 ? P.pt[0].irc : (t == 1 ? P.pt[1].irc : P.pt[2].irc);
    q.iomgrc = t == 0 ? P.pt[0].iomgrc : (t == 1 ? P.pt[1].iomgrc : P.pt[2].iomgrc);
    return q;
}

// The factors of one pair's hard acceleration and jerk, for a particle at
// (xi, vi) and a neighbour at (xj, vj) of mass mj: with q = xi - xj,
// u = vi - vj, fa = G mj (1 - K) / s^3, c1 = 3 (q.u) / s^2 and
// fb = G mj (dK/ds) (q.u) / s^4 (one square root and one division: 1/s,
// then its powers).
__device__ __forceinline__ void pair_factors(const double xi[3], const double vi[3],
                                             double xj0, double xj1, double xj2,
                                             double vj0, double vj1, double vj2,
                                             double mj, const HardPar &P, int t,
                                             double &fa, double &c1, double &fb,
                                             double q[3], double u[3])
{
    const PairPar pp = pair_of(P, t);
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        q[c] = dsub(xi[c], c == 0 ? xj0 : c == 1 ? xj1 : xj2);
        u[c] = dsub(vi[c], c == 0 ? vj0 : c == 1 ? vj1 : vj2);
    }
    const double s2 = dfma(q[0], q[0], dfma(q[1], q[1], dfma(q[2], q[2], pp.eps2)));
    const double s = dsqrt(s2);
    const double ri = ddiv(1.0, s);
    const double ri2 = dmul(ri, ri);
    const double ri3 = dmul(ri2, ri);
    const double xk = dmul(dfma(s, pp.irc, -P.gamma), P.iomg);
    const double w = dsub(1.0, K_of_x(xk));
    const double dKds = dmul(dK_of_x(xk), pp.iomgrc);
    const double rv = dot3(q[0], q[1], q[2], u[0], u[1], u[2]);
    const double gm = dmul(P.G, mj);
    fa = dmul(dmul(gm, w), ri3);
    c1 = dmul(dmul(3.0, rv), ri2);
    fb = dmul(dmul(gm, dmul(dmul(dKds, rv), ri)), ri3);
}

// The pair's terms subtracted into acc and jrk, with tq = u - c1 q:
//   acc -= fa q,  jrk -= fa tq - fb q.
__device__ __forceinline__ void pair_apply(double fa, double fb, const double q[3],
                                           const double tq[3], double acc[3],
                                           double jrk[3])
{
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        acc[c] = dfma(-fa, q[c], acc[c]);
        jrk[c] = dfma(-fa, tq[c], dfma(fb, q[c], jrk[c]));
    }
}

// Hard acceleration and jerk of a particle at (xi, vi) from one neighbour at
// (xj, vj) of mass mj, subtracted into acc and jrk.
__device__ __forceinline__ void pair_add(const double xi[3], const double vi[3],
                                         double xj0, double xj1, double xj2,
                                         double vj0, double vj1, double vj2,
                                         double mj, const HardPar &P, int t,
                                         double acc[3], double jrk[3])
{
    double fa, c1, fb, q[3], u[3], tq[3];
    pair_factors(xi, vi, xj0, xj1, xj2, vj0, vj1, vj2, mj, P, t, fa, c1, fb, q, u);
#pragma unroll
    for (int c = 0; c < 3; ++c) tq[c] = dfma(-c1, q[c], u[c]);
    pair_apply(fa, fb, q, tq, acc, jrk);
}

__device__ __forceinline__ void load3(const double *p, int n, int i, double r[3])
{
#pragma unroll
    for (int c = 0; c < 3; ++c) r[c] = p[(size_t)c * n + i];
}

__device__ __forceinline__ void store3(double *p, int n, int i, const double r[3])
{
#pragma unroll
    for (int c = 0; c < 3; ++c) p[(size_t)c * n + i] = r[c];
}

// Hard acceleration and jerk of particle i (SoA arrays of length 3n) over
// its neighbour row, in row order.
// x and v may be the predicted arrays that other lanes of the warp wrote in
// this launch: plain (coherent) loads, no read-only cache.
__device__ void hard_one(int i, int n, const double *x, const double *v,
                         const double *__restrict__ m,
                         const long long *__restrict__ off,
                         const int *__restrict__ idx, const HardPar &P,
                         double *a, double *jk, long long *pairs)
{
    double acc[3] = {0.0, 0.0, 0.0}, jrk[3] = {0.0, 0.0, 0.0};
    double xi[3], vi[3];
    load3(x, n, i, xi);
    load3(v, n, i, vi);
    const long long e0 = off[i], e1 = off[i + 1];
    const int ti = i >= P.nfs;
    for (long long e = e0; e < e1; ++e) {
        const int j = idx[e];
        pair_add(xi, vi, x[j], x[(size_t)n + j], x[2 * (size_t)n + j], v[j],
                 v[(size_t)n + j], v[2 * (size_t)n + j], m[j], P,
                 ti + (j >= P.nfs), acc, jrk);
    }
    *pairs += e1 - e0;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        a[c] = acc[c];
        jk[c] = jrk[c];
    }
}

__global__ void __launch_bounds__(HB)
k_hard_force(int n, const double *__restrict__ x, const double *__restrict__ v,
             const double *__restrict__ m, const long long *__restrict__ off,
             const int *__restrict__ idx, HardPar P, double *__restrict__ a,
             double *__restrict__ jk)
{
    for (int i = blockIdx.x * HB + threadIdx.x; i < n; i += gridDim.x * HB) {
        double ai[3], ji[3];
        long long pairs = 0;
        hard_one(i, n, x, v, m, off, idx, P, ai, ji, &pairs);
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            a[(size_t)c * n + i] = ai[c];
            jk[(size_t)c * n + i] = ji[c];
        }
    }
}

// ---------------------------------------------------------------- components

__device__ __forceinline__ int uf_find(int *parent, int x, long long *rounds,
                                       long long lim)
{
    // path halving; the writes only shorten paths and are benign under races
    for (;;) {
        const int p = atomicAdd(parent + x, 0);
        if (p == x) return x;
        const int gp = atomicAdd(parent + p, 0);
        if (gp != p) atomicCAS(parent + x, p, gp);
        x = gp;
        if (++*rounds > lim) return -1;
    }
}

__global__ void __launch_bounds__(HB) k_uf_init(int n, int *parent)
{
    for (int i = blockIdx.x * HB + threadIdx.x; i < n; i += gridDim.x * HB)
        parent[i] = i;
}

// One thread per row: every edge (i, j > i) joins the two roots, the larger
// hooked under the smaller, so each component's root ends as its smallest
// index whatever the order of the hooks.
__global__ void __launch_bounds__(HB)
k_uf_union(int n, const long long *__restrict__ off, const int *__restrict__ idx,
           int *parent, P3TDevState *st, long long lim)
{
    for (int i = blockIdx.x * HB + threadIdx.x; i < n; i += gridDim.x * HB) {
        for (long long e = off[i]; e < off[i + 1]; ++e) {
            const int j = idx[e];
            if (j <= i) continue;
            long long rounds = 0;
            for (;;) {
                int ri = uf_find(parent, i, &rounds, lim);
                int rj = uf_find(parent, j, &rounds, lim);
                if (ri < 0 || rj < 0) {
                    p3t_raise(st, P3T_ERR_TIMEOUT);
                    return;
                }
                if (ri == rj) break;
                if (ri > rj) {
                    const int t = ri;
                    ri = rj;
                    rj = t;
                }
                if (atomicCAS(parent + rj, rj, ri) == rj) break;
                if (++rounds > lim) {
                    p3t_raise(st, P3T_ERR_TIMEOUT);
                    return;
                }
            }
        }
    }
}

// label = root; component sizes counted at the root (non-isolated only).
__global__ void __launch_bounds__(HB)
k_uf_label(int n, const long long *__restrict__ off, int *parent,
           int *__restrict__ csize, P3TDevState *st, long long lim)
{
    for (int i = blockIdx.x * HB + threadIdx.x; i < n; i += gridDim.x * HB) {
        long long rounds = 0;
        const int r = uf_find(parent, i, &rounds, lim);
        if (r < 0) {
            p3t_raise(st, P3T_ERR_TIMEOUT);
            continue;
        }
        if (off[i + 1] > off[i]) atomicAdd(csize + r, 1);
    }
}

__global__ void __launch_bounds__(HB)
k_comp_fill(int n, const long long *__restrict__ off, int *parent,
            const long long *__restrict__ cstart, int *__restrict__ cfill,
            int *__restrict__ member, P3TDevState *st, long long lim)
{
    for (int i = blockIdx.x * HB + threadIdx.x; i < n; i += gridDim.x * HB) {
        if (off[i + 1] == off[i]) continue;
        long long rounds = 0;
        const int r = uf_find(parent, i, &rounds, lim);
        if (r < 0) {
            p3t_raise(st, P3T_ERR_TIMEOUT);
            continue;
        }
        member[cstart[r] + atomicAdd(cfill + r, 1)] = i;
    }
}

// The component roots in one dense list, in 33 size classes x 32 level
// buckets: first the components of more than 32 particles, then sizes 32,
// 31, ..., 1, and deepest first within a class (the depth of a component is
// the deepest first-step level of its members, held at the root in clev;
// levels from 31 on share the last bucket).  A counting sort: histogram,
// one-warp scan, scatter; the order inside a bucket is arbitrary and no
// result depends on it.
//
// Each class is a queue.  A component of more than 32 particles is one work
// item (one warp, lanes over its members).  A class of s <= 32 particles
// has work items of floor(32 / s) components: a warp that packs that many
// components side by side, one lane per particle, and takes the next
// component of the queue into a slot as soon as the slot's component is
// done (so a warp stays with a class while its queue lasts, and items that
// find the queue empty end at once).  Items go out in rounds: each round
// gives every class a share of the warps proportional to its items (at
// least one), so that the classes run side by side, each from its deepest
// components on, and a warp meets the end of a queue about once per hard
// step instead of once per class.  When a queue runs dry its warps' slots
// idle until the warp's longest component is done; handed out class by
// class, every warp met that drain at every class (30 % of the lanes of a
// 2^20 hard step idle in it).
//
// FP64 on B300: one warp per SM sub-partition already keeps its FP64 unit
// busy (a dependent add takes ~63 cycles, about the unit's time for one
// warp instruction), so more warps only share the unit and slow the
// deepest components, whose block steps are a serial chain.  k_herm_pack
// therefore runs HW = 4 warps per block and HBS blocks per SM, held there by
// padding the block's shared memory.
constexpr int HW = 4;
#ifndef P3T_HERM_BLOCKS_PER_SM
#define P3T_HERM_BLOCKS_PER_SM 1
#endif
constexpr int HBS = P3T_HERM_BLOCKS_PER_SM;
constexpr int NLB = 32;  // level buckets
constexpr int NS = 33;   // size classes: more than 32, then s = 32 .. 1
constexpr int NB = NLB * NS;
static_assert(NB == P3T_HERM_BUCKETS, "bucket scratch");
static_assert(NB % 32 == 0, "one-warp scan");
// bucket scratch (ints): counts, root starts (NB + 1), fill counters, the
// classes' shares of a round as exclusive prefix sums (NS + 1), queue heads
// per class, the number of rounds (NS + 1 reserved), then a 64-bit counter
constexpr int BK_COUNT = 0, BK_RSTART = NB, BK_RFILL = 2 * NB + 1,
              BK_SHARE = 3 * NB + 1, BK_NEXT = 3 * NB + NS + 2,
              BK_ROUNDS = 3 * NB + 2 * NS + 2,
              BK_WORK = (3 * NB + 3 * NS + 3 + 1) & ~1;
static_assert(BK_WORK + 2 <= 2 * P3T_HERM_BUCKET_LL, "bucket scratch size");

__device__ __forceinline__ int class_size(int co) { return co == 0 ? 0 : NS - co; }

__global__ void __launch_bounds__(HB)
k_comp_level(int n, const long long *__restrict__ off, int *parent,
             const int *__restrict__ lev, int *__restrict__ clev, P3TDevState *st,
             long long lim)
{
    for (int i = blockIdx.x * HB + threadIdx.x; i < n; i += gridDim.x * HB) {
        if (off[i + 1] == off[i]) continue;
        long long rounds = 0;
        const int r = uf_find(parent, i, &rounds, lim);
        if (r < 0) {
            p3t_raise(st, P3T_ERR_TIMEOUT);
            continue;
        }
        atomicMax(clev + r, lev[i]);
    }
}

__device__ __forceinline__ int root_bucket(int size, int lv)
{
    const int co = size > 32 ? 0 : NS - size;                 // class order
    return co * NLB + NLB - 1 - (lv < NLB - 1 ? lv : NLB - 1);  // deepest first
}

__global__ void __launch_bounds__(HB)
k_root_hist(int n, const int *__restrict__ parent, const int *__restrict__ csize,
            const int *__restrict__ clev, int *__restrict__ bk)
{
    __shared__ int h[NB];
    for (int b = threadIdx.x; b < NB; b += HB) h[b] = 0;
    __syncthreads();
    for (int i = blockIdx.x * HB + threadIdx.x; i < n; i += gridDim.x * HB)
        if (parent[i] == i && csize[i] > 0)
            atomicAdd(&h[root_bucket(csize[i], clev[i])], 1);
    __syncthreads();
    for (int b = threadIdx.x; b < NB; b += HB)
        if (h[b]) atomicAdd(bk + BK_COUNT + b, h[b]);
}

// counts -> root starts and fill counters (exclusive); then the rounds of
// work items: a class with c items (c components of more than 32
// particles, else ceil(components / floor(32 / s))) gets
// max(1, round(warps c / all items)) items per round, and there are as many
// rounds as the class needing most takes
__global__ void k_root_scan(int *bk, int warps)
{
    constexpr int PER = NB / 32;
    const int *bcount = bk + BK_COUNT;
    int *rstart = bk + BK_RSTART, *rfill = bk + BK_RFILL, *share = bk + BK_SHARE;
    const int lane = threadIdx.x;
    int sr = 0;
    for (int q = 0; q < PER; ++q) sr += bcount[lane * PER + q];
    int er = warp_incl_scan(sr) - sr;
    for (int q = 0; q < PER; ++q) {
        const int b = lane * PER + q;
        rstart[b] = er;
        rfill[b] = er;
        er += bcount[b];
    }
    if (lane == 31) rstart[NB] = er;
    __syncwarp();
    if (lane == 0) {
        long long all = 0;
        for (int co = 0; co < NS; ++co) {
            const int count = rstart[(co + 1) * NLB] - rstart[co * NLB];
            const int s = class_size(co);
            all += s == 0 ? count : (count + 32 / s - 1) / (32 / s);
        }
        int run = 0, rounds = 0;
        for (int co = 0; co < NS; ++co) {
            share[co] = run;
            const int count = rstart[(co + 1) * NLB] - rstart[co * NLB];
            const int s = class_size(co);
            if (count == 0) continue;
            const int items = s == 0 ? count : (count + 32 / s - 1) / (32 / s);
            int sh = (int)(((long long)warps * items + all / 2) / all);
            sh = sh < 1 ? 1 : sh;
            run += sh;
            const int need = (items + sh - 1) / sh;
            rounds = need > rounds ? need : rounds;
        }
        share[NS] = run;
        bk[BK_ROUNDS] = rounds;
    }
}

__global__ void __launch_bounds__(HB)
k_root_scatter(int n, const int *__restrict__ parent, const int *__restrict__ csize,
               const int *__restrict__ clev, int *bk, int *__restrict__ roots)
{
    int *rfill = bk + BK_RFILL;
    for (int i = blockIdx.x * HB + threadIdx.x; i < n; i += gridDim.x * HB)
        if (parent[i] == i && csize[i] > 0)
            roots[atomicAdd(rfill + root_bucket(csize[i], clev[i]), 1)] = i;
}

// ------------------------------------------------------------------ Hermite

struct HermPar {
    HardPar f;
    double eta2[2], eta_s2[2];  // per species: eta^2 (Eq. 18), eta_s^2 (Eq. 20)
    double dt_soft, dt_max, tick;
    double dm2;            // dt_max^2
    double idt_max;        // 1 / dt_max: 1 / h = 2^k / dt_max exactly
    double a0c[2];         // per species: alpha G / r_cut^2, a_0 = a0c m_i
    double c6, c24, c120;  // 1/6, 1/24, 1/120
    // Products of dt_max (or 1/dt_max) and the constants in the order the
    // corrector forms them at level 0: (1/dt_max)^2, (1/dt_max)^3,
    // dt_max^3/6, dt_max^4/24, dt_max^5/120 and 6 dt_max.  At level k each
    // is the level-0 value times an exact power of two, so when every one
    // stays normal over [0, kmax] (fast) the corrector takes them by
    // exponent arithmetic, bit for bit the rounded products.
    double ih2_0, ih3_0, h3c6_0, h4c24_0, h5c120_0, h6_0;
    long long T;  // dt_soft in ticks
    long long max_block;  // block steps allowed per component
    int kmax;
    int fast;
};

// x 2^n for x and x 2^n normal: the exponent field moved.
__device__ __forceinline__ double scale2n(double x, int n)
{
    return __longlong_as_double(__double_as_longlong(x) + ((long long)n << 52));
}

// Level of a step dt of at most eta sqrt(num / den), tested in squares (no
// division, no outer square root): dt^2 den <= e with e = eta^2 num.  The
// smallest k in [kmin, kmax] with (dt_max 2^-k)^2 den <= e (kmax when none
// is); capped counts a step for which even kmax fails.
__device__ __forceinline__ int level_sq(double den, double e, const HermPar &H,
                                        int kmin, long long &capped)
{
    // (dt_max 2^-k)^2 den is P 4^-k with P = dt_max^2 den when every
    // dt_max^2 4^-k stays normal (fast), and P 4^-k <= e is a comparison of
    // exponents and mantissas: with d the exponent difference of P and e,
    // it holds for 2k > d, and for 2k = d when P's mantissa is at most e's
    if (H.fast) {
        const double P = dmul(H.dm2, den);
        if (P == 0.0) return kmin;  // no hard force: no limit
        const long long bp = __double_as_longlong(P), be = __double_as_longlong(e);
        const int ep = (int)((bp >> 52) & 0x7ff), ee = (int)((be >> 52) & 0x7ff);
        if (bp > 0 && be > 0 && ep > 0 && ep < 0x7ff && ee > 0 && ee < 0x7ff) {
            const long long mm = (1LL << 52) - 1;
            const int d = ep - ee + ((bp & mm) > (be & mm) ? 1 : 0);
            int k = (d + 1) >> 1;  // ceil(d / 2)
            k = k > kmin ? k : kmin;
            if (k > H.kmax) {
                ++capped;
                k = H.kmax;
            }
            return k;
        }
    }
    int k = kmin;
    double q = scale2(H.dm2, -2 * k);
    while (k < H.kmax && dmul(q, den) > e) {
        ++k;
        q = dmul(q, 0.25);
    }
    if (k == H.kmax && dmul(q, den) > e) ++capped;
    return k;
}

// Forces at t = 0 and first-step levels (Eq. 20) of every particle
// with neighbours: one thread per entry of the member list (*total entries),
// so that no lane idles on an isolated particle.
__global__ void __launch_bounds__(HB)
k_herm_init(int n, const double *__restrict__ x, const double *__restrict__ v,
            const double *__restrict__ m, const long long *__restrict__ off,
            const int *__restrict__ idx, const int *__restrict__ member,
            const long long *__restrict__ total, HermPar H,
            double *__restrict__ a, double *__restrict__ jk,
            long long *__restrict__ t, int *__restrict__ lev, P3TDevState *st)
{
    long long pairs = 0, capped = 0;
    const long long nm = *total;
    for (long long q = blockIdx.x * HB + threadIdx.x; q < nm; q += gridDim.x * HB) {
        const int i = member[q];
        t[i] = 0;
        double ai[3], ji[3];
        hard_one(i, n, x, v, m, off, idx, H.f, ai, ji, &pairs);
        store3(a, n, i, ai);
        store3(jk, n, i, ji);
        // Eq. 20: dt^2 |j|^2 <= eta_s^2 (|a|^2 + a0^2)
        const int sp = i >= H.f.nfs;
        const double a0 = dmul(H.a0c[sp], m[i]);
        const double jj = dot3(ji[0], ji[1], ji[2], ji[0], ji[1], ji[2]);
        const double e = dmul(H.eta_s2[sp], dfma(a0, a0, dot3(ai[0], ai[1], ai[2], ai[0], ai[1], ai[2])));
        lev[i] = level_sq(jj, e, H, 0, capped);
    }
    if (pairs) atomicAdd((unsigned long long *)&st->herm[2], (unsigned long long)pairs);
    if (capped) atomicAdd((unsigned long long *)&st->herm[3], (unsigned long long)capped);
}

__device__ __forceinline__ long long warp_min_ll(long long v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const long long w = __shfl_xor_sync(0xffffffffu, v, o);
        v = w < v ? w : v;
    }
    return v;
}

// Third-order prediction over d = (t_n - t) in time units.
__device__ __forceinline__ void predict_reg(const double x[3], const double v[3],
                                            const double a[3], const double jk[3],
                                            double d, const HermPar &H,
                                            double xp[3], double vp[3])
{
    const double d2 = dmul(dmul(d, d), 0.5);
    const double d3 = dmul(dmul(dmul(d, d), d), H.c6);
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        xp[c] = dfma(jk[c], d3, dfma(a[c], d2, dfma(v[c], d, x[c])));
        vp[c] = dfma(jk[c], d2, dfma(a[c], d, v[c]));
    }
}

// Correction at tn of a particle due then: from its prediction (xp, vp), the
// force and jerk (a, jk) at the start of its step and (a1, j1) at tn, the new
// x and v; a, jk become a1, j1; then its next level (Eq. 18).
__device__ __forceinline__ void correct_reg(double x[3], double v[3], double a[3],
                                            double jk[3], const double xp[3],
                                            const double vp[3], const double a1[3],
                                            const double j1[3], double mi,
                                            int sp, long long tn,
                                            const HermPar &H, long long &t,
                                            int &lev, long long &capped)
{
    // h = 2^(kmax - lev) ticks = dt_max 2^-lev and 1/h = 2^lev / dt_max,
    // both exact scalings (the parameter checks keep them normal), so they
    // equal the rounded product and quotient
    const double h = scale2(H.dt_max, -lev);
    double ih2, ih3, h3c6, h4c24, h5c120, h6;
    if (H.fast) {  // the same products, by exponent arithmetic
        ih2 = scale2n(H.ih2_0, 2 * lev);
        ih3 = scale2n(H.ih3_0, 3 * lev);
        h3c6 = scale2n(H.h3c6_0, -3 * lev);
        h4c24 = scale2n(H.h4c24_0, -4 * lev);
        h5c120 = scale2n(H.h5c120_0, -5 * lev);
        h6 = scale2n(H.h6_0, -lev);
    } else {
        const double ih = scale2(H.idt_max, lev);
        ih2 = dmul(ih, ih);
        ih3 = dmul(ih2, ih);
        const double h2 = dmul(h, h), h3 = dmul(h2, h), h4 = dmul(h3, h),
                     h5 = dmul(h4, h);
        h3c6 = dmul(h3, H.c6);
        h4c24 = dmul(h4, H.c24);
        h5c120 = dmul(h5, H.c120);
        h6 = dmul(6.0, h);
    }
    double a2[3], a3[3], a2e[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const double j0 = jk[c];
        const double da = dsub(a[c], a1[c]);
        a2[c] = dmul(dfma(-h, dfma(4.0, j0, dmul(2.0, j1[c])), dmul(-6.0, da)), ih2);
        a3[c] = dmul(dfma(h6, dadd(j0, j1[c]), dmul(12.0, da)), ih3);
        x[c] = dfma(a3[c], h5c120, dfma(a2[c], h4c24, xp[c]));
        v[c] = dfma(a3[c], h4c24, dfma(a2[c], h3c6, vp[c]));
        a[c] = a1[c];
        jk[c] = j1[c];
        a2e[c] = dfma(a3[c], h, a2[c]);
    }
    t = tn;
    if (tn == H.T) return;
    // Eq. 18, with sqrt(A) sqrt(B) taken as sqrt(A B), in squares, and the
    // denominator's first term |a^(1)| |a^(3)| (the printed |a^(0)| |a^(3)|
    // is not of the dimension of |a^(2)|^2):
    // dt^2 (sqrt(|j|^2 |a3|^2) + |a2|^2) <= eta^2 (sqrt((|a|^2 + a0^2) |a2|^2) + |j|^2)
    const double a0 = dmul(H.a0c[sp], mi);
    const double aa = dot3(a1[0], a1[1], a1[2], a1[0], a1[1], a1[2]);
    const double jj = dot3(j1[0], j1[1], j1[2], j1[0], j1[1], j1[2]);
    const double a2sq = dot3(a2e[0], a2e[1], a2e[2], a2e[0], a2e[1], a2e[2]);
    const double num = dadd(dsqrt(dmul(dfma(a0, a0, aa), a2sq)), jj);
    const double den = dadd(dsqrt(dmul(jj, dot3(a3[0], a3[1], a3[2], a3[0], a3[1], a3[2]))),
                            a2sq);
    const int kmin = lev > 0 ? lev - 1 : 0;
    int k = level_sq(den, dmul(H.eta2[sp], num), H, kmin, capped);
    while (tn % (1LL << (H.kmax - k)) != 0) ++k;
    lev = k;
}

// Prediction of particle i to tick tn, state in global memory.
__device__ __forceinline__ void predict_one(int i, int n, long long tn,
                                            const HermPar &H, const double *x,
                                            const double *v, const double *a,
                                            const double *jk, double *xp,
                                            double *vp, const long long *t)
{
    double xi[3], vi[3], ai[3], ji[3], xq[3], vq[3];
    load3(x, n, i, xi);
    load3(v, n, i, vi);
    load3(a, n, i, ai);
    load3(jk, n, i, ji);
    predict_reg(xi, vi, ai, ji, dmul((double)(tn - t[i]), H.tick), H, xq, vq);
    store3(xp, n, i, xq);
    store3(vp, n, i, vq);
}

// Evaluation at tn from the predicted arrays and correction of particle i
// (due at tn), state in global memory.
__device__ __forceinline__ void correct_one(
    int i, int n, long long tn, const HermPar &H, double *x, double *v,
    const double *__restrict__ m, const long long *__restrict__ off,
    const int *__restrict__ idx, double *a, double *jk, const double *xp,
    const double *vp, long long *t, int *lev, long long &pairs,
    long long &capped)
{
    double a1[3], j1[3], ai[3], ji[3], xq[3], vq[3], xn[3], vn[3];
    hard_one(i, n, xp, vp, m, off, idx, H.f, a1, j1, &pairs);
    load3(a, n, i, ai);
    load3(jk, n, i, ji);
    load3(xp, n, i, xq);
    load3(vp, n, i, vq);
    long long ti = t[i];
    int li = lev[i];
    correct_reg(xn, vn, ai, ji, xq, vq, a1, j1, m[i], i >= H.f.nfs, tn, H, ti,
                li, capped);
    store3(x, n, i, xn);
    store3(v, n, i, vn);
    store3(a, n, i, ai);
    store3(jk, n, i, ji);
    t[i] = ti;
    lev[i] = li;
}

// One hard step of one component of more than 32 particles by a whole warp:
// lanes over the members.  The state arrays are shared by the lanes (each
// lane writes its members, all read the neighbours' predictions), so they
// are plain pointers; __syncwarp orders the phases.
__device__ void integrate_warp(int size, long long base, int lane, int n,
                               double *x, double *v, const double *__restrict__ m,
                               const long long *__restrict__ off,
                               const int *__restrict__ idx,
                               const int *__restrict__ member, const HermPar &H,
                               double *a, double *jk, double *xp, double *vp,
                               long long *t, int *lev, P3TDevState *st,
                               long long &nblk, long long &nstep,
                               long long &pairs, long long &capped,
                               long long &maxblk)
{
    for (long long it = 0;; ++it) {
        if (it >= H.max_block) {
            if (lane == 0) p3t_raise(st, P3T_ERR_TIMEOUT);
            return;
        }
        long long tmin = H.T;
        bool live = false;
        for (int q = lane; q < size; q += 32) {
            const int i = member[base + q];
            if (t[i] == H.T) continue;
            const long long e = t[i] + (1LL << (H.kmax - lev[i]));
            tmin = e < tmin ? e : tmin;
            live = true;
        }
        if (!__any_sync(0xffffffffu, live)) {
            maxblk = it > maxblk ? it : maxblk;
            return;
        }
        const long long tn = warp_min_ll(tmin);
        if (lane == 0) ++nblk;
        for (int q = lane; q < size; q += 32)
            predict_one(member[base + q], n, tn, H, x, v, a, jk, xp, vp, t);
        __syncwarp();
        for (int q = lane; q < size; q += 32) {
            const int i = member[base + q];
            if (t[i] + (1LL << (H.kmax - lev[i])) != tn) continue;
            correct_one(i, n, tn, H, x, v, m, off, idx, a, jk, xp, vp, t, lev,
                        pairs, capped);
            ++nstep;
        }
        __syncwarp();
    }
}

// Predictions and masses of the particles of one packed warp, by lane.
struct LaneSmem {
    double xp[3][32], vp[3][32], m[32];
};

// neighbour rows up to this length are held as lane numbers, 5 bits each
constexpr int ROW_PACK = 12;
// pair terms of one block step of a packed warp (8 doubles each: fa, fb, q,
// u - c1 q); a block step with more pairs (components of more than 16
// particles, densely connected, all due) takes the per-lane loop
constexpr int FCAP = 512;
constexpr int FTERMS = 8;

// The queue of one class of components of s <= 32 particles, served by one
// warp with floor(32 / s) slots: slot q = lane / s holds a component, lane
// q s + r its r-th member.  Each lane keeps its particle's state in
// registers; the block steps of the slots run in lock-step, each slot with
// its own t_n (the least t_i + dt_i over its lanes), and the predictions
// pass through shared memory.  A slot whose component reaches dt_soft
// writes it back and takes the next root of the queue (*next counts the
// roots handed out); the warp leaves when the queue is empty and its slots
// are done.  loc[i] receives the lane of particle i, so that the rows
// (global indices) turn into lane numbers; with symmetric rows every
// neighbour is a member of the same component, and the mask to 5 bits only
// keeps the shared-memory reads in bounds for rows that are not.
__device__ void integrate_class(int s, const int *__restrict__ croots, int count,
                                unsigned *next, int lane, int n, double *x,
                                double *v, const double *__restrict__ m,
                                const long long *__restrict__ off,
                                const int *__restrict__ idx,
                                const long long *__restrict__ cstart,
                                const int *__restrict__ member, const HermPar &H,
                                const double *__restrict__ ga,
                                const double *__restrict__ gj,
                                const int *__restrict__ glev, int *loc,
                                LaneSmem &S, double *F, P3TDevState *st,
                                long long &nblk,
                                long long &nstep, long long &pairs,
                                long long &capped, long long &ncomp,
                                int &maxsize, long long &maxblk)
{
    const unsigned full = 0xffffffffu;
    const int slot = lane / s, mi = lane - slot * s, head = slot * s;
    bool retired = slot >= 32 / s;  // lanes past the last whole slot never work
    bool have = false;              // the lane holds a particle in flight
    int i = 0, lev = 0;
    long long t = 0, e0 = 0, len = 0, blk = 0;
    unsigned long long row = 0;
    double xs[3] = {0.0, 0.0, 0.0}, vs[3] = {0.0, 0.0, 0.0};
    double as[3] = {0.0, 0.0, 0.0}, js[3] = {0.0, 0.0, 0.0}, mass = 0.0;
    for (;;) {
        // empty slots take the next component of the queue
        int r = -1;
        if (!have && !retired && mi == 0) {
            const unsigned k = atomicAdd(next, 1u);
            if (k < (unsigned)count) r = croots[k];
        }
        r = __shfl_sync(full, r, head);
        const bool fresh = r >= 0;
        if (!have && !fresh) retired = true;
        if (fresh) {
            i = member[cstart[r] + mi];
            load3(x, n, i, xs);
            load3(v, n, i, vs);
            load3(ga, n, i, as);
            load3(gj, n, i, js);
            t = 0;
            lev = glev[i];
            mass = m[i];
            e0 = off[i];
            len = off[i + 1] - e0;
            loc[i] = lane;
            S.m[lane] = mass;
            have = true;
            blk = 0;
            if (mi == 0) {
                ++ncomp;
                maxsize = s > maxsize ? s : maxsize;
            }
        }
        if (!__any_sync(full, have)) break;
        // black holes among the lanes (pair types, Sect. 3.2.2)
        const unsigned bhm = __ballot_sync(full, have && i >= H.f.nfs);
        __syncwarp();
        if (fresh && len <= ROW_PACK) {
            row = 0;
            for (int q = 0; q < (int)len; ++q)
                row |= (unsigned long long)(loc[idx[e0 + q]] & 31) << (5 * q);
        }
        // one block step of every slot in flight
        const long long e = have ? t + (1LL << (H.kmax - lev)) : LLONG_MAX;
        long long tn = e;  // least over the slot: tree over lanes head..head+s-1
        for (int o = 1; o < s; o <<= 1) {
            const long long w = __shfl_down_sync(full, tn, o);
            if (mi + o < s && w < tn) tn = w;
        }
        tn = __shfl_sync(full, tn, head);
        if (have && mi == 0) ++blk;
        double xp[3], vp[3];
        if (have) {
            predict_reg(xs, vs, as, js, dmul((double)(tn - t), H.tick), H, xp, vp);
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                S.xp[c][lane] = xp[c];
                S.vp[c][lane] = vp[c];
            }
        }
        __syncwarp();
        // The pairs of the due particles, numbered over the warp by a scan
        // of their row lengths, are spread over all lanes: lane l computes
        // the terms of pairs l, l + 32, ... (its owner found by a binary
        // search over the scan) into F: fa, fb, q and u - c1 q.  Each due
        // lane then applies its row in row order with the same operations
        // as pair_add, so the result is the per-lane loop's bit for bit, in
        // ceil(pairs / 32) rounds of the costly part instead of the longest
        // row's length, and only the fused sums per pair in row order.
        const bool due = have && e == tn;
        const int ln = due ? (int)len : 0;
        const int incl = warp_incl_scan(ln), ex = incl - ln;
        const int T = __shfl_sync(full, incl, 31);
        const bool spread = T <= FCAP;  // warp-uniform
        if (spread) {
            for (int base = 0; base < T; base += 32) {
                const int k = base + lane;
                int o = 0;  // the largest lane whose first pair is at or before k
#pragma unroll
                for (int step = 16; step > 0; step >>= 1) {
                    const int cand = o + step;
                    if (__shfl_sync(full, ex, cand) <= k) o = cand;
                }
                const unsigned long long orow = __shfl_sync(full, row, o);
                const long long oe0 = __shfl_sync(full, e0, o);
                const long long olen = __shfl_sync(full, len, o);
                const int oi = __shfl_sync(full, i, o), oex = __shfl_sync(full, ex, o);
                if (k < T) {
                    const int q = k - oex;
                    const int jl = olen <= ROW_PACK ? (int)((orow >> (5 * q)) & 31)
                                                    : loc[idx[oe0 + q]] & 31;
                    const double xo[3] = {S.xp[0][o], S.xp[1][o], S.xp[2][o]};
                    const double vo[3] = {S.vp[0][o], S.vp[1][o], S.vp[2][o]};
                    double fa, c1, fb, q3[3], u3[3];
                    pair_factors(xo, vo, S.xp[0][jl], S.xp[1][jl], S.xp[2][jl],
                                 S.vp[0][jl], S.vp[1][jl], S.vp[2][jl], S.m[jl],
                                 H.f, (oi >= H.f.nfs) + (int)((bhm >> jl) & 1u),
                                 fa, c1, fb, q3, u3);
                    F[k] = fa;
                    F[FCAP + k] = fb;
#pragma unroll
                    for (int c = 0; c < 3; ++c) {
                        F[(2 + c) * FCAP + k] = q3[c];
                        F[(5 + c) * FCAP + k] = dfma(-c1, q3[c], u3[c]);
                    }
                }
            }
            __syncwarp();
        }
        if (due) {
            double a1[3] = {0.0, 0.0, 0.0}, j1[3] = {0.0, 0.0, 0.0};
            for (long long q = 0; q < len; ++q) {
                const int jl = len <= ROW_PACK ? (int)((row >> (5 * q)) & 31)
                                               : loc[idx[e0 + q]] & 31;
                if (spread) {
                    const int k = ex + (int)q;
                    const double q3[3] = {F[2 * FCAP + k], F[3 * FCAP + k],
                                          F[4 * FCAP + k]};
                    const double t3[3] = {F[5 * FCAP + k], F[6 * FCAP + k],
                                          F[7 * FCAP + k]};
                    pair_apply(F[k], F[FCAP + k], q3, t3, a1, j1);
                } else {
                    pair_add(xp, vp, S.xp[0][jl], S.xp[1][jl], S.xp[2][jl],
                             S.vp[0][jl], S.vp[1][jl], S.vp[2][jl], S.m[jl], H.f,
                             (i >= H.f.nfs) + (int)((bhm >> jl) & 1u), a1, j1);
                }
            }
            pairs += len;
            correct_reg(xs, vs, as, js, xp, vp, a1, j1, mass, i >= H.f.nfs, tn, H,
                        t, lev, capped);
            ++nstep;
        }
        // every member is due at t_n = dt_soft: the component is done
        if (have && tn == H.T) {
            store3(x, n, i, xs);
            store3(v, n, i, vs);
            have = false;
            if (mi == 0) {
                nblk += blk;
                maxblk = blk > maxblk ? blk : maxblk;
            }
        }
        if (__any_sync(full, have && blk >= H.max_block)) {
            if (lane == 0) p3t_raise(st, P3T_ERR_TIMEOUT);
            break;
        }
        __syncwarp();  // F and the predictions are rewritten next step
    }
}

// All components of a hard step: warps take work items in order (the big
// components, deepest first, one warp each; then the queues of the packed
// classes, largest size first).
__global__ void __launch_bounds__(HW * 32)
k_herm_pack(int n, double *x, double *v, const double *__restrict__ m,
            const long long *__restrict__ off, const int *__restrict__ idx,
            const int *__restrict__ roots, int *bk, const int *__restrict__ csize,
            const long long *__restrict__ cstart, const int *__restrict__ member,
            HermPar H, double *a, double *jk, double *xp, double *vp,
            long long *t, int *lev, int *loc, P3TDevState *st)
{
    __shared__ LaneSmem smem[HW];
    extern __shared__ double hdyn[];  // pair terms, FTERMS FCAP per warp
    if (st->error) return;
    const int lane = threadIdx.x & 31;
    LaneSmem &S = smem[threadIdx.x >> 5];
    double *F = hdyn + (size_t)(threadIdx.x >> 5) * FTERMS * FCAP;
    const int *rstart = bk + BK_RSTART, *share = bk + BK_SHARE;
    unsigned *next = (unsigned *)(bk + BK_NEXT);
    unsigned long long *work = (unsigned long long *)(bk + BK_WORK);
    const int per = share[NS];  // items per round (0: no components)
    const long long nitems = (long long)per * bk[BK_ROUNDS];
    long long nblk = 0, nstep = 0, pairs = 0, capped = 0, ncomp = 0, maxblk = 0;
    int maxsize = 0;
    for (;;) {
        long long item = 0;
        if (lane == 0) item = (long long)atomicAdd(work, 1ull);
        item = __shfl_sync(0xffffffffu, item, 0);
        if (item >= nitems) break;
        // the class and the item's rank in it
        const int round = (int)(item / per), pos = (int)(item - (long long)round * per);
        int co = 0;
        while (share[co + 1] <= pos) ++co;
        const int k = round * (share[co + 1] - share[co]) + pos - share[co];
        const int r0 = rstart[co * NLB], count = rstart[(co + 1) * NLB] - r0;
        if (co == 0) {
            if (k >= count) continue;
            const int r = roots[r0 + k];
            const int size = csize[r];
            if (lane == 0) {
                ++ncomp;
                maxsize = size > maxsize ? size : maxsize;
            }
            integrate_warp(size, cstart[r], lane, n, x, v, m, off, idx, member,
                           H, a, jk, xp, vp, t, lev, st, nblk, nstep, pairs,
                           capped, maxblk);
        } else {
            integrate_class(class_size(co), roots + r0, count, next + co, lane, n,
                            x, v, m, off, idx, cstart, member, H, a, jk, lev, loc,
                            S, F, st, nblk, nstep, pairs, capped, ncomp, maxsize,
                            maxblk);
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        nblk += __shfl_xor_sync(0xffffffffu, nblk, o);
        nstep += __shfl_xor_sync(0xffffffffu, nstep, o);
        pairs += __shfl_xor_sync(0xffffffffu, pairs, o);
        capped += __shfl_xor_sync(0xffffffffu, capped, o);
        ncomp += __shfl_xor_sync(0xffffffffu, ncomp, o);
        maxsize = max(maxsize, __shfl_xor_sync(0xffffffffu, maxsize, o));
        maxblk = max(maxblk, __shfl_xor_sync(0xffffffffu, maxblk, o));
    }
    if (lane == 0) {
        if (nblk) atomicAdd((unsigned long long *)&st->herm[0], (unsigned long long)nblk);
        if (nstep) atomicAdd((unsigned long long *)&st->herm[1], (unsigned long long)nstep);
        if (pairs) atomicAdd((unsigned long long *)&st->herm[2], (unsigned long long)pairs);
        if (capped) atomicAdd((unsigned long long *)&st->herm[3], (unsigned long long)capped);
        if (ncomp) atomicAdd((unsigned long long *)&st->herm[4], (unsigned long long)ncomp);
        if (maxsize) atomicMax((unsigned long long *)&st->herm[5], (unsigned long long)maxsize);
        if (maxblk) atomicMax((unsigned long long *)&st->herm[6], (unsigned long long)maxblk);
    }
}

// Isolated particles drift: x <- x + dt_soft v (Sect. 2.2, step 5).
__global__ void __launch_bounds__(HB)
k_drift_isolated(int n, double *__restrict__ x, const double *__restrict__ v,
                 const long long *__restrict__ off, double dt)
{
    for (int i = blockIdx.x * HB + threadIdx.x; i < n; i += gridDim.x * HB) {
        if (off[i + 1] != off[i]) continue;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const size_t k = (size_t)c * n + i;
            x[k] = dadd(x[k], dmul(dt, v[k]));
        }
    }
}

__global__ void k_herm_reset(P3TDevState *st)
{
    if (threadIdx.x == 0 && blockIdx.x == 0)
        for (int k = 0; k < 7; ++k) st->herm[k] = 0;
}

int grid_for(long long n, int sms)
{
    long long b = (n + HB - 1) / HB;
    if (b > (long long)sms * 8) b = (long long)sms * 8;
    return b < 1 ? 1 : (int)b;
}

}  // namespace

// Dynamic shared memory that holds k_herm_pack at HBS blocks per SM: the
// SM's shared memory split HBS ways, less the per-block reserve and the
// static part, lowered until the occupancy calculator agrees; it also holds
// the warps' pair terms (FTERMS FCAP doubles per warp).  Host only; called
// where the hard-step scratch is allocated (never under capture).
int p3t_hard_setup(p3t_ctx *c)
{
    int dev = 0, per_sm = 0, reserved = 0, optin = 0;
    P3T_CUDA_TRY(cudaGetDevice(&dev));
    P3T_CUDA_TRY(cudaDeviceGetAttribute(&per_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev));
    P3T_CUDA_TRY(cudaDeviceGetAttribute(&reserved, cudaDevAttrReservedSharedMemoryPerBlock, dev));
    P3T_CUDA_TRY(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
    const int fixed = (int)sizeof(LaneSmem) * HW;
    int pad = per_sm / HBS - reserved - fixed;
    if (pad > optin - fixed) pad = optin - fixed;
    if (pad < 0) pad = 0;
    P3T_CUDA_TRY(cudaFuncSetAttribute(k_herm_pack,
                                      cudaFuncAttributeMaxDynamicSharedMemorySize, pad));
    for (; pad > 0; pad -= 1024 < pad ? 1024 : pad) {
        int nb = 0;
        P3T_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_herm_pack,
                                                                   HW * 32, pad));
        if (nb >= HBS) break;
    }
    // the padding also holds the warps' pair terms
    if (pad < (int)(HW * FTERMS * FCAP * sizeof(double))) return P3T_ERR_STATE;
    c->herm_pad = pad;
    return P3T_OK;
}

extern "C" int p3t_hard_force(int64_t n, const double *pos, const double *vel,
                              const double *mass, const int64_t *offsets,
                              const int32_t *idx, double G, double eps,
                              double r_cut, double gamma, double *acc,
                              double *jerk, void *stream)
{
    if (n < 0 || n > INT32_MAX - 1) return P3T_ERR_INVALID;
    if (n > 0 && (!pos || !vel || !mass || !offsets || !acc || !jerk))
        return P3T_ERR_INVALID;
    if (!(r_cut >= P3T_R_OUT_MIN) || !(gamma >= 0.0 && gamma < 1.0) ||
        !(eps >= 0.0) || !(G > 0.0))
        return P3T_ERR_INVALID;
    if (n == 0) return P3T_OK;
    int dev = 0, sms = 0;
    P3T_CUDA_TRY(cudaGetDevice(&dev));
    P3T_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const HardPar P = hard_par(G, eps, r_cut, gamma);
    k_hard_force<<<grid_for(n, sms), HB, 0, (cudaStream_t)stream>>>(
        (int)n, pos, vel, mass, (const long long *)offsets, idx, P, acc, jerk);
    p3t_count_launches(1);
    P3T_CUDA_TRY(cudaGetLastError());
    return P3T_OK;
}

int p3t_run_hard_step(p3t_ctx *c, int n, double *pos, double *vel,
                      const double *mass, const long long *off, const int *idx,
                      const p3t_hermite_params *hp, cudaStream_t s)
{
    HermPar H;
    H.f = hard_par(c->p.G, c->p.eps, c->p.r_out, c->p.gamma);
    const double eta_s = hp->eta / 10.0;
    H.eta2[0] = H.eta2[1] = hp->eta * hp->eta;
    H.eta_s2[0] = H.eta_s2[1] = eta_s * eta_s;
    H.a0c[0] = H.a0c[1] = hp->alpha * c->p.G / (c->p.r_out * c->p.r_out);
    if (c->n_bh > 0) {
        // two species (Sect. 3.2.2): black holes from n - n_bh on; a black
        // hole's a_0 takes its cut-off with the stars
        H.f.pt[1] = pair_par(c->sp.eps_bh, c->sp.r_cut_bh, c->p.gamma);
        H.f.pt[2] = pair_par(0.0, INFINITY, c->p.gamma);
        H.f.nfs = n - (int)c->n_bh;
        H.a0c[1] = hp->alpha * c->p.G / (c->sp.r_cut_bh * c->sp.r_cut_bh);
        const double eta_sb = c->sp.eta_bh / 10.0;
        H.eta2[1] = c->sp.eta_bh * c->sp.eta_bh;
        H.eta_s2[1] = eta_sb * eta_sb;
    }
    H.c6 = 1.0 / 6.0;
    H.c24 = 1.0 / 24.0;
    H.c120 = 1.0 / 120.0;
    H.dt_soft = hp->dt_soft;
    H.dt_max = ldexp(hp->dt_soft, -hp->log2_soft_over_max);
    H.tick = ldexp(H.dt_max, -hp->kmax);
    H.dm2 = H.dt_max * H.dt_max;
    H.idt_max = 1.0 / H.dt_max;
    H.T = 1LL << (hp->log2_soft_over_max + hp->kmax);
    H.kmax = hp->kmax;
    {
        // the corrector's products at level 0, formed as the kernel forms
        // them at any level; fast when all of them, and dt_max^2 4^-k,
        // stay normal over [0, kmax]
        const double dt = H.dt_max, ih = H.idt_max;
        const double h2 = dt * dt, h3 = h2 * dt, h4 = h3 * dt, h5 = h4 * dt;
        H.ih2_0 = ih * ih;
        H.ih3_0 = H.ih2_0 * ih;
        H.h3c6_0 = h3 * H.c6;
        H.h4c24_0 = h4 * H.c24;
        H.h5c120_0 = h5 * H.c120;
        H.h6_0 = 6.0 * dt;
        const int K = H.kmax;
        const double lo[] = {ldexp(dt, -K), ldexp(h2, -2 * K), ldexp(h3, -3 * K),
                             ldexp(h4, -4 * K), ldexp(h5, -5 * K),
                             ldexp(H.h3c6_0, -3 * K), ldexp(H.h4c24_0, -4 * K),
                             ldexp(H.h5c120_0, -5 * K), ldexp(H.h6_0, -K),
                             ldexp(H.dm2, -2 * K), ih, H.ih2_0, H.ih3_0};
        const double hi[] = {dt, h2, h3, h4, h5, H.h3c6_0, H.h4c24_0, H.h5c120_0,
                             H.h6_0, H.dm2, ldexp(ih, K), ldexp(H.ih2_0, 2 * K),
                             ldexp(H.ih3_0, 3 * K)};
        H.fast = 1;
        for (int q = 0; q < (int)(sizeof(lo) / sizeof(lo[0])); ++q)
            if (!(lo[q] >= DBL_MIN && hi[q] <= DBL_MAX)) H.fast = 0;
    }
    H.max_block = c->lim_block;
    const int g = grid_for(n, c->sms);
    k_herm_reset<<<1, 32, 0, s>>>(c->st);
    k_uf_init<<<g, HB, 0, s>>>(n, c->hparent);
    k_uf_union<<<g, HB, 0, s>>>(n, off, idx, c->hparent, c->st, c->lim_uf);
    P3T_CUDA_TRY(cudaMemsetAsync(c->hcsize, 0, sizeof(int) * (size_t)n, s));
    P3T_CUDA_TRY(cudaMemsetAsync(c->hcfill, 0, sizeof(int) * (size_t)n, s));
    k_uf_label<<<g, HB, 0, s>>>(n, off, c->hparent, c->hcsize, c->st, c->lim_uf);
    int rc = p3t_scan_ll(c, c->hcsize, c->hcstart, n, s);
    if (rc != P3T_OK) return rc;
    k_comp_fill<<<g, HB, 0, s>>>(n, off, c->hparent, c->hcstart, c->hcfill,
                                 c->hmember, c->st, c->lim_uf);
    k_herm_init<<<g, HB, 0, s>>>(n, pos, vel, mass, off, idx, c->hmember,
                                 c->hcstart + n, H, c->ha, c->hj, c->ht,
                                 c->hlev, c->st);
    // component roots bucketed by depth and size, then packed into work
    // items (the fill counters are free again and hold the component levels)
    P3T_CUDA_TRY(cudaMemsetAsync(c->hcfill, 0, sizeof(int) * (size_t)n, s));
    int *bk = (int *)c->hbucket;
    P3T_CUDA_TRY(cudaMemsetAsync(c->hbucket, 0, sizeof(long long) * P3T_HERM_BUCKET_LL, s));
    k_comp_level<<<g, HB, 0, s>>>(n, off, c->hparent, c->hlev, c->hcfill, c->st,
                                  c->lim_uf);
    k_root_hist<<<g, HB, 0, s>>>(n, c->hparent, c->hcsize, c->hcfill, bk);
    k_root_scan<<<1, 32, 0, s>>>(bk, c->sms * HBS * HW);
    k_root_scatter<<<g, HB, 0, s>>>(n, c->hparent, c->hcsize, c->hcfill, bk,
                                    c->hroots);
    // every component, deepest first, from one dynamically shared list
    k_herm_pack<<<c->sms * HBS, HW * 32, c->herm_pad, s>>>(
        n, pos, vel, mass, off, idx, c->hroots, bk, c->hcsize, c->hcstart,
        c->hmember, H, c->ha, c->hj, c->hxp, c->hvp, c->ht, c->hlev, c->hloc,
        c->st);
    k_drift_isolated<<<g, HB, 0, s>>>(n, pos, vel, off, hp->dt_soft);
    p3t_count_launches(12);  // the scan counts its own
    P3T_CUDA_TRY(cudaGetLastError());
    return P3T_OK;
}
