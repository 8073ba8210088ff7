// Force evaluation over the interaction lists (the hot loop).
//
// For particle i of group g (Eq. 8, the soft force, per unit mass):
//   a_i = sum_{c in cells(g)}  G [ M d/s^3 - Q d/s^5 + (5/2)(d.Q.d) d/s^7 ]
//       + sum_{j in far(g)}    G m_j d/s^3
//       + sum_{j in near(g)}   G m_j K(s) d/s^3
// with d = x_src - x_i, s^2 = |d|^2 + eps^2 (Eq. 2), K of Eq. 12-15; the cell
// term is the softened quadrupole expansion about the cell's centre of mass
// (traceless Q_ab = sum m (3 d_a d_b - |d|^2 delta_ab)).  Self pairs have
// d = 0 and contribute exactly zero.
//
// Layout of the work: one warp per group (groups fetched dynamically), two
// i-particles per lane (group size <= 64; groups of at most 32 evaluate only
// the first).  The warp walks the tree for its
// group (the same traversal and opening test as the list walk in
// p3t_walk.cu) and feeds what it finds into three small rings in shared
// memory: accepted cells, far leaf ranges, near leaf ranges.  Whenever a ring
// holds a tile (64 cells or 32 particles) its sources are staged in shared
// memory as group-relative FP32 vectors, (x_hi - c) + x_lo, so that no
// absolute coordinate enters the FP32 arithmetic, and every lane applies
// them to each of its particles two sources at a time: one packed FP32x2
// instruction evaluates a particle against a pair of staged sources (a
// broadcast read).  Walking and evaluating in one kernel means the
// interaction lists never go through HBM and the walk's memory latency hides
// behind other warps' arithmetic; the walk is software-pipelined by one
// batch, so that a batch's box records are in flight while the previous
// batch's tiles are evaluated.  Partial sums of a tile are added into (hi,
// lo) pairs by compensated (Kahan) addition, so the summation error is
// essentially that of 32-term FP32 sums.
#include <math.h>

#include "p3t_internal.cuh"

namespace {

#ifndef P3T_PC_UNROLL
#define P3T_PC_UNROLL 4
#endif
constexpr int kPcUnroll = P3T_PC_UNROLL;  // unroll of the cell-tile loop (pairs)

struct ForceConsts {
    float eps2;    // eps^2
    float kA, kB;  // x = s * kA + kB = (s / r_cut - gamma) / (1 - gamma)
    float G;
    double h2;     // h * h (FP64, exact predicate)
    double r_out, gamma, w_in;  // potential: W = w_in * y below r_in
};

__device__ __forceinline__ float4 far_pad()
{
    return make_float4(1e15f, 1e15f, 1e15f, 0.0f);
}

// Compensated addition of v to the sum (hi, lo), Kahan's form: the rounding
// error of hi + v, recovered as v - ((hi + v) - hi), goes into lo.  It is
// exact whenever |hi| >= |v|, which holds after a group's first tiles (a
// tile's partial sum is one of many); the terms themselves carry FP32
// rounding, so no more exactness is needed.
// Asynchronous 16-byte copy global -> shared (cp.async; no register holds
// the data while it is in flight).
__device__ __forceinline__ void cp_async16(void *smem, const void *gmem)
{
    const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 16;" ::"r"(sa), "l"(gmem));
}

__device__ __forceinline__ void two_sum_add(float &hi, float &lo, float v)
{
    float s = __fadd_rn(hi, v);
    float err = __fsub_rn(v, __fsub_rn(s, hi));
    hi = s;
    lo = __fadd_rn(lo, err);
}

struct Acc3 {
    float hx, hy, hz, lx, ly, lz;
    __device__ __forceinline__ void zero() { hx = hy = hz = lx = ly = lz = 0.0f; }
    __device__ __forceinline__ void add(float x, float y, float z)
    {
        two_sum_add(hx, lx, x);
        two_sum_add(hy, ly, y);
        two_sum_add(hz, lz, z);
    }
};

// Every term is evaluated for one i-particle against two consecutive staged
// sources at once, with the FP32x2 instructions of sm_100 and later (one issue
// slot for two FMAs); each half rounds exactly like the scalar operation.
// The sources are staged in shared memory pair-interleaved (two components
// of both sources of a pair in 16 bytes), so one 128-bit load gives two
// components of both sources, and the particle's coordinates are
// held as broadcast pairs.
typedef float2 f2;
__device__ __forceinline__ f2 add2(f2 a, f2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ f2 mul2(f2 a, f2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ f2 fma2(f2 a, f2 b, f2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ f2 dup2(float a) { return make_float2(a, a); }
// 1/sqrt(x) by the hardware approximation with subnormal inputs flushed
// (rsqrt.approx.ftz.f32).  Used where x >= (near radius)^2 > 0 or x is the
// padding's ~1e30, so no input is subnormal and the flush changes nothing;
// it saves the subnormal guard that rsqrtf carries.
__device__ __forceinline__ float rsqrt_ftz(float x)
{
    float r;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}
__device__ __forceinline__ f2 rsqrt2(f2 a) { return make_float2(rsqrt_ftz(a.x), rsqrt_ftz(a.y)); }

// Cell sources (components of two cells): position relative to the group
// centre, mass and the negated traceless quadrupole Q' = -Q.  With Q',
// q' = Q' d = -Q d and (d.Q'.d) = -(d.Q.d), so
//   a = M d/s^3 - Q d/s^5 + (5/2)(d.Q.d) d/s^7
//     = [M / s^3 - (5/2) (d.Q'.d) / s^7] d + q' / s^5
//     = (1 / s^5) (b d + q'),   b = M s^2 - (5/2) (d.Q'.d) / s^2,
// which needs no sign flips and no 1/s^7: 30 FP32x2 instructions per pair of
// cells.  (nx, ny, nz) = minus the particle's coordinates.
struct CellPair {
    f2 X, Y, Z, M, Qxx, Qyy, Qzz, Qxy, Qxz, Qyz;
};

template <bool POT>
__device__ __forceinline__ void pc_term2(f2 nx, f2 ny, f2 nz,
                                         const CellPair &c, f2 eps2, f2 &ax,
                                         f2 &ay, f2 &az, f2 &pp)
{
    const f2 dx = add2(c.X, nx), dy = add2(c.Y, ny), dz = add2(c.Z, nz);
    const f2 s2 = fma2(dx, dx, fma2(dy, dy, fma2(dz, dz, eps2)));
    const f2 ri = rsqrt2(s2);
    const f2 ri2 = mul2(ri, ri);
    const f2 qx = fma2(c.Qxx, dx, fma2(c.Qxy, dy, mul2(c.Qxz, dz)));
    const f2 qy = fma2(c.Qxy, dx, fma2(c.Qyy, dy, mul2(c.Qyz, dz)));
    const f2 qz = fma2(c.Qxz, dx, fma2(c.Qyz, dy, mul2(c.Qzz, dz)));
    const f2 dqd = fma2(dx, qx, fma2(dy, qy, mul2(dz, qz)));
    const f2 ri5 = mul2(mul2(ri, ri2), ri2);
    const f2 b = fma2(mul2(dup2(-2.5f), dqd), ri2, mul2(c.M, s2));
    ax = fma2(ri5, fma2(b, dx, qx), ax);
    ay = fma2(ri5, fma2(b, dy, qy), ay);
    az = fma2(ri5, fma2(b, dz, qz), az);
    if (POT)  // phi = -(M/s + (1/2)(d.Q.d)/s^5), summed with its sign flipped
        pp = add2(pp, fma2(mul2(dup2(-0.5f), dqd), ri5, mul2(c.M, ri)));
}

// Particle sources (two particles): position relative to the group centre
// and mass.
struct PartPair {
    f2 X, Y, Z, M;
};

// far particle term (K = 1); pp accumulates m/s for the potential
template <bool POT>
__device__ __forceinline__ void pp_far2(f2 nx, f2 ny, f2 nz, const PartPair &p,
                                        f2 eps2, f2 &ax, f2 &ay, f2 &az,
                                        f2 &pp)
{
    const f2 dx = add2(p.X, nx), dy = add2(p.Y, ny), dz = add2(p.Z, nz);
    const f2 s2 = fma2(dx, dx, fma2(dy, dy, fma2(dz, dz, eps2)));
    const f2 ri = rsqrt2(s2);
    const f2 mr = mul2(p.M, ri);
    const f2 ri2 = mul2(ri, ri);
    const f2 f = mul2(mr, ri2);
    ax = fma2(f, dx, ax);
    ay = fma2(f, dy, ay);
    az = fma2(f, dz, az);
    if (POT) pp = add2(pp, mr);
}

// near particle term with the cut-off K; returns the softened distances
__device__ __forceinline__ f2 pp_near2(f2 nx, f2 ny, f2 nz, const PartPair &p,
                                       f2 eps2, f2 kA, f2 kB, f2 &ax, f2 &ay,
                                       f2 &az)
{
    const f2 dx = add2(p.X, nx), dy = add2(p.Y, ny), dz = add2(p.Z, nz);
    const f2 r2 = fma2(dx, dx, fma2(dy, dy, mul2(dz, dz)));
    const f2 s2 = add2(r2, eps2);
    const f2 ri = make_float2(s2.x > 0.0f ? rsqrtf(s2.x) : 0.0f,
                              s2.y > 0.0f ? rsqrtf(s2.y) : 0.0f);
    const f2 s = mul2(s2, ri);
    f2 x = fma2(s, kA, kB);
    x = make_float2(__saturatef(x.x), __saturatef(x.y));
    const f2 x2 = mul2(x, x);
    const f2 x4 = mul2(x2, x2);
    f2 q = fma2(dup2(-20.0f), x, dup2(70.0f));
    q = fma2(q, x, dup2(-84.0f));
    q = fma2(q, x, dup2(35.0f));
    const f2 K = mul2(q, x4);
    // ordered so that K = 0 with a huge 1/s never forms 0 * inf
    f2 f = mul2(p.M, K);
    f = mul2(f, ri);
    f = mul2(f, ri);
    f = mul2(f, ri);
    ax = fma2(f, dx, ax);
    ay = fma2(f, dy, ay);
    az = fma2(f, dz, az);
    return s;
}

// W(s / r_cut) / s for the potential (Eq. 6, Eq. 16 with G's numerator sign
// reversed), FP64; only pairs with r_in <= s < r_cut reach the middle branch.
__device__ double w_over_s(double s, const ForceConsts &k)
{
    const double g = k.gamma;
    double y = s / k.r_out;
    if (y >= 1.0) return 1.0 / s;
    if (y < g) return k.w_in / k.r_out;
    double g2 = g * g, g3 = g2 * g, g4 = g3 * g, g5 = g4 * g, g6 = g5 * g,
           g7 = g6 * g;
    double d = 1.0 - g, d7 = d * d * d * d * d * d * d;
    auto Gf = [&](double t) {
        double t2 = t * t, t3 = t2 * t, t4 = t3 * t, t5 = t4 * t, t6 = t5 * t,
               t7 = t6 * t;
        double num = (-10.0 / 3.0) * t7 + 14.0 * (g + 1.0) * t6
                     - 21.0 * (g2 + 3.0 * g + 1.0) * t5
                     + (35.0 * (g3 + 9.0 * g2 + 9.0 * g + 1.0) / 3.0) * t4
                     - 70.0 * (g3 + 3.0 * g2 + g) * t3
                     + 210.0 * (g3 + g2) * t2 - 140.0 * g3 * t * log(t)
                     + (g7 - 7.0 * g6 + 21.0 * g5 - 35.0 * g4);
        return -num / d7;
    };
    double W = Gf(y) + (1.0 - Gf(1.0)) * y;
    return W / s;
}

__device__ __forceinline__ float4 rel4(float4 hi, float4 lo, float4 c)
{
    return make_float4(__fadd_rn(__fsub_rn(hi.x, c.x), lo.x),
                       __fadd_rn(__fsub_rn(hi.y, c.y), lo.y),
                       __fadd_rn(__fsub_rn(hi.z, c.z), lo.z), hi.w);
}

// Warps (groups in flight) per block of the walk + force kernel are a
// template parameter (2, 4 or 8), chosen per context by the autotuner; 4 by
// default.  P3T_FORCE_MIN_BLOCKS: the resident blocks per SM its registers
// are sized for (0: the compiler chooses).
#ifndef P3T_FORCE_MIN_BLOCKS
#define P3T_FORCE_MIN_BLOCKS 0
#endif
constexpr int FSTACK = 768;  // walk stack entries per warp (child ranges)
constexpr int RING = 128;    // leaf-range ring capacity; never more than 95 used
constexpr int CRING = 128;   // cell ring capacity; never more than 127 used
constexpr int WB = 64;       // cells per walk batch (two per lane)
constexpr int CTILE = 64;    // cells per tile (two staged per lane)
constexpr int PTILE = 32;    // particles per tile (one staged per lane)

// components of the staged sources (cells use all ten, particles the first
// four): X Y Z M -Qxx -Qyy -Qzz -Qxy -Qxz -Qyz
constexpr int NCOMP = 10;

struct __align__(16) WarpSmem {
    float t[NCOMP][CTILE];          // staged sources, pair-interleaved (see cell_tile)
    int stack[FSTACK];              // packed child ranges: child * 8 + nchild-1
    int cb[WB];                     // cells of the current walk batch
    float4 box[2][WB];              // their box records (wmin, wmax), by slot
    float4 raw[3][CTILE];           // force records of a requested cell tile
    int pc[CRING];                  // accepted cells
    int2 pf[RING];                  // far leaf ranges (first, count)
    int2 pn[RING];                  // near leaf ranges
    int tj[PTILE];                  // sorted ids of staged particles
    float4 gmn, gmx, ct;            // the group's box and centre
};

struct RangeRing {
    int head, nr, np;  // first entry, ranges held, particles held
};

// Appends one range per flagged lane to a ring of leaf ranges.
__device__ __forceinline__ void ring_push_ranges(int2 *ring, RangeRing &r,
                                                 bool flag, int first,
                                                 int count, int lane)
{
    const unsigned m = __ballot_sync(0xffffffffu, flag);
    if (flag) ring[(r.head + r.nr + __popc(m & lanemask_lt())) & (RING - 1)] =
        make_int2(first, count);
    const int c = __reduce_add_sync(0xffffffffu, flag ? count : 0);
    r.nr += __popc(m);
    r.np += c;
}

// Takes the next `take` (<= 32, <= r.np) particle ids off the front of a
// ring of ranges; returns this lane's id (lane < take) and writes it to
// tj[lane].  Lane p finds the range holding tile position p by a binary
// search over the ranges' inclusive prefix counts (held one per lane), so no
// lane loops over a range.
__device__ __forceinline__ int ring_take(int2 *ring, RangeRing &r, int take,
                                         int *tj, int lane)
{
    const bool have = lane < r.nr;
    int2 g = have ? ring[(r.head + lane) & (RING - 1)] : make_int2(0, 0);
    int inc = warp_incl_scan(g.y);
    // the first range whose inclusive count exceeds p = lane: inc rises
    // strictly over the ranges (none is empty) and stays at their total on
    // the lanes past them, which is at least take > p
    int lo = 0, hi = 31;
#pragma unroll
    for (int step = 0; step < 5; ++step) {
        const int mid = (lo + hi) >> 1;
        const bool right = __shfl_sync(0xffffffffu, inc, mid) <= lane;
        lo = right ? mid + 1 : lo;
        hi = right ? hi : mid;
    }
    const int own = min(lo, 31);
    const int ox = __shfl_sync(0xffffffffu, g.x, own);
    const int oy = __shfl_sync(0xffffffffu, g.y, own);
    const int oinc = __shfl_sync(0xffffffffu, inc, own);
    const int id = ox + (lane - (oinc - oy));
    if (lane < take) tj[lane] = id;
    const unsigned full = __ballot_sync(0xffffffffu, have && inc <= take);
    const int nfull = __popc(full);
    // the range straddling the tile boundary keeps its remainder
    const int exc = inc - g.y;
    if (lane == nfull && have && exc < take) {
        int used = take - exc;
        ring[(r.head + lane) & (RING - 1)] = make_int2(g.x + used, g.y - used);
    }
    __syncwarp();
    r.head = (r.head + nfull) & (RING - 1);
    r.nr -= nfull;
    r.np -= take;
    return id;
}

// Recording of the sources a group evaluates (the inspection entry point
// p3t_force_lists; the timed kernels are the instantiations without it).
// Every staged tile appends one record per real source: the group in bits
// 33-62, the kind (0 cell, 1 near particle, 2 far particle) in bits 31-32 and
// the cell id or sorted particle id in bits 0-30; records past cap are
// counted, not written.
struct Rec {
    long long *buf;
    long long cap;
    unsigned long long *cnt;
    int g;
};

__device__ __forceinline__ void rec_tile(const Rec &R, int take, int lane,
                                         int kind, int id, int slot0 = 0)
{
    unsigned long long base = 0;
    const int nt = take - slot0 < 32 ? take - slot0 : 32;  // this round's sources
    if (nt <= 0) return;
    if (lane == 0) base = atomicAdd(R.cnt, (unsigned long long)nt);
    base = __shfl_sync(0xffffffffu, base, 0);
    if (lane < nt && base + lane < (unsigned long long)R.cap)
        R.buf[base + lane] = ((long long)R.g << 33) | ((long long)kind << 31) | id;
}

template <bool POT>
struct GroupAcc {
    Acc3 a0, a1;
    float ph0, pl0, ph1, pl1;
};

// The lane's two particles, group-relative and negated, each coordinate as a
// broadcast pair.
struct IPair {
    f2 x0, y0, z0, x1, y1, z1;
};

// Tile partial sums of one particle: the two halves of each pair hold the
// sums over even and odd sources.
struct Part3 {
    f2 x, y, z, p;
    __device__ __forceinline__ void zero() { x = y = z = p = dup2(0.f); }
};

template <bool POT>
__device__ __forceinline__ void tile_end(GroupAcc<POT> &A, const Part3 &u,
                                         const Part3 &v, float sgn)
{
    A.a0.add(u.x.x + u.x.y, u.y.x + u.y.y, u.z.x + u.z.y);
    A.a1.add(v.x.x + v.x.y, v.y.x + v.y.y, v.z.x + v.z.y);
    if (POT) {
        two_sum_add(A.ph0, A.pl0, sgn * (u.p.x + u.p.y));
        two_sum_add(A.ph1, A.pl1, sgn * (v.p.x + v.p.y));
    }
}

// Cells 2p and 2p + 1 of the staged tile (j = 2p).
__device__ __forceinline__ CellPair cell_pair(const WarpSmem &S, int j)
{
    CellPair c;
    const float4 *t4 = reinterpret_cast<const float4 *>(&S.t[0][0]) + (j >> 1) * 5;
    const float4 A = t4[0], B = t4[1], C = t4[2], D = t4[3], E = t4[4];
    c.X = make_float2(A.x, A.y);   c.Y = make_float2(A.z, A.w);
    c.Z = make_float2(B.x, B.y);   c.M = make_float2(B.z, B.w);
    c.Qxx = make_float2(C.x, C.y); c.Qyy = make_float2(C.z, C.w);
    c.Qzz = make_float2(D.x, D.y); c.Qxy = make_float2(D.z, D.w);
    c.Qxz = make_float2(E.x, E.y); c.Qyz = make_float2(E.z, E.w);
    return c;
}

// Staged form of one cell (slot of the tile): position relative to the group
// centre, mass and -Q, from its force records (hi com + M, lo com + Qxx,
// Qyy Qxy Qxz Qyz), written pair-interleaved: the cells 2p and 2p+1 fill 20
// consecutive floats, components (2k, 2k+1) of both in float4 k, so one
// 128-bit load gives two components of the pair.  Empty slots are far
// padding with no mass.
__device__ __forceinline__ void stage_cell(WarpSmem &S, int slot, bool have,
                                           float4 a, float4 bb, float4 cc)
{
    const float4 ct = S.ct;
    float v[NCOMP];
    if (have) {
        v[0] = __fadd_rn(__fsub_rn(a.x, ct.x), bb.x);
        v[1] = __fadd_rn(__fsub_rn(a.y, ct.y), bb.y);
        v[2] = __fadd_rn(__fsub_rn(a.z, ct.z), bb.z);
        v[3] = a.w;
        v[4] = -bb.w;          // -Qxx
        v[5] = -cc.x;          // -Qyy
        v[6] = bb.w + cc.x;    // -Qzz = Qxx + Qyy (traceless)
        v[7] = -cc.y;          // -Qxy
        v[8] = -cc.z;          // -Qxz
        v[9] = -cc.w;          // -Qyz
    } else {
        const float4 fp = far_pad();
        v[0] = fp.x; v[1] = fp.y; v[2] = fp.z;
#pragma unroll
        for (int q = 3; q < NCOMP; ++q) v[q] = 0.0f;
    }
    float *t = &S.t[0][0];
    const int pr = slot >> 1, hf = slot & 1;
#pragma unroll
    for (int k = 0; k < NCOMP / 2; ++k) {
        t[pr * 20 + 4 * k + hf] = v[2 * k];
        t[pr * 20 + 4 * k + 2 + hf] = v[2 * k + 1];
    }
}

// Evaluation of the staged cell tile (64 cells, or 32 when jend = 32) for the
// lane's particles.  TWO: the lane holds a second particle (slot 32 +
// lane); groups of at most 32 particles skip it.
template <bool POT, bool TWO>
__device__ __forceinline__ void cell_eval(const WarpSmem &S, int jend,
                                          const IPair &P, float eps2,
                                          GroupAcc<POT> &A)
{
    Part3 u, w;
    u.zero();
    w.zero();
    const f2 e2 = dup2(eps2);
#pragma unroll kPcUnroll
    for (int j = 0; j < jend; j += 2) {
        const CellPair c = cell_pair(S, j);
        pc_term2<POT>(P.x0, P.y0, P.z0, c, e2, u.x, u.y, u.z, u.p);
        if (TWO) pc_term2<POT>(P.x1, P.y1, P.z1, c, e2, w.x, w.y, w.z, w.p);
    }
    tile_end<POT>(A, u, w, -1.0f);
}

// One tile of up to CTILE = 64 accepted cells from the ring, two per lane
// (slots lane and lane + 32), loaded and staged at once (the walk's last,
// partial tiles); a tile of at most 32 cells evaluates only the first half.
template <bool POT, bool TWO, bool REC>
__device__ __forceinline__ void cell_tile(WarpSmem &S, int &head, int &n,
                                          int take, const float4 *cf0,
                                          const float4 *cf1, const float4 *cf2,
                                          const IPair &P,
                                          float eps2, GroupAcc<POT> &A, int lane,
                                          const Rec &R)
{
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        const int slot = lane + 32 * h;
        const int c = slot < take ? S.pc[(head + slot) & (CRING - 1)] : 0;
        if (REC) rec_tile(R, take, lane, 0, c, 32 * h);
        float4 a = make_float4(0.f, 0.f, 0.f, 0.f), bb = a, cc = a;
        if (slot < take) {
            a = cf0[c];
            bb = cf1[c];
            cc = cf2[c];
        }
        stage_cell(S, slot, slot < take, a, bb, cc);
    }
    head = (head + take) & (CRING - 1);
    n -= take;
    __syncwarp();
    cell_eval<POT, TWO>(S, take > 32 ? 64 : 32, P, eps2, A);
    __syncwarp();
}

// A full tile of CTILE cells taken from the ring and its force records
// requested into S.raw by cp.async; staged and evaluated by cell_raw_tile
// after the next wait, one walk iteration later, so that the records'
// latency hides behind the warp's other work.
template <bool REC>
__device__ __forceinline__ void cell_request(WarpSmem &S, int &head, int &n,
                                             const float4 *cf0,
                                             const float4 *cf1,
                                             const float4 *cf2, int lane,
                                             const Rec &R)
{
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        const int slot = lane + 32 * h;
        const int c = S.pc[(head + slot) & (CRING - 1)];
        if (REC) rec_tile(R, CTILE, lane, 0, c, 32 * h);
        cp_async16(&S.raw[0][slot], cf0 + c);
        cp_async16(&S.raw[1][slot], cf1 + c);
        cp_async16(&S.raw[2][slot], cf2 + c);
    }
    asm volatile("cp.async.commit_group;");
    head = (head + CTILE) & (CRING - 1);
    n -= CTILE;
}

// The requested tile (its copies complete), staged and evaluated.
template <bool POT, bool TWO>
__device__ __forceinline__ void cell_raw_tile(WarpSmem &S, const IPair &P,
                                              float eps2, GroupAcc<POT> &A,
                                              int lane)
{
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        const int slot = lane + 32 * h;
        stage_cell(S, slot, true, S.raw[0][slot], S.raw[1][slot], S.raw[2][slot]);
    }
    __syncwarp();
    cell_eval<POT, TWO>(S, CTILE, P, eps2, A);
    __syncwarp();
}

// Staged particles j and j + 1 (j even).
__device__ __forceinline__ PartPair part_pair(const WarpSmem &S, int j)
{
    PartPair p;
    const float4 *t4 = reinterpret_cast<const float4 *>(&S.t[0][0]) + (j >> 1) * 2;
    const float4 A = t4[0], B = t4[1];
    p.X = make_float2(A.x, A.y);
    p.Y = make_float2(A.z, A.w);
    p.Z = make_float2(B.x, B.y);
    p.M = make_float2(B.z, B.w);
    return p;
}

// One tile of up to PTILE = 32 particles from a ring of leaf ranges (TWO as
// for cell_tile).
template <bool NEAR, bool POT, bool TWO, bool REC>
__device__ __forceinline__ void particle_tile(
    WarpSmem &S, int2 *ring, RangeRing &r, int take, const float4 *phi,
    const float4 *plo, const IPair &P, int k0, int k1,
    const ForceConsts &k, GroupAcc<POT> &A, int lane, const Rec &R)
{
    const int j = ring_take(ring, r, take, S.tj, lane);
    if (REC) rec_tile(R, take, lane, NEAR ? 1 : 2, j);
    float4 v;
    if (lane < take) {
        v = rel4(phi[j], plo[j], S.ct);
    } else {
        v = far_pad();
        S.tj[lane] = -1;
    }
    {  // pair-interleaved, as for cells: (X, Y) and (Z, M) of a pair per float4
        float *t = &S.t[0][0];
        const int pr = lane >> 1, hf = lane & 1;
        t[pr * 8 + hf] = v.x;
        t[pr * 8 + 2 + hf] = v.y;
        t[pr * 8 + 4 + hf] = v.z;
        t[pr * 8 + 6 + hf] = v.w;
    }
    __syncwarp();
    Part3 u, w;
    u.zero();
    w.zero();
    const f2 e2 = dup2(k.eps2);
    if (NEAR) {
        const f2 kA = dup2(k.kA), kB = dup2(k.kB);
        float tp0 = 0.f, tp1 = 0.f;
#pragma unroll 2
        for (int j = 0; j < PTILE; j += 2) {
            const PartPair p = part_pair(S, j);
            const f2 s0 = pp_near2(P.x0, P.y0, P.z0, p, e2, kA, kB, u.x, u.y, u.z);
            const f2 s1 = TWO ? pp_near2(P.x1, P.y1, P.z1, p, e2, kA, kB, w.x, w.y, w.z)
                              : dup2(0.f);
            if (POT) {
                const int ja = S.tj[j], jb = S.tj[j + 1];
                if (ja >= 0 && ja != k0) tp0 -= p.M.x * (float)w_over_s((double)s0.x, k);
                if (jb >= 0 && jb != k0) tp0 -= p.M.y * (float)w_over_s((double)s0.y, k);
                if (TWO && ja >= 0 && ja != k1)
                    tp1 -= p.M.x * (float)w_over_s((double)s1.x, k);
                if (TWO && jb >= 0 && jb != k1)
                    tp1 -= p.M.y * (float)w_over_s((double)s1.y, k);
            }
        }
        if (POT) {
            u.p = make_float2(tp0, 0.f);
            w.p = make_float2(tp1, 0.f);
        }
        tile_end<POT>(A, u, w, 1.0f);
    } else {
#pragma unroll 8
        for (int j = 0; j < PTILE; j += 2) {
            const PartPair p = part_pair(S, j);
            pp_far2<POT>(P.x0, P.y0, P.z0, p, e2, u.x, u.y, u.z, u.p);
            if (TWO) pp_far2<POT>(P.x1, P.y1, P.z1, p, e2, w.x, w.y, w.z, w.p);
        }
        tile_end<POT>(A, u, w, -1.0f);
    }
    __syncwarp();
}

// Evaluates the full particle tiles during the walk (the full cell tiles go
// through cell_request / cell_raw_tile), and at its end (last) every tile
// left over, partial ones included.
template <bool POT, bool TWO, bool REC>
__device__ __forceinline__ void drain(WarpSmem &S, bool last, int &pc_head,
                                      int &pc_n, RangeRing &rf, RangeRing &rn,
                                      const float4 *cf0, const float4 *cf1,
                                      const float4 *cf2, const float4 *phi,
                                      const float4 *plo, const IPair &P,
                                      int k0, int k1, const ForceConsts &kg,
                                      GroupAcc<POT> &A, int lane, const Rec &R)
{
    while (last && pc_n >= 1)  // during the walk full cell tiles are requested
        cell_tile<POT, TWO, REC>(S, pc_head, pc_n, min(pc_n, CTILE), cf0, cf1,
                                 cf2, P, kg.eps2, A, lane, R);
    while (rf.np >= (last ? 1 : PTILE))
        particle_tile<false, POT, TWO, REC>(S, S.pf, rf, min(rf.np, PTILE), phi,
                                            plo, P, k0, k1, kg, A, lane, R);
    while (rn.np >= (last ? 1 : PTILE))
        particle_tile<true, POT, TWO, REC>(S, S.pn, rn, min(rn.np, PTILE), phi,
                                           plo, P, k0, k1, kg, A, lane, R);
}

// Pops child ranges from the top of the walk stack until they hold at most
// WB = 64 cells, lists them in S.cb and requests their box records into
// S.box with cp.async; returns the batch size (warp-uniform, 0 when the
// stack is empty).  The lane's cells are slots lane and lane + 32.
__device__ __forceinline__ int pop_batch(WarpSmem &S, int &top,
                                         const float4 *__restrict__ wmin,
                                         const float4 *__restrict__ wmax,
                                         int lane)
{
    const unsigned full = 0xffffffffu;
    if (top == 0) return 0;
    int rx = 0, ry = 0;
    if (lane < top) {
        int e = S.stack[top - 1 - lane];
        rx = e >> 3;
        ry = (e & 7) + 1;
    }
    int inc = warp_incl_scan(ry);
    bool take = lane < top && inc <= WB;
    int ntake = __popc(__ballot_sync(full, take));
    const int total = __shfl_sync(full, inc, ntake - 1);
    if (take)
        for (int t = 0; t < ry; ++t) S.cb[inc - ry + t] = rx + t;
    top -= ntake;
    __syncwarp();
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        const int slot = lane + 32 * h;
        if (slot < total) {
            const int c = S.cb[slot];
            cp_async16(&S.box[0][slot], wmin + c);
            cp_async16(&S.box[1][slot], wmax + c);
        }
    }
    asm volatile("cp.async.commit_group;");
    return total;
}

template <bool POT, bool REC, int FW>
__global__ void __launch_bounds__(FW * 32, P3T_FORCE_MIN_BLOCKS)
k_walk_force(const int *__restrict__ gclus,
             const ClusterConsts *__restrict__ ccs,
             const int2 *__restrict__ grange,
             const float4 *__restrict__ gmin, const float4 *__restrict__ gmax,
             const float4 *__restrict__ gctr, const float4 *__restrict__ wmin,
             const float4 *__restrict__ wmax, const int4 *__restrict__ node,
             float theta2, const float4 *__restrict__ phi,
             const float4 *__restrict__ plo, const float4 *__restrict__ cf0,
             const float4 *__restrict__ cf1, const float4 *__restrict__ cf2,
             const int *__restrict__ order, int n, ForceConsts k,
             const int *__restrict__ gperm, float *__restrict__ gcost,
             int *__restrict__ pgroup, float *__restrict__ acc,
             double *__restrict__ pot, P3TDevState *st,
             long long *__restrict__ rec, long long rec_cap, long long lim_walk)
{
    __shared__ WarpSmem smem[FW];
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const unsigned full = 0xffffffffu, lt = lanemask_lt();
    WarpSmem &S = smem[w];
    if (st->error) return;  // no valid tree
    const int G = st->ngroup;
    for (;;) {
        int g = 0;
        if (lane == 0) g = (int)atomicAdd(&st->work, 1u);
        g = __shfl_sync(full, g, 0);
        if (g >= G) break;
        g = gperm[g];
        const Rec R = {rec, rec_cap, (unsigned long long *)&st->rec_n, g};
        const int2 gr = grange[g];
        const float4 ct = gctr[g];
        __syncwarp();  // the previous group's reads of S are done
        if (lane == 0) {
            S.gmn = gmin[g];
            S.gmx = gmax[g];
            S.ct = ct;
        }
        const int cl = gclus[g];
        const ClusterConsts cc = ccs[cl];
        ForceConsts kg = k;
        kg.eps2 = cc.eps2;
        kg.kA = cc.kA;
        kg.kB = cc.kB;
        kg.h2 = cc.h2;
        kg.r_out = cc.r_out;
        kg.w_in = cc.w_in;
        const float hg2 = cc.hg2;
        const int k0 = gr.x + lane, k1 = gr.x + 32 + lane;
        const bool v0 = lane < gr.y, v1 = lane + 32 < gr.y;
        const bool two = gr.y > 32;  // warp-uniform
        const float4 p0 = v0 ? rel4(phi[k0], plo[k0], ct) : far_pad();
        const float4 p1 = v1 ? rel4(phi[k1], plo[k1], ct) : far_pad();
        const IPair P = {dup2(-p0.x), dup2(-p0.y), dup2(-p0.z),
                         dup2(-p1.x), dup2(-p1.y), dup2(-p1.z)};
        GroupAcc<POT> A;
        A.a0.zero();
        A.a1.zero();
        A.ph0 = A.pl0 = A.ph1 = A.pl1 = 0.f;
        int pc_head = 0, pc_n = 0;
        RangeRing rf = {0, 0, 0}, rn = {0, 0, 0};
        int cnt_pc = 0, cnt_pn = 0, cnt_pf = 0;

        if (lane == 0) S.stack[0] = cl * 8;  // the cluster's root, one cell
        int top = 1;
        long long iter = 0;
        bool overflow = false, timeout = false;
        __syncwarp();
        // The walk is software-pipelined by one batch: the next batch (up to
        // 64 cells, two per lane) is popped and its box records copied into
        // shared memory by cp.async before the full tiles are evaluated, so
        // the records' latency hides behind the warp's own arithmetic and no
        // register holds them.  The batches, and so the tiles, are those of
        // the plain loop (pop, test, push, evaluate), in the same order.
        int total = pop_batch(S, top, wmin, wmax, lane);
        bool pend = false;  // a cell tile's records requested into S.raw
        while (total > 0) {
            if (++iter > lim_walk) {  // a finite tree stays far below the default
                timeout = true;
                break;
            }
            asm volatile("cp.async.wait_all;" ::: "memory");
            __syncwarp();
            bool is_pc[2], near[2], farl[2], open[2];
            int cid[2], child[2], nchild[2], pfirst[2], pcount[2];
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int slot = lane + 32 * h;
                is_pc[h] = near[h] = farl[h] = open[h] = false;
                cid[h] = slot < total ? S.cb[slot] : -1;
                child[h] = nchild[h] = pfirst[h] = pcount[h] = 0;
                if (cid[h] >= 0) {
                    const float4 cmn = S.box[0][slot], cmx = S.box[1][slot];
                    float d2 = box_d2(S.gmn, S.gmx, cmn, cmx);
                    float l = box_side(cmn, cmx);
                    if (mac_accept(d2, l, theta2, hg2)) {
                        is_pc[h] = true;
                    } else {
                        child[h] = __float_as_int(cmn.w);
                        nchild[h] = __float_as_int(cmx.w);
                        if (nchild[h] <= 0) {  // a leaf: first particle, -count
                            pfirst[h] = child[h];
                            pcount[h] = -nchild[h];
                            near[h] = d2 <= hg2;
                            farl[h] = !near[h];
                        } else {
                            open[h] = true;
                        }
                    }
                }
            }
            // accepted cells -> cell ring, leaves -> particle rings, opened
            // cells -> stack; slot order (lane, then lane + 32)
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                unsigned m = __ballot_sync(full, is_pc[h]);
                if (is_pc[h]) S.pc[(pc_head + pc_n + __popc(m & lt)) & (CRING - 1)] = cid[h];
                pc_n += __popc(m);
                cnt_pc += __popc(m);
                int before = rn.np;
                ring_push_ranges(S.pn, rn, near[h], pfirst[h], pcount[h], lane);
                cnt_pn += rn.np - before;
                before = rf.np;
                ring_push_ranges(S.pf, rf, farl[h], pfirst[h], pcount[h], lane);
                cnt_pf += rf.np - before;
            }
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                unsigned mo = __ballot_sync(full, open[h]);
                int np = __popc(mo);
                if (top + np > FSTACK) {
                    overflow = true;
                    break;
                }
                if (open[h]) S.stack[top + __popc(mo & lt)] = child[h] * 8 + (nchild[h] - 1);
                top += np;
            }
            if (overflow) break;
            __syncwarp();
            // the next batch, requested now
            total = pop_batch(S, top, wmin, wmax, lane);
            // the cell tile requested one iteration ago, then the next one
            if (pend) {
                if (two) cell_raw_tile<POT, true>(S, P, kg.eps2, A, lane);
                else cell_raw_tile<POT, false>(S, P, kg.eps2, A, lane);
                pend = false;
            }
            if (pc_n >= CTILE) {
                cell_request<REC>(S, pc_head, pc_n, cf0, cf1, cf2, lane, R);
                pend = true;
            }
            // evaluate every full particle tile
            if (two)
                drain<POT, true, REC>(S, false, pc_head, pc_n, rf, rn, cf0, cf1,
                                      cf2, phi, plo, P, k0, k1, kg, A, lane, R);
            else
                drain<POT, false, REC>(S, false, pc_head, pc_n, rf, rn, cf0, cf1,
                                       cf2, phi, plo, P, k0, k1, kg, A, lane, R);
        }
        if (overflow || timeout) {
            // the abandoned batch's copies land before S.box is reused
            asm volatile("cp.async.wait_all;" ::: "memory");
            __syncwarp();
            if (lane == 0) p3t_raise(st, timeout ? P3T_ERR_TIMEOUT : P3T_ERR_CAPACITY);
            continue;
        }
        // the requested tile and the partial tiles left over
        asm volatile("cp.async.wait_all;" ::: "memory");
        __syncwarp();
        if (pend) {
            if (two) cell_raw_tile<POT, true>(S, P, kg.eps2, A, lane);
            else cell_raw_tile<POT, false>(S, P, kg.eps2, A, lane);
        }
        if (two)
            drain<POT, true, REC>(S, true, pc_head, pc_n, rf, rn, cf0, cf1, cf2,
                                  phi, plo, P, k0, k1, kg, A, lane, R);
        else
            drain<POT, false, REC>(S, true, pc_head, pc_n, rf, rn, cf0, cf1, cf2,
                                   phi, plo, P, k0, k1, kg, A, lane, R);
        // ---- write back in the caller's order ----
        const float Gc = k.G;
        // work of this group per particle slot of a lane, and the group of
        // its particles, for the evaluation order of the next build (weights:
        // the instruction counts per source of the cell, far and near tiles;
        // the next build multiplies by the slots of the new group, so that a
        // group estimated from a group of the other size class is not off by
        // a factor of two)
        if (lane == 0)
            gcost[g] = 8.0f * cnt_pc + 3.0f * cnt_pf + 5.5f * cnt_pn;
        if (v0) {
            int o = order[k0];
            pgroup[o] = g;
            acc[o] = Gc * (A.a0.hx + A.a0.lx);
            acc[(size_t)n + o] = Gc * (A.a0.hy + A.a0.ly);
            acc[2 * (size_t)n + o] = Gc * (A.a0.hz + A.a0.lz);
            if (POT) pot[o] = (double)Gc * ((double)A.ph0 + (double)A.pl0);
        }
        if (v1) {
            int o = order[k1];
            pgroup[o] = g;
            acc[o] = Gc * (A.a1.hx + A.a1.lx);
            acc[(size_t)n + o] = Gc * (A.a1.hy + A.a1.ly);
            acc[2 * (size_t)n + o] = Gc * (A.a1.hz + A.a1.lz);
            if (POT) pot[o] = (double)Gc * ((double)A.ph1 + (double)A.pl1);
        }
        if (lane == 0) {
            const long long m = gr.y;
            atomicAdd((unsigned long long *)&st->tot[0], (unsigned long long)cnt_pc);
            atomicAdd((unsigned long long *)&st->tot[1], (unsigned long long)cnt_pn);
            atomicAdd((unsigned long long *)&st->tot[2], (unsigned long long)cnt_pf);
            atomicAdd((unsigned long long *)&st->int_pc, (unsigned long long)(m * cnt_pc));
            atomicAdd((unsigned long long *)&st->int_pp,
                      (unsigned long long)(m * (cnt_pn + cnt_pf)));
            atomicAdd((unsigned long long *)&st->int_ppn, (unsigned long long)(m * cnt_pn));
            atomicAdd((unsigned long long *)&st->cum_int[0], (unsigned long long)(m * cnt_pc));
            atomicAdd((unsigned long long *)&st->cum_int[1],
                      (unsigned long long)(m * (cnt_pn + cnt_pf)));
            atomicAdd((unsigned long long *)&st->cum_int[2], (unsigned long long)(m * cnt_pn));
        }
    }
}

// Resets the per-call counters of a force evaluation and marks the group
// costs it records as those of this n.
__global__ void k_force_reset(P3TDevState *st, int n)
{
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        st->work = 0;
        st->cost_n = n;
        st->cost_groups = st->ngroup;
        st->tot[0] = st->tot[1] = st->tot[2] = 0;
        st->int_pc = st->int_pp = st->int_ppn = 0;
        st->rec_n = 0;
    }
}

ForceConsts make_consts(const p3t_params &p)
{
    ForceConsts k;
    k.eps2 = (float)(p.eps * p.eps);
    k.kA = (float)(1.0 / ((1.0 - p.gamma) * p.r_out));
    k.kB = (float)(-p.gamma / (1.0 - p.gamma));
    k.G = (float)p.G;
    double h = p.h > 0.0 ? p.h : p.r_out;
    k.h2 = h * h;
    k.r_out = p.r_out;
    k.gamma = p.gamma;
    double g = p.gamma;
    if (g > 0.0) {
        double g2 = g * g, g3 = g2 * g, g4 = g3 * g, g5 = g4 * g, g6 = g5 * g;
        double gm1 = g - 1.0;
        double gm17 = gm1 * gm1 * gm1 * gm1 * gm1 * gm1 * gm1;
        k.w_in = 7.0 * (g6 - 9.0 * g5 + 45.0 * g4 - 60.0 * g3 * log(g)
                        - 45.0 * g2 + 9.0 * g - 1.0) / (3.0 * gm17);
    } else {
        k.w_in = 7.0 / 3.0;
    }
    return k;
}

// ---- two species (Sect. 3.2.2): black hole-star soft forces ----
// The tree evaluates star-star pairs (and zero between black holes, whose
// cluster has K = 0).  Each black hole-star pair is evaluated once, in FP64,
// by the star's thread (sorted order: stars first, then the black holes):
// with d = x_b - x_i, s^2 = |d|^2 + eps_bh^2 and y = s / r_cut_bh,
//   a_i += G m_b K(y) d / s^3,   a_b -= G m_i K(y) d / s^3,
//   phi_i -= G m_b W(y) / s,     phi_b -= G m_i W(y) / s.
// The black holes' terms are summed per block, then per black hole over the
// blocks in block order (deterministic).
constexpr int SFB = 256;

__device__ __forceinline__ double k_of_x64(double x)
{
    if (x <= 0.0) return 0.0;
    if (x >= 1.0) return 1.0;
    const double x2 = x * x;
    return x2 * x2 * fma(fma(fma(-20.0, x, 70.0), x, -84.0), x, 35.0);
}

__global__ void __launch_bounds__(SFB)
k_sp_soft(int n, int nfs, int nbh, const double *__restrict__ xs,
          const double *__restrict__ ms, const int *__restrict__ order,
          ForceConsts kb, double G, double eps2, float *__restrict__ acc,
          double *__restrict__ pot, double *__restrict__ part)
{
    __shared__ double red[SFB / 32][4];
    const int k = blockIdx.x * SFB + threadIdx.x;
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const bool star = k < nfs;
    const double xi = star ? xs[k] : 0.0, yi = star ? xs[(size_t)n + k] : 0.0,
                 zi = star ? xs[2 * (size_t)n + k] : 0.0;
    const double mi = star ? ms[k] : 0.0;
    const double irc = 1.0 / kb.r_out, iomg = 1.0 / (1.0 - kb.gamma);
    double ax = 0.0, ay = 0.0, az = 0.0, ph = 0.0;
    for (int b = 0; b < nbh; ++b) {
        const int kk = nfs + b;
        const double dx = xs[kk] - xi, dy = xs[(size_t)n + kk] - yi,
                     dz = xs[2 * (size_t)n + kk] - zi;
        const double s2 = dx * dx + dy * dy + dz * dz + eps2;
        const double sq = sqrt(s2);
        double f = 0.0, wos = 0.0;
        if (star) {
            // K = 0 inside r_in: a coincident pair (s = 0 with eps_bh = 0)
            // contributes no force, and its potential has a finite limit
            const double K = k_of_x64((sq * irc - kb.gamma) * iomg);
            f = K > 0.0 ? G * K / (s2 * sq) : 0.0;
            if (pot) wos = G * w_over_s(sq, kb);
        }
        const double mb = ms[kk];
        ax += mb * f * dx;
        ay += mb * f * dy;
        az += mb * f * dz;
        ph -= mb * wos;
        double r[4] = {-mi * f * dx, -mi * f * dy, -mi * f * dz, -mi * wos};
#pragma unroll
        for (int c = 0; c < 4; ++c)
#pragma unroll
            for (int o = 16; o > 0; o >>= 1)
                r[c] += __shfl_xor_sync(0xffffffffu, r[c], o);
        if (lane == 0)
#pragma unroll
            for (int c = 0; c < 4; ++c) red[w][c] = r[c];
        __syncthreads();
        if (threadIdx.x < 4) {
            double t = 0.0;
            for (int q = 0; q < SFB / 32; ++q) t += red[q][threadIdx.x];
            part[((size_t)blockIdx.x * nbh + b) * 4 + threadIdx.x] = t;
        }
        __syncthreads();
    }
    if (star) {
        const int o = order[k];
        acc[o] = (float)((double)acc[o] + ax);
        acc[(size_t)n + o] = (float)((double)acc[(size_t)n + o] + ay);
        acc[2 * (size_t)n + o] = (float)((double)acc[2 * (size_t)n + o] + az);
        if (pot) pot[o] += ph;
    }
}

// One warp per black hole: its terms summed over the blocks of k_sp_soft.
__global__ void k_sp_soft_bh(int n, int nfs, int nbh, int nblk,
                             const int *__restrict__ order,
                             const double *__restrict__ part,
                             float *__restrict__ acc, double *__restrict__ pot)
{
    const int b = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (b >= nbh) return;
    double r[4] = {0.0, 0.0, 0.0, 0.0};
    for (int q = lane; q < nblk; q += 32)
#pragma unroll
        for (int c = 0; c < 4; ++c) r[c] += part[((size_t)q * nbh + b) * 4 + c];
#pragma unroll
    for (int c = 0; c < 4; ++c)
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) r[c] += __shfl_xor_sync(0xffffffffu, r[c], o);
    if (lane == 0) {
        const int o = order[nfs + b];
        acc[o] = (float)((double)acc[o] + r[0]);
        acc[(size_t)n + o] = (float)((double)acc[(size_t)n + o] + r[1]);
        acc[2 * (size_t)n + o] = (float)((double)acc[2 * (size_t)n + o] + r[2]);
        if (pot) pot[o] += r[3];
    }
}

}  // namespace

int p3t_run_force(p3t_ctx *c, float *acc, double *pot, cudaStream_t s,
                  long long *rec, long long rec_cap)
{
    const int n = (int)c->n;
    k_force_reset<<<1, 32, 0, s>>>(c->st, n);
    p3t_count_launches(1);
    // the group count is read on the device; size the grid from the bound
    const int64_t G = (n + 15) / 16 + c->nclus;
    ForceConsts k = make_consts(c->p);
    float theta2, hg2;
    p3t_mac_constants(&c->p, &theta2, &hg2);
    const int fw = c->force_warps == 2 || c->force_warps == 8 ? c->force_warps : 4;
    int blocks = (int)((G + fw - 1) / fw);
    // enough blocks to fill every SM, whatever fits per SM
    if (blocks > c->sms * 64 / fw) blocks = c->sms * 64 / fw;
#define P3T_FORCE_ARGS                                                         \
    c->gclus, c->cc, c->grange, c->gmin, c->gmax, c->gctr, c->wmin, c->wmax,   \
        c->node, theta2, c->phi, c->plo, c->cf0, c->cf1, c->cf2, c->order, n,  \
        k, c->gperm, c->gcost, c->pgroup, acc, pot, c->st, rec, rec_cap,   \
        c->lim_walk
#define P3T_FORCE_LAUNCH(POT, REC, W)                                          \
    k_walk_force<POT, REC, W><<<blocks, (W) * 32, 0, s>>>(P3T_FORCE_ARGS)
    if (rec)
        P3T_FORCE_LAUNCH(false, true, 4);
    else if (fw == 2) {
        if (pot) P3T_FORCE_LAUNCH(true, false, 2);
        else P3T_FORCE_LAUNCH(false, false, 2);
    } else if (fw == 8) {
        if (pot) P3T_FORCE_LAUNCH(true, false, 8);
        else P3T_FORCE_LAUNCH(false, false, 8);
    } else {
        if (pot) P3T_FORCE_LAUNCH(true, false, 4);
        else P3T_FORCE_LAUNCH(false, false, 4);
    }
#undef P3T_FORCE_LAUNCH
#undef P3T_FORCE_ARGS
    p3t_count_launches(1);
    if (c->n_bh > 0) {
        const int nbh = (int)c->n_bh, nfs = n - nbh;
        const int nblk = (nfs + SFB - 1) / SFB;
        p3t_params q = c->p;
        q.r_out = c->sp.r_cut_bh;
        const ForceConsts kb = make_consts(q);
        k_sp_soft<<<nblk, SFB, 0, s>>>(n, nfs, nbh, c->xs, c->ms, c->order, kb,
                                       c->p.G, c->sp.eps_bh * c->sp.eps_bh, acc,
                                       pot, c->sp_part);
        k_sp_soft_bh<<<1, 32 * 32, 0, s>>>(n, nfs, nbh, nblk, c->order,
                                           c->sp_part, acc, pot);
        p3t_count_launches(2);
    }
    P3T_CUDA_TRY(cudaGetLastError());
    return P3T_OK;
}
