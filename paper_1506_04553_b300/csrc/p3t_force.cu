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
// i-particles per lane (group size <= 64).  The warp walks the tree for its
// group (the same traversal and opening test as the list walk in
// p3t_walk.cu) and feeds what it finds into three small rings in shared
// memory: accepted cells, far leaf ranges, near leaf ranges.  Whenever a ring
// holds 32 sources they are staged in shared memory as group-relative FP32
// vectors, (x_hi - c) + x_lo, so that no absolute coordinate enters the FP32
// arithmetic, and every lane applies each staged source (a broadcast read) to
// both of its particles.  Walking and evaluating in one kernel means the
// interaction lists never go through HBM and the walk's memory latency hides
// behind other warps' arithmetic.  Partial sums of a tile are added into
// (hi, lo) pairs with an error-free two-sum, so the summation error is that
// of 32-term FP32 sums.
#include <math.h>

#include "p3t_internal.cuh"

namespace {

constexpr int FW = 4;  // warps (groups in flight) per block

#ifndef P3T_PC_UNROLL
#define P3T_PC_UNROLL 8
#endif
constexpr int kPcUnroll = P3T_PC_UNROLL;  // unroll of the cell-tile loop

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

__device__ __forceinline__ void two_sum_add(float &hi, float &lo, float v)
{
    float s = __fadd_rn(hi, v);
    float bb = __fsub_rn(s, hi);
    float err = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bb)), __fsub_rn(v, bb));
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

// cell term; A = (d_com.xyz, M), B = (Qxx, Qyy, Qzz, Qxy), C = (Qxz, Qyz, -, -)
__device__ __forceinline__ void pc_term(float xi, float yi, float zi, float4 A,
                                        float4 B, float4 C, float eps2,
                                        float &ax, float &ay, float &az)
{
    float dx = A.x - xi, dy = A.y - yi, dz = A.z - zi;
    float s2 = fmaf(dx, dx, fmaf(dy, dy, fmaf(dz, dz, eps2)));
    float ri = rsqrtf(s2);
    float ri2 = ri * ri;
    float qx = fmaf(B.x, dx, fmaf(B.w, dy, C.x * dz));
    float qy = fmaf(B.w, dx, fmaf(B.y, dy, C.y * dz));
    float qz = fmaf(C.x, dx, fmaf(C.y, dy, B.z * dz));
    float dqd = fmaf(dx, qx, fmaf(dy, qy, dz * qz));
    float ri3 = ri * ri2;
    float ri5 = ri3 * ri2;
    float ri7 = ri5 * ri2;
    float a = fmaf(2.5f * dqd, ri7, A.w * ri3);
    ax = fmaf(a, dx, ax);
    ay = fmaf(a, dy, ay);
    az = fmaf(a, dz, az);
    ax = fmaf(-ri5, qx, ax);
    ay = fmaf(-ri5, qy, ay);
    az = fmaf(-ri5, qz, az);
}

__device__ __forceinline__ float pc_pot(float xi, float yi, float zi, float4 A,
                                        float4 B, float4 C, float eps2)
{
    float dx = A.x - xi, dy = A.y - yi, dz = A.z - zi;
    float s2 = fmaf(dx, dx, fmaf(dy, dy, fmaf(dz, dz, eps2)));
    float ri = rsqrtf(s2);
    float ri2 = ri * ri;
    float qx = fmaf(B.x, dx, fmaf(B.w, dy, C.x * dz));
    float qy = fmaf(B.w, dx, fmaf(B.y, dy, C.y * dz));
    float qz = fmaf(C.x, dx, fmaf(C.y, dy, B.z * dz));
    float dqd = fmaf(dx, qx, fmaf(dy, qy, dz * qz));
    float ri5 = ri * ri2 * ri2;
    return -(A.w * ri + 0.5f * dqd * ri5);
}

// far particle term (K = 1)
__device__ __forceinline__ void pp_far(float xi, float yi, float zi, float4 A,
                                       float eps2, float &ax, float &ay,
                                       float &az)
{
    float dx = A.x - xi, dy = A.y - yi, dz = A.z - zi;
    float s2 = fmaf(dx, dx, fmaf(dy, dy, fmaf(dz, dz, eps2)));
    float ri = rsqrtf(s2);
    float mr = A.w * ri;
    float ri2 = ri * ri;
    float f = mr * ri2;
    ax = fmaf(f, dx, ax);
    ay = fmaf(f, dy, ay);
    az = fmaf(f, dz, az);
}

// near particle term with the cut-off K; returns r^2 (unsoftened, FP32)
__device__ __forceinline__ float pp_near(float xi, float yi, float zi,
                                         float4 A, const ForceConsts &k,
                                         float &ax, float &ay, float &az,
                                         float &s_out)
{
    float dx = A.x - xi, dy = A.y - yi, dz = A.z - zi;
    float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
    float s2 = r2 + k.eps2;
    float ri = s2 > 0.0f ? rsqrtf(s2) : 0.0f;
    float s = s2 * ri;
    float x = __saturatef(fmaf(s, k.kA, k.kB));
    float x2 = x * x;
    float x4 = x2 * x2;
    float p = fmaf(-20.0f, x, 70.0f);
    p = fmaf(p, x, -84.0f);
    p = fmaf(p, x, 35.0f);
    float K = p * x4;
    // ordered so that K = 0 with a huge 1/s never forms 0 * inf
    float f = A.w * K;
    f = f * ri;
    f = f * ri;
    f = f * ri;
    ax = fmaf(f, dx, ax);
    ay = fmaf(f, dy, ay);
    az = fmaf(f, dz, az);
    s_out = s;
    return r2;
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


// Resident blocks per SM the force kernel's registers are sized for (0: let
// the compiler choose).
#ifndef P3T_FORCE_MIN_BLOCKS
#define P3T_FORCE_MIN_BLOCKS 0
#endif
constexpr int FSTACK = 768;  // walk stack entries per warp (child ranges)
constexpr int RING = 64;     // ring capacity (entries); never more than 63 used

struct __align__(16) WarpSmem {
    float4 t0[32], t1[32], t2[32];  // staged sources
    int stack[FSTACK];              // packed child ranges: child * 8 + nchild-1
    int cb[32];                     // cells of the current walk batch
    int pc[RING];                   // accepted cells
    int2 pf[RING];                  // far leaf ranges (first, count)
    int2 pn[RING];                  // near leaf ranges
    int tj[32];                     // sorted ids of staged particles
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
    int c = flag ? count : 0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
    r.nr += __popc(m);
    r.np += c;
}

// Takes the next `take` (<= 32, <= r.np) particle ids off the front of a
// ring of ranges into tj[0..take).
__device__ __forceinline__ void ring_take(int2 *ring, RangeRing &r, int take,
                                         int *tj, int lane)
{
    const bool have = lane < r.nr;
    int2 g = have ? ring[(r.head + lane) & (RING - 1)] : make_int2(0, 0);
    int inc = warp_incl_scan(g.y);
    int exc = inc - g.y;
    if (have && exc < take) {
        int stop = min(inc, take);
        for (int p = exc; p < stop; ++p) tj[p] = g.x + (p - exc);
    }
    const unsigned full = __ballot_sync(0xffffffffu, have && inc <= take);
    const int nfull = __popc(full);
    // the range straddling the tile boundary keeps its remainder
    if (lane == nfull && have && exc < take) {
        int used = take - exc;
        ring[(r.head + lane) & (RING - 1)] = make_int2(g.x + used, g.y - used);
    }
    __syncwarp();
    r.head = (r.head + nfull) & (RING - 1);
    r.nr -= nfull;
    r.np -= take;
}

template <bool POT>
struct GroupAcc {
    Acc3 a0, a1;
    float ph0, pl0, ph1, pl1;
};

// One tile of up to 32 accepted cells.
template <bool POT>
__device__ __forceinline__ void cell_tile(WarpSmem &S, int &head, int &n,
                                          int take, const float4 *cf0,
                                          const float4 *cf1, const float4 *cf2,
                                          float4 ct, float4 p0, float4 p1,
                                          float eps2, GroupAcc<POT> &A, int lane)
{
    if (lane < take) {
        int c = S.pc[(head + lane) & (RING - 1)];
        float4 a = cf0[c], bb = cf1[c], cc = cf2[c];
        S.t0[lane] = make_float4(__fadd_rn(__fsub_rn(a.x, ct.x), bb.x),
                                 __fadd_rn(__fsub_rn(a.y, ct.y), bb.y),
                                 __fadd_rn(__fsub_rn(a.z, ct.z), bb.z), a.w);
        S.t1[lane] = make_float4(bb.w, cc.x, -(bb.w + cc.x), cc.y);
        S.t2[lane] = make_float4(cc.z, cc.w, 0.0f, 0.0f);
    } else {
        S.t0[lane] = far_pad();
        S.t1[lane] = make_float4(0.f, 0.f, 0.f, 0.f);
        S.t2[lane] = make_float4(0.f, 0.f, 0.f, 0.f);
    }
    head = (head + take) & (RING - 1);
    n -= take;
    __syncwarp();
    float tx0 = 0.f, ty0 = 0.f, tz0 = 0.f, tx1 = 0.f, ty1 = 0.f, tz1 = 0.f,
          tp0 = 0.f, tp1 = 0.f;
#pragma unroll kPcUnroll
    for (int j = 0; j < 32; ++j) {
        const float4 a = S.t0[j], bq = S.t1[j], cq = S.t2[j];
        pc_term(p0.x, p0.y, p0.z, a, bq, cq, eps2, tx0, ty0, tz0);
        pc_term(p1.x, p1.y, p1.z, a, bq, cq, eps2, tx1, ty1, tz1);
        if (POT) {
            tp0 += pc_pot(p0.x, p0.y, p0.z, a, bq, cq, eps2);
            tp1 += pc_pot(p1.x, p1.y, p1.z, a, bq, cq, eps2);
        }
    }
    A.a0.add(tx0, ty0, tz0);
    A.a1.add(tx1, ty1, tz1);
    if (POT) {
        two_sum_add(A.ph0, A.pl0, tp0);
        two_sum_add(A.ph1, A.pl1, tp1);
    }
    __syncwarp();
}

// One tile of up to 32 particles from a ring of leaf ranges.
template <bool NEAR, bool POT>
__device__ __forceinline__ void particle_tile(
    WarpSmem &S, int2 *ring, RangeRing &r, int take, const float4 *phi,
    const float4 *plo, float4 ct, float4 p0, float4 p1, int k0, int k1,
    const ForceConsts &k, GroupAcc<POT> &A, int lane)
{
    ring_take(ring, r, take, S.tj, lane);
    if (lane < take) {
        int j = S.tj[lane];
        S.t0[lane] = rel4(phi[j], plo[j], ct);
    } else {
        S.t0[lane] = far_pad();
        S.tj[lane] = -1;
    }
    __syncwarp();
    float tx0 = 0.f, ty0 = 0.f, tz0 = 0.f, tx1 = 0.f, ty1 = 0.f, tz1 = 0.f,
          tp0 = 0.f, tp1 = 0.f;
    if (NEAR) {
#pragma unroll 4
        for (int j = 0; j < 32; ++j) {
            const float4 a = S.t0[j];
            float s0, s1;
            pp_near(p0.x, p0.y, p0.z, a, k, tx0, ty0, tz0, s0);
            pp_near(p1.x, p1.y, p1.z, a, k, tx1, ty1, tz1, s1);
            if (POT) {
                const int kj = S.tj[j];
                if (kj >= 0 && kj != k0) tp0 -= a.w * (float)w_over_s((double)s0, k);
                if (kj >= 0 && kj != k1) tp1 -= a.w * (float)w_over_s((double)s1, k);
            }
        }
    } else {
#pragma unroll 8
        for (int j = 0; j < 32; ++j) {
            const float4 a = S.t0[j];
            pp_far(p0.x, p0.y, p0.z, a, k.eps2, tx0, ty0, tz0);
            pp_far(p1.x, p1.y, p1.z, a, k.eps2, tx1, ty1, tz1);
            if (POT) {
                float dx = a.x - p0.x, dy = a.y - p0.y, dz = a.z - p0.z;
                tp0 -= a.w * rsqrtf(fmaf(dx, dx, fmaf(dy, dy, fmaf(dz, dz, k.eps2))));
                dx = a.x - p1.x; dy = a.y - p1.y; dz = a.z - p1.z;
                tp1 -= a.w * rsqrtf(fmaf(dx, dx, fmaf(dy, dy, fmaf(dz, dz, k.eps2))));
            }
        }
    }
    A.a0.add(tx0, ty0, tz0);
    A.a1.add(tx1, ty1, tz1);
    if (POT) {
        two_sum_add(A.ph0, A.pl0, tp0);
        two_sum_add(A.ph1, A.pl1, tp1);
    }
    __syncwarp();
}

template <bool POT>
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
             float *__restrict__ acc, double *__restrict__ pot,
             P3TDevState *st)
{
    __shared__ WarpSmem smem[FW];
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const unsigned full = 0xffffffffu, lt = lanemask_lt();
    WarpSmem &S = smem[w];
    const int G = st->ngroup;
    for (;;) {
        int g = 0;
        if (lane == 0) g = (int)atomicAdd(&st->work, 1u);
        g = __shfl_sync(full, g, 0);
        if (g >= G) break;
        const int2 gr = grange[g];
        const float4 ct = gctr[g];
        const float4 gmn = gmin[g], gmx = gmax[g];
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
        const float4 p0 = v0 ? rel4(phi[k0], plo[k0], ct) : far_pad();
        const float4 p1 = v1 ? rel4(phi[k1], plo[k1], ct) : far_pad();
        GroupAcc<POT> A;
        A.a0.zero();
        A.a1.zero();
        A.ph0 = A.pl0 = A.ph1 = A.pl1 = 0.f;
        int pc_head = 0, pc_n = 0;
        RangeRing rf = {0, 0, 0}, rn = {0, 0, 0};
        long long cnt_pc = 0, cnt_pn = 0, cnt_pf = 0;

        if (lane == 0) S.stack[0] = cl * 8;  // the cluster's root, one cell
        int top = 1;
        int iter = 0;
        bool overflow = false;
        __syncwarp();
        while (top > 0) {
            if (++iter > (1 << 24)) {  // a finite tree never gets here
                overflow = true;
                break;
            }
            // pop child ranges from the top holding at most 32 cells
            int rx = 0, ry = 0;
            if (lane < top) {
                int e = S.stack[top - 1 - lane];
                rx = e >> 3;
                ry = (e & 7) + 1;
            }
            int inc = warp_incl_scan(ry);
            bool take = lane < top && inc <= 32;
            int ntake = __popc(__ballot_sync(full, take));
            int total = __shfl_sync(full, inc, ntake - 1);
            if (take)
                for (int t = 0; t < ry; ++t) S.cb[inc - ry + t] = rx + t;
            top -= ntake;
            __syncwarp();
            const int c = lane < total ? S.cb[lane] : -1;
            __syncwarp();

            bool is_pc = false, near = false, farl = false, open = false;
            int child = 0, nchild = 0, pfirst = 0, pcount = 0;
            if (c >= 0) {
                const float4 cmn = wmin[c], cmx = wmax[c];
                float d2 = box_d2(gmn, gmx, cmn, cmx);
                float l = box_side(cmn, cmx);
                if (mac_accept(d2, l, theta2, hg2)) {
                    is_pc = true;
                } else {
                    child = __float_as_int(cmn.w);
                    nchild = __float_as_int(cmx.w);
                    if (nchild == 0) {
                        int4 nd = node[c];
                        pfirst = nd.x;
                        pcount = nd.y;
                        near = d2 <= hg2;
                        farl = !near;
                    } else {
                        open = true;
                    }
                }
            }
            // accepted cells -> cell ring
            {
                unsigned m = __ballot_sync(full, is_pc);
                if (is_pc) S.pc[(pc_head + pc_n + __popc(m & lt)) & (RING - 1)] = c;
                pc_n += __popc(m);
                cnt_pc += __popc(m);
            }
            // leaves -> particle rings
            {
                int before = rn.np;
                ring_push_ranges(S.pn, rn, near, pfirst, pcount, lane);
                cnt_pn += rn.np - before;
                before = rf.np;
                ring_push_ranges(S.pf, rf, farl, pfirst, pcount, lane);
                cnt_pf += rf.np - before;
            }
            // opened cells -> stack
            {
                unsigned mo = __ballot_sync(full, open);
                int np = __popc(mo);
                if (top + np > FSTACK) {
                    overflow = true;
                    break;
                }
                if (open) S.stack[top + __popc(mo & lt)] = child * 8 + (nchild - 1);
                top += np;
            }
            __syncwarp();
            // evaluate every full tile
            while (pc_n >= 32)
                cell_tile<POT>(S, pc_head, pc_n, 32, cf0, cf1, cf2, ct, p0, p1,
                               kg.eps2, A, lane);
            while (rf.np >= 32)
                particle_tile<false, POT>(S, S.pf, rf, 32, phi, plo, ct, p0, p1,
                                          k0, k1, kg, A, lane);
            while (rn.np >= 32)
                particle_tile<true, POT>(S, S.pn, rn, 32, phi, plo, ct, p0, p1,
                                         k0, k1, kg, A, lane);
        }
        if (overflow) {
            if (lane == 0) p3t_raise(st, P3T_ERR_CAPACITY);
            continue;
        }
        // the partial tiles left over
        if (pc_n > 0)
            cell_tile<POT>(S, pc_head, pc_n, pc_n, cf0, cf1, cf2, ct, p0, p1,
                           kg.eps2, A, lane);
        if (rf.np > 0)
            particle_tile<false, POT>(S, S.pf, rf, rf.np, phi, plo, ct, p0, p1,
                                      k0, k1, kg, A, lane);
        if (rn.np > 0)
            particle_tile<true, POT>(S, S.pn, rn, rn.np, phi, plo, ct, p0, p1,
                                     k0, k1, kg, A, lane);
        // ---- write back in the caller's order ----
        const float Gc = k.G;
        if (v0) {
            int o = order[k0];
            acc[o] = Gc * (A.a0.hx + A.a0.lx);
            acc[(size_t)n + o] = Gc * (A.a0.hy + A.a0.ly);
            acc[2 * (size_t)n + o] = Gc * (A.a0.hz + A.a0.lz);
            if (POT) pot[o] = (double)Gc * ((double)A.ph0 + (double)A.pl0);
        }
        if (v1) {
            int o = order[k1];
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

// Resets the per-call counters of a force evaluation.
__global__ void k_force_reset(P3TDevState *st)
{
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        st->work = 0;
        st->tot[0] = st->tot[1] = st->tot[2] = 0;
        st->int_pc = st->int_pp = st->int_ppn = 0;
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

}  // namespace

int p3t_run_force(p3t_ctx *c, float *acc, double *pot, cudaStream_t s)
{
    const int n = (int)c->n;
    k_force_reset<<<1, 32, 0, s>>>(c->st);
    p3t_count_launches(1);
    // the group count is read on the device; size the grid from the bound
    const int64_t G = (n + 15) / 16 + c->nclus;
    ForceConsts k = make_consts(c->p);
    float theta2, hg2;
    p3t_mac_constants(&c->p, &theta2, &hg2);
    int blocks = (int)((G + FW - 1) / FW);
    if (blocks > c->sms * 16) blocks = c->sms * 16;
    if (pot)
        k_walk_force<true><<<blocks, FW * 32, 0, s>>>(
            c->gclus, c->cc, c->grange, c->gmin, c->gmax, c->gctr, c->wmin,
            c->wmax, c->node, theta2, c->phi, c->plo, c->cf0, c->cf1, c->cf2,
            c->order, n, k, acc, pot, c->st);
    else
        k_walk_force<false><<<blocks, FW * 32, 0, s>>>(
            c->gclus, c->cc, c->grange, c->gmin, c->gmax, c->gctr, c->wmin,
            c->wmax, c->node, theta2, c->phi, c->plo, c->cf0, c->cf1, c->cf2,
            c->order, n, k, acc, pot, c->st);
    p3t_count_launches(1);
    P3T_CUDA_TRY(cudaGetLastError());
    return P3T_OK;
}
