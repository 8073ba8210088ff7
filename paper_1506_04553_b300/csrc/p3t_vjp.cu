// Backward pass: vector-Jacobian product of the tree force.
//
// For L = sum_i w_i . a_i with the tree topology, the groups and the
// interaction sets held fixed (no counterpart in the paper; derived from
// Eq. 8 and the softened quadrupole expansion), this file computes dL/dx and
// dL/dm for every particle.
//   pair term, d = x_j - x_i, s^2 = |d|^2 + eps^2:
//     f = G m_j K d / s^3,  J = df/dd = G m_j [phi I + psi d d^T],
//     phi = K / s^3,  psi = K'(s) / s^4 - 3 K / s^5
//     dL/dx_i -= J w_i,  dL/dx_j += J w_i,  dL/dm_j += G phi (w_i . d)
//   cell term, d = com - x_i:
//     f = G [M d / s^3 - Q d / s^5 + (5/2)(d.Q.d) d / s^7]
//     dL/dx_i -= J^T w_i and the cell adjoints dL/dcom += J^T w_i,
//     dL/dM += G (w_i . d) / s^3, dL/dQ (symmetric part)
//       = G [-(w d^T + d w^T) / (2 s^5) + (5/2)(w . d) d d^T / s^7]
//   cell adjoints -> members k (e = x_k - com):
//     dL/dx_k += (m_k / M) dL/dcom + m_k (6 S e - 2 tr(S) e)
//     dL/dm_k += dL/dM + e . dL/dcom / M + 3 e.S.e - |e|^2 tr(S)
//
// k_walk_vjp walks each group exactly as the force kernel does (shared
// walk in p3t_walkcore.cuh, so the interaction sets are recomputed, not
// stored).  The group's particles are staged once per group in shared
// memory, in group-relative coordinates.  For a tile of up to 64 sources
// (cells, or particles of leaves) each lane owns two sources, held as the
// two halves of every FP32x2 operand, and sweeps the particles one at a time
// (each broadcast to both halves).  The sources' adjoints stay in the lane's
// registers and go to FP64 atomics once per tile; the particle-side products
// (3 per particle, the lane's two sources added) are summed over the lanes
// by a warp reduce-scatter, four particles at a time, and kept by the
// particle's owner lane in two-sum (hi, lo) FP32 accumulators.  Two sources
// per lane halve the reduce-scatter per source and particle.
// The cell adjoints then reach the member particles in FP64: with
// T = 3 S - tr(S) I and e = x_k - com (so 6 S e - 2 tr(S) e = 2 T e and
// 3 e.S.e - |e|^2 tr(S) = e.T.e), the sums over a particle's ancestors are
// a quadratic form in x_k.  One thread per leaf adds its ancestors' terms
// about the leaf's centre of mass r (delta = com - r, x' = x_k - r):
//   P = sum dL/dcom / M,  Ts = sum T,  Tc = sum T delta,
//   a = sum (dL/dM - delta . dL/dcom / M + delta.T.delta)
// and every member gets dL/dx_k += m_k (P + 2 (Ts x' - Tc)) and
// dL/dm_k += a + x'.P + x'.Ts.x' - 2 x'.Tc.
#include <math.h>

#include "p3t_walkcore.cuh"

namespace {

using p3t_walk::Smem;

#ifndef P3T_VJP_MIN_BLOCKS
#define P3T_VJP_MIN_BLOCKS 0
#endif
// The warps per block of k_walk_vjp are a template parameter (2 or 4),
// chosen per context by the autotuner; 4 by default.
// Particles per i-side reduce-scatter.  Eight would save 1.5 instructions
// per particle, but the eight-fold unrolled tiles no longer fit the
// instruction cache (stalls for lack of an instruction: 0.35 -> 1.2 per
// issue, 30.9 -> 33.8 ms at 2^20).
constexpr int NPC = 4;
constexpr int GMAX = 64;  // particle slots of a group

struct VjpConsts {
    float eps2, kA, kB;
    double G;
};

typedef float2 f2;
__device__ __forceinline__ f2 add2(f2 a, f2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ f2 mul2(f2 a, f2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ f2 fma2(f2 a, f2 b, f2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ f2 dup2(float a) { return make_float2(a, a); }

// 1/sqrt(x) with subnormal inputs flushed (rsqrt.approx.ftz.f32); used only
// where x >= (near radius)^2 > 0 or x is a padding distance of ~1e31.
__device__ __forceinline__ float rsqrt_ftz(float x)
{
    float r;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

// Padding: absent sources sit at -PAD, absent particles at +PAD, so that no
// padded pair has a zero distance; masses and weights of padding are zero.
constexpr float PAD = 1e15f;

__device__ __forceinline__ float4 rel(float4 hi, float4 lo, float4 c)
{
    return make_float4(__fadd_rn(__fsub_rn(hi.x, c.x), lo.x),
                       __fadd_rn(__fsub_rn(hi.y, c.y), lo.y),
                       __fadd_rn(__fsub_rn(hi.z, c.z), lo.z), hi.w);
}

__device__ __forceinline__ void two_sum_add(float &hi, float &lo, float v)
{
    float s = __fadd_rn(hi, v);
    float bb = __fsub_rn(s, hi);
    float err = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bb)), __fsub_rn(v, bb));
    hi = s;
    lo = __fadd_rn(lo, err);
}

// Warp reduce-scatter of NS sources x NV values held by every lane: after
// the call a[0][0..NV) of lane l holds the warp-wide totals of source
// src_of<NS>(l); the 32/NS lanes sharing that source hold the same totals.
// log2(NS) levels exchange half of the remaining sources with a partner,
// the remaining levels are a butterfly over NV values.
template <int NS>
__device__ __forceinline__ int src_of(int lane)
{
    int s = 0;
#pragma unroll
    for (int b = 0; (1 << b) < NS; ++b) s = 2 * s + ((lane >> (4 - b)) & 1);
    return s;
}

template <int NS, int NV>
__device__ __forceinline__ void reduce_scatter(float (&a)[NS][NV], int lane)
{
#pragma unroll
    for (int b = 0; (1 << b) < NS; ++b) {
        const int mask = 16 >> b;
        const int half = NS >> (b + 1);
        const bool upper = (lane & mask) != 0;
#pragma unroll
        for (int q = 0; q < half; ++q)
#pragma unroll
            for (int v = 0; v < NV; ++v) {
                const float lo = a[q][v], hi = a[q + half][v];
                const float send = upper ? lo : hi;
                const float keep = upper ? hi : lo;
                a[q][v] = keep + __shfl_xor_sync(0xffffffffu, send, mask);
            }
    }
#pragma unroll
    for (int mask = 16 / NS; mask > 0; mask >>= 1)
#pragma unroll
        for (int v = 0; v < NV; ++v)
            a[0][v] += __shfl_xor_sync(0xffffffffu, a[0][v], mask);
}

// Value v of a[0] without dynamic register indexing.
template <int NV>
__device__ __forceinline__ float pick(const float (&a)[NV], int v)
{
    float r = a[0];
#pragma unroll
    for (int q = 1; q < NV; ++q) r = (v == q) ? a[q] : r;
    return r;
}

// The group's particles, staged once per group: negated group-relative
// positions and weights, slot = particle index in the group, each value
// duplicated (slot p fills 12 floats: nx, nx, ny, ny, ..., wz, wz), so that
// three 128-bit loads give a particle as broadcast pairs; and the
// particle-side tile sums.
struct __align__(16) VjpSmem {
    float pd[GMAX * 12];
    float ts[3][GMAX];
};

__device__ __forceinline__ void stage_slot(VjpSmem *V, int slot, float nx,
                                           float ny, float nz, float wx,
                                           float wy, float wz)
{
    float4 *d = reinterpret_cast<float4 *>(V->pd) + slot * 3;
    d[0] = make_float4(nx, nx, ny, ny);
    d[1] = make_float4(nz, nz, wx, wx);
    d[2] = make_float4(wy, wy, wz, wz);
}

// A particle as broadcast pairs.
struct PPair {
    f2 nx, ny, nz, wx, wy, wz;
};

__device__ __forceinline__ PPair load_dup(const VjpSmem *V, int j)
{
    const float4 *t4 = reinterpret_cast<const float4 *>(V->pd) + j * 3;
    const float4 A = t4[0], B = t4[1], C = t4[2];
    PPair r;
    r.nx = make_float2(A.x, A.y);
    r.ny = make_float2(A.z, A.w);
    r.nz = make_float2(B.x, B.y);
    r.wx = make_float2(B.z, B.w);
    r.wy = make_float2(C.x, C.y);
    r.wz = make_float2(C.z, C.w);
    return r;
}

// Two cells (the halves) against one particle (broadcast pairs).
struct CellSrc {
    f2 X, Y, Z, M, M3, Qxx, Qyy, Qzz, Qxy, Qxz, Qyz;  // M3 = -3 M
};

// J^T w per half (jx, jy, jz) and the cell adjoints
// acc = (dL/dM, dL/dcom xyz, 2S xx yy zz xy xz yz) per half, all without G.
__device__ __forceinline__ void cell_pair(const CellSrc &c, f2 nx, f2 ny,
                                          f2 nz, f2 wx, f2 wy, f2 wz, f2 eps2,
                                          f2 (&acc)[10], f2 &jx, f2 &jy,
                                          f2 &jz)
{
    const f2 dx = add2(c.X, nx), dy = add2(c.Y, ny), dz = add2(c.Z, nz);
    const f2 s2 = fma2(dx, dx, fma2(dy, dy, fma2(dz, dz, eps2)));
    const f2 ri = make_float2(rsqrt_ftz(s2.x), rsqrt_ftz(s2.y));
    const f2 ri2 = mul2(ri, ri);
    const f2 ri3 = mul2(ri, ri2), ri5 = mul2(ri3, ri2), ri7 = mul2(ri5, ri2);
    // Q = [[Qxx, Qxy, Qxz], [Qxy, Qyy, Qyz], [Qxz, Qyz, Qzz]]
    const f2 qx = fma2(c.Qxx, dx, fma2(c.Qxy, dy, mul2(c.Qxz, dz)));
    const f2 qy = fma2(c.Qxy, dx, fma2(c.Qyy, dy, mul2(c.Qyz, dz)));
    const f2 qz = fma2(c.Qxz, dx, fma2(c.Qyz, dy, mul2(c.Qzz, dz)));
    const f2 dqd = fma2(dx, qx, fma2(dy, qy, mul2(dz, qz)));
    const f2 wd = fma2(wx, dx, fma2(wy, dy, mul2(wz, dz)));
    const f2 wqd = fma2(wx, qx, fma2(wy, qy, mul2(wz, qz)));
    // J^T w = cw w + cd d + cq q - Qw / s^5 with
    //   cw = M / s^3 + (5/2) dQd / s^7,   cq = 5 wd / s^7,
    //   cd = -3 M wd / s^5 + 5 wQd / s^7 - (35/2) dQd wd / s^9
    //      = [-3 M wd + (5 wQd - (35/2) dQd wd / s^2) / s^2] / s^5;
    // with v = -w / s^5 and u = cq d + v, cq q - Qw / s^5 = Q u, so
    //   J^T w = cw w + cd d + Q u
    const f2 cw = fma2(mul2(dup2(2.5f), dqd), ri7, mul2(c.M, ri3));
    const f2 cdi = fma2(mul2(mul2(dqd, wd), ri2), dup2(-17.5f), mul2(dup2(5.0f), wqd));
    const f2 cd = mul2(fma2(cdi, ri2, mul2(c.M3, wd)), ri5);
    const f2 cq = mul2(dup2(5.0f), mul2(wd, ri7));  // 5 wd / s^7
    const f2 nri5 = mul2(dup2(-1.0f), ri5);
    const f2 vx = mul2(nri5, wx), vy = mul2(nri5, wy), vz = mul2(nri5, wz);
    const f2 ux = fma2(cq, dx, vx), uy = fma2(cq, dy, vy), uz = fma2(cq, dz, vz);
    jx = fma2(cw, wx, fma2(cd, dx, fma2(c.Qxx, ux, fma2(c.Qxy, uy, mul2(c.Qxz, uz)))));
    jy = fma2(cw, wy, fma2(cd, dy, fma2(c.Qxy, ux, fma2(c.Qyy, uy, mul2(c.Qyz, uz)))));
    jz = fma2(cw, wz, fma2(cd, dz, fma2(c.Qxz, ux, fma2(c.Qyz, uy, mul2(c.Qzz, uz)))));
    acc[0] = fma2(wd, ri3, acc[0]);
    acc[1] = add2(acc[1], jx);
    acc[2] = add2(acc[2], jy);
    acc[3] = add2(acc[3], jz);
    // 2S = -(w d^T + d w^T) / s^5 + 5 wd d d^T / s^7 (twice the adjoint: its
    // factors are those of J^T w): 2S_ab = d_a u_b + v_a d_b,
    // 2S_aa = d_a (u_a + v_a)
    acc[4] = fma2(dx, add2(ux, vx), acc[4]);
    acc[5] = fma2(dy, add2(uy, vy), acc[5]);
    acc[6] = fma2(dz, add2(uz, vz), acc[6]);
    acc[7] = fma2(dx, uy, fma2(vx, dy, acc[7]));
    acc[8] = fma2(dx, uz, fma2(vx, dz, acc[8]));
    acc[9] = fma2(dy, uz, fma2(vy, dz, acc[9]));
}

// Two source particles (the halves) against one particle (broadcast pairs).
struct PartSrc {
    f2 X, Y, Z, m;
};

// J w per half (jx, jy, jz) and the source adjoints acc = (dL/dx_j xyz,
// dL/dm_j) per half, all without G.  selfx / selfy: the half's source is the
// particle itself (contributes 0).
template <bool NEAR>
__device__ __forceinline__ void pair_pair(const PartSrc &p, f2 nx, f2 ny,
                                          f2 nz, f2 wx, f2 wy, f2 wz,
                                          bool selfx, bool selfy, f2 eps2,
                                          f2 kA, f2 kB, f2 (&acc)[4], f2 &jx,
                                          f2 &jy, f2 &jz)
{
    const f2 dx = add2(p.X, nx), dy = add2(p.Y, ny), dz = add2(p.Z, nz);
    const f2 s2 = fma2(dx, dx, fma2(dy, dy, fma2(dz, dz, eps2)));
    f2 ri;
    if (NEAR)
        ri = make_float2((s2.x > 0.0f && !selfx) ? rsqrtf(s2.x) : 0.0f,
                         (s2.y > 0.0f && !selfy) ? rsqrtf(s2.y) : 0.0f);
    else  // far leaves: s^2 >= (near radius)^2, never the particle itself
        ri = make_float2(rsqrt_ftz(s2.x), rsqrt_ftz(s2.y));
    const f2 ri2 = mul2(ri, ri);
    const f2 ri3 = mul2(ri2, ri);
    f2 phi, psi;
    if (NEAR) {
        const f2 sv = mul2(s2, ri);
        f2 x = fma2(sv, kA, kB);
        x = make_float2(__saturatef(x.x), __saturatef(x.y));
        const f2 x2 = mul2(x, x), x4 = mul2(x2, x2);
        f2 pk = fma2(dup2(-20.0f), x, dup2(70.0f));
        pk = fma2(pk, x, dup2(-84.0f));
        pk = fma2(pk, x, dup2(35.0f));
        const f2 K = mul2(pk, x4);
        const f2 omx = fma2(x, dup2(-1.0f), dup2(1.0f));
        const f2 Kp = mul2(mul2(mul2(dup2(140.0f), mul2(x2, x)),
                                mul2(mul2(omx, omx), omx)), kA);
        // products ordered so that K = 0 with a huge 1/s never forms 0*inf
        phi = mul2(mul2(mul2(K, ri), ri), ri);
        psi = fma2(dup2(-3.0f), mul2(mul2(phi, ri), ri),
                   mul2(mul2(mul2(mul2(Kp, ri), ri), ri), ri));
    } else {
        phi = ri3;
        psi = mul2(mul2(dup2(-3.0f), ri3), ri2);
    }
    const f2 wd = fma2(wx, dx, fma2(wy, dy, mul2(wz, dz)));
    const f2 mphi = mul2(p.m, phi);
    const f2 mpw = mul2(mul2(p.m, psi), wd);
    jx = fma2(mphi, wx, mul2(mpw, dx));
    jy = fma2(mphi, wy, mul2(mpw, dy));
    jz = fma2(mphi, wz, mul2(mpw, dz));
    acc[0] = add2(acc[0], jx);
    acc[1] = add2(acc[1], jy);
    acc[2] = add2(acc[2], jz);
    acc[3] = fma2(phi, wd, acc[3]);
}

// Per-lane state of one group.  Lane l owns particle slots l and l + 32.
struct VjpEval {
    VjpSmem *V;
    int lane, gfirst, npart;  // npart: particles swept (multiple of NPC)
    float4 ct;
    float ih[2][3], il[2][3];  // owner's dL/dx sums (without G, sign: + J w)
    const float4 *phi, *plo, *cf0, *cf1, *cf2;
    const int *order;
    double *gpos, *gmass, *cadj;
    int n;
    VjpConsts k;

    // Particle-side products of NPC particles starting at particle ch (the
    // lane's two sources already added): summed over the lanes and stored
    // in the tile sums.
    __device__ __forceinline__ void flush(float (&r)[NPC][3], int ch)
    {
        reduce_scatter<NPC, 3>(r, lane);
        const int v = lane & (32 / NPC - 1);
        if (v < 3) V->ts[v][ch + src_of<NPC>(lane)] = pick<3>(r[0], v);
    }

    // The owners add the tile sums of their particles.
    __device__ __forceinline__ void tile_end()
    {
        __syncwarp();
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            two_sum_add(ih[0][c], il[0][c], V->ts[c][lane]);
            two_sum_add(ih[1][c], il[1][c], V->ts[c][lane + 32]);
        }
        __syncwarp();
    }

    // Cell tile: ids in S.tj[0..take), take <= 64; lane l owns cells l and
    // l + 32, the halves of every FP32x2 operand.
    __device__ __forceinline__ void cells(Smem &S, int take)
    {
        float v[2][11];  // X Y Z M -3M Qxx Qyy Qzz Qxy Qxz Qyz
        int cid[2];
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int slot = lane + 32 * h;
            cid[h] = slot < take ? S.tj[slot] : -1;
            if (cid[h] >= 0) {
                const float4 a = cf0[cid[h]], bb = cf1[cid[h]], cc = cf2[cid[h]];
                v[h][0] = __fadd_rn(__fsub_rn(a.x, ct.x), bb.x);
                v[h][1] = __fadd_rn(__fsub_rn(a.y, ct.y), bb.y);
                v[h][2] = __fadd_rn(__fsub_rn(a.z, ct.z), bb.z);
                v[h][3] = a.w;
                v[h][4] = -3.0f * a.w;
                v[h][5] = bb.w;
                v[h][6] = cc.x;
                v[h][7] = -(bb.w + cc.x);
                v[h][8] = cc.y;
                v[h][9] = cc.z;
                v[h][10] = cc.w;
            } else {
                v[h][0] = v[h][1] = v[h][2] = -PAD;
#pragma unroll
                for (int q = 3; q < 11; ++q) v[h][q] = 0.0f;
            }
        }
        CellSrc c;
        c.X = make_float2(v[0][0], v[1][0]);
        c.Y = make_float2(v[0][1], v[1][1]);
        c.Z = make_float2(v[0][2], v[1][2]);
        c.M = make_float2(v[0][3], v[1][3]);
        c.M3 = make_float2(v[0][4], v[1][4]);
        c.Qxx = make_float2(v[0][5], v[1][5]);
        c.Qyy = make_float2(v[0][6], v[1][6]);
        c.Qzz = make_float2(v[0][7], v[1][7]);
        c.Qxy = make_float2(v[0][8], v[1][8]);
        c.Qxz = make_float2(v[0][9], v[1][9]);
        c.Qyz = make_float2(v[0][10], v[1][10]);
        __syncwarp();  // S.tj is rewritten by the walk after the tile
        f2 acc[10];
#pragma unroll
        for (int q = 0; q < 10; ++q) acc[q] = dup2(0.0f);
        const f2 e2 = dup2(k.eps2);
        for (int ch = 0; ch < npart; ch += NPC) {
            float r[NPC][3];
#pragma unroll
            for (int u = 0; u < NPC; ++u) {
                f2 jx, jy, jz;
                const PPair q = load_dup(V, ch + u);
                cell_pair(c, q.nx, q.ny, q.nz, q.wx, q.wy, q.wz, e2, acc, jx, jy,
                          jz);
                r[u][0] = __fadd_rn(jx.x, jx.y);
                r[u][1] = __fadd_rn(jy.x, jy.y);
                r[u][2] = __fadd_rn(jz.x, jz.y);
            }
            flush(r, ch);
        }
        tile_end();
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            if (cid[h] >= 0) {
                double *dst = cadj + (size_t)cid[h] * 10;
#pragma unroll
                for (int q = 0; q < 10; ++q)
                    atomicAdd(dst + q, k.G * (double)(h == 0 ? acc[q].x : acc[q].y));
            }
        }
    }

    // Particle tile: ids in S.tj[0..take), take <= 64; lane l owns sources
    // l and l + 32, the halves of every FP32x2 operand.
    template <bool NEAR>
    __device__ __forceinline__ void particles(Smem &S, int take)
    {
        float v[2][4];  // X Y Z m
        int sj[2];
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int slot = lane + 32 * h;
            sj[h] = slot < take ? S.tj[slot] : -1;
            if (sj[h] >= 0) {
                const float4 a = rel(phi[sj[h]], plo[sj[h]], ct);
                v[h][0] = a.x;
                v[h][1] = a.y;
                v[h][2] = a.z;
                v[h][3] = a.w;
            } else {
                v[h][0] = v[h][1] = v[h][2] = -PAD;
                v[h][3] = 0.0f;
            }
        }
        PartSrc p;
        p.X = make_float2(v[0][0], v[1][0]);
        p.Y = make_float2(v[0][1], v[1][1]);
        p.Z = make_float2(v[0][2], v[1][2]);
        p.m = make_float2(v[0][3], v[1][3]);
        __syncwarp();  // S.tj is rewritten by the walk after the tile
        f2 acc[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) acc[q] = dup2(0.0f);
        const f2 e2 = dup2(k.eps2), kA = dup2(k.kA), kB = dup2(k.kB);
        // the sources' slots if they are in the group (else negative)
        const int self0 = sj[0] - gfirst, self1 = sj[1] - gfirst;
        for (int ch = 0; ch < npart; ch += NPC) {
            float r[NPC][3];
#pragma unroll
            for (int u = 0; u < NPC; ++u) {
                const int j = ch + u;
                f2 jx, jy, jz;
                const PPair q = load_dup(V, j);
                pair_pair<NEAR>(p, q.nx, q.ny, q.nz, q.wx, q.wy, q.wz,
                                self0 == j, self1 == j, e2, kA, kB, acc, jx,
                                jy, jz);
                r[u][0] = __fadd_rn(jx.x, jx.y);
                r[u][1] = __fadd_rn(jy.x, jy.y);
                r[u][2] = __fadd_rn(jz.x, jz.y);
            }
            flush(r, ch);
        }
        tile_end();
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            if (sj[h] >= 0) {
                const int o = order[sj[h]];
#pragma unroll
                for (int q = 0; q < 3; ++q)
                    atomicAdd(gpos + (size_t)q * n + o,
                              k.G * (double)(h == 0 ? acc[q].x : acc[q].y));
                atomicAdd(gmass + o, k.G * (double)(h == 0 ? acc[3].x : acc[3].y));
            }
        }
    }
};

template <int VW>
__global__ void __launch_bounds__(VW * 32, P3T_VJP_MIN_BLOCKS)
k_walk_vjp(const int *__restrict__ gclus,
           const ClusterConsts *__restrict__ ccs,
           const int2 *__restrict__ grange,
           const float4 *__restrict__ gmin, const float4 *__restrict__ gmax,
           const float4 *__restrict__ gctr, const float4 *__restrict__ wmin,
           const float4 *__restrict__ wmax,
           float theta2, const float4 *__restrict__ phi,
           const float4 *__restrict__ plo, const float4 *__restrict__ cf0,
           const float4 *__restrict__ cf1, const float4 *__restrict__ cf2,
           const int *__restrict__ order, int n, VjpConsts k,
           const float *__restrict__ w, double *__restrict__ gpos,
           double *__restrict__ gmass, double *__restrict__ cadj,
           const int *__restrict__ gperm, P3TDevState *st, long long lim_walk)
{
    __shared__ Smem smem[VW];
    __shared__ VjpSmem vsm[VW];
    const int wi = threadIdx.x >> 5, lane = threadIdx.x & 31;
    Smem &S = smem[wi];
    if (st->error) return;  // no valid tree
    const int G = st->ngroup;
    for (;;) {
        int g = 0;
        if (lane == 0) g = (int)atomicAdd(&st->work_vjp, 1u);
        g = __shfl_sync(0xffffffffu, g, 0);
        if (g >= G) break;
        g = gperm[g];
        const int2 gr = grange[g];
        const int cl = gclus[g];
        const ClusterConsts cc = ccs[cl];
        VjpEval ev;
        ev.V = &vsm[wi];
        ev.lane = lane;
        ev.gfirst = gr.x;
        ev.npart = ((gr.y + NPC - 1) / NPC) * NPC;
        ev.ct = gctr[g];
        // stage the group's particles; slots past the group are padding
        __syncwarp();  // the previous group's reads of vsm are done
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int slot = lane + 32 * h;
            float4 p = make_float4(PAD, PAD, PAD, 0.0f);
            float3 wv = make_float3(0.0f, 0.0f, 0.0f);
            if (slot < gr.y) {
                const int kk = gr.x + slot, o = order[kk];
                p = rel(phi[kk], plo[kk], ev.ct);
                wv = make_float3(w[o], w[(size_t)n + o], w[2 * (size_t)n + o]);
            }
            stage_slot(ev.V, slot, -p.x, -p.y, -p.z, wv.x, wv.y, wv.z);
            for (int c = 0; c < 3; ++c) ev.ih[h][c] = ev.il[h][c] = 0.0f;
        }
        __syncwarp();
        ev.phi = phi;
        ev.plo = plo;
        ev.cf0 = cf0;
        ev.cf1 = cf1;
        ev.cf2 = cf2;
        ev.order = order;
        ev.gpos = gpos;
        ev.gmass = gmass;
        ev.cadj = cadj;
        ev.n = n;
        ev.k = k;
        ev.k.eps2 = cc.eps2;
        ev.k.kA = cc.kA;
        ev.k.kB = cc.kB;
        long long cnt[3] = {0, 0, 0};
        const int wst = p3t_walk::walk_group(S, gmin[g], gmax[g], wmin, wmax,
                                             theta2, cc.hg2, cl, lane, ev, cnt,
                                             lim_walk);
        if (wst != P3T_OK) {
            if (lane == 0) p3t_raise(st, wst);
            continue;
        }
        // dL/dx_i = -G sum J w over the particle's sources
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int slot = lane + 32 * h;
            if (slot < gr.y) {
                const int o = order[gr.x + slot];
                for (int q = 0; q < 3; ++q)
                    atomicAdd(&gpos[(size_t)q * n + o],
                              -k.G * ((double)ev.ih[h][q] + (double)ev.il[h][q]));
            }
        }
    }
}

// Cell adjoints (aM, acom[3] / M, 2S xx yy zz xy xz yz) pushed to the member
// particles, FP64; one thread per leaf climbs to the root summing the
// coefficients of the quadratic form about the leaf's centre of mass, then
// evaluates it for each member (every particle lies in exactly one leaf).
__global__ void __launch_bounds__(256)
k_vjp_leaves(const P3TDevState *__restrict__ st, int n,
             const int *__restrict__ leaf_sorted, const int4 *__restrict__ node,
             const int *__restrict__ parent, const double *__restrict__ ccom,
             const double *__restrict__ xs, const double *__restrict__ ms,
             const int *__restrict__ order, const double *__restrict__ cadj,
             double *__restrict__ gpos, double *__restrict__ gmass)
{
    if (st->error) return;
    const int nl = st->nleaf;
    for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < nl;
         q += gridDim.x * blockDim.x) {
        const int leaf = leaf_sorted[q];
        const double r[3] = {ccom[3 * leaf], ccom[3 * leaf + 1], ccom[3 * leaf + 2]};
        double P[3] = {0.0, 0.0, 0.0}, Tc[3] = {0.0, 0.0, 0.0};
        double Ts[6] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0};  // xx yy zz xy xz yz
        double a = 0.0;
        int c = leaf;
        for (int up = 0; up <= P3T_MAX_LEVEL && c >= 0; ++up) {
            const double *A = cadj + (size_t)c * 10;
            bool any = false;
#pragma unroll
            for (int v = 0; v < 10; ++v) any |= A[v] != 0.0;
            if (any) {
                const double d[3] = {ccom[3 * c] - r[0], ccom[3 * c + 1] - r[1],
                                     ccom[3 * c + 2] - r[2]};
                // T = 3 S - tr(S) I, A[4..9] holding 2S
                const double tr = 0.5 * (A[4] + A[5] + A[6]);
                const double T[6] = {1.5 * A[4] - tr, 1.5 * A[5] - tr, 1.5 * A[6] - tr,
                                     1.5 * A[7], 1.5 * A[8], 1.5 * A[9]};
                const double Td[3] = {T[0] * d[0] + T[3] * d[1] + T[4] * d[2],
                                      T[3] * d[0] + T[1] * d[1] + T[5] * d[2],
                                      T[4] * d[0] + T[5] * d[1] + T[2] * d[2]};
#pragma unroll
                for (int v = 0; v < 3; ++v) {
                    P[v] += A[1 + v];
                    Tc[v] += Td[v];
                }
#pragma unroll
                for (int v = 0; v < 6; ++v) Ts[v] += T[v];
                a += A[0] - (d[0] * A[1] + d[1] * A[2] + d[2] * A[3]) +
                     (d[0] * Td[0] + d[1] * Td[1] + d[2] * Td[2]);
            }
            c = parent[c];
        }
        const int4 nd = node[leaf];
        for (int k = nd.x; k < nd.x + nd.y; ++k) {
            const double x[3] = {xs[k] - r[0], xs[(size_t)n + k] - r[1],
                                 xs[2 * (size_t)n + k] - r[2]};
            const double Tx[3] = {Ts[0] * x[0] + Ts[3] * x[1] + Ts[4] * x[2],
                                  Ts[3] * x[0] + Ts[1] * x[1] + Ts[5] * x[2],
                                  Ts[4] * x[0] + Ts[5] * x[1] + Ts[2] * x[2]};
            const double mk = ms[k];
            const int o = order[k];
#pragma unroll
            for (int v = 0; v < 3; ++v)
                gpos[(size_t)v * n + o] += mk * (P[v] + 2.0 * (Tx[v] - Tc[v]));
            gmass[o] += a + (x[0] * P[0] + x[1] * P[1] + x[2] * P[2]) +
                        (x[0] * Tx[0] + x[1] * Tx[1] + x[2] * Tx[2]) -
                        2.0 * (x[0] * Tc[0] + x[1] * Tc[1] + x[2] * Tc[2]);
        }
    }
}

// Cell adjoints prepared for the push: dL/dcom divided by M once per cell,
// so that the push, which visits every cell on every particle's path, does
// no division.
__global__ void k_vjp_prep(const P3TDevState *__restrict__ st,
                           const double *__restrict__ cM, double *__restrict__ cadj)
{
    const int nc = st->ncell;
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < nc;
         c += gridDim.x * blockDim.x) {
        double *A = cadj + (size_t)c * 10;
        const double a1 = A[1], a2 = A[2], a3 = A[3];
        if (a1 != 0.0 || a2 != 0.0 || a3 != 0.0) {
            const double iM = 1.0 / cM[c];
            A[1] = a1 * iM;
            A[2] = a2 * iM;
            A[3] = a3 * iM;
        }
    }
}

__global__ void k_vjp_reset(P3TDevState *st)
{
    if (threadIdx.x == 0 && blockIdx.x == 0) st->work_vjp = 0;
}

}  // namespace

// dL/dx (gpos, double[3][n]) and dL/dm (gmass, double[n]) for the weights w
// (float[3][n]); cadj is scratch of 10 doubles per cell.
int p3t_run_vjp(p3t_ctx *c, const float *w, double *gpos, double *gmass,
                double *cadj, cudaStream_t s)
{
    const int n = (int)c->n;
    const int64_t G = (n + 15) / 16 + c->nclus;  // bound; the count is on the device
    const int64_t C = c->cap_cells;
    P3T_CUDA_TRY(cudaMemsetAsync(gpos, 0, sizeof(double) * 3 * (size_t)n, s));
    P3T_CUDA_TRY(cudaMemsetAsync(gmass, 0, sizeof(double) * (size_t)n, s));
    P3T_CUDA_TRY(cudaMemsetAsync(cadj, 0, sizeof(double) * 10 * (size_t)C, s));
    float theta2, hg2;
    p3t_mac_constants(&c->p, &theta2, &hg2);
    VjpConsts k;
    k.eps2 = (float)(c->p.eps * c->p.eps);
    k.kA = (float)(1.0 / ((1.0 - c->p.gamma) * c->p.r_out));
    k.kB = (float)(-c->p.gamma / (1.0 - c->p.gamma));
    k.G = c->p.G;
    const int vw = c->vjp_warps == 2 ? 2 : 4;
    int blocks = (int)((G + vw - 1) / vw);
    if (blocks > c->sms * 64 / vw) blocks = c->sms * 64 / vw;
    k_vjp_reset<<<1, 32, 0, s>>>(c->st);
    const int slot = p3t_prof_open(c, P3T_PH_VJPWALK, s);
#define P3T_VJP_ARGS                                                           \
    c->gclus, c->cc, c->grange, c->gmin, c->gmax, c->gctr, c->wmin, c->wmax,   \
        theta2, c->phi, c->plo, c->cf0, c->cf1, c->cf2, c->order, n, k, w,     \
        gpos, gmass, cadj, c->gperm, c->st, c->lim_walk
    if (vw == 2)
        k_walk_vjp<2><<<blocks, 2 * 32, 0, s>>>(P3T_VJP_ARGS);
    else
        k_walk_vjp<4><<<blocks, 4 * 32, 0, s>>>(P3T_VJP_ARGS);
#undef P3T_VJP_ARGS
    p3t_prof_close(c, slot, s);
    k_vjp_prep<<<c->sms * 8, 256, 0, s>>>(c->st, c->cM, cadj);
    k_vjp_leaves<<<c->sms * 8, 256, 0, s>>>(c->st, n, c->leaf_sorted, c->node,
                                            c->parent, c->ccom, c->xs, c->ms,
                                            c->order, cadj, gpos, gmass);
    p3t_count_launches(4);
    P3T_CUDA_TRY(cudaGetLastError());
    return P3T_OK;
}
