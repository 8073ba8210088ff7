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
// stored) and evaluates the Jacobian products in FP32 group-relative
// coordinates; contributions to sources are summed over the warp and added
// to FP64 accumulators with atomics.  k_vjp_push then sends every cell
// adjoint to the member particles in FP64: one thread per particle descends
// from the root to its leaf and applies the adjoint of each cell on the way.
#include <math.h>

#include "p3t_walkcore.cuh"

namespace {

using p3t_walk::Smem;

constexpr int VW = 4;  // warps per block

struct VjpConsts {
    float eps2, kA, kB;
    double G;
};

__device__ __forceinline__ float4 vpad()
{
    return make_float4(1e15f, 1e15f, 1e15f, 0.0f);
}

__device__ __forceinline__ float4 rel(float4 hi, float4 lo, float4 c)
{
    return make_float4(__fadd_rn(__fsub_rn(hi.x, c.x), lo.x),
                       __fadd_rn(__fsub_rn(hi.y, c.y), lo.y),
                       __fadd_rn(__fsub_rn(hi.z, c.z), lo.z), hi.w);
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

// Per-lane state of one group: two particles per lane.
struct VjpEval {
    float4 p0, p1;        // group-relative positions
    float3 w0, w1;        // weights (zero for empty slots)
    int k0, k1;           // sorted ids
    double g0[3], g1[3];  // dL/dx of the lane's particles (without G)
    float4 ct;
    const float4 *phi, *plo, *cf0, *cf1, *cf2;
    const int *order;
    double *gpos, *gmass, *cadj;
    int n, lane;
    VjpConsts k;

    // Cell tile: ids in S.tj[0..take).
    __device__ __forceinline__ void cells(Smem &S, int take)
    {
        if (lane < take) {
            const int c = S.tj[lane];
            float4 a = cf0[c], bb = cf1[c], cc = cf2[c];
            S.t0[lane] = make_float4(__fadd_rn(__fsub_rn(a.x, ct.x), bb.x),
                                     __fadd_rn(__fsub_rn(a.y, ct.y), bb.y),
                                     __fadd_rn(__fsub_rn(a.z, ct.z), bb.z), a.w);
            S.t1[lane] = make_float4(bb.w, cc.x, -(bb.w + cc.x), cc.y);
            S.t2[lane] = make_float4(cc.z, cc.w, 0.0f, 0.0f);
        }
        __syncwarp();
        float s0[3] = {0.f, 0.f, 0.f}, s1[3] = {0.f, 0.f, 0.f};
        constexpr int NS = 2, NV = 10, LPS = 32 / NS;
        for (int j = 0; j < take; j += NS) {
            float acc[NS][NV];
#pragma unroll
            for (int u = 0; u < NS; ++u) {
#pragma unroll
                for (int q = 0; q < NV; ++q) acc[u][q] = 0.f;
                if (j + u < take) {
                    const float4 a = S.t0[j + u], B = S.t1[j + u], Cq = S.t2[j + u];
                    cell_one(a, B, Cq, p0, w0, s0, acc[u]);
                    cell_one(a, B, Cq, p1, w1, s1, acc[u]);
                }
            }
            reduce_scatter<NS, NV>(acc, lane);
            const int src = j + src_of<NS>(lane);
            if (src < take) {
                const size_t base = (size_t)S.tj[src] * 10;
                for (int v = lane & (LPS - 1); v < NV; v += LPS)
                    atomicAdd(&cadj[base + v], k.G * (double)pick<NV>(acc[0], v));
            }
        }
        for (int q = 0; q < 3; ++q) {
            g0[q] += (double)s0[q];
            g1[q] += (double)s1[q];
        }
        __syncwarp();
    }

    // One particle against one cell: i-side sum into s, cell adjoints
    // (aM, acom[3], S xx yy zz xy xz yz) into acc.
    __device__ __forceinline__ void cell_one(float4 a, float4 B, float4 Cq,
                                             float4 p, float3 w, float *s,
                                             float *acc)
    {
        const float dx = a.x - p.x, dy = a.y - p.y, dz = a.z - p.z;
        const float s2 = fmaf(dx, dx, fmaf(dy, dy, fmaf(dz, dz, k.eps2)));
        const float ri = rsqrtf(s2);
        const float ri2 = ri * ri;
        const float ri3 = ri * ri2, ri5 = ri3 * ri2, ri7 = ri5 * ri2,
                    ri9 = ri7 * ri2;
        // Q = [[B.x, B.w, Cq.x], [B.w, B.y, Cq.y], [Cq.x, Cq.y, B.z]]
        const float qx = fmaf(B.x, dx, fmaf(B.w, dy, Cq.x * dz));
        const float qy = fmaf(B.w, dx, fmaf(B.y, dy, Cq.y * dz));
        const float qz = fmaf(Cq.x, dx, fmaf(Cq.y, dy, B.z * dz));
        const float wqx = fmaf(B.x, w.x, fmaf(B.w, w.y, Cq.x * w.z));
        const float wqy = fmaf(B.w, w.x, fmaf(B.y, w.y, Cq.y * w.z));
        const float wqz = fmaf(Cq.x, w.x, fmaf(Cq.y, w.y, B.z * w.z));
        const float dqd = fmaf(dx, qx, fmaf(dy, qy, dz * qz));
        const float wd = fmaf(w.x, dx, fmaf(w.y, dy, w.z * dz));
        const float wqd = fmaf(w.x, qx, fmaf(w.y, qy, w.z * qz));
        const float M = a.w;
        // J^T w = M (w ri3 - 3 wd d ri5) - (Q w ri5 - 5 wQd d ri7)
        //         + 2.5 (2 wd Qd ri7 + dQd w ri7 - 7 dQd wd d ri9)
        const float cw = M * ri3 + 2.5f * dqd * ri7;
        const float cd = -3.0f * M * wd * ri5 + 5.0f * wqd * ri7
                         - 17.5f * dqd * wd * ri9;
        const float cq = 5.0f * wd * ri7;
        const float jx = cw * w.x + cd * dx + cq * qx - ri5 * wqx;
        const float jy = cw * w.y + cd * dy + cq * qy - ri5 * wqy;
        const float jz = cw * w.z + cd * dz + cq * qz - ri5 * wqz;
        s[0] -= jx;
        s[1] -= jy;
        s[2] -= jz;
        acc[0] += wd * ri3;
        acc[1] += jx;
        acc[2] += jy;
        acc[3] += jz;
        const float h5 = -0.5f * ri5, t7 = 2.5f * wd * ri7;
        acc[4] += 2.0f * h5 * w.x * dx + t7 * dx * dx;
        acc[5] += 2.0f * h5 * w.y * dy + t7 * dy * dy;
        acc[6] += 2.0f * h5 * w.z * dz + t7 * dz * dz;
        acc[7] += h5 * (w.x * dy + w.y * dx) + t7 * dx * dy;
        acc[8] += h5 * (w.x * dz + w.z * dx) + t7 * dx * dz;
        acc[9] += h5 * (w.y * dz + w.z * dy) + t7 * dy * dz;
    }

    // Particle tile: sorted ids in S.tj[0..take).
    template <bool NEAR>
    __device__ __forceinline__ void particles(Smem &S, int take)
    {
        if (lane < take) {
            const int j = S.tj[lane];
            S.t0[lane] = rel(phi[j], plo[j], ct);
        }
        __syncwarp();
        float s0[3] = {0.f, 0.f, 0.f}, s1[3] = {0.f, 0.f, 0.f};
        constexpr int NS = 8, NV = 4;
        for (int j = 0; j < take; j += NS) {
            float acc[NS][NV];
#pragma unroll
            for (int u = 0; u < NS; ++u) {
#pragma unroll
                for (int q = 0; q < NV; ++q) acc[u][q] = 0.f;
                if (j + u < take) {
                    const float4 a = S.t0[j + u];
                    const int kj = S.tj[j + u];
                    pair_one<NEAR>(a, kj == k0, p0, w0, s0, acc[u]);
                    pair_one<NEAR>(a, kj == k1, p1, w1, s1, acc[u]);
                }
            }
            reduce_scatter<NS, NV>(acc, lane);
            const int src = j + src_of<NS>(lane);
            if (src < take) {
                const int v = lane & 3;  // 32 / NS = 4 lanes per source
                const int o = order[S.tj[src]];
                double *dst = v < 3 ? gpos + (size_t)v * n + o : gmass + o;
                atomicAdd(dst, k.G * (double)pick<NV>(acc[0], v));
            }
        }
        for (int q = 0; q < 3; ++q) {
            g0[q] += (double)s0[q];
            g1[q] += (double)s1[q];
        }
        __syncwarp();
    }

    // One particle against one source particle (self pairs contribute 0).
    template <bool NEAR>
    __device__ __forceinline__ void pair_one(float4 a, bool self, float4 p,
                                             float3 w, float *s, float *acc)
    {
        const float dx = a.x - p.x, dy = a.y - p.y, dz = a.z - p.z;
        const float s2 = fmaf(dx, dx, fmaf(dy, dy, fmaf(dz, dz, k.eps2)));
        const float ri = (s2 > 0.0f && !self) ? rsqrtf(s2) : 0.0f;
        const float ri2 = ri * ri;
        const float ri3 = ri2 * ri;
        float phi_, psi;
        if (NEAR) {
            const float sv = s2 * ri;
            const float x = __saturatef(fmaf(sv, k.kA, k.kB));
            const float x2 = x * x, x4 = x2 * x2;
            float pk = fmaf(-20.0f, x, 70.0f);
            pk = fmaf(pk, x, -84.0f);
            pk = fmaf(pk, x, 35.0f);
            const float K = pk * x4;
            const float omx = 1.0f - x;
            const float Kp = 140.0f * (x2 * x) * (omx * omx * omx) * k.kA;
            // products ordered so that K = 0 with a huge 1/s never forms 0*inf
            phi_ = ((K * ri) * ri) * ri;
            psi = ((((Kp * ri) * ri) * ri) * ri) - 3.0f * (((phi_ * ri) * ri));
        } else {
            phi_ = ri3;
            psi = -3.0f * ri3 * ri2;
        }
        const float wd = fmaf(w.x, dx, fmaf(w.y, dy, w.z * dz));
        const float m = a.w;
        const float jx = m * fmaf(phi_, w.x, psi * wd * dx);
        const float jy = m * fmaf(phi_, w.y, psi * wd * dy);
        const float jz = m * fmaf(phi_, w.z, psi * wd * dz);
        s[0] -= jx;
        s[1] -= jy;
        s[2] -= jz;
        acc[0] += jx;
        acc[1] += jy;
        acc[2] += jz;
        acc[3] += phi_ * wd;
    }
};

__global__ void __launch_bounds__(VW * 32)
k_walk_vjp(const int *__restrict__ gclus,
           const ClusterConsts *__restrict__ ccs,
           const int2 *__restrict__ grange,
           const float4 *__restrict__ gmin, const float4 *__restrict__ gmax,
           const float4 *__restrict__ gctr, const float4 *__restrict__ wmin,
           const float4 *__restrict__ wmax, const int4 *__restrict__ node,
           float theta2, const float4 *__restrict__ phi,
           const float4 *__restrict__ plo, const float4 *__restrict__ cf0,
           const float4 *__restrict__ cf1, const float4 *__restrict__ cf2,
           const int *__restrict__ order, int n, VjpConsts k,
           const float *__restrict__ w, double *__restrict__ gpos,
           double *__restrict__ gmass, double *__restrict__ cadj,
           const int *__restrict__ gperm, P3TDevState *st)
{
    __shared__ Smem smem[VW];
    const int wi = threadIdx.x >> 5, lane = threadIdx.x & 31;
    Smem &S = smem[wi];
    if (st->error) return;  // no valid tree
    const int G = st->ngroup;
    for (;;) {
        int g = 0;
        if (lane == 0) g = (int)atomicAdd(&st->work, 1u);
        g = __shfl_sync(0xffffffffu, g, 0);
        if (g >= G) break;
        g = gperm[g];
        const int2 gr = grange[g];
        const int cl = gclus[g];
        const ClusterConsts cc = ccs[cl];
        VjpEval ev;
        ev.ct = gctr[g];
        ev.k0 = gr.x + lane;
        ev.k1 = gr.x + 32 + lane;
        const bool v0 = lane < gr.y, v1 = lane + 32 < gr.y;
        const int o0 = v0 ? order[ev.k0] : 0, o1 = v1 ? order[ev.k1] : 0;
        ev.p0 = v0 ? rel(phi[ev.k0], plo[ev.k0], ev.ct) : vpad();
        ev.p1 = v1 ? rel(phi[ev.k1], plo[ev.k1], ev.ct) : vpad();
        ev.w0 = v0 ? make_float3(w[o0], w[(size_t)n + o0], w[2 * (size_t)n + o0])
                   : make_float3(0.f, 0.f, 0.f);
        ev.w1 = v1 ? make_float3(w[o1], w[(size_t)n + o1], w[2 * (size_t)n + o1])
                   : make_float3(0.f, 0.f, 0.f);
        for (int q = 0; q < 3; ++q) ev.g0[q] = ev.g1[q] = 0.0;
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
        ev.lane = lane;
        ev.k = k;
        ev.k.eps2 = cc.eps2;
        ev.k.kA = cc.kA;
        ev.k.kB = cc.kB;
        long long cnt[3] = {0, 0, 0};
        if (!p3t_walk::walk_group(S, gmin[g], gmax[g], wmin, wmax, node,
                                  theta2, cc.hg2, cl, lane, ev, cnt)) {
            if (lane == 0) p3t_raise(st, P3T_ERR_CAPACITY);
            continue;
        }
        if (v0)
            for (int q = 0; q < 3; ++q)
                atomicAdd(&gpos[(size_t)q * n + o0], k.G * ev.g0[q]);
        if (v1)
            for (int q = 0; q < 3; ++q)
                atomicAdd(&gpos[(size_t)q * n + o1], k.G * ev.g1[q]);
    }
}

// Cell adjoints (aM, acom[3], S xx yy zz xy xz yz) pushed to the member
// particles, FP64; one thread per particle (sorted id k) walks from the root
// down to its leaf.
__global__ void __launch_bounds__(256)
k_vjp_push(int n, int nc, const long long *__restrict__ off,
           const int4 *__restrict__ node, const double *__restrict__ cM,
           const double *__restrict__ ccom, const double *__restrict__ xs,
           const double *__restrict__ ms, const int *__restrict__ order,
           const double *__restrict__ cadj, double *__restrict__ gpos,
           double *__restrict__ gmass)
{
    const int kk = blockIdx.x * blockDim.x + threadIdx.x;
    if (kk >= n) return;
    const double x[3] = {xs[kk], xs[(size_t)n + kk], xs[2 * (size_t)n + kk]};
    const double mk = ms[kk];
    double gx[3] = {0.0, 0.0, 0.0}, gm = 0.0;
    int c = 0;  // root of the particle's cluster (sorted order keeps clusters)
    if (nc > 1) {
        int lo = 0, hi = nc;
        while (hi - lo > 1) {
            int mid = (lo + hi) >> 1;
            if (off[mid] <= kk)
                lo = mid;
            else
                hi = mid;
        }
        c = lo;
    }
    for (int depth = 0; depth <= P3T_MAX_LEVEL; ++depth) {
        const double *A = cadj + (size_t)c * 10;
        bool any = false;
#pragma unroll
        for (int q = 0; q < 10; ++q) any |= A[q] != 0.0;
        if (any) {
            const double M = cM[c];
            const double e[3] = {x[0] - ccom[3 * c], x[1] - ccom[3 * c + 1],
                                 x[2] - ccom[3 * c + 2]};
            const double Sxx = A[4], Syy = A[5], Szz = A[6], Sxy = A[7],
                         Sxz = A[8], Syz = A[9];
            const double tr = Sxx + Syy + Szz;
            const double Se[3] = {Sxx * e[0] + Sxy * e[1] + Sxz * e[2],
                                  Sxy * e[0] + Syy * e[1] + Syz * e[2],
                                  Sxz * e[0] + Syz * e[1] + Szz * e[2]};
            const double eSe = e[0] * Se[0] + e[1] * Se[1] + e[2] * Se[2];
            const double ee = e[0] * e[0] + e[1] * e[1] + e[2] * e[2];
            const double eac = e[0] * A[1] + e[1] * A[2] + e[2] * A[3];
            for (int q = 0; q < 3; ++q)
                gx[q] += (mk / M) * A[1 + q] + mk * (6.0 * Se[q] - 2.0 * tr * e[q]);
            gm += A[0] + eac / M + 3.0 * eSe - ee * tr;
        }
        const int4 nd = node[c];
        const int nch = nd.w & 255;
        if (nch == 0) break;
        int next = nd.z;
        for (int q = 0; q < nch; ++q) {
            const int4 ch = node[nd.z + q];
            if (kk >= ch.x && kk < ch.x + ch.y) next = nd.z + q;
        }
        c = next;
    }
    const int o = order[kk];
    for (int q = 0; q < 3; ++q) gpos[(size_t)q * n + o] += gx[q];
    gmass[o] += gm;
}

__global__ void k_vjp_reset(P3TDevState *st)
{
    if (threadIdx.x == 0 && blockIdx.x == 0) st->work = 0;
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
    int blocks = (int)((G + VW - 1) / VW);
    if (blocks > c->sms * 16) blocks = c->sms * 16;
    k_vjp_reset<<<1, 32, 0, s>>>(c->st);
    k_walk_vjp<<<blocks, VW * 32, 0, s>>>(
        c->gclus, c->cc, c->grange, c->gmin, c->gmax, c->gctr, c->wmin,
        c->wmax, c->node, theta2, c->phi, c->plo, c->cf0, c->cf1, c->cf2,
        c->order, n, k, w,
        gpos, gmass, cadj, c->gperm, c->st);
    k_vjp_push<<<(n + 255) / 256, 256, 0, s>>>(n, c->nclus,
                                               (const long long *)c->clus_off,
                                               c->node, c->cM, c->ccom,
                                               c->xs, c->ms, c->order, cadj,
                                               gpos, gmass);
    p3t_count_launches(3);
    P3T_CUDA_TRY(cudaGetLastError());
    return P3T_OK;
}
