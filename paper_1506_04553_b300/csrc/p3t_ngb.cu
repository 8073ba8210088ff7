// Neighbour lists (Sect. 2.2: for every particle, the particles within a
// distance h; h = r_cut + dr_buff).
//
// j is a neighbour of i iff j != i and ((dx*dx + dy*dy) + dz*dz) < h*h in
// FP64 with dx = x_i - x_j.  Every such pair lies in a leaf whose member box
// is within the guard distance of the group's box (the opening test never
// accepts a cell closer than max(h, r_cut), and the guard box distance of an
// ancestor never exceeds that of its descendants), so a walk that opens only
// cells with d2 <= hg2 meets every candidate.  Pairs are screened in FP32
// with group-relative coordinates against the group's radius hs2, which
// exceeds h^2 by more than the FP32 error of r^2, and the survivors are
// decided by the FP64 predicate above: the result is exact.
//
// The counting walk also keeps the first P3T_NGB_SLOTS neighbours of every
// particle and lists the groups with a longer row.  After the counts are
// scanned into CSR offsets, the short rows are sorted and copied from the
// kept neighbours; the walk runs a second time only over the listed groups,
// to fill the long rows, which are sorted afterwards.  Rows are sorted by
// original index.
#include "p3t_internal.cuh"

namespace {

constexpr int NW = 4;        // warps per block
constexpr int NSTACK = 768;  // walk stack entries per warp
constexpr int NRING = 64;

__device__ __forceinline__ bool exact_ngb(const double *__restrict__ xs,
                                          int n, int ki, int kj, double h2)
{
    double dx = __dsub_rn(xs[ki], xs[kj]);
    double dy = __dsub_rn(xs[(size_t)n + ki], xs[(size_t)n + kj]);
    double dz = __dsub_rn(xs[2 * (size_t)n + ki], xs[2 * (size_t)n + kj]);
    double r2 = __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)),
                          __dmul_rn(dz, dz));
    return r2 < h2;
}

__device__ __forceinline__ float4 rel4n(float4 hi, float4 lo, float4 c)
{
    return make_float4(__fadd_rn(__fsub_rn(hi.x, c.x), lo.x),
                       __fadd_rn(__fsub_rn(hi.y, c.y), lo.y),
                       __fadd_rn(__fsub_rn(hi.z, c.z), lo.z), hi.w);
}

struct __align__(16) NgbSmem {
    float4 t0[32];
    int tj[32];
    int stack[NSTACK];
    int cb[32];
    int2 ring[NRING];
};

constexpr int SL = P3T_NGB_SLOTS;

// Screens the staged tile against the lane's two particles.  Counting:
// neighbours beyond the count c go to the particle's slots while c < SL.
// Filling (long rows only, b0 / b1): neighbours go to the CSR row at w.
template <bool FILL>
__device__ __forceinline__ void ngb_tile(NgbSmem &S, int nk, float4 p0, float4 p1,
                                         bool v0, bool v1, int k0, int k1,
                                         float hs2, const double *xs, int n,
                                         double h2, const int *order,
                                         int &c0, int &c1, long long &w0,
                                         long long &w1, bool b0, bool b1,
                                         int *s0, int *s1, int *idx,
                                         long long cap, P3TDevState *st)
{
    for (int j = 0; j < nk; ++j) {
        const float4 a = S.t0[j];
        const int kj = S.tj[j];
        float dx = a.x - p0.x, dy = a.y - p0.y, dz = a.z - p0.z;
        float r20 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
        dx = a.x - p1.x; dy = a.y - p1.y; dz = a.z - p1.z;
        float r21 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
        if (r20 < hs2 && v0 && kj >= 0 && kj != k0 && exact_ngb(xs, n, k0, kj, h2)) {
            if (FILL) {
                if (b0) {
                    if (w0 < cap) idx[w0] = order[kj];
                    else p3t_raise(st, P3T_ERR_CAPACITY);
                    ++w0;
                }
            } else if (c0 < SL) {
                s0[c0] = order[kj];
            }
            ++c0;
        }
        if (r21 < hs2 && v1 && kj >= 0 && kj != k1 && exact_ngb(xs, n, k1, kj, h2)) {
            if (FILL) {
                if (b1) {
                    if (w1 < cap) idx[w1] = order[kj];
                    else p3t_raise(st, P3T_ERR_CAPACITY);
                    ++w1;
                }
            } else if (c1 < SL) {
                s1[c1] = order[kj];
            }
            ++c1;
        }
    }
}

template <bool FILL>
__global__ void __launch_bounds__(NW * 32)
k_ngb_walk(const int *__restrict__ gclus,
           const ClusterConsts *__restrict__ ccs,
           const int2 *__restrict__ grange,
           const float4 *__restrict__ gmin, const float4 *__restrict__ gmax,
           const float4 *__restrict__ gctr, const float4 *__restrict__ wmin,
           const float4 *__restrict__ wmax, const int4 *__restrict__ node,
           const float4 *__restrict__ phi,
           const float4 *__restrict__ plo, const int *__restrict__ order,
           const double *__restrict__ xs, int n,
           int *__restrict__ cnt, const long long *__restrict__ row_off,
           int *__restrict__ idx, long long cap, const int *__restrict__ gperm,
           int *__restrict__ slots, int *__restrict__ ovf, P3TDevState *st,
           long long lim_walk)
{
    __shared__ NgbSmem smem[NW];
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const unsigned full = 0xffffffffu, lt = lanemask_lt();
    NgbSmem &S = smem[w];
    if (st->error) return;  // no valid tree
    // counting: every group, in the work order; filling: the listed groups
    const int G = FILL ? st->novf : st->ngroup;
    for (;;) {
        int g = 0;
        if (lane == 0) g = (int)atomicAdd(&st->work_ngb, 1u);
        g = __shfl_sync(full, g, 0);
        if (g >= G) break;
        g = FILL ? ovf[g] : gperm[g];
        const int2 gr = grange[g];
        const float4 ct = gctr[g];
        const float4 gmn = gmin[g], gmx = gmax[g];
        const float hs2 = gmn.w;
        const int cl = gclus[g];
        // a neighbour of a group particle lies within R + h of the group's
        // centre (R: gmx.w, a sphere about the centre holding the group);
        // candidates outside, with a 1% margin in the square, are dropped
        // when staged
        const float rfl = gmx.w + sqrtf((float)ccs[cl].h2);
        const float rf2 = 1.01f * rfl * rfl;
        const float hg2 = ccs[cl].hg2;
        const double h2 = ccs[cl].h2;
        const int k0 = gr.x + lane, k1 = gr.x + 32 + lane;
        const bool v0 = lane < gr.y, v1 = lane + 32 < gr.y;
        const float4 p0 = v0 ? rel4n(phi[k0], plo[k0], ct) : make_float4(1e15f, 1e15f, 1e15f, 0.f);
        const float4 p1 = v1 ? rel4n(phi[k1], plo[k1], ct) : make_float4(1e15f, 1e15f, 1e15f, 0.f);
        int c0 = 0, c1 = 0;
        const int o0 = v0 ? order[k0] : 0, o1 = v1 ? order[k1] : 0;
        long long w0 = 0, w1 = 0;
        bool b0 = false, b1 = false;
        if (FILL) {
            if (v0) {
                w0 = row_off[o0];
                b0 = row_off[o0 + 1] - w0 > SL;
            }
            if (v1) {
                w1 = row_off[o1];
                b1 = row_off[o1 + 1] - w1 > SL;
            }
        }
        int *s0 = slots + (size_t)o0 * SL, *s1 = slots + (size_t)o1 * SL;
        int head = 0, nr = 0, np = 0;  // ring of near leaf ranges
        if (lane == 0) S.stack[0] = cl * 8;  // the cluster's root
        int top = 1;
        long long iter = 0;
        bool bad = false, timeout = false;
        __syncwarp();
        for (;;) {
            // drain full tiles (and everything once the walk is done)
            while (np >= 32 || (top == 0 && np > 0)) {
                const int take = min(np, 32);
                const bool have = lane < nr;
                int2 r = have ? S.ring[(head + lane) & (NRING - 1)] : make_int2(0, 0);
                int inc = warp_incl_scan(r.y);
                int exc = inc - r.y;
                if (have && exc < take) {
                    int stop = min(inc, take);
                    for (int q = exc; q < stop; ++q) S.tj[q] = r.x + (q - exc);
                }
                const int nfull = __popc(__ballot_sync(full, have && inc <= take));
                if (lane == nfull && have && exc < take) {
                    int used = take - exc;
                    S.ring[(head + lane) & (NRING - 1)] = make_int2(r.x + used, r.y - used);
                }
                __syncwarp();
                head = (head + nfull) & (NRING - 1);
                nr -= nfull;
                np -= take;
                float4 pv = make_float4(1e15f, 1e15f, 1e15f, 0.f);
                int jv = -1;
                if (lane < take) {
                    jv = S.tj[lane];
                    pv = rel4n(phi[jv], plo[jv], ct);
                }
                const bool keep = lane < take &&
                                  fmaf(pv.x, pv.x, fmaf(pv.y, pv.y, pv.z * pv.z)) < rf2;
                const unsigned km = __ballot_sync(full, keep);
                __syncwarp();  // every lane has read its S.tj entry
                if (keep) {
                    const int q = __popc(km & lt);
                    S.t0[q] = pv;
                    S.tj[q] = jv;
                }
                __syncwarp();
                ngb_tile<FILL>(S, __popc(km), p0, p1, v0, v1, k0, k1, hs2, xs, n, h2, order,
                               c0, c1, w0, w1, b0, b1, s0, s1, idx, cap, st);
                __syncwarp();
            }
            if (top == 0) break;
            if (++iter > lim_walk) {  // a finite tree stays far below the default
                timeout = true;
                break;
            }
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
            bool near = false, open = false;
            int child = 0, nchild = 0, pfirst = 0, pcount = 0;
            if (c >= 0) {
                const float4 cmn = wmin[c], cmx = wmax[c];
                if (box_d2(gmn, gmx, cmn, cmx) <= hg2) {
                    child = __float_as_int(cmn.w);
                    nchild = __float_as_int(cmx.w);
                    if (nchild <= 0) {  // a leaf: first particle, -count
                        pfirst = child;
                        pcount = -nchild;
                        near = true;
                    } else {
                        open = true;
                    }
                }
            }
            {
                unsigned m = __ballot_sync(full, near);
                if (near)
                    S.ring[(head + nr + __popc(m & lt)) & (NRING - 1)] =
                        make_int2(pfirst, pcount);
                int x = near ? pcount : 0;
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(full, x, o);
                nr += __popc(m);
                np += x;
            }
            {
                unsigned mo = __ballot_sync(full, open);
                int q = __popc(mo);
                if (top + q > NSTACK) {
                    bad = true;
                    break;
                }
                if (open) S.stack[top + __popc(mo & lt)] = child * 8 + (nchild - 1);
                top += q;
            }
            __syncwarp();
        }
        if (bad || timeout) {
            if (lane == 0) p3t_raise(st, timeout ? P3T_ERR_TIMEOUT : P3T_ERR_CAPACITY);
            continue;
        }
        if (!FILL) {
            if (v0) cnt[o0] = c0;
            if (v1) cnt[o1] = c1;
            if (__any_sync(full, c0 > SL || c1 > SL) && lane == 0)
                ovf[atomicAdd(&st->novf, 1)] = g;
        }
    }
}

// Short rows (at most SL): the kept neighbours, sorted ascending in
// registers, copied to the CSR row.
__global__ void k_ngb_gather(int n, const long long *__restrict__ row_off,
                             const int *__restrict__ slots,
                             int *__restrict__ idx, long long cap,
                             P3TDevState *st)
{
    if (st->error) return;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += gridDim.x * blockDim.x) {
        const long long b = row_off[i];
        const int len = (int)(row_off[i + 1] - b);
        if (len == 0 || len > SL) continue;
        if (b + len > cap) {
            p3t_raise(st, P3T_ERR_CAPACITY);
            continue;
        }
        int v[SL];
#pragma unroll
        for (int q = 0; q < SL; ++q) v[q] = q < len ? slots[(size_t)i * SL + q] : INT_MAX;
#pragma unroll
        for (int a = 1; a < SL; ++a)  // insertion sort, fixed shape
#pragma unroll
            for (int q = a; q > 0; --q)
                if (v[q - 1] > v[q]) {
                    const int t = v[q - 1];
                    v[q - 1] = v[q];
                    v[q] = t;
                }
#pragma unroll
        for (int q = 0; q < SL; ++q)
            if (q < len) idx[b + q] = v[q];
    }
}

// Sorts each long CSR row ascending (insertion sort per thread).
__global__ void k_ngb_sort(int n, const long long *__restrict__ row_off,
                           int *__restrict__ idx, long long cap)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += gridDim.x * blockDim.x) {
        long long b = row_off[i], e = row_off[i + 1];
        if (e > cap || e - b <= SL) continue;
        for (long long a = b + 1; a < e; ++a) {
            int v = idx[a];
            long long q = a - 1;
            while (q >= b && idx[q] > v) {
                idx[q + 1] = idx[q];
                --q;
            }
            idx[q + 1] = v;
        }
    }
}

__global__ void k_work_reset(P3TDevState *st, int fill)
{
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        st->work_ngb = 0;
        if (!fill) st->novf = 0;
    }
}

// ---- two species (Sect. 3.2.2): rows with the black holes ----
// The tree gives the star-star rows (the black holes form a cluster of their
// own whose neighbour radius admits no pair).  The black hole-star pairs
// within h_bh and the black hole pairs (always neighbours) are added here,
// in ascending index order: a star's row is its tree row, then the black
// holes (indices n_fs .. n-1, the largest); a black hole's row is its stars
// (one thread per star, in index order, ranked by warp ballots and per-block
// offsets), then the other black holes.  At most 32 black holes.
constexpr int SPB = 256;  // threads per block of the star passes

// sorted position of every index (inv) and of every black hole (bhpos)
__global__ void k_sp_inv(int n, int nfs, const int *__restrict__ order,
                         int *__restrict__ inv, int *__restrict__ bhpos)
{
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n;
         k += gridDim.x * blockDim.x) {
        const int o = order[k];
        inv[o] = k;
        if (o >= nfs) bhpos[o - nfs] = k;
    }
}

// Per star (thread o of block o / SPB): its row length (tree row plus black
// holes within h_bh) and, per black hole, the block's count of such stars.
__global__ void __launch_bounds__(SPB)
k_sp_count(int n, int nfs, int nbh, const double *__restrict__ xs,
           const int *__restrict__ inv, const int *__restrict__ bhpos,
           const long long *__restrict__ toff, double h2, int *__restrict__ cnt,
           int *__restrict__ blockcnt)
{
    __shared__ int wc[SPB / 32][32];
    const int o = blockIdx.x * SPB + threadIdx.x;
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const bool star = o < nfs;
    const int k = star ? inv[o] : 0;
    int mine = 0;
    for (int b = 0; b < nbh; ++b) {
        const bool f = star && exact_ngb(xs, n, k, bhpos[b], h2);
        mine += f;
        const unsigned m = __ballot_sync(0xffffffffu, f);
        if (lane == 0) wc[w][b] = __popc(m);
    }
    if (star) cnt[o] = (int)(toff[o + 1] - toff[o]) + mine;
    __syncthreads();
    if (threadIdx.x < nbh) {
        int t = 0;
        for (int q = 0; q < SPB / 32; ++q) t += wc[q][threadIdx.x];
        blockcnt[(size_t)blockIdx.x * nbh + threadIdx.x] = t;
    }
}

// One warp per black hole: exclusive scan of its per-block counts, and the
// length of its row (the stars, then the other black holes).
__global__ void k_sp_scan_bh(int nblk, int nfs, int nbh, int *__restrict__ blockcnt,
                             int *__restrict__ cnt)
{
    const int b = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (b >= nbh) return;
    int run = 0;
    for (int q0 = 0; q0 < nblk; q0 += 32) {
        const int q = q0 + lane;
        const int v = q < nblk ? blockcnt[(size_t)q * nbh + b] : 0;
        const int inc = warp_incl_scan(v);
        if (q < nblk) blockcnt[(size_t)q * nbh + b] = run + inc - v;
        run += __shfl_sync(0xffffffffu, inc, 31);
    }
    if (lane == 0) cnt[nfs + b] = run + (nbh - 1);
}

// Rows: every star copies its tree row and appends its black holes; every
// star within h_bh of black hole b writes its index at its rank in b's row;
// thread b < nbh of block 0 appends the other black holes to row n_fs + b.
__global__ void __launch_bounds__(SPB)
k_sp_fill(int n, int nfs, int nbh, const double *__restrict__ xs,
          const int *__restrict__ inv, const int *__restrict__ bhpos,
          const long long *__restrict__ toff, const int *__restrict__ tidx,
          long long tcap, double h2, const int *__restrict__ blockcnt,
          const long long *__restrict__ off, int *__restrict__ idx,
          long long cap, P3TDevState *st)
{
    __shared__ int wc[SPB / 32][32];
    const int o = blockIdx.x * SPB + threadIdx.x;
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const bool star = o < nfs;
    const int k = star ? inv[o] : 0;
    unsigned mine = 0;
    for (int b = 0; b < nbh; ++b) {
        const bool f = star && exact_ngb(xs, n, k, bhpos[b], h2);
        mine |= (unsigned)f << b;
        const unsigned m = __ballot_sync(0xffffffffu, f);
        if (lane == 0) wc[w][b] = __popc(m);
    }
    __syncthreads();
    if (star) {
        if (off[o + 1] > cap || toff[o + 1] > tcap) {
            p3t_raise(st, P3T_ERR_CAPACITY);
        } else {
            long long p = off[o];
            for (long long e = toff[o]; e < toff[o + 1]; ++e) idx[p++] = tidx[e];
            for (int b = 0; b < nbh; ++b)
                if ((mine >> b) & 1u) idx[p++] = nfs + b;
        }
    }
    for (int b = 0; b < nbh; ++b) {
        const bool f = (mine >> b) & 1u;
        const unsigned m = __ballot_sync(0xffffffffu, f);  // same as above
        if (!f) continue;
        int before = 0;
        for (int q = 0; q < w; ++q) before += wc[q][b];
        const long long pos = off[nfs + b] + blockcnt[(size_t)blockIdx.x * nbh + b] +
                              before + __popc(m & lanemask_lt());
        if (pos < cap)
            idx[pos] = o;
        else
            p3t_raise(st, P3T_ERR_CAPACITY);
    }
    if (blockIdx.x == 0 && threadIdx.x < nbh) {
        const int b = threadIdx.x;
        const long long e = off[nfs + b + 1];
        if (e > cap) {
            p3t_raise(st, P3T_ERR_CAPACITY);
        } else {
            long long p = e - (nbh - 1);
            for (int b2 = 0; b2 < nbh; ++b2)
                if (b2 != b) idx[p++] = nfs + b2;
        }
    }
}

}  // namespace

// fill == 0: per-particle counts into c->ngb_cnt (and the kept neighbours);
// fill == 1: CSR rows (short rows from the kept neighbours, long rows by a
// second walk over the listed groups).
int p3t_run_ngb(p3t_ctx *c, int fill, const long long *row_off, int *idx,
                long long cap, cudaStream_t s)
{
    const int n = (int)c->n;
    const int64_t G = (n + 15) / 16 + c->nclus;  // bound; the count is on the device
    int blocks = (int)((G + NW - 1) / NW);
    if (blocks > c->sms * 16) blocks = c->sms * 16;
    int nb = (n + 255) / 256;
    if (nb > c->sms * 8) nb = c->sms * 8;
    if (nb < 1) nb = 1;
    k_work_reset<<<1, 32, 0, s>>>(c->st, fill);
    if (fill) {
        k_ngb_gather<<<nb, 256, 0, s>>>(n, row_off, c->ngb_slots, idx, cap, c->st);
        k_ngb_walk<true><<<blocks, NW * 32, 0, s>>>(
            c->gclus, c->cc, c->grange, c->gmin, c->gmax, c->gctr, c->wmin,
            c->wmax, c->node, c->phi, c->plo, c->order, c->xs, n, c->ngb_cnt,
            row_off, idx, cap, c->gperm, c->ngb_slots, c->ngb_ovf, c->st,
            c->lim_walk);
        k_ngb_sort<<<nb, 256, 0, s>>>(n, row_off, idx, cap);
        p3t_count_launches(4);
    } else {
        k_ngb_walk<false><<<blocks, NW * 32, 0, s>>>(
            c->gclus, c->cc, c->grange, c->gmin, c->gmax, c->gctr, c->wmin,
            c->wmax, c->node, c->phi, c->plo, c->order, c->xs, n, c->ngb_cnt,
            row_off, idx, cap, c->gperm, c->ngb_slots, c->ngb_ovf, c->st,
            c->lim_walk);
        p3t_count_launches(2);
    }
    P3T_CUDA_TRY(cudaGetLastError());
    return P3T_OK;
}

// Neighbour lists with two species: the tree rows into the context's scratch
// (sp_off, sp_idx), then the merged rows into the caller's arrays.  needed !=
// NULL: synchronous, with capacity checks on both (the scratch grows unless
// P3T_FLAG_NO_SYNC is set).
int p3t_run_ngb_species(p3t_ctx *c, long long *offsets, int *idx, long long cap,
                        long long *needed, cudaStream_t s)
{
    const int n = (int)c->n, nbh = (int)c->n_bh, nfs = n - nbh;
    int rc = p3t_run_ngb(c, 0, nullptr, nullptr, 0, s);
    if (rc == P3T_OK) rc = p3t_scan_ll(c, c->ngb_cnt, c->sp_off, n, s);
    if (rc != P3T_OK) return rc;
    if (needed) {
        long long tnnz = 0;
        P3T_CUDA_TRY(cudaMemcpyAsync(&tnnz, c->sp_off + n, sizeof(long long),
                                     cudaMemcpyDeviceToHost, s));
        P3T_CUDA_TRY(cudaStreamSynchronize(s));
        if (tnnz > c->cap_sp_idx) {
            if (c->p.flags & P3T_FLAG_NO_SYNC) return P3T_ERR_CAPACITY;
            const int64_t want = tnnz + tnnz / 4 + 1024;
            if (c->sp_idx) cudaFree(c->sp_idx);
            c->sp_idx = nullptr;
            c->cap_sp_idx = 0;
            P3T_CUDA_TRY(cudaMalloc((void **)&c->sp_idx, (size_t)want * sizeof(int)));
            c->cap_sp_idx = want;
        }
    }
    rc = p3t_run_ngb(c, 1, c->sp_off, c->sp_idx, c->cap_sp_idx, s);
    if (rc != P3T_OK) return rc;
    const int g = (n + SPB - 1) / SPB;
    const int nblk = (nfs + SPB - 1) / SPB;
    const double h2 = c->sp.h_bh * c->sp.h_bh;
    int *bhpos = c->sp_bh, *blockcnt = c->sp_bh + 32;
    k_sp_inv<<<g, SPB, 0, s>>>(n, nfs, c->order, c->sp_inv, bhpos);
    k_sp_count<<<nblk, SPB, 0, s>>>(n, nfs, nbh, c->xs, c->sp_inv, bhpos,
                                    c->sp_off, h2, c->ngb_cnt, blockcnt);
    k_sp_scan_bh<<<1, 32 * 32, 0, s>>>(nblk, nfs, nbh, blockcnt, c->ngb_cnt);
    p3t_count_launches(3);
    rc = p3t_scan_ll(c, c->ngb_cnt, offsets, n, s);
    if (rc != P3T_OK) return rc;
    if (needed) {
        long long nnz = 0;
        P3T_CUDA_TRY(cudaMemcpyAsync(&nnz, offsets + n, sizeof(long long),
                                     cudaMemcpyDeviceToHost, s));
        P3T_CUDA_TRY(cudaStreamSynchronize(s));
        *needed = nnz;
        if (nnz > cap) return P3T_ERR_CAPACITY;
    }
    k_sp_fill<<<nblk, SPB, 0, s>>>(n, nfs, nbh, c->xs, c->sp_inv, bhpos,
                                   c->sp_off, c->sp_idx, c->cap_sp_idx, h2,
                                   blockcnt, offsets, idx, cap, c->st);
    p3t_count_launches(1);
    P3T_CUDA_TRY(cudaGetLastError());
    return P3T_OK;
}
