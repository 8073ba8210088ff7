// Tree walk: interaction lists per group (Sect. 2.2, Barnes-Hut with the
// opening criterion theta).
//
// Opening test (the paper names the parameter, not its form).  For the FP32
// outward-rounded member boxes of group g and cell c, in FP32 with one
// rounding per operation and in this order:
//     gap_a = max(max(cmin_a - gmax_a, gmin_a - cmax_a), 0)
//     d2    = (gap_x*gap_x + gap_y*gap_y) + gap_z*gap_z
//     l     = max(max(cmax_x - cmin_x, cmax_y - cmin_y), cmax_z - cmin_z)
//     accept  <=>  l*l < theta2*d2  and  d2 > hg2
// theta2 = fl(theta)^2 and hg2 = fl(max(h, r_cut))^2 * (1 + 2^-10).  An
// accepted cell goes to the cell list (evaluated with K = 1, since every
// pair it stands for is farther apart than max(h, r_cut)); a leaf that is not
// accepted puts its particles on the near list (d2 <= hg2: K < 1 and
// neighbours possible) or the far list (K = 1); any other cell is opened.
//
// One warp per group.  The warp keeps a stack of child ranges (first child,
// number of children) in shared memory; each iteration pops ranges from the
// top until they hold at most 32 cells, tests one cell per lane, appends
// accepted cells and leaf particles with warp prefix sums, and pushes the
// ranges of opened cells.  Each iteration that grows the stack descends one
// level, so the stack never holds more than 32 ranges per level (672 for 21
// levels); the capacity below is 1024 and an overflow raises an error.
//
// The walk runs twice: a counting pass (per-group list lengths, then a scan
// into offsets) and a filling pass that writes the lists.
#include "p3t_internal.cuh"

namespace {

constexpr int WALK_WARPS = 4;
constexpr int WALK_STACK = 1024;

template <bool FILL>
__global__ void __launch_bounds__(WALK_WARPS * 32)
k_walk(int ngroup, const int *__restrict__ gclus,
       const ClusterConsts *__restrict__ ccs, const int2 *__restrict__ grange,
       const float4 *__restrict__ gmin, const float4 *__restrict__ gmax,
       const float4 *__restrict__ wmin, const float4 *__restrict__ wmax,
       const int4 *__restrict__ node, float theta2,
       long long *__restrict__ cnt, const long long *__restrict__ off,
       int *__restrict__ pc_list, int *__restrict__ ppn_list,
       int *__restrict__ ppf_list, P3TDevState *st, long long lim_walk)
{
    __shared__ int2 stack[WALK_WARPS][WALK_STACK];
    __shared__ int buf[WALK_WARPS][32];
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const unsigned full = 0xffffffffu, lt = lanemask_lt();
    int2 *stk = stack[w];
    int *cb = buf[w];
    for (int g = blockIdx.x * WALK_WARPS + w; g < ngroup;
         g += gridDim.x * WALK_WARPS) {
        const float4 gmn = gmin[g], gmx = gmax[g];
        const int cl = gclus[g];
        const float hg2 = ccs[cl].hg2;
        long long npc = 0, nppn = 0, nppf = 0;
        long long o_pc = 0, o_ppn = 0, o_ppf = 0;
        if (FILL) {
            o_pc = off[g];
            o_ppn = off[(ngroup + 1) + g];
            o_ppf = off[2 * (ngroup + 1) + g];
        }
        if (lane == 0) stk[0] = make_int2(cl, 1);  // the cluster's root
        int top = 1;
        bool overflow = false, timeout = false;
        long long iter = 0;
        __syncwarp();
        while (top > 0) {
            if (++iter > lim_walk) {  // a finite tree stays far below the default
                timeout = true;
                break;
            }
            // pop child ranges from the top holding at most 32 cells
            int2 r = lane < top ? stk[top - 1 - lane] : make_int2(0, 0);
            int inc = warp_incl_scan(r.y);
            bool take = lane < top && inc <= 32;
            unsigned tk = __ballot_sync(full, take);
            int ntake = __popc(tk);
            int total = __shfl_sync(full, inc, ntake - 1);
            if (take)
                for (int t = 0; t < r.y; ++t) cb[inc - r.y + t] = r.x + t;
            top -= ntake;
            __syncwarp();
            const int c = lane < total ? cb[lane] : -1;
            __syncwarp();

            bool is_pc = false, near = false, far = false, open = false;
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
                    if (nchild <= 0) {  // a leaf: first particle, -count
                        pfirst = child;
                        pcount = -nchild;
                        near = d2 <= hg2;
                        far = !near;
                    } else {
                        open = true;
                    }
                }
            }
            // cell list
            unsigned m = __ballot_sync(full, is_pc);
            if (FILL && is_pc) pc_list[o_pc + npc + __popc(m & lt)] = c;
            npc += __popc(m);
            // near / far particle lists
            {
                int x = near ? pcount : 0;
                int ix = warp_incl_scan(x);
                int tot = __shfl_sync(full, ix, 31);
                if (FILL && near) {
                    long long b = o_ppn + nppn + (ix - x);
                    for (int t = 0; t < pcount; ++t) ppn_list[b + t] = pfirst + t;
                }
                nppn += tot;
            }
            {
                int x = far ? pcount : 0;
                int ix = warp_incl_scan(x);
                int tot = __shfl_sync(full, ix, 31);
                if (FILL && far) {
                    long long b = o_ppf + nppf + (ix - x);
                    for (int t = 0; t < pcount; ++t) ppf_list[b + t] = pfirst + t;
                }
                nppf += tot;
            }
            // push opened ranges
            unsigned mo = __ballot_sync(full, open);
            int np = __popc(mo);
            if (top + np > WALK_STACK) {
                overflow = true;
                break;
            }
            if (open) stk[top + __popc(mo & lt)] = make_int2(child, nchild);
            top += np;
            if (lane == 0) atomicMax(&st->max_stack, top);
            __syncwarp();
        }
        if (overflow || timeout) {
            if (lane == 0) p3t_raise(st, timeout ? P3T_ERR_TIMEOUT : P3T_ERR_CAPACITY);
            npc = nppn = nppf = 0;
        }
        if (!FILL && lane == 0) {
            cnt[g] = npc;
            cnt[ngroup + g] = nppn;
            cnt[2 * ngroup + g] = nppf;
        }
        __syncwarp();
    }
}

// Exclusive scan of the three per-group counts into offsets (n+1 entries
// each, rows of length ngroup+1), list totals and interaction counts.
// One block; each thread scans a contiguous chunk.
constexpr int SCAN_T = 1024;

__global__ void __launch_bounds__(SCAN_T)
k_scan_lists(int ngroup, const long long *__restrict__ cnt,
             const int2 *__restrict__ grange, long long *__restrict__ off,
             P3TDevState *st)
{
    __shared__ long long part[SCAN_T];
    __shared__ long long ipart[3][SCAN_T];
    const int t = threadIdx.x;
    const int chunk = (ngroup + SCAN_T - 1) / SCAN_T;
    const int b = t * chunk;
    const int e = min(ngroup, b + chunk);
    for (int L = 0; L < 3; ++L) {
        const long long *c = cnt + (long long)L * ngroup;
        long long *o = off + (long long)L * (ngroup + 1);
        long long s = 0, ip = 0;
        for (int g = b; g < e; ++g) {
            s += c[g];
            ip += c[g] * (long long)grange[g].y;
        }
        part[t] = s;
        if (L == 0) ipart[0][t] = ip;
        else if (L == 1) { ipart[1][t] = ip; ipart[2][t] = ip; }
        else ipart[1][t] += ip;
        __syncthreads();
        if (t == 0) {
            long long run = 0;
            for (int q = 0; q < SCAN_T; ++q) {
                long long v = part[q];
                part[q] = run;
                run += v;
            }
            st->tot[L] = run;
            o[ngroup] = run;
        }
        __syncthreads();
        long long run = part[t];
        for (int g = b; g < e; ++g) {
            o[g] = run;
            run += c[g];
        }
        __syncthreads();
    }
    if (t == 0) {
        long long a = 0, p = 0, pn = 0;
        for (int q = 0; q < SCAN_T; ++q) {
            a += ipart[0][q];
            p += ipart[1][q];
            pn += ipart[2][q];
        }
        st->int_pc = a;
        st->int_pp = p;
        st->int_ppn = pn;
    }
}

}  // namespace

void p3t_mac_constants(const p3t_params *p, float *theta2, float *hg2)
{
    float th = (float)p->theta;
    *theta2 = th * th;
    double hh = p->h > 0.0 ? p->h : p->r_out;
    float hg = (float)(hh > p->r_out ? hh : p->r_out);
    float hs = hg * hg;
    *hg2 = hs * 1.0009765625f;
}

int p3t_run_walk(p3t_ctx *c, int fill, cudaStream_t s)
{
    const int G = c->hst->ngroup;
    if (G == 0) return P3T_OK;
    float theta2, hg2;
    p3t_mac_constants(&c->p, &theta2, &hg2);
    int blocks = (G + WALK_WARPS - 1) / WALK_WARPS;
    int maxb = c->sms * 8;
    if (blocks > maxb) blocks = maxb;
    if (fill)
        k_walk<true><<<blocks, WALK_WARPS * 32, 0, s>>>(
            G, c->gclus, c->cc, c->grange, c->gmin, c->gmax, c->wmin, c->wmax,
            c->node, theta2, c->lcnt, c->loff, c->list[0], c->list[1],
            c->list[2], c->st, c->lim_walk);
    else
        k_walk<false><<<blocks, WALK_WARPS * 32, 0, s>>>(
            G, c->gclus, c->cc, c->grange, c->gmin, c->gmax, c->wmin, c->wmax,
            c->node, theta2, c->lcnt, c->loff, c->list[0], c->list[1],
            c->list[2], c->st, c->lim_walk);
    p3t_count_launches(1);
    P3T_CUDA_TRY(cudaGetLastError());
    return P3T_OK;
}

int p3t_scan_lists(p3t_ctx *c, cudaStream_t s)
{
    const int G = c->hst->ngroup;
    if (G == 0) return P3T_OK;
    k_scan_lists<<<1, SCAN_T, 0, s>>>(G, c->lcnt, c->grange, c->loff, c->st);
    p3t_count_launches(1);
    P3T_CUDA_TRY(cudaGetLastError());
    return P3T_OK;
}
