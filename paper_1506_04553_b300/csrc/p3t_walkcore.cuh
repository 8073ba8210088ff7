// Per-group tree walk shared by kernels that evaluate interactions as the
// walk finds them (one warp per group).
//
// The warp keeps a stack of child ranges (first child, number of children)
// in shared memory.  Each iteration pops ranges from the top until they hold
// at most 32 cells, tests one cell per lane with the opening test of
// p3t_internal.cuh, and sends what it finds to three rings in shared memory:
// accepted cells, far leaf ranges (K = 1) and near leaf ranges (K < 1
// possible).  Whenever a ring holds 32 sources the caller's evaluator is
// invoked on a tile of 32; the partial tiles are evaluated when the walk
// ends.  The traversal and the test are those of the list walk in
// p3t_walk.cu, so the sources met are the same sets.
#pragma once
#include "p3t_internal.cuh"

namespace p3t_walk {

constexpr int STACK = 768;  // child ranges per warp
constexpr int RING = 64;    // ring capacity; at most 63 entries are held

struct __align__(16) Smem {
    int stack[STACK];               // packed child ranges: child*8 + nchild-1
    int cb[32];                     // cells of the current walk batch
    int pc[RING];                   // accepted cells
    int2 pf[RING];                  // far leaf ranges (first, count)
    int2 pn[RING];                  // near leaf ranges
    int tj[32];                     // ids of the staged sources
};

struct RangeRing {
    int head, nr, np;  // first entry, ranges held, particles held
};

struct CellRing {
    int head, n;
};

// Appends one range per flagged lane.
__device__ __forceinline__ void push_ranges(int2 *ring, RangeRing &r,
                                            bool flag, int first, int count)
{
    const unsigned m = __ballot_sync(0xffffffffu, flag);
    if (flag)
        ring[(r.head + r.nr + __popc(m & lanemask_lt())) & (RING - 1)] =
            make_int2(first, count);
    const int c = __reduce_add_sync(0xffffffffu, flag ? count : 0);
    r.nr += __popc(m);
    r.np += c;
}

// Moves the next `take` (<= 32, <= r.np) particle ids off the front of a ring
// of ranges into tj[0..take).  Lane p finds the range holding position p by a
// binary search over the ranges' inclusive prefix counts (one per lane):
// they rise strictly over the ranges (none is empty) and stay at their total,
// at least take > p, on the lanes past them.
__device__ __forceinline__ void take_particles(int2 *ring, RangeRing &r,
                                               int take, int *tj, int lane)
{
    const bool have = lane < r.nr;
    int2 g = have ? ring[(r.head + lane) & (RING - 1)] : make_int2(0, 0);
    int inc = warp_incl_scan(g.y);
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
    if (lane < take) tj[lane] = ox + (lane - (oinc - oy));
    const unsigned full = __ballot_sync(0xffffffffu, have && inc <= take);
    const int nfull = __popc(full);
    const int exc = inc - g.y;
    if (lane == nfull && have && exc < take) {
        int used = take - exc;
        ring[(r.head + lane) & (RING - 1)] = make_int2(g.x + used, g.y - used);
    }
    __syncwarp();
    r.head = (r.head + nfull) & (RING - 1);
    r.nr -= nfull;
    r.np -= take;
}

// Moves the next `take` accepted cells into tj[0..take).
__device__ __forceinline__ void take_cells(Smem &S, CellRing &r, int take,
                                           int lane)
{
    if (lane < take) S.tj[lane] = S.pc[(r.head + lane) & (RING - 1)];
    __syncwarp();
    r.head = (r.head + take) & (RING - 1);
    r.n -= take;
}

// Pops child ranges from the top of the stack until they hold at most 32
// cells; returns this lane's cell of the batch (-1 past its end) and the
// batch size in total (warp-uniform, 0 when the stack is empty).
__device__ __forceinline__ int pop_batch(Smem &S, int &top, int &total,
                                         int lane)
{
    const unsigned full = 0xffffffffu;
    if (top == 0) {
        total = 0;
        return -1;
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
    total = __shfl_sync(full, inc, ntake - 1);
    if (take)
        for (int t = 0; t < ry; ++t) S.cb[inc - ry + t] = rx + t;
    top -= ntake;
    __syncwarp();
    const int c = lane < total ? S.cb[lane] : -1;
    __syncwarp();
    return c;
}

// Walks the tree of cell `root` (the group's cluster) for one group.  The
// evaluator supplies
//   ev.cells(S, take)            tile of `take` cells, ids in S.tj
//   ev.particles<NEAR>(S, take)  tile of `take` particles, ids in S.tj
// Returns P3T_OK, P3T_ERR_CAPACITY when the stack overflowed or
// P3T_ERR_TIMEOUT after lim iterations (the group is left unfinished).
// cnt[0..2] receive the numbers of cells, near and far particles met.  The
// walk is software-pipelined by one batch: the next batch is popped and its
// box records requested before the full tiles are evaluated (the batches and
// tiles are those of the plain pop-test-push-evaluate loop, in its order).
// A leaf's box records carry its particle range (first particle in
// wmin.w, minus the count in wmax.w), so no second load is needed.
template <class Ev>
__device__ __forceinline__ int walk_group(
    Smem &S, float4 gmn, float4 gmx, const float4 *__restrict__ wmin,
    const float4 *__restrict__ wmax, float theta2, float hg2, int root,
    int lane, Ev &ev, long long cnt[3], long long lim)
{
    const unsigned full = 0xffffffffu, lt = lanemask_lt();
    CellRing rc = {0, 0};
    RangeRing rf = {0, 0, 0}, rn = {0, 0, 0};
    if (lane == 0) S.stack[0] = root * 8;  // the group's root, one cell
    int top = 1;
    long long iter = 0;
    __syncwarp();
    int total = 0;
    int c = pop_batch(S, top, total, lane);
    float4 cmn = make_float4(0.f, 0.f, 0.f, 0.f), cmx = cmn;
    if (c >= 0) {
        cmn = wmin[c];
        cmx = wmax[c];
    }
    while (total > 0) {
        if (++iter > lim) return P3T_ERR_TIMEOUT;  // a finite tree stays far below
        bool is_pc = false, near = false, farl = false, open = false;
        int child = 0, nchild = 0, pfirst = 0, pcount = 0;
        if (c >= 0) {
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
                    farl = !near;
                } else {
                    open = true;
                }
            }
        }
        {
            unsigned m = __ballot_sync(full, is_pc);
            if (is_pc) S.pc[(rc.head + rc.n + __popc(m & lt)) & (RING - 1)] = c;
            rc.n += __popc(m);
            cnt[0] += __popc(m);
        }
        {
            int before = rn.np;
            push_ranges(S.pn, rn, near, pfirst, pcount);
            cnt[1] += rn.np - before;
            before = rf.np;
            push_ranges(S.pf, rf, farl, pfirst, pcount);
            cnt[2] += rf.np - before;
        }
        {
            unsigned mo = __ballot_sync(full, open);
            int np = __popc(mo);
            if (top + np > STACK) return P3T_ERR_CAPACITY;
            if (open) S.stack[top + __popc(mo & lt)] = child * 8 + (nchild - 1);
            top += np;
        }
        __syncwarp();
        c = pop_batch(S, top, total, lane);
        if (c >= 0) {
            cmn = wmin[c];
            cmx = wmax[c];
        }
        while (rc.n >= 32) {
            take_cells(S, rc, 32, lane);
            ev.cells(S, 32);
        }
        while (rf.np >= 32) {
            take_particles(S.pf, rf, 32, S.tj, lane);
            ev.template particles<false>(S, 32);
        }
        while (rn.np >= 32) {
            take_particles(S.pn, rn, 32, S.tj, lane);
            ev.template particles<true>(S, 32);
        }
    }
    if (rc.n > 0) {
        const int t = rc.n;
        take_cells(S, rc, t, lane);
        ev.cells(S, t);
    }
    if (rf.np > 0) {
        const int t = rf.np;
        take_particles(S.pf, rf, t, S.tj, lane);
        ev.template particles<false>(S, t);
    }
    if (rn.np > 0) {
        const int t = rn.np;
        take_particles(S.pn, rn, t, S.tj, lane);
        ev.template particles<true>(S, t);
    }
    return P3T_OK;
}

}  // namespace p3t_walk
