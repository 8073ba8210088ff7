// Per-group tree walk shared by kernels that evaluate interactions as the
// walk finds them (one warp per group).
//
// The warp keeps a stack of child ranges (first child, number of children)
// in shared memory.  Each iteration pops ranges from the top until they hold
// at most 64 cells, tests two cells per lane with the opening test of
// p3t_internal.cuh, and sends what it finds to three rings in shared memory:
// accepted cells, far leaf ranges (K = 1) and near leaf ranges (K < 1
// possible).  Whenever a ring holds a tile (64 cells or 64 particles) the
// caller's evaluator is invoked on it; the partial tiles are evaluated
// when the walk ends.  The traversal and the test are those of the list walk
// in p3t_walk.cu, so the sources met are the same sets.
#pragma once
#include "p3t_internal.cuh"

namespace p3t_walk {

constexpr int STACK = 768;  // child ranges per warp
constexpr int RING = 128;   // ring capacity; at most 127 entries are held
constexpr int WB = 64;      // cells per walk batch (two per lane)
constexpr int CTILE = 64;   // cells per tile (two per lane)
constexpr int PTILE = 64;   // particles per tile (two per lane)
// A ring holds less than a tile when a batch starts and gains at most one
// entry per cell of the batch (a leaf range holds at least one particle).
static_assert(RING >= CTILE - 1 + WB && RING >= PTILE - 1 + WB,
              "ring too small for a tile plus a batch");

struct __align__(16) Smem {
    int stack[STACK];               // packed child ranges: child*8 + nchild-1
    int cb[WB];                     // cells of the current walk batch
    float4 box[2][WB];              // their box records (wmin, wmax), by slot
    int pc[RING];                   // accepted cells
    int2 pf[RING];                  // far leaf ranges (first, count)
    int2 pn[RING];                  // near leaf ranges
    int tj[64];                     // ids of the sources of a tile
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

// Moves the next `take` (<= PTILE) particle ids off the front of a ring of
// ranges into tj[0..take), in rounds of 32.
__device__ __forceinline__ void take_tile(int2 *ring, RangeRing &r, int take,
                                          int *tj, int lane)
{
#pragma unroll
    for (int h = 0; h < PTILE / 32; ++h)
        if (take > 32 * h)
            take_particles(ring, r, min(take - 32 * h, 32), tj + 32 * h, lane);
}

// Moves the next `take` (<= CTILE) accepted cells into tj[0..take).
__device__ __forceinline__ void take_cells(Smem &S, CellRing &r, int take,
                                           int lane)
{
#pragma unroll
    for (int h = 0; h < CTILE / 32; ++h) {
        const int slot = lane + 32 * h;
        if (slot < take) S.tj[slot] = S.pc[(r.head + slot) & (RING - 1)];
    }
    __syncwarp();
    r.head = (r.head + take) & (RING - 1);
    r.n -= take;
}

// Asynchronous 16-byte copy global -> shared (cp.async).
__device__ __forceinline__ void cp_async16(void *smem, const void *gmem)
{
    const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 16;" ::"r"(sa), "l"(gmem));
}

// Pops child ranges from the top of the stack until they hold at most WB =
// 64 cells, lists them in S.cb and requests their box records into S.box
// with cp.async; returns the batch size (warp-uniform, 0 when the stack is
// empty).  The lane's cells are slots lane and lane + 32.
__device__ __forceinline__ int pop_batch(Smem &S, int &top,
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

// Walks the tree of cell `root` (the group's cluster) for one group.  The
// evaluator supplies
//   ev.cells(S, take)            tile of `take` (<= CTILE) cells, ids in S.tj
//   ev.particles<NEAR>(S, take)  tile of `take` (<= PTILE) particles, ids in
//                                S.tj
// Returns P3T_OK, P3T_ERR_CAPACITY when the stack overflowed or
// P3T_ERR_TIMEOUT after lim iterations (the group is left unfinished).
// cnt[0..2] receive the numbers of cells, near and far particles met.  The
// walk takes batches of up to 64 cells (two per lane) and is
// software-pipelined by one batch: the next batch is popped and its box
// records copied into shared memory by cp.async before the full tiles are
// evaluated (the batches and tiles are those of the plain
// pop-test-push-evaluate loop, in its order).  A leaf's box records carry
// its particle range (first particle in wmin.w, minus the count in wmax.w),
// so no second load is needed.
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
    int total = pop_batch(S, top, wmin, wmax, lane);
    int status = P3T_OK;
    while (total > 0) {
        if (++iter > lim) {  // a finite tree stays far below
            status = P3T_ERR_TIMEOUT;
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
                float d2 = box_d2(gmn, gmx, cmn, cmx);
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
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            unsigned m = __ballot_sync(full, is_pc[h]);
            if (is_pc[h]) S.pc[(rc.head + rc.n + __popc(m & lt)) & (RING - 1)] = cid[h];
            rc.n += __popc(m);
            cnt[0] += __popc(m);
            int before = rn.np;
            push_ranges(S.pn, rn, near[h], pfirst[h], pcount[h]);
            cnt[1] += rn.np - before;
            before = rf.np;
            push_ranges(S.pf, rf, farl[h], pfirst[h], pcount[h]);
            cnt[2] += rf.np - before;
        }
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            unsigned mo = __ballot_sync(full, open[h]);
            int np = __popc(mo);
            if (top + np > STACK) {
                status = P3T_ERR_CAPACITY;
                break;
            }
            if (open[h]) S.stack[top + __popc(mo & lt)] = child[h] * 8 + (nchild[h] - 1);
            top += np;
        }
        if (status != P3T_OK) break;
        __syncwarp();
        total = pop_batch(S, top, wmin, wmax, lane);
        while (rc.n >= CTILE) {
            take_cells(S, rc, CTILE, lane);
            ev.cells(S, CTILE);
        }
        while (rf.np >= PTILE) {
            take_tile(S.pf, rf, PTILE, S.tj, lane);
            ev.template particles<false>(S, PTILE);
        }
        while (rn.np >= PTILE) {
            take_tile(S.pn, rn, PTILE, S.tj, lane);
            ev.template particles<true>(S, PTILE);
        }
    }
    if (status != P3T_OK) {
        // the abandoned batch's copies land before S.box is reused
        asm volatile("cp.async.wait_all;" ::: "memory");
        __syncwarp();
        return status;
    }
    if (rc.n > 0) {
        const int t = rc.n;
        take_cells(S, rc, t, lane);
        ev.cells(S, t);
    }
    if (rf.np > 0) {
        const int t = rf.np;
        take_tile(S.pf, rf, t, S.tj, lane);
        ev.template particles<false>(S, t);
    }
    if (rn.np > 0) {
        const int t = rn.np;
        take_tile(S.pn, rn, t, S.tj, lane);
        ev.template particles<true>(S, t);
    }
    return P3T_OK;
}

}  // namespace p3t_walk
