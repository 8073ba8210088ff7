// C ABI of libp3t: context, memory management and the entry points declared
// in include/p3t.h.
#include <float.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include <atomic>
#include <new>

#include "p3t_internal.cuh"

static std::atomic<long long> g_launches{0};

void p3t_count_launches(long long k) { g_launches.fetch_add(k); }

int p3t_prof_open(p3t_ctx *c, int phase, cudaStream_t s)
{
    if (!c->prof_on) return -1;
    P3TEvents &e = c->prof;
    if (e.used == e.cap) {
        int cap = e.cap ? 2 * e.cap : 64;
        cudaEvent_t *ev = (cudaEvent_t *)realloc(e.ev, 2 * cap * sizeof(cudaEvent_t));
        int *ph = (int *)realloc(e.phase, cap * sizeof(int));
        if (!ev || !ph) return -1;
        e.ev = ev;
        e.phase = ph;
        for (int k = 2 * e.cap; k < 2 * cap; ++k)
            if (cudaEventCreate(&e.ev[k]) != cudaSuccess) return -1;
        e.cap = cap;
    }
    int slot = e.used++;
    e.phase[slot] = phase;
    cudaEventRecord(e.ev[2 * slot], s);
    return slot;
}

void p3t_prof_close(p3t_ctx *c, int slot, cudaStream_t s)
{
    if (slot < 0) return;
    cudaEventRecord(c->prof.ev[2 * slot + 1], s);
}

// Resolves recorded event pairs into the per-phase totals.
static int prof_resolve(p3t_ctx *c)
{
    P3TEvents &e = c->prof;
    for (int k = 0; k < e.used; ++k) {
        if (cudaEventSynchronize(e.ev[2 * k + 1]) != cudaSuccess) return P3T_ERR_CUDA;
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, e.ev[2 * k], e.ev[2 * k + 1]) != cudaSuccess)
            return P3T_ERR_CUDA;
        c->prof_ms[e.phase[k]] += ms;
        c->prof_calls[e.phase[k]] += 1;
    }
    e.used = 0;
    return P3T_OK;
}

void p3t_cluster_consts(const p3t_params *p, double r_out, double eps,
                        double h, ClusterConsts *k)
{
    double hh = h > 0.0 ? h : r_out;
    k->eps2 = (float)(eps * eps);
    k->kA = (float)(1.0 / ((1.0 - p->gamma) * r_out));
    k->kB = (float)(-p->gamma / (1.0 - p->gamma));
    float hg = (float)(hh > r_out ? hh : r_out);
    float hs = hg * hg;
    k->hg2 = hs * 1.0009765625f;
    k->h = hh;
    k->h2 = hh * hh;
    k->r_out = r_out;
    double g = p->gamma;
    if (g > 0.0) {
        double g2 = g * g, g3 = g2 * g, g4 = g3 * g, g5 = g4 * g, g6 = g5 * g;
        double gm1 = g - 1.0;
        double gm17 = gm1 * gm1 * gm1 * gm1 * gm1 * gm1 * gm1;
        k->w_in = 7.0 * (g6 - 9.0 * g5 + 45.0 * g4 - 60.0 * g3 * log(g)
                         - 45.0 * g2 + 9.0 * g - 1.0) / (3.0 * gm17);
    } else {
        k->w_in = 7.0 / 3.0;
    }
}

namespace {

template <class T>
int grow(T *&ptr, int64_t &cap_slot, int64_t want, size_t per)
{
    (void)cap_slot;
    if (ptr) cudaFree(ptr);
    ptr = nullptr;
    if (want <= 0) want = 1;
    P3T_CUDA_TRY(cudaMalloc((void **)&ptr, (size_t)want * per));
    return P3T_OK;
}

#define P3T_TRY(expr)                \
    do {                             \
        int r__ = (expr);            \
        if (r__ != P3T_OK) return r__; \
    } while (0)

int check_params(const p3t_params *p)
{
    if (!p) return P3T_ERR_INVALID;
    if (!(p->theta >= 0.0) || !isfinite(p->theta)) return P3T_ERR_INVALID;
    if (!(p->r_out >= P3T_R_OUT_MIN) || !isfinite(p->r_out)) return P3T_ERR_INVALID;
    if (!(p->gamma >= 0.0 && p->gamma < 1.0)) return P3T_ERR_INVALID;
    if (!(p->eps >= 0.0) || !isfinite(p->eps)) return P3T_ERR_INVALID;
    if (!(p->h >= 0.0) || !isfinite(p->h)) return P3T_ERR_INVALID;
    if (!(p->G > 0.0) || !isfinite(p->G)) return P3T_ERR_INVALID;
    if (p->n_leaf < 1 || p->n_leaf > 64) return P3T_ERR_INVALID;
    if (p->n_group < 1 || p->n_group > 64) return P3T_ERR_INVALID;
    return P3T_OK;
}

int ensure_clusters(p3t_ctx *c, int nc)
{
    if (nc <= c->cap_clus) return P3T_OK;
    int cap = nc + 16;
    if (c->clus_off_h) cudaFreeHost(c->clus_off_h);
    if (c->cc_h) cudaFreeHost(c->cc_h);
    c->clus_off_h = nullptr;
    c->cc_h = nullptr;
    P3T_CUDA_TRY(cudaMallocHost((void **)&c->clus_off_h, (cap + 1) * sizeof(int64_t)));
    P3T_CUDA_TRY(cudaMallocHost((void **)&c->cc_h, cap * sizeof(ClusterConsts)));
    free(c->clus_par);
    c->clus_par = (double *)calloc(3 * (size_t)cap, sizeof(double));
    if (!c->clus_par) return P3T_ERR_CUDA;
    int64_t d = 0;
    P3T_TRY(grow(c->clus_off, d, cap + 1, sizeof(int64_t)));
    P3T_TRY(grow(c->cc, d, cap, sizeof(ClusterConsts)));
    P3T_TRY(grow(c->clus_box, d, 8 * (int64_t)cap, sizeof(double)));
    c->cap_clus = cap;
    return P3T_OK;
}

// Writes the per-cluster constants of the current layout to pinned memory
// and queues their upload.
int upload_clusters(p3t_ctx *c, cudaStream_t s)
{
    for (int k = 0; k < c->nclus; ++k) {
        double r = c->p.r_out, e = c->p.eps, h = c->p.h;
        if (c->ensemble) {
            if (c->clus_par[k] > 0.0) r = c->clus_par[k];
            if (c->clus_par[c->cap_clus + k] >= 0.0) e = c->clus_par[c->cap_clus + k];
            if (c->clus_par[2 * c->cap_clus + k] > 0.0) h = c->clus_par[2 * c->cap_clus + k];
        }
        p3t_cluster_consts(&c->p, r, e, h, &c->cc_h[k]);
    }
    P3T_CUDA_TRY(cudaMemcpyAsync(c->clus_off, c->clus_off_h,
                                 (c->nclus + 1) * sizeof(int64_t),
                                 cudaMemcpyHostToDevice, s));
    P3T_CUDA_TRY(cudaMemcpyAsync(c->cc, c->cc_h, c->nclus * sizeof(ClusterConsts),
                                 cudaMemcpyHostToDevice, s));
    return P3T_OK;
}

int ensure_particles(p3t_ctx *c, int64_t n)
{
    if (n <= c->cap_n) return P3T_OK;
    int64_t cap = n + n / 8 + 1024;
    int64_t d = 0;
    P3T_TRY(grow(c->key_a, d, cap, sizeof(u64)));
    P3T_TRY(grow(c->key_b, d, cap, sizeof(u64)));
    P3T_TRY(grow(c->idx_a, d, cap, sizeof(int)));
    P3T_TRY(grow(c->idx_b, d, cap, sizeof(int)));
    P3T_TRY(grow(c->order, d, cap, sizeof(int)));
    P3T_TRY(grow(c->xs, d, 3 * cap, sizeof(double)));
    P3T_TRY(grow(c->ms, d, cap, sizeof(double)));
    P3T_TRY(grow(c->phi, d, cap, sizeof(float4)));
    P3T_TRY(grow(c->plo, d, cap, sizeof(float4)));
    P3T_TRY(grow(c->ngb_cnt, d, cap, sizeof(int)));
    P3T_TRY(grow(c->ngb_slots, d, P3T_NGB_SLOTS * cap, sizeof(int)));
    P3T_TRY(grow(c->ngb_ovf, d, cap, sizeof(int)));
    c->cap_tiles = p3t_sort_tiles(cap);
    P3T_TRY(grow(c->rs_counts, d, 256 * c->cap_tiles, sizeof(int)));
    c->cap_scan = p3t_scan_blocks(cap) + 2;
    P3T_TRY(grow(c->scan_part, d, c->cap_scan, sizeof(long long)));
    // groups: at most one per particle
    c->cap_groups = cap;
    P3T_TRY(grow(c->grange, d, cap, sizeof(int2)));
    P3T_TRY(grow(c->gmin, d, cap, sizeof(float4)));
    P3T_TRY(grow(c->gmax, d, cap, sizeof(float4)));
    P3T_TRY(grow(c->gctr, d, cap, sizeof(float4)));
    P3T_TRY(grow(c->lcnt, d, 3 * cap, sizeof(long long)));
    P3T_TRY(grow(c->loff, d, 3 * (cap + 1), sizeof(long long)));
    P3T_TRY(grow(c->pclus, d, cap, sizeof(int)));
    P3T_TRY(grow(c->gclus, d, cap, sizeof(int)));
    P3T_TRY(grow(c->gperm, d, cap, sizeof(int)));
    P3T_TRY(grow(c->gcost, d, cap, sizeof(float)));
    P3T_TRY(grow(c->pgroup, d, cap, sizeof(int)));
    // the recorded group costs went with the old arrays
    P3T_CUDA_TRY(cudaMemset(&c->st->cost_n, 0, sizeof(int)));
    c->cap_n = cap;
    return P3T_OK;
}

int ensure_cells(p3t_ctx *c, int64_t want)
{
    if (want <= c->cap_cells) return P3T_OK;
    int64_t cap = want;
    int64_t d = 0;
    P3T_TRY(grow(c->node, d, cap, sizeof(int4)));
    P3T_TRY(grow(c->parent, d, cap, sizeof(int)));
    P3T_TRY(grow(c->leaf_list, d, cap, sizeof(int)));
    P3T_TRY(grow(c->leaf_sorted, d, cap, sizeof(int)));
    P3T_TRY(grow(c->cpend, d, cap, sizeof(int)));
    P3T_TRY(grow(c->cM, d, cap, sizeof(double)));
    P3T_TRY(grow(c->ccom, d, 3 * cap, sizeof(double)));
    P3T_TRY(grow(c->cQ, d, 6 * cap, sizeof(double)));
    P3T_TRY(grow(c->cbmin, d, 3 * cap, sizeof(double)));
    P3T_TRY(grow(c->cbmax, d, 3 * cap, sizeof(double)));
    P3T_TRY(grow(c->wmin, d, cap, sizeof(float4)));
    P3T_TRY(grow(c->wmax, d, cap, sizeof(float4)));
    P3T_TRY(grow(c->cf0, d, cap, sizeof(float4)));
    P3T_TRY(grow(c->cf1, d, cap, sizeof(float4)));
    P3T_TRY(grow(c->cf2, d, cap, sizeof(float4)));
    c->cap_cells = cap;
    return P3T_OK;
}

// Grows the cell arrays while keeping the current tree (copied over).
int ensure_cells_keep(p3t_ctx *c, int64_t want)
{
    if (want <= c->cap_cells) return P3T_OK;
    p3t_ctx old = *c;
    c->node = nullptr; c->parent = nullptr; c->cM = nullptr; c->ccom = nullptr;
    c->cQ = nullptr; c->cbmin = nullptr; c->cbmax = nullptr; c->wmin = nullptr;
    c->wmax = nullptr; c->cf0 = nullptr; c->cf1 = nullptr; c->cf2 = nullptr;
    c->cap_cells = 0;
    P3T_TRY(ensure_cells(c, want));
    const size_t C = (size_t)old.cap_cells;
    struct { void *dst, *src; size_t bytes; } cp[] = {
        {c->node, old.node, C * sizeof(int4)}, {c->parent, old.parent, C * 4},
        {c->cM, old.cM, C * 8}, {c->ccom, old.ccom, 3 * C * 8},
        {c->cQ, old.cQ, 6 * C * 8}, {c->cbmin, old.cbmin, 3 * C * 8},
        {c->cbmax, old.cbmax, 3 * C * 8}, {c->wmin, old.wmin, C * 16},
        {c->wmax, old.wmax, C * 16}, {c->cf0, old.cf0, C * 16},
        {c->cf1, old.cf1, C * 16}, {c->cf2, old.cf2, C * 16}};
    for (auto &e : cp) {
        P3T_CUDA_TRY(cudaMemcpy(e.dst, e.src, e.bytes, cudaMemcpyDeviceToDevice));
        cudaFree(e.src);
    }
    return P3T_OK;
}

int ensure_list(p3t_ctx *c, int L, int64_t want)
{
    if (want <= c->cap_list[L]) return P3T_OK;
    int64_t cap = want + want / 4 + 1024;
    int64_t d = 0;
    P3T_TRY(grow(c->list[L], d, cap, sizeof(int)));
    c->cap_list[L] = cap;
    return P3T_OK;
}

int sync_state(p3t_ctx *c, cudaStream_t s)
{
    P3T_CUDA_TRY(cudaMemcpyAsync(c->hst, c->st, sizeof(P3TDevState),
                                 cudaMemcpyDeviceToHost, s));
    P3T_CUDA_TRY(cudaStreamSynchronize(s));
    return P3T_OK;
}

int clear_error(p3t_ctx *c, cudaStream_t s)
{
    P3T_CUDA_TRY(cudaMemsetAsync(&c->st->error, 0, sizeof(int), s));
    return P3T_OK;
}

void free_all(p3t_ctx *c)
{
    void *ptrs[] = {c->st, c->key_a, c->key_b, c->idx_a, c->idx_b, c->order,
                    c->xs, c->ms, c->phi, c->plo, c->ngb_cnt, c->ngb_slots, c->ngb_ovf, c->rs_counts,
                    c->rs_totals, c->bbox_part, c->node, c->parent, c->cM,
                    c->ccom, c->cQ, c->cbmin, c->cbmax, c->wmin, c->wmax,
                    c->cf0, c->cf1, c->cf2, c->grange, c->gmin, c->gmax,
                    c->gctr, c->lcnt, c->loff, c->list[0], c->list[1],
                    c->list[2], c->scan_part, c->red_part, c->cadj,
                    c->clus_off, c->cc, c->clus_box, c->pclus, c->gclus,
                    c->gperm, c->gcost, c->pgroup, c->leaf_list, c->leaf_sorted, c->cpend, c->hparent, c->hcsize,
                    c->hcfill, c->hmember, c->hlev, c->hcstart, c->ht, c->ha,
                    c->hj, c->hxp, c->hvp, c->hroots, c->hloc, c->hbucket,
                    c->sp_off, c->sp_idx, c->sp_inv, c->sp_bh, c->sp_part};
    for (void *p : ptrs)
        if (p) cudaFree(p);
    if (c->hst) cudaFreeHost(c->hst);
    if (c->clus_off_h) cudaFreeHost(c->clus_off_h);
    if (c->cc_h) cudaFreeHost(c->cc_h);
    free(c->clus_par);
    for (int k = 0; k < 2 * c->prof.cap; ++k) cudaEventDestroy(c->prof.ev[k]);
    free(c->prof.ev);
    free(c->prof.phase);
}

}  // namespace

extern "C" {

int p3t_default_params(p3t_params *p)
{
    if (!p) return P3T_ERR_INVALID;
    memset(p, 0, sizeof(*p));
    p->theta = 0.4;
    p->r_out = 1.0 / 64.0;
    p->gamma = 0.1;
    p->eps = 0.0;
    p->h = 0.0;
    p->G = 1.0;
    p->n_leaf = 16;
    p->n_group = 64;
    p->flags = 0;
    return P3T_OK;
}

int p3t_create(p3t_ctx **out, const p3t_params *p)
{
    if (!out) return P3T_ERR_INVALID;
    *out = nullptr;
    P3T_TRY(check_params(p));
    p3t_ctx *c = new (std::nothrow) p3t_ctx;
    if (!c) return P3T_ERR_CUDA;
    memset(c, 0, sizeof(*c));
    c->p = *p;
    if (cudaGetDevice(&c->device) != cudaSuccess) {
        delete c;
        return P3T_ERR_CUDA;
    }
    cudaDeviceGetAttribute(&c->sms, cudaDevAttrMultiProcessorCount, c->device);
    if (c->sms <= 0) c->sms = 148;
    c->lim_walk = P3T_LIM_WALK;
    c->lim_uf = P3T_LIM_UF;
    c->lim_block = P3T_LIM_BLOCK;
    int64_t d = 0;
    int rc = P3T_OK;
    if ((rc = grow(c->st, d, 1, sizeof(P3TDevState))) != P3T_OK ||
        cudaMallocHost((void **)&c->hst, sizeof(P3TDevState)) != cudaSuccess ||
        (rc = grow(c->rs_totals, d, 256, sizeof(int))) != P3T_OK ||
        (rc = grow(c->bbox_part, d, 6 * c->sms * 4, sizeof(double))) != P3T_OK ||
        (rc = grow(c->red_part, d, 2 * c->sms * 4, sizeof(double))) != P3T_OK) {
        free_all(c);
        delete c;
        return rc ? rc : P3T_ERR_CUDA;
    }
    if (ensure_clusters(c, 1) != P3T_OK) {
        free_all(c);
        delete c;
        return P3T_ERR_CUDA;
    }
    c->nclus = 1;
    if (cudaMemset(c->st, 0, sizeof(P3TDevState)) != cudaSuccess) {
        free_all(c);
        delete c;
        return P3T_ERR_CUDA;
    }
    memset(c->hst, 0, sizeof(P3TDevState));
    *out = c;
    return P3T_OK;
}

int p3t_destroy(p3t_ctx *c)
{
    if (!c) return P3T_OK;
    cudaDeviceSynchronize();
    free_all(c);
    delete c;
    return P3T_OK;
}

int p3t_set_params(p3t_ctx *c, const p3t_params *p)
{
    if (!c) return P3T_ERR_INVALID;
    P3T_TRY(check_params(p));
    c->p = *p;
    c->lists_valid = 0;
    return P3T_OK;
}

int p3t_build_tree(p3t_ctx *c, int64_t n, const double *pos,
                   const double *mass, void *stream)
{
    if (!c || n < 0 || n > 0x7fffff00LL) return P3T_ERR_INVALID;
    if (n > 0 && (!pos || !mass)) return P3T_ERR_INVALID;
    cudaStream_t s = (cudaStream_t)stream;
    const bool no_sync = (c->p.flags & P3T_FLAG_NO_SYNC) != 0;
    if (c->ensemble && n != c->clus_off_h[c->nclus]) return P3T_ERR_INVALID;
    c->built = 0;
    c->lists_valid = 0;
    c->n = n;
    if (n == 0) {
        memset(c->hst, 0, sizeof(P3TDevState));
        P3T_CUDA_TRY(cudaMemcpyAsync(c->st, c->hst, sizeof(P3TDevState),
                                     cudaMemcpyHostToDevice, s));
        c->built = 1;
        return P3T_OK;
    }
    if (!c->ensemble) {
        c->nclus = 1;
        c->clus_off_h[0] = 0;
        c->clus_off_h[1] = n;
    }
    if (no_sync) {
        // nothing may be allocated or waited for: capacities must suffice
        if (n > c->cap_n || c->cap_cells == 0) return P3T_ERR_CAPACITY;
    } else {
        P3T_TRY(ensure_particles(c, n));
        int64_t first = n / 2 + 64;
        if (c->lim_cells > 0 && first > c->lim_cells) first = c->lim_cells;
        if (c->cap_cells < first) P3T_TRY(ensure_cells(c, first));
    }
    P3T_TRY(upload_clusters(c, s));
    for (int attempt = 0; attempt < 8; ++attempt) {
        P3T_TRY(clear_error(c, s));
        int slot = p3t_prof_open(c, P3T_PH_BUILD, s);
        int rc = p3t_build_levels(c, (int)n, s, pos, mass);
        p3t_prof_close(c, slot, s);
        P3T_TRY(rc);
        if (no_sync) {
            // errors (a cell capacity overflow included) latch on the device
            c->built = 1;
            return P3T_OK;
        }
        P3T_TRY(sync_state(c, s));
        if (c->hst->error == 0) {
            // leave room for later builds that may not allocate
            c->need_cells = c->hst->ncell;
            int64_t want = c->hst->ncell + c->hst->ncell / 2 + 64;
            if (c->lim_cells > 0 && want > c->lim_cells) want = c->lim_cells;
            if (want > c->cap_cells) P3T_TRY(ensure_cells_keep(c, want));
            c->built = 1;
            return P3T_OK;
        }
        if (c->hst->error != P3T_ERR_CAPACITY) {  // returned once, then cleared
            const int e = c->hst->error;
            P3T_TRY(clear_error(c, s));
            return e;
        }
        c->need_cells = c->hst->need_cells;
        int64_t want = 2 * c->cap_cells;
        if (c->hst->need_cells > want) want = c->hst->need_cells;
        if (c->lim_cells > 0 && want > c->lim_cells) {
            if (c->cap_cells >= c->lim_cells) {
                P3T_TRY(clear_error(c, s));
                return P3T_ERR_CAPACITY;
            }
            want = c->lim_cells;
        }
        P3T_TRY(ensure_cells(c, want));
    }
    return P3T_ERR_CAPACITY;
}

int p3t_set_ensemble(p3t_ctx *c, int32_t n_clusters, const int64_t *off,
                     const double *r_out, const double *eps, const double *h)
{
    if (!c || n_clusters < 0) return P3T_ERR_INVALID;
    c->n_bh = 0;
    if (n_clusters == 0) {
        c->ensemble = 0;
        c->built = 0;
        return P3T_OK;
    }
    if (!off || off[0] != 0) return P3T_ERR_INVALID;
    for (int k = 0; k < n_clusters; ++k) {
        if (off[k + 1] <= off[k]) return P3T_ERR_INVALID;
        if (r_out && !(r_out[k] >= P3T_R_OUT_MIN && isfinite(r_out[k]))) return P3T_ERR_INVALID;
        if (eps && !(eps[k] >= 0.0 && isfinite(eps[k]))) return P3T_ERR_INVALID;
        if (h && !(h[k] >= 0.0 && isfinite(h[k]))) return P3T_ERR_INVALID;
    }
    if (off[n_clusters] > 0x7fffff00LL) return P3T_ERR_INVALID;
    P3T_TRY(ensure_clusters(c, n_clusters));
    c->nclus = n_clusters;
    for (int k = 0; k <= n_clusters; ++k) c->clus_off_h[k] = off[k];
    for (int k = 0; k < n_clusters; ++k) {
        c->clus_par[k] = r_out ? r_out[k] : 0.0;
        c->clus_par[c->cap_clus + k] = eps ? eps[k] : -1.0;
        c->clus_par[2 * c->cap_clus + k] = h ? h[k] : 0.0;
    }
    c->ensemble = 1;
    c->built = 0;
    return P3T_OK;
}

int p3t_set_species(p3t_ctx *c, int64_t n, int64_t n_bh, const p3t_species *sp)
{
    if (!c || n_bh < 0) return P3T_ERR_INVALID;
    if (n_bh == 0) return p3t_set_ensemble(c, 0, nullptr, nullptr, nullptr, nullptr);
    if (!sp || n_bh > 32 || n_bh >= n || n > 0x7fffff00LL) return P3T_ERR_INVALID;
    if (!(sp->r_cut_bh >= P3T_R_OUT_MIN) || !isfinite(sp->r_cut_bh) ||
        !(sp->eps_bh >= 0.0) || !isfinite(sp->eps_bh) || !(sp->h_bh >= 0.0) ||
        !isfinite(sp->h_bh) || !(sp->eta_bh > 0.0) || !isfinite(sp->eta_bh))
        return P3T_ERR_INVALID;
    // two clusters: the stars with the context's r_out, eps and h (the
    // per-cluster values 0, -1, 0 select them), the black holes with K = 0
    // (r_out 1e10) and a neighbour radius that admits no pair (its square
    // underflows to 0): the black hole-star pairs and the black hole pairs
    // are added by the species kernels
    P3T_TRY(ensure_clusters(c, 2));
    c->nclus = 2;
    c->clus_off_h[0] = 0;
    c->clus_off_h[1] = n - n_bh;
    c->clus_off_h[2] = n;
    c->clus_par[0] = 0.0;
    c->clus_par[1] = 1e10;
    c->clus_par[c->cap_clus + 0] = -1.0;
    c->clus_par[c->cap_clus + 1] = 0.0;
    c->clus_par[2 * c->cap_clus + 0] = 0.0;
    c->clus_par[2 * c->cap_clus + 1] = 1e-300;
    const int64_t nblk = (n - n_bh + 255) / 256;
    int64_t d = 0;
    P3T_TRY(grow(c->sp_off, d, n + 1, sizeof(long long)));
    P3T_TRY(grow(c->sp_inv, d, n, sizeof(int)));
    P3T_TRY(grow(c->sp_bh, d, 32 + nblk * n_bh, sizeof(int)));
    P3T_TRY(grow(c->sp_part, d, 4 * nblk * n_bh, sizeof(double)));
    c->ensemble = 1;
    c->built = 0;
    c->n_bh = n_bh;
    c->sp = *sp;
    return P3T_OK;
}

int p3t_long_force(p3t_ctx *c, float *acc, double *pot, void *stream)
{
    if (!c) return P3T_ERR_INVALID;
    if (!c->built) return P3T_ERR_STATE;
    if (c->n == 0) return P3T_OK;
    if (!acc) return P3T_ERR_INVALID;
    cudaStream_t s = (cudaStream_t)stream;
    int slot = p3t_prof_open(c, P3T_PH_FORCE, s);
    int rc = p3t_run_force(c, acc, pot, s);
    p3t_prof_close(c, slot, s);
    return rc;
}

int p3t_set_limits(p3t_ctx *c, const p3t_limits *l)
{
    if (!c) return P3T_ERR_INVALID;
    c->lim_walk = (l && l->walk_iters > 0) ? l->walk_iters : P3T_LIM_WALK;
    c->lim_uf = (l && l->uf_rounds > 0) ? l->uf_rounds : P3T_LIM_UF;
    c->lim_block = (l && l->block_steps > 0) ? l->block_steps : P3T_LIM_BLOCK;
    c->lim_cells = (l && l->max_cells > 0) ? l->max_cells : 0;
    return P3T_OK;
}

int p3t_force_lists(p3t_ctx *c, float *acc, int64_t *rec, int64_t cap,
                    int64_t *count, void *stream)
{
    if (!c || !count || cap < 1 || !rec) return P3T_ERR_INVALID;
    if (!c->built) return P3T_ERR_STATE;
    *count = 0;
    if (c->n == 0) return P3T_OK;
    if (!acc) return P3T_ERR_INVALID;
    cudaStream_t s = (cudaStream_t)stream;
    P3T_TRY(p3t_run_force(c, acc, nullptr, s, (long long *)rec, cap));
    P3T_TRY(sync_state(c, s));
    if (c->hst->error) {
        const int e = c->hst->error;
        P3T_TRY(clear_error(c, s));
        return e;
    }
    *count = c->hst->rec_n;
    return *count > cap ? P3T_ERR_CAPACITY : P3T_OK;
}

int p3t_long_force_vjp(p3t_ctx *c, const float *w, double *grad_pos,
                       double *grad_mass, void *stream)
{
    if (!c) return P3T_ERR_INVALID;
    if (!c->built) return P3T_ERR_STATE;
    if (c->n == 0) return P3T_OK;
    if (!w || !grad_pos || !grad_mass) return P3T_ERR_INVALID;
    if (c->n_bh > 0) return P3T_ERR_STATE;  // no gradient of the species terms
    const int64_t need = 10 * (int64_t)c->cap_cells;
    if (need > c->cap_cadj) {
        if (c->p.flags & P3T_FLAG_NO_SYNC) return P3T_ERR_CAPACITY;
        int64_t d = 0;
        P3T_TRY(grow(c->cadj, d, need + need / 4, sizeof(double)));
        c->cap_cadj = need + need / 4;
    }
    cudaStream_t s = (cudaStream_t)stream;
    int slot = p3t_prof_open(c, P3T_PH_WALK, s);
    int rc = p3t_run_vjp(c, w, grad_pos, grad_mass, c->cadj, s);
    p3t_prof_close(c, slot, s);
    return rc;
}

int ensure_hermite(p3t_ctx *c, int64_t n)
{
    if (n > c->cap_herm) {
        if (c->p.flags & P3T_FLAG_NO_SYNC) return P3T_ERR_CAPACITY;
        const int64_t cap = n + n / 8 + 1024;
        int64_t d = 0;
        P3T_TRY(grow(c->hparent, d, cap, sizeof(int)));
        P3T_TRY(grow(c->hcsize, d, cap, sizeof(int)));
        P3T_TRY(grow(c->hcfill, d, cap, sizeof(int)));
        P3T_TRY(grow(c->hmember, d, cap, sizeof(int)));
        P3T_TRY(grow(c->hlev, d, cap, sizeof(int)));
        P3T_TRY(grow(c->hcstart, d, cap + 1, sizeof(long long)));
        P3T_TRY(grow(c->hroots, d, cap, sizeof(int)));
        P3T_TRY(grow(c->hloc, d, cap, sizeof(int)));
        P3T_TRY(grow(c->hbucket, d, P3T_HERM_BUCKET_LL, sizeof(long long)));
        P3T_TRY(grow(c->ht, d, cap, sizeof(long long)));
        P3T_TRY(grow(c->ha, d, 3 * cap, sizeof(double)));
        P3T_TRY(grow(c->hj, d, 3 * cap, sizeof(double)));
        P3T_TRY(grow(c->hxp, d, 3 * cap, sizeof(double)));
        P3T_TRY(grow(c->hvp, d, 3 * cap, sizeof(double)));
        P3T_TRY(p3t_hard_setup(c));
        c->cap_herm = cap;
    }
    const int64_t nb = p3t_scan_blocks(n) + 2;
    if (nb > c->cap_scan) {
        if (c->p.flags & P3T_FLAG_NO_SYNC) return P3T_ERR_CAPACITY;
        int64_t d = 0;
        P3T_TRY(grow(c->scan_part, d, nb, sizeof(long long)));
        c->cap_scan = nb;
    }
    return P3T_OK;
}

int p3t_hard_step(p3t_ctx *c, int64_t n, double *pos, double *vel,
                  const double *mass, const int64_t *offsets,
                  const int32_t *idx, const p3t_hermite_params *hp,
                  void *stream)
{
    if (!c || !hp || n < 0 || n > INT32_MAX - 1) return P3T_ERR_INVALID;
    // an ensemble layout only as the two species, with their n
    if (c->ensemble && (c->n_bh == 0 || n != c->clus_off_h[c->nclus]))
        return P3T_ERR_INVALID;
    if (n > 0 && (!pos || !vel || !mass || !offsets || !idx))
        return P3T_ERR_INVALID;
    if (!(hp->eta > 0.0) || !isfinite(hp->eta) || !(hp->alpha >= 0.0) ||
        !isfinite(hp->alpha) || !(hp->dt_soft > 0.0) || !isfinite(hp->dt_soft) ||
        hp->log2_soft_over_max < 0 || hp->log2_soft_over_max > 30 ||
        hp->kmax < 1 || hp->log2_soft_over_max + hp->kmax > 58)
        return P3T_ERR_INVALID;
    // the tick dt_soft 2^-(p + kmax) and 1 / dt_max stay normal, so that
    // steps and their inverses are exact power-of-two scalings
    if (!(ldexp(hp->dt_soft, -(hp->log2_soft_over_max + hp->kmax)) >= DBL_MIN) ||
        !(hp->dt_soft <= 1e300))
        return P3T_ERR_INVALID;
    if (n == 0) return P3T_OK;
    P3T_TRY(ensure_hermite(c, n));
    return p3t_run_hard_step(c, (int)n, pos, vel, mass,
                             (const long long *)offsets, idx, hp,
                             (cudaStream_t)stream);
}

int p3t_check(p3t_ctx *c, void *stream)
{
    if (!c) return P3T_ERR_INVALID;
    cudaStream_t s = (cudaStream_t)stream;
    P3T_TRY(sync_state(c, s));
    int e = c->hst->error;
    if (e) P3T_TRY(clear_error(c, s));
    return e;
}

int p3t_neighbours(p3t_ctx *c, int64_t *offsets, int32_t *idx, int64_t cap,
                   int64_t *needed, void *stream)
{
    if (!c || !offsets || cap < 0 || (cap > 0 && !idx)) return P3T_ERR_INVALID;
    if (!c->built) return P3T_ERR_STATE;
    cudaStream_t s = (cudaStream_t)stream;
    const int n = (int)c->n;
    if (n == 0) {
        P3T_CUDA_TRY(cudaMemsetAsync(offsets, 0, sizeof(int64_t), s));
        if (needed) *needed = 0;
        return P3T_OK;
    }
    int slot = p3t_prof_open(c, P3T_PH_NGB, s);
    if (c->n_bh > 0) {
        long long nnz = 0;
        int rc = p3t_run_ngb_species(c, (long long *)offsets, idx, cap,
                                     needed ? &nnz : nullptr, s);
        p3t_prof_close(c, slot, s);
        if (needed) {
            *needed = nnz;
            if (rc == P3T_OK) {
                rc = sync_state(c, s);
                if (rc == P3T_OK && c->hst->error) {
                    rc = c->hst->error;
                    clear_error(c, s);
                }
            }
        }
        return rc;
    }
    int rc = p3t_run_ngb(c, 0, nullptr, nullptr, 0, s);
    if (rc == P3T_OK)
        rc = p3t_scan_ll(c, c->ngb_cnt, (long long *)offsets, n, s);
    if (rc == P3T_OK && needed) {
        long long nnz = 0;
        if (cudaMemcpyAsync(&nnz, offsets + n, sizeof(long long),
                            cudaMemcpyDeviceToHost, s) != cudaSuccess ||
            cudaStreamSynchronize(s) != cudaSuccess)
            rc = P3T_ERR_CUDA;
        *needed = nnz;
        c->hst->nnz = nnz;
        if (rc == P3T_OK && nnz > cap) rc = P3T_ERR_CAPACITY;
    }
    if (rc == P3T_OK)
        rc = p3t_run_ngb(c, 1, (const long long *)offsets, idx, cap, s);
    p3t_prof_close(c, slot, s);
    if (rc == P3T_OK && needed) {
        long long nnz = c->hst->nnz;
        rc = sync_state(c, s);
        c->hst->nnz = nnz;
        if (rc == P3T_OK && c->hst->error) {
            rc = c->hst->error;
            clear_error(c, s);
        }
    }
    return rc;
}

int p3t_energy(p3t_ctx *c, int64_t n, const double *mass, const double *vel,
               const double *pot, double *out, void *stream)
{
    if (!c || n < 0 || !out || (n > 0 && (!mass || !vel)))
        return P3T_ERR_INVALID;
    cudaStream_t s = (cudaStream_t)stream;
    if (n == 0) {
        P3T_CUDA_TRY(cudaMemsetAsync(out, 0, 2 * sizeof(double), s));
        return P3T_OK;
    }
    return p3t_energy_launch(c, (long long)n, mass, vel, pot, out, s);
}

int p3t_get_stats(p3t_ctx *c, p3t_stats *o)
{
    if (!c || !o) return P3T_ERR_INVALID;
    if (cudaDeviceSynchronize() != cudaSuccess) return P3T_ERR_CUDA;
    long long nnz = c->hst->nnz;
    P3T_CUDA_TRY(cudaMemcpy(c->hst, c->st, sizeof(P3TDevState),
                            cudaMemcpyDeviceToHost));
    c->hst->nnz = nnz;
    memset(o, 0, sizeof(*o));
    o->n = c->n;
    o->herm_block_steps = c->hst->herm[0];
    o->herm_particle_steps = c->hst->herm[1];
    o->herm_pairs = c->hst->herm[2];
    o->herm_capped = c->hst->herm[3];
    o->herm_components = c->hst->herm[4];
    o->herm_max_component = c->hst->herm[5];
    o->herm_max_block_steps = c->hst->herm[6];
    if (c->n == 0) return P3T_OK;
    o->need_cells = c->need_cells;
    o->n_cells = c->hst->ncell;
    o->n_groups = c->hst->ngroup;
    o->n_levels = c->hst->max_level + 1;
    o->list_pc = c->hst->tot[0];
    o->list_pp_near = c->hst->tot[1];
    o->list_pp_far = c->hst->tot[2];
    o->int_pc = c->hst->int_pc;
    o->int_pp = c->hst->int_pp;
    o->int_pp_near = c->hst->int_ppn;
    o->max_walk_stack = c->hst->max_stack;
    o->nnz = nnz;
    return P3T_OK;
}

int p3t_get_order(p3t_ctx *c, uint64_t *key, int32_t *order)
{
    if (!c || !c->built) return P3T_ERR_STATE;
    size_t n = (size_t)c->n;
    if (n == 0) return P3T_OK;
    if (key)
        P3T_CUDA_TRY(cudaMemcpy(key, c->key_a, n * 8, cudaMemcpyDeviceToHost));
    if (order)
        P3T_CUDA_TRY(cudaMemcpy(order, c->order, n * 4, cudaMemcpyDeviceToHost));
    return P3T_OK;
}

int p3t_get_root(p3t_ctx *c, double *lo, double *size)
{
    if (!c || !c->built) return P3T_ERR_STATE;
    P3T_CUDA_TRY(cudaDeviceSynchronize());
    P3T_CUDA_TRY(cudaMemcpy(c->hst, c->st, sizeof(P3TDevState),
                            cudaMemcpyDeviceToHost));
    if (lo)
        for (int a = 0; a < 3; ++a) lo[a] = c->hst->lo[a];
    if (size) *size = c->hst->size;
    return P3T_OK;
}

int p3t_get_cells(p3t_ctx *c, int32_t *level, int32_t *first, int32_t *count,
                  int32_t *child, int32_t *nchild, double *M, double *com,
                  double *Q, float *fmin, float *fmax)
{
    if (!c || !c->built) return P3T_ERR_STATE;
    const size_t C = c->n ? (size_t)c->hst->ncell : 0;
    if (C == 0) return P3T_OK;
    int4 *node = (int4 *)malloc(C * sizeof(int4));
    float4 *a = (float4 *)malloc(C * sizeof(float4));
    float4 *b = (float4 *)malloc(C * sizeof(float4));
    if (!node || !a || !b) {
        free(node); free(a); free(b);
        return P3T_ERR_CUDA;
    }
    int rc = P3T_OK;
    if (cudaMemcpy(node, c->node, C * sizeof(int4), cudaMemcpyDeviceToHost) != cudaSuccess ||
        cudaMemcpy(a, c->wmin, C * sizeof(float4), cudaMemcpyDeviceToHost) != cudaSuccess ||
        cudaMemcpy(b, c->wmax, C * sizeof(float4), cudaMemcpyDeviceToHost) != cudaSuccess ||
        (M && cudaMemcpy(M, c->cM, C * 8, cudaMemcpyDeviceToHost) != cudaSuccess) ||
        (com && cudaMemcpy(com, c->ccom, 3 * C * 8, cudaMemcpyDeviceToHost) != cudaSuccess) ||
        (Q && cudaMemcpy(Q, c->cQ, 6 * C * 8, cudaMemcpyDeviceToHost) != cudaSuccess))
        rc = P3T_ERR_CUDA;
    if (rc == P3T_OK)
        for (size_t k = 0; k < C; ++k) {
            if (level) level[k] = node[k].w >> 8;
            if (first) first[k] = node[k].x;
            if (count) count[k] = node[k].y;
            if (child) child[k] = node[k].z;
            if (nchild) nchild[k] = node[k].w & 255;
            if (fmin) {
                fmin[3 * k] = a[k].x; fmin[3 * k + 1] = a[k].y; fmin[3 * k + 2] = a[k].z;
            }
            if (fmax) {
                fmax[3 * k] = b[k].x; fmax[3 * k + 1] = b[k].y; fmax[3 * k + 2] = b[k].z;
            }
        }
    free(node);
    free(a);
    free(b);
    return rc;
}

int p3t_get_groups(p3t_ctx *c, int32_t *first, int32_t *count, float *fmin,
                   float *fmax)
{
    if (!c || !c->built) return P3T_ERR_STATE;
    const size_t G = c->n ? (size_t)c->hst->ngroup : 0;
    if (G == 0) return P3T_OK;
    int2 *r = (int2 *)malloc(G * sizeof(int2));
    float4 *a = (float4 *)malloc(G * sizeof(float4));
    float4 *b = (float4 *)malloc(G * sizeof(float4));
    int rc = P3T_OK;
    if (!r || !a || !b ||
        cudaMemcpy(r, c->grange, G * sizeof(int2), cudaMemcpyDeviceToHost) != cudaSuccess ||
        cudaMemcpy(a, c->gmin, G * sizeof(float4), cudaMemcpyDeviceToHost) != cudaSuccess ||
        cudaMemcpy(b, c->gmax, G * sizeof(float4), cudaMemcpyDeviceToHost) != cudaSuccess)
        rc = P3T_ERR_CUDA;
    if (rc == P3T_OK)
        for (size_t g = 0; g < G; ++g) {
            if (first) first[g] = r[g].x;
            if (count) count[g] = r[g].y;
            if (fmin) { fmin[3 * g] = a[g].x; fmin[3 * g + 1] = a[g].y; fmin[3 * g + 2] = a[g].z; }
            if (fmax) { fmax[3 * g] = b[g].x; fmax[3 * g + 1] = b[g].y; fmax[3 * g + 2] = b[g].z; }
        }
    free(r);
    free(a);
    free(b);
    return rc;
}

int p3t_get_lists(p3t_ctx *c, int64_t *pc_off, int32_t *pc, int64_t *ppn_off,
                  int32_t *ppn, int64_t *ppf_off, int32_t *ppf)
{
    if (!c || !c->built) return P3T_ERR_STATE;
    const size_t G = c->n ? (size_t)c->hst->ngroup : 0;
    if (G == 0) return P3T_OK;
    if (!c->lists_valid) {
        cudaStream_t s = 0;
        P3T_TRY(clear_error(c, s));
        P3T_TRY(p3t_run_walk(c, 0, s));
        P3T_TRY(p3t_scan_lists(c, s));
        P3T_TRY(sync_state(c, s));
        if (c->hst->error) {  // returned once, then cleared
            const int e = c->hst->error;
            P3T_TRY(clear_error(c, s));
            return e;
        }
        for (int L = 0; L < 3; ++L) {
            P3T_TRY(ensure_list(c, L, c->hst->tot[L]));
            c->list_tot[L] = c->hst->tot[L];
        }
        P3T_TRY(p3t_run_walk(c, 1, s));
        P3T_CUDA_TRY(cudaStreamSynchronize(s));
        c->lists_valid = 1;
    }
    int64_t *offs[3] = {pc_off, ppn_off, ppf_off};
    int32_t *lists[3] = {pc, ppn, ppf};
    for (int L = 0; L < 3; ++L) {
        int64_t *o = offs[L];
        int64_t tot = c->list_tot[L];
        if (o)
            P3T_CUDA_TRY(cudaMemcpy(o, c->loff + (size_t)L * (G + 1),
                                    (G + 1) * 8, cudaMemcpyDeviceToHost));
        if (lists[L] && tot > 0)
            P3T_CUDA_TRY(cudaMemcpy(lists[L], c->list[L], (size_t)tot * 4,
                                    cudaMemcpyDeviceToHost));
    }
    return P3T_OK;
}

int p3t_profile_enable(p3t_ctx *c, int on)
{
    if (!c) return P3T_ERR_INVALID;
    c->prof_on = on ? 1 : 0;
    return P3T_OK;
}

int p3t_get_profile(p3t_ctx *c, p3t_profile *o, int reset)
{
    if (!c || !o) return P3T_ERR_INVALID;
    int rc = prof_resolve(c);
    if (rc) return rc;
    o->build_ms = c->prof_ms[P3T_PH_BUILD];
    o->walk_ms = c->prof_ms[P3T_PH_WALK];
    o->force_ms = c->prof_ms[P3T_PH_FORCE];
    o->ngb_ms = c->prof_ms[P3T_PH_NGB];
    o->builds = c->prof_calls[P3T_PH_BUILD];
    o->walks = c->prof_calls[P3T_PH_WALK];
    o->forces = c->prof_calls[P3T_PH_FORCE];
    o->ngbs = c->prof_calls[P3T_PH_NGB];
    o->vjp_walk_ms = c->prof_ms[P3T_PH_VJPWALK];
    o->build_keys_ms = c->prof_ms[P3T_PH_B_KEYS];
    o->build_sort_ms = c->prof_ms[P3T_PH_B_SORT];
    o->build_split_ms = c->prof_ms[P3T_PH_B_SPLIT];
    o->build_moments_ms = c->prof_ms[P3T_PH_B_MOMENTS];
    o->build_groups_ms = c->prof_ms[P3T_PH_B_GROUPS];
    o->vjp_walks = c->prof_calls[P3T_PH_VJPWALK];
    if (c->built && c->n > 0) {
        long long cum[3];
        P3T_CUDA_TRY(cudaMemcpy(cum, c->st->cum_int, sizeof(cum),
                                cudaMemcpyDeviceToHost));
        o->int_pc = cum[0];
        o->int_pp = cum[1];
        o->int_pp_near = cum[2];
        if (reset)
            P3T_CUDA_TRY(cudaMemset(c->st->cum_int, 0, sizeof(cum)));
    } else {
        o->int_pc = o->int_pp = o->int_pp_near = 0;
    }
    if (reset) {
        for (int k = 0; k < P3T_NPH; ++k) {
            c->prof_ms[k] = 0.0;
            c->prof_calls[k] = 0;
        }
    }
    return P3T_OK;
}

int64_t p3t_launch_count(void) { return g_launches.load(); }

const char *p3t_status_string(int s)
{
    switch (s) {
    case P3T_OK: return "ok";
    case P3T_ERR_INVALID: return "invalid argument or input";
    case P3T_ERR_CAPACITY: return "capacity exceeded";
    case P3T_ERR_CUDA: return "CUDA error";
    case P3T_ERR_TIMEOUT: return "device wait timed out";
    case P3T_ERR_STATE: return "call out of order";
    default: return "unknown status";
    }
}

}  // extern "C"

// ---- autotuning of the group and leaf sizes --------------------------------
// One timed configuration of the autotuner: the best of `reps` runs of
// build + force (+ backward with weights w), after one untimed run that
// sizes every buffer.
static int tune_time(p3t_ctx *c, int64_t n, const double *pos,
                     const double *mass, const float *w, float *acc,
                     double *gpos, double *gmass, int reps, void *stream,
                     cudaEvent_t e0, cudaEvent_t e1, double *ms)
{
    cudaStream_t s = (cudaStream_t)stream;
    *ms = 1e300;
    for (int r = -1; r < reps; ++r) {
        if (r >= 0) cudaEventRecord(e0, s);
        P3T_TRY(p3t_build_tree(c, n, pos, mass, stream));
        P3T_TRY(p3t_long_force(c, acc, nullptr, stream));
        if (w) P3T_TRY(p3t_long_force_vjp(c, w, gpos, gmass, stream));
        if (r < 0) {
            P3T_TRY(p3t_check(c, stream));
            continue;
        }
        cudaEventRecord(e1, s);
        if (cudaEventSynchronize(e1) != cudaSuccess) return P3T_ERR_CUDA;
        float t = 0.f;
        cudaEventElapsedTime(&t, e0, e1);
        if (t < *ms) *ms = t;
    }
    return p3t_check(c, stream);
}

extern "C" int p3t_autotune(p3t_ctx *c, int64_t n, const double *pos,
                            const double *mass, const float *w, int reps,
                            void *stream, p3t_tune *out)
{
    if (!c || n <= 0 || !pos || !mass || reps < 1 || !out) return P3T_ERR_INVALID;
    if (c->p.flags & P3T_FLAG_NO_SYNC) return P3T_ERR_STATE;
    if (w && c->n_bh > 0) return P3T_ERR_STATE;  // no backward with species
    cudaStream_t s = (cudaStream_t)stream;
    static const int groups[] = {32, 48, 64};
    static const int leaves[] = {8, 16, 32};
    static const int fwarps[] = {2, 4, 8};
    static const int vwarps[] = {2, 4};
    const p3t_params keep = c->p;
    const int keep_fw = c->force_warps, keep_vw = c->vjp_warps;
    memset(out, 0, sizeof(*out));
    float *acc = nullptr, *ref = nullptr;
    double *gpos = nullptr, *gmass = nullptr;
    void *scr = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    int rc = P3T_OK;
    if (cudaMalloc(&acc, sizeof(float) * 3 * n) != cudaSuccess ||
        cudaMalloc(&ref, sizeof(float) * 3 * n) != cudaSuccess ||
        (w && cudaMalloc(&gpos, sizeof(double) * 3 * n) != cudaSuccess) ||
        (w && cudaMalloc(&gmass, sizeof(double) * n) != cudaSuccess) ||
        cudaMalloc(&scr, p3t_force_err_scratch(c)) != cudaSuccess ||
        cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)
        rc = P3T_ERR_CUDA;
    // reference: the starting configuration at half the opening angle
    if (rc == P3T_OK) {
        c->p.theta = 0.5 * keep.theta;
        rc = p3t_build_tree(c, n, pos, mass, stream);
        if (rc == P3T_OK) rc = p3t_long_force(c, ref, nullptr, stream);
        if (rc == P3T_OK) rc = p3t_check(c, stream);
        c->p = keep;
    }
    double base_med = 0.0, base_max = 0.0, best = 1e300;
    int bg = keep.n_group, bl = keep.n_leaf;
    double best_med = 0.0, best_max = 0.0;
    for (int gi = 0; gi < 3 && rc == P3T_OK; ++gi)
        for (int li = 0; li < 3 && rc == P3T_OK; ++li) {
            c->p.n_group = groups[gi];
            c->p.n_leaf = leaves[li];
            double t = 0.0, med = 0.0, mx = 0.0;
            rc = tune_time(c, n, pos, mass, w, acc, gpos, gmass, reps, stream, e0,
                           e1, &t);
            if (rc == P3T_OK) rc = p3t_force_err(c, n, acc, ref, scr, &med, &mx, s);
            if (rc != P3T_OK) break;
            ++out->evaluated;
            if (groups[gi] == keep.n_group && leaves[li] == keep.n_leaf) {
                base_med = med;
                base_max = mx;
            }
            out->cand_ms[gi * 3 + li] = t;
            out->cand_err_median[gi * 3 + li] = med;
            out->cand_err_max[gi * 3 + li] = mx;
        }
    // the accuracy check: no worse than the starting configuration by more
    // than the stated factors (the starting configuration always passes)
    for (int q = 0; q < 9 && rc == P3T_OK; ++q) {
        const bool start = groups[q / 3] == keep.n_group && leaves[q % 3] == keep.n_leaf;
        const bool ok = start || (out->cand_err_median[q] <= P3T_TUNE_MEDIAN_FACTOR * base_med &&
                                  out->cand_err_max[q] <= P3T_TUNE_MAX_FACTOR * base_max);
        if (!ok) {
            ++out->rejected;
            continue;
        }
        if (out->cand_ms[q] < best) {
            best = out->cand_ms[q];
            bg = groups[q / 3];
            bl = leaves[q % 3];
            best_med = out->cand_err_median[q];
            best_max = out->cand_err_max[q];
        }
    }
    // block shapes of the walk kernels for the chosen sizes (they change no
    // arithmetic, so no accuracy check)
    int bfw = keep_fw ? keep_fw : 4, bvw = keep_vw ? keep_vw : 4;
    c->p = keep;
    c->p.n_group = bg;
    c->p.n_leaf = bl;
    for (int fi = 0; fi < 3 && rc == P3T_OK; ++fi)
        for (int vi = 0; vi < (w ? 2 : 1) && rc == P3T_OK; ++vi) {
            c->force_warps = fwarps[fi];
            c->vjp_warps = w ? vwarps[vi] : bvw;
            double t = 0.0;
            rc = tune_time(c, n, pos, mass, w, acc, gpos, gmass, reps, stream, e0,
                           e1, &t);
            if (rc != P3T_OK) break;
            ++out->evaluated;
            if (t < best) {
                best = t;
                bfw = c->force_warps;
                bvw = c->vjp_warps;
            }
        }
    c->force_warps = rc == P3T_OK ? bfw : keep_fw;
    c->vjp_warps = rc == P3T_OK ? bvw : keep_vw;
    if (rc != P3T_OK) {
        c->p = keep;
    } else {
        out->n_group = bg;
        out->n_leaf = bl;
        out->force_warps = bfw;
        out->vjp_warps = bvw;
        out->ms = best;
        out->err_median = best_med;
        out->err_max = best_max;
        out->base_err_median = base_med;
        out->base_err_max = base_max;
        rc = p3t_build_tree(c, n, pos, mass, stream);
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFree(acc);
    cudaFree(ref);
    cudaFree(gpos);
    cudaFree(gmass);
    cudaFree(scr);
    return rc;
}
