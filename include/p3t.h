/*
 * p3t.h -- C ABI of libp3t, the tree side of the P3T (particle-particle
 * particle-tree) scheme of Iwasawa, Portegies Zwart & Makino,
 * arXiv:1506.04553, on one NVIDIA B300 (sm_103a).
 *
 * The library evaluates the long-range ("soft") gravitational acceleration
 *     a_soft,i = -sum_{j != i} G m_j K(s_ij) q_ij / s_ij^3          (Eq. 8)
 * with q_ij = q_i - q_j and s_ij = sqrt(|q_ij|^2 + eps^2)            (Eq. 2-3)
 * and the cut-off function K(x) of Eq. 12-15, by a Barnes-Hut octree to
 * quadrupole order, and gives every particle its list of neighbours within a
 * radius h, the two products the GPU tree library hands to the host-side
 * Hermite part in Sect. 2.2.  It also provides the velocity kick and drift of
 * the second-order splitting of Eq. 11 and of the step procedure of
 * Sect. 2.2.
 *
 * Conventions for every entry point:
 *   - Every function returns an int status (P3T_OK or a P3T_ERR_* code).
 *   - Particle arrays are DEVICE pointers in the caller's particle order.
 *     Three-vectors are structure-of-arrays: x[0..n), y[0..n), z[0..n)
 *     contiguous (a (3, n) row-major array).
 *   - The caller owns every pointer it passes; the context owns the tree,
 *     the interaction lists and all other scratch.  Nothing the caller passes
 *     is retained after a call returns (build_tree copies what it needs).
 *   - `stream` is a cudaStream_t (NULL = legacy default stream).  All device
 *     work of a call is issued on that stream.
 *   - A context belongs to one device (the current device at p3t_create) and
 *     must not be used by two host threads at once.
 */
#ifndef P3T_H
#define P3T_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ---- */
#define P3T_OK 0
#define P3T_ERR_INVALID 1  /* bad parameter, n < 0, NULL pointer, NaN/Inf
                              coordinate, non-positive or non-finite mass */
#define P3T_ERR_CAPACITY 2 /* caller buffer too small; *needed says how big */
#define P3T_ERR_CUDA 3     /* a CUDA runtime call failed */
#define P3T_ERR_TIMEOUT 4  /* a bounded device-side wait expired */
#define P3T_ERR_STATE 5    /* call out of order (e.g. force before build) */

/* ---- flags ---- */
/* p3t_build_tree neither allocates nor synchronises; capacities must have
 * been sized by an earlier build without the flag (which keeps 50% headroom
 * of cells), and a capacity overflow latches P3T_ERR_CAPACITY on the device
 * (p3t_check).  With it every call of a step only enqueues work on the
 * stream, so the step can be captured into a CUDA graph. */
#define P3T_FLAG_NO_SYNC 1

typedef struct p3t_ctx p3t_ctx;

/* Parameters.  Names follow the paper: r_out is r_cut of Eq. 12-15 and
 * Table 1, gamma = r_in / r_cut (Eq. 15; 0.1 in every run of the paper),
 * eps the Plummer softening of Eq. 2, theta the opening criterion of
 * Table 1, h the neighbour radius of Sect. 2.2 (h = r_cut + dr_buff). */
/* Smallest accepted r_out.  Every source evaluated without the cut-off
 * lies at least r_out away, so its squared distance is a normal FP32 number
 * (the force kernel's reciprocal square root flushes subnormal inputs). */
#define P3T_R_OUT_MIN 1e-15

typedef struct p3t_params {
    double theta;    /* opening parameter, >= 0 (0 = direct summation) */
    double r_out;    /* outer cut-off radius r_cut, >= P3T_R_OUT_MIN */
    double gamma;    /* r_in / r_cut, in [0, 1) */
    double eps;      /* Plummer softening, >= 0 */
    double h;        /* neighbour radius, >= 0; 0 means h = r_out */
    double G;        /* gravitational constant, > 0 */
    int32_t n_leaf;  /* a cell with more than n_leaf particles is split
                        (1..64; default 16) */
    int32_t n_group; /* particles sharing one interaction list (1..64;
                        default 64) */
    int32_t flags;   /* P3T_FLAG_* */
    int32_t reserved;
} p3t_params;

/* Fills *p with the defaults: theta 0.4, r_out 1/64, gamma 0.1, eps 0,
 * h 0 (= r_out), G 1, n_leaf 16, n_group 64, flags 0. */
int p3t_default_params(p3t_params *p);

/* Creates a context on the current device.  *ctx receives the handle.
 * Errors: P3T_ERR_INVALID (NULL or out-of-range parameter). */
int p3t_create(p3t_ctx **ctx, const p3t_params *p);

/* Releases the context and all device memory it owns.  NULL is a no-op. */
int p3t_destroy(p3t_ctx *ctx);

/* Replaces the parameters.  n_leaf / n_group changes take effect at the next
 * p3t_build_tree; the others at the next p3t_long_force. */
int p3t_set_params(p3t_ctx *ctx, const p3t_params *p);

/* Builds the octree (Sect. 2.2: Barnes-Hut tree "up to the quadrupole
 * moment") for n particles.
 *   pos  : device, double[3][n] (SoA), the particle positions q_i
 *   mass : device, double[n], m_i > 0
 * Steps: root cube, 63-bit Morton keys (21 bits per axis), stable radix sort
 * by (key, index), level-wise split of every cell holding more than n_leaf
 * particles, FP64 monopole + traceless quadrupole moments per cell, groups
 * of n_group consecutive particles cut from containers (cells of at most
 * 16 n_group particles whose parent holds more).  The context keeps
 * Morton-ordered copies, so
 * pos and mass may change after the call returns.  n == 0 builds an empty
 * tree.  Synchronises `stream` once at the end (to size later launches).
 * Errors: P3T_ERR_INVALID (n < 0, NULL pointer with n > 0, non-finite
 * coordinate, mass not finite and positive), P3T_ERR_CUDA. */
int p3t_build_tree(p3t_ctx *ctx, int64_t n, const double *pos,
                   const double *mass, void *stream);

/* Ensembles: the particle arrays hold n_clusters independent clusters,
 * cluster k at [off[k], off[k+1]) (host int64, off[0] = 0, every cluster
 * non-empty).  Each cluster gets its own root cube, octree and groups, and
 * interacts only with itself (no forces or neighbours across clusters).
 * r_out, eps, h: host double[n_clusters] per-cluster values, or NULL for the
 * context's parameters.  Applies from the next p3t_build_tree, whose n must
 * be off[n_clusters].  n_clusters = 0 returns to a single cluster.  The
 * paper integrates one cluster; ensembles are a service of the library.
 * Errors: P3T_ERR_INVALID. */
int p3t_set_ensemble(p3t_ctx *ctx, int32_t n_clusters, const int64_t *off,
                     const double *r_out, const double *eps, const double *h);

/* Two species (Sect. 3.2.2): stars and black holes, with a cut-off per kind
 * of pair. */
typedef struct p3t_species {
    double r_cut_bh; /* cut-off of a black hole-star pair (paper: 1/32) */
    double eps_bh;   /* softening of a black hole-star pair (paper: 1e-4) */
    double h_bh;     /* neighbour radius of a black hole-star pair
                        (r_cut_bh + dr_buff), >= 0 */
    double eta_bh;   /* Hermite accuracy parameter of the black holes
                        (paper: 0.03); the stars use p3t_hermite_params.eta */
} p3t_species;

/* The last n_bh of the n particles are black holes (1 <= n_bh <= 32 and
 * n_bh < n; n_bh = 0 switches species off).  Pairs of stars keep the context's r_out, eps and
 * h.  A black hole and a star: r_cut_bh, eps_bh, h_bh.  Two black holes: the
 * force is not split (F_soft = 0, all of it hard), not softened, and they
 * are always neighbours.  Applies from the next p3t_build_tree, whose n must
 * be this n:
 *  - p3t_build_tree: one tree over the stars, one over the black holes;
 *  - p3t_long_force: star pairs by the tree; black hole-star pairs by direct
 *    FP64 summation, added to the result; nothing between black holes (the
 *    potential between black holes is W(s / 1e10) / s, below 3e-10 G m);
 *  - p3t_neighbours: a star's row is its stars by the tree, then the black
 *    holes within h_bh (their indices are the largest, so rows stay
 *    ascending); a black hole's row is the stars within h_bh, then every
 *    other black hole;
 *  - p3t_hard_step: pair constants by pair type; eta and a_0 per species, a
 *    black hole's a_0 = alpha G m / r_cut_bh^2.
 * Replaces any ensemble layout (p3t_set_ensemble replaces it in turn).
 * p3t_long_force_vjp returns P3T_ERR_STATE while species are set.
 * Errors: P3T_ERR_INVALID. */
int p3t_set_species(p3t_ctx *ctx, int64_t n, int64_t n_bh,
                    const p3t_species *sp);

/* Autotuner (a service of the library; the paper has none).  Chooses the
 * group size and leaf size (n_group in {32, 48, 64} x n_leaf in {8, 16, 32})
 * and then the block shape of the walk kernels (warps per block of the
 * walk + force kernel in {2, 4, 8} and, with weights, of the backward kernel
 * in {2, 4}) by timing, on the given particles, the step the workload runs:
 * p3t_build_tree + p3t_long_force, plus p3t_long_force_vjp with the weights
 * w when w is not NULL (device float[3][n]); each configuration the best of
 * `reps` runs after one untimed run.
 * Accuracy check: the reference is the force of the starting configuration
 * at half the opening angle theta / 2 (its tree error is several times
 * smaller).  A (n_group, n_leaf) candidate is kept only if the median and
 * the maximum over particles of |a - a_ref| / max(|a_ref|, 1e-3 rms|a_ref|)
 * are at most P3T_TUNE_MEDIAN_FACTOR and P3T_TUNE_MAX_FACTOR times those of
 * the starting configuration (which is always kept); the block shape changes
 * no arithmetic.  The fastest kept configuration goes into the context (its
 * n_group and n_leaf into the parameters) and the tree is left built with it.
 * Allocates and frees its scratch (3 n floats for the reference and the
 * candidates' forces, 4 n doubles of gradients with w) and synchronises:
 * must not be called with P3T_FLAG_NO_SYNC.
 * Errors: P3T_ERR_INVALID, P3T_ERR_STATE (NO_SYNC; w with species), and
 * those of the timed calls (the context's parameters are then restored). */
#define P3T_TUNE_MEDIAN_FACTOR 1.25
#define P3T_TUNE_MAX_FACTOR 2.0
typedef struct p3t_tune {
    int32_t n_group, n_leaf;   /* chosen sizes */
    int32_t force_warps;       /* chosen warps per block, walk + force */
    int32_t vjp_warps;         /* chosen warps per block, backward */
    double ms;                 /* the chosen configuration's time (ms) */
    double err_median, err_max;          /* its error against the reference */
    double base_err_median, base_err_max; /* the starting configuration's */
    int32_t evaluated;         /* configurations timed */
    int32_t rejected;          /* (n_group, n_leaf) pairs failing the check */
    double cand_ms[9];         /* per pair (n_group index x 3 + n_leaf index) */
    double cand_err_median[9];
    double cand_err_max[9];
} p3t_tune;
int p3t_autotune(p3t_ctx *ctx, int64_t n, const double *pos,
                 const double *mass, const float *w, int reps, void *stream,
                 p3t_tune *out);

/* Long-range acceleration a_soft (Eq. 8) of every particle by the tree.
 *   acc : device, float[3][n] (SoA), written in the caller's order
 *   pot : device, double[n] or NULL; if given, the soft potential
 *         phi_i = -sum_j G m_j W(s_ij / r_cut) / s_ij (Eq. 6, Eq. 16)
 * Each group of particles walks the tree with the opening test (a cell is
 * accepted only when its box is farther than max(h, r_cut) from the group's
 * box and its size is below theta times that distance) and its interactions
 * are evaluated as they are found: cells as softened quadrupoles with K = 1,
 * leaf particles pair by pair with K.  No host synchronisation: errors found
 * by the kernels (P3T_ERR_CAPACITY if a walk stack overflows) are latched on
 * the device and returned by the next p3t_check, p3t_build_tree or
 * synchronising p3t_neighbours call.
 * Errors: P3T_ERR_STATE (no tree), P3T_ERR_INVALID (acc NULL with n > 0),
 * P3T_ERR_CUDA. */
int p3t_long_force(p3t_ctx *ctx, float *acc, double *pot, void *stream);

/* Backward pass of p3t_long_force: for weights w_i (the gradient of a loss
 * with respect to the accelerations), computes dL/dx_i and dL/dm_i of
 * L = sum_i w_i . a_i with the tree topology, the groups and the
 * interaction sets of the current tree held fixed.  The paper has no
 * backward pass; the derivative follows Eq. 8 (pair terms, including dK/ds
 * from Eq. 12-15) and the softened quadrupole cell terms, with the cell
 * moments' dependence on member positions and masses.  The interaction sets
 * are recomputed by the same walk as the forward pass, not stored.
 *   w         : device, float[3][n] (SoA, caller's order)
 *   grad_pos  : device, double[3][n], overwritten
 *   grad_mass : device, double[n], overwritten
 * Uses context-owned scratch (10 doubles per cell).  No host
 * synchronisation; walk-stack overflows latch P3T_ERR_CAPACITY (p3t_check).
 * Errors: P3T_ERR_STATE (no tree), P3T_ERR_INVALID (NULL with n > 0),
 * P3T_ERR_CUDA. */
int p3t_long_force_vjp(p3t_ctx *ctx, const float *w, double *grad_pos,
                       double *grad_mass, void *stream);

/* ---- the hard part (Sect. 2.1-2.2): F_hard over the neighbour lists ----
 *
 * Hard acceleration and jerk of every particle from its neighbour row (the
 * CSR lists of p3t_neighbours: offsets int64[n+1], ascending original
 * indices idx): with q = x_i - x_j, u = v_i - v_j, s^2 = |q|^2 + eps^2
 * (Eq. 2) and the pair weight 1 - K(s) of Eq. 7 (K of Eq. 12-15, r_cut,
 * gamma = r_in / r_cut),
 *   a_i  = -sum_j G m_j (1-K) q / s^3,
 *   da_i = -sum_j G m_j [(1-K)(u - 3 (q.u) q / s^2) / s^3
 *                        - (dK/ds)((q.u)/s) q / s^3].
 * pos, vel: device double[3][n] (SoA, original order); mass device
 * double[n]; acc, jerk: device double[3][n] written.  FP64, one rounding
 * per operation in a fixed order.  Stream-ordered, no synchronisation, no
 * allocation.  Errors: P3T_ERR_INVALID (n < 0, NULL pointers with n > 0,
 * r_cut < P3T_R_OUT_MIN, gamma outside [0, 1), eps < 0, G <= 0). */
int p3t_hard_force(int64_t n, const double *pos, const double *vel,
                   const double *mass, const int64_t *offsets,
                   const int32_t *idx, double G, double eps, double r_cut,
                   double gamma, double *acc, double *jerk, void *stream);

/* Parameters of the Hermite integration of the hard part. */
typedef struct p3t_hermite_params {
    double eta;      /* accuracy parameter of Eq. 18 (Table 1: 0.1);
                        the first step uses eta / 10 (Eq. 20) */
    double alpha;    /* a_0 = alpha G m_i / r_cut^2 (Eq. 19; 0.1) */
    double dt_soft;  /* the soft step: the hard part runs over [0, dt_soft];
                        at most 1e300, and dt_soft 2^-(p + kmax) must be a
                        normal double */
    int32_t log2_soft_over_max; /* p: dt_max = dt_soft 2^-p (Table 1: 2) */
    int32_t kmax;    /* finest level: steps down to dt_max 2^-kmax (1..58-p) */
} p3t_hermite_params;

/* One hard step of the P3T procedure (Sect. 2.2, steps 5 and 6): particles
 * with an empty neighbour row are isolated and drift, x <- x + dt_soft v;
 * every other particle is integrated over dt_soft under H_hard (pair forces
 * of p3t_hard_force over its row, using the context's G, eps, r_out and
 * gamma; with species set, eps and r_out per pair type and eta per species,
 * see p3t_set_species) with the fourth-order Hermite scheme and individual block
 * timesteps (Makino & Aarseth 1992):
 *   - time in integer ticks of dt_max 2^-kmax; a particle at level k steps
 *     dt_max 2^-k and its time is a multiple of its step;
 *   - first levels from Eq. 20 (eta / 10), later from
 *     Eq. 18 with a^(2), a^(3) from the Hermite interpolation and
 *     |a^(1)| |a^(3)| + |a^(2)|^2 as its denominator (the printed
 *     |a^(0)| |a^(3)| is not a time^-2 term beside |a^(2)|^2), both
 *     tested in squares (dt^2 den <= eta^2 num: no division); a
 *     step may at most double and is halved until the current time is a
 *     multiple of it;
 *   - each block step predicts positions and velocities to the next time
 *     (third order), evaluates the particles due then from the predicted
 *     values and corrects them (fourth order).
 * The rows must be symmetric (those of p3t_neighbours are; other rows give
 * undefined positions) and must hold every particle that comes within r_cut
 * during dt_soft (h = r_cut + buffer).  The connected components of the
 * neighbour graph are integrated independently: those of up to 32
 * particles packed into warps, one particle per lane, larger ones one warp
 * each.  pos and vel (device double[3][n]) are updated in place; mass
 * device double[n].  Stream-ordered, no host synchronisation; scratch
 * (about 145 B per particle) is allocated on the
 * first call for a larger n.  Counters in p3t_stats (herm_*).
 * Errors: P3T_ERR_INVALID (arguments, parameters, ensemble layout),
 * P3T_ERR_CUDA; P3T_ERR_TIMEOUT (latched, see p3t_check) when a component
 * needs more than 2^26 block steps or the component search does not
 * settle. */
int p3t_hard_step(p3t_ctx *ctx, int64_t n, double *pos, double *vel,
                  const double *mass, const int64_t *offsets,
                  const int32_t *idx, const p3t_hermite_params *hp,
                  void *stream);

/* Synchronises `stream` and returns (and clears) the first error latched by
 * a kernel of this context since the last check, or P3T_OK. */
int p3t_check(p3t_ctx *ctx, void *stream);

/* Neighbour lists (Sect. 2.2) of the particles of the current tree, in CSR
 * form: the neighbours of particle i are idx[offsets[i] .. offsets[i+1]),
 * ascending original indices.  j is a neighbour of i iff j != i and
 * ((dx*dx + dy*dy) + dz*dz) < h*h evaluated in FP64 with dx = x_i - x_j
 * (unsoftened distance, strict inequality).
 *   offsets : device, int64[n + 1]
 *   idx     : device, int32[cap]
 *   cap     : capacity of idx
 *   needed  : host int64*, receives the total count (nnz); may be NULL, in
 *             which case no host synchronisation happens and a too-small
 *             cap is latched (nothing is written past cap) and reported by
 *             the next p3t_check.
 * May run concurrently with p3t_long_force on another stream, after the
 * same p3t_build_tree (both only read the tree; each walk has its own
 * device work counter): the neighbour walk then fills the SMs that the
 * force kernel's tail leaves idle.
 * With species set (p3t_set_species) the radius depends on the pair type
 * and the rows are built through context scratch for the star rows, which
 * grows only when `needed` is given: call once with `needed` before
 * capturing calls without it in a CUDA graph.
 * Errors: P3T_ERR_CAPACITY (nnz > cap; offsets valid, idx undefined),
 * P3T_ERR_STATE (no tree), P3T_ERR_CUDA. */
int p3t_neighbours(p3t_ctx *ctx, int64_t *offsets, int32_t *idx, int64_t cap,
                   int64_t *needed, void *stream);

/* Velocity kick by the soft force (Eq. 11; Sect. 2.2 steps 4 and 8):
 * v <- v + dt * a, elementwise in FP64 (no fused multiply-add).
 *   vel : device, double[3][n];  acc : device, float[3][n].
 * Errors: P3T_ERR_INVALID (n < 0 or NULL with n > 0), P3T_ERR_CUDA. */
int p3t_kick(int64_t n, double *vel, const float *acc, double dt, void *stream);

/* Drift (Sect. 2.2 step 5): x <- x + dt * v, elementwise in FP64.
 *   pos : device, double[3][n];  vel : device, double[3][n]. */
int p3t_drift(int64_t n, double *pos, const double *vel, double dt,
              void *stream);

/* Energies in FP64: out[0] = E_kin = 1/2 sum m_i |v_i|^2 and, if pot is not
 * NULL, out[1] = 1/2 sum m_i phi_i (else 0).  out is a DEVICE double[2].
 * Uses scratch owned by ctx. */
int p3t_energy(p3t_ctx *ctx, int64_t n, const double *mass, const double *vel,
               const double *pot, double *out, void *stream);

/* The same energy sums as p3t_energy for callers that cannot allocate device
 * memory: code that runs while a stream is being captured into a CUDA graph,
 * or inside a host application whose device memory is entirely owned by
 * another allocator (a pre-reserved pool), may not call cudaMalloc, and a
 * p3t_ctx (which allocates) may not be available to it.  The paper has no
 * counterpart; this is a service of the library.
 * Scratch: a static device array of P3T_ENERGY_NOALLOC_MAX_PARTIALS block
 * partial sums (two doubles each, 16 KiB) that every GPU loading the library
 * keeps until exit; no cudaMalloc, cudaFree or allocating library routine is
 * called.  The launch uses min(ceil(n / 256), 4 x SM count) blocks, so any n
 * fits as long as the device has at most 256 SMs.
 *   n    : 0 <= n <= P3T_ENERGY_NOALLOC_MAX_N (INT32_MAX, the most
 *          particles the library indexes: neighbour indices are int32);
 *          larger n is rejected with P3T_ERR_CAPACITY.  The kernel indexes
 *          in 64 bits, so no accepted n overflows it.
 *   mass, vel, pot, out : as p3t_energy (device pointers; pot may be NULL)
 * The first call on a device looks up the scratch address for that device
 * (cudaGetSymbolAddress); make that first call before any stream capture.
 * All calls share the one array and it keeps the last call's contents (every
 * partial a call reads is written by that call first, so nothing needs
 * clearing); calls that overlap on the GPU (different streams, no ordering)
 * race on it and must be serialised by the caller.
 * Errors: P3T_ERR_INVALID (NULL pointer with n > 0, n < 0),
 * P3T_ERR_CAPACITY (n too large, or more partials than the array holds),
 * P3T_ERR_CUDA. */
#define P3T_ENERGY_NOALLOC_MAX_PARTIALS 1024
#define P3T_ENERGY_NOALLOC_MAX_N 2147483647LL
int p3t_energy_noalloc(int64_t n, const double *mass, const double *vel,
                       const double *pot, double *out, void *stream);

/* Counters of the last build / force evaluation (host struct). */
typedef struct p3t_stats {
    int64_t n;
    int64_t n_cells;
    int64_t n_groups;
    int64_t n_levels;     /* deepest level + 1 */
    int64_t list_pc;      /* cell entries over all group lists */
    int64_t list_pp_near; /* particle entries with K < 1 possible */
    int64_t list_pp_far;  /* particle entries with K = 1 */
    int64_t int_pc;       /* particle-cell interactions (sum over groups of
                             group size x cell list length) */
    int64_t int_pp;       /* particle-particle interactions, self included */
    int64_t int_pp_near;  /* the part of int_pp from near lists */
    int64_t max_walk_stack; /* deepest walk stack (child ranges) seen by the
                               inspection walk of p3t_get_lists; the walks
                               of the force, neighbour and backward kernels
                               traverse identically and hold 768 */
    int64_t nnz;          /* neighbour pairs (after p3t_neighbours) */
    /* last p3t_hard_step */
    int64_t herm_block_steps;    /* block steps, summed over components */
    int64_t herm_particle_steps; /* particle steps (force evaluations) */
    int64_t herm_pairs;          /* pair evaluations, first forces included */
    int64_t herm_capped;         /* steps whose level hit kmax */
    int64_t herm_components;     /* connected components integrated */
    int64_t herm_max_component;  /* particles in the largest one */
    int64_t herm_max_block_steps; /* most block steps of one component */
    int64_t need_cells;  /* cells the last p3t_build_tree needed (its count
                            when it succeeded; at least what the failing level
                            asked for when a p3t_limits cell bound stopped it) */
} p3t_stats;
int p3t_get_stats(p3t_ctx *ctx, p3t_stats *s);

/* ---- profiling ----
 * With profiling on, CUDA events are recorded on the caller's stream around
 * each phase; p3t_get_profile synchronises and returns the accumulated
 * device time of every phase since the last reset. */
typedef struct p3t_profile {
    double build_ms;   /* p3t_build_tree, all kernels */
    double walk_ms;    /* p3t_long_force_vjp (walk + Jacobian products +
                          push of cell adjoints) */
    double force_ms;   /* p3t_long_force: the fused walk + force kernel */
    double ngb_ms;     /* p3t_neighbours: near walks, scan, row sort */
    int64_t builds, walks, forces, ngbs; /* number of timed calls */
    int64_t int_pc, int_pp, int_pp_near; /* interactions evaluated by
                                            p3t_long_force since the last
                                            reset */
    double vjp_walk_ms;  /* the backward's walk + Jacobian kernel alone (part
                            of walk_ms) */
    int64_t vjp_walks;
    /* parts of build_ms: root box and keys; radix sort and gather of the
     * Morton-ordered copies; octree split and leaf order; moments; groups,
     * their boxes and evaluation order */
    double build_keys_ms, build_sort_ms, build_split_ms, build_moments_ms,
        build_groups_ms;
} p3t_profile;
int p3t_profile_enable(p3t_ctx *ctx, int on);
int p3t_get_profile(p3t_ctx *ctx, p3t_profile *out, int reset);

/* Number of kernels this library has launched since it was loaded (all
 * contexts, all entry points). */
int64_t p3t_launch_count(void);

/* Measured arithmetic ceilings of the current device, for the roofline of
 * the force kernel beside its nominal FP32 peak.  Runs register-only loops
 * over every SM: independent FP32 FMA chains (scalar, and FP32x2 as the
 * force kernel issues them) and chains of the hardware reciprocal square
 * root.  Each loop is timed with CUDA events after one warm-up launch, for
 * about 10 ms, on a private stream; the call synchronises the device work it
 * launched and allocates (and frees) one small output buffer.
 * fma_flops, fma2_flops: flop/s (an FMA counts 2); rsqrt_ops: 1/sqrt per
 * second.  Any pointer may be NULL.  Errors: P3T_ERR_CUDA. */
int p3t_alu_peaks(double *fma_flops, double *fma2_flops, double *rsqrt_ops);

/* FP64 figures of the current device that set the design of the hard
 * part's Hermite kernel (p3t_hard_step): dfma_ops, FP64 FMAs per second
 * over every SM (independent register chains, CUDA-event timed after a
 * warm-up launch, about 10 ms); add_cycles, div_cycles, sqrt_cycles, the
 * latency in SM clock cycles of one dependent IEEE add, division and square
 * root (correctly rounded, as the hard part uses them) in one warp, timed
 * with the SM clock over 4096 operations.  Private stream, synchronised;
 * allocates and frees two small buffers.  Any pointer may be NULL.
 * Errors: P3T_ERR_CUDA. */
int p3t_fp64_peaks(double *dfma_ops, double *add_cycles, double *div_cycles,
                   double *sqrt_cycles);

/* ---- inspection (tests and tools; each call synchronises and copies to
 * HOST buffers sized from p3t_get_stats) ---- */

/* Sorted Morton keys and the original index of each sorted particle. */
int p3t_get_order(p3t_ctx *ctx, uint64_t *key, int32_t *order);

/* Root cube: lo[3] and side. */
int p3t_get_root(p3t_ctx *ctx, double *lo, double *size);

/* Cells (any order; children of a cell are contiguous and in Morton order):
 * level, first sorted particle, count, first child (-1 for a leaf), number of
 * children, FP64 mass, centre of mass [3], quadrupole [6] (xx yy zz xy xz yz,
 * traceless, about the centre of mass), FP32 outward-rounded member box
 * fmin[3], fmax[3].  Any pointer may be NULL. */
int p3t_get_cells(p3t_ctx *ctx, int32_t *level, int32_t *first,
                  int32_t *count, int32_t *child, int32_t *nchild, double *M,
                  double *com, double *Q, float *fmin, float *fmax);

/* Groups: first sorted particle and count of each group (any order), and
 * the FP32 outward-rounded member box. */
int p3t_get_groups(p3t_ctx *ctx, int32_t *first, int32_t *count, float *fmin,
                   float *fmax);

/* Interaction lists of the current tree and parameters, CSR per group (group
 * order as p3t_get_groups): cells (cell ids as p3t_get_cells), near particles
 * and far particles (sorted particle ids).  Offsets have n_groups + 1
 * entries.  The lists are made by a separate walk with the same traversal
 * and opening test as the force kernel (run on the first call after a build
 * or a parameter change); call once with the list pointers NULL to learn the
 * sizes from the offsets' last entries, then again to copy the lists. */
int p3t_get_lists(p3t_ctx *ctx, int64_t *pc_off, int32_t *pc,
                  int64_t *ppn_off, int32_t *ppn, int64_t *ppf_off,
                  int32_t *ppf);

/* Bounds of the kernels' loops and bounded waits, and of the cells a build may
 * allocate: a service for tests and for callers that want a failure rather
 * than a long wait.  The paper has no counterpart.  A value <= 0 selects the
 * default.
 *   walk_iters  : iterations of one group's tree walk in the force,
 *                 neighbour, backward and inspection walks (default 2^24;
 *                 a walk of a finite tree needs a few hundred to a few
 *                 thousand); past it the group is abandoned and
 *                 P3T_ERR_TIMEOUT latched
 *   uf_rounds   : rounds of the lock-free union-find of p3t_hard_step per
 *                 edge and lookup (default 2^20): P3T_ERR_TIMEOUT
 *   block_steps : block steps of one component in p3t_hard_step (default
 *                 2^26): P3T_ERR_TIMEOUT
 *   max_cells   : cells p3t_build_tree may allocate (default: no bound); a
 *                 tree that needs more returns P3T_ERR_CAPACITY, and
 *                 p3t_stats.need_cells says how many the failing level asked
 *                 for
 * A kernel that reaches a bound stops that work item and returns normally;
 * the latched error is returned by p3t_check (or the next synchronising
 * call), after which the context is usable again. */
typedef struct p3t_limits {
    int64_t walk_iters;
    int64_t uf_rounds;
    int64_t block_steps;
    int64_t max_cells;
} p3t_limits;

/* Sets the bounds (NULL: all defaults).  Errors: P3T_ERR_INVALID (ctx NULL). */
int p3t_set_limits(p3t_ctx *ctx, const p3t_limits *lim);

/* The sources the fused walk + force kernel itself evaluates, per group: runs
 * p3t_long_force (acc as there, device float[3][n], written) with a recording
 * instantiation of the kernel that appends, for every staged tile, one record
 * per source to rec (device int64[cap]): the group (numbering of
 * p3t_get_groups) in bits 33-62, the kind (0 accepted cell, 1 near-leaf
 * particle, 2 far-leaf particle) in bits 31-32, and the cell id (numbering
 * of p3t_get_cells) or sorted particle id in bits 0-30.  Records are in no
 * particular order; *count (host) receives their number.  The timed path
 * uses the instantiation without recording.  Synchronises.
 * Errors: P3T_ERR_CAPACITY (*count > cap; the first cap records written),
 * P3T_ERR_INVALID (cap < 1, NULL pointers), P3T_ERR_STATE (no tree), and
 * those of p3t_long_force. */
int p3t_force_lists(p3t_ctx *ctx, float *acc, int64_t *rec, int64_t cap,
                    int64_t *count, void *stream);

/* Human-readable name of a status code. */
const char *p3t_status_string(int status);

#ifdef __cplusplus
}
#endif
#endif /* P3T_H */
