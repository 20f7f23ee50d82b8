/*
 * rpyfmm.h -- C ABI of the GB300 RPY matvec library (librpyfmm.so).
 *
 * Operation (Sec. 1 of "RPYFMM: Parallel adaptive fast multipole method for
 * Rotne-Prager-Yamakawa tensor in biomolecular hydrodynamics simulations"):
 *
 *     u_i = sum_j D_ij F_j,        i = 1..N,
 *
 * with the RPY tensor D: the self term kT/(6 pi eta a) I, the far branch
 * (Eq. "rpy-far", r >= 2a) and the overlap branch (r < 2a; the standard form
 * kT/(6 pi eta a)[(1 - 9r/(32a)) I + (3/(32a)) r(x)r / r], which the paper
 * prints garbled).  Pairs in adjacent leaves are summed directly; all other
 * pairs go through the four Laplace potentials of Sec. 2 (Eq. 2.8, with the
 * dipole term read as -C2 grad L_C), evaluated by an adaptive FMM whose
 * multipole-to-local step uses plane-wave (exponential) expansions along six
 * directions (Sec. 1, Sec. 3.2 Fig. "op": M-to-I, I-to-I, I-to-L).
 *
 * Conventions for every entry point:
 *  - Arrays marked "device" are CUDA device pointers owned by the caller;
 *    arrays marked "host" are ordinary host memory owned by the caller.
 *    Positions, forces and velocities are N x 3 row-major FP64 (x, y, z per
 *    bead) in the caller's bead order.
 *  - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *    stream).  Work is enqueued on it; entry points that must read sizes
 *    back (tree builds) synchronise that stream before returning.
 *  - A tree handle owns all device workspace it needs; rpy_matvec allocates
 *    nothing.  Handles are not thread-safe: one host thread per handle at a
 *    time; different handles may be used concurrently on different streams.
 *  - kT_over_eta is kT/eta; D is linear in it, D_ii = kT_over_eta/(6 pi a) I.
 *  - Every function returns an rpy_status (0 = success).  Invalid arguments
 *    are rejected before any device work.  Errors found on the device
 *    during an asynchronous call are reported by the next call that
 *    synchronises (rpy_tree_sync, rpy_tree_stats, a build).
 *  - There is no CPU fallback: without a CUDA device every compute entry
 *    point returns RPY_ERR_NODEVICE.
 */
#ifndef RPYFMM_H
#define RPYFMM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct rpy_tree_s *rpy_tree;

typedef enum {
    RPY_OK = 0,
    RPY_ERR_INVALID = -1,    /* bad argument (n < 1, a <= 0, NULL pointer, ...) */
    RPY_ERR_DIGITS = -2,     /* digits not in {3, 6, 9}, or 9 with RPY_FP32 */
    RPY_ERR_OOM = -3,        /* device allocation failed */
    RPY_ERR_CUDA = -4,       /* a CUDA call failed; see rpy_last_cuda_error() */
    RPY_ERR_TIMEOUT = -5,    /* a bounded device wait gave up */
    RPY_ERR_NONFINITE = -6,  /* a position is NaN or infinite */
    RPY_ERR_STATE = -7,      /* handle in the wrong state (freed, mismatched sizes) */
    RPY_ERR_NODEVICE = -8,   /* no CUDA device visible */
    RPY_ERR_INTERNAL = -9    /* internal capacity exceeded (reported, never silent) */
} rpy_status;

typedef enum {
    RPY_FP64 = 0,            /* every stage in FP64 */
    RPY_FP32 = 1             /* precision form: near field and translations in FP32 with
                                compensated accumulation; bounding cube, Morton keys,
                                r ~ 0 overlap pairs and the final per-bead sum in FP64 */
} rpy_precision;

/* Build parameters.  Zero fields take the defaults listed. */
typedef struct {
    int digits;       /* 3, 6 or 9: relative-L2 accuracy setting (required) */
    int precision;    /* rpy_precision; default RPY_FP64 */
    int leaf_cap;     /* refinement limit: a box splits while it holds more beads
                         (Sec. 4.2 "threshold"); 0 = default for the setting */
    int order_p;      /* expansion order p; 0 = default for the setting */
    int max_level;    /* deepest level allowed, 1..21; 0 = 21 */
    int flags;        /* bit 0 (RPY_FLAG_NO_GRAPH): never replay the matvec as a CUDA graph;
                         bit 1 (RPY_FLAG_FRAME_PASSES): run M2X / X2X / X2L one plane-wave
                         frame (two of the six directions) at a time, with a third of the
                         plane-wave memory; chosen automatically when the buffers of all
                         six directions would exceed 64 GB;
                         bit 2 (RPY_FLAG_EVAL_PER_POTENTIAL): evaluate Eq. (2.8) at the beads
                         per Laplace potential (approach 1 of Sec. 2: 12 expansions per
                         bead) instead of one expansion per velocity component (approach 2,
                         the default: 6 expansions per bead);
                         bit 3 (RPY_FLAG_BOX_ORIGIN) / bit 4 (RPY_FLAG_CUBE_ORIGIN): where the
                         fourth charge set q4 = F . (r - o) of Sec. 2 takes its origin o.  Box
                         origin: every expansion carries q4 about its own box centre, moved
                         along with each translation (M2M, X2X, L2L), so its values stay of
                         the size of the box's own moments; cube origin: one origin per system
                         (the bounding-cube centre), which leaves the far-field combination
                         grad L4 - sum_k x_k grad L_k of Eq. (2.8) to cancel terms of size
                         |x - o| |grad L|.  Default: box origin for RPY_FP32 at 6 digits, cube
                         origin for RPY_FP64 and at 3 digits (whose rounding stays far below
                         the setting there); at most one of the two bits;
                         bit 5 (RPY_FLAG_CARTESIAN): the polynomial far field that the paper's
                         Sec. 5 proposes for low accuracy: Cartesian Taylor expansions of total
                         degree order_p (default 8, at most 10) with a direct multipole-to-local
                         step over the V lists instead of spherical harmonics and plane waves;
                         every W- and X-list interaction is summed directly; 3 digits only
                         (RPY_ERR_DIGITS otherwise); rpy_laplace_far is not available on such a
                         tree (RPY_ERR_STATE);
                         other bits must be 0 */
    int direct_w;     /* W-list boxes with at most this many beads are summed directly
                         instead of by multipole evaluation: 0 = automatic
                         (about 1.8 (p+3)(p+4)/2), -1 = never */
    int direct_x;     /* X-list pairs whose target box holds at most this many beads are
                         summed directly instead of by source-to-local expansion:
                         0 = automatic (about 0.6 (p+1)(p+2)/2), -1 = never */
    int quad;         /* plane-wave quadrature rule of M2X / X2X / X2L: 0 = the rule of
                         `digits`; 3, 4, 5, 6 or 9 = the rule built for that many digits
                         (max relative error of the 1/r representation 3.6e-4, 3.6e-5,
                         2.8e-6, 4.0e-7, 2.3e-10 over the V-list region; 134, 218, 323,
                         464, 1168 stored plane waves per direction) */
} rpy_build_params;

enum { RPY_FLAG_NO_GRAPH = 1, RPY_FLAG_FRAME_PASSES = 2, RPY_FLAG_EVAL_PER_POTENTIAL = 4, RPY_FLAG_BOX_ORIGIN = 8,
       RPY_FLAG_CUBE_ORIGIN = 16, RPY_FLAG_CARTESIAN = 32 };

/* Statistics of a built tree (host struct filled by rpy_tree_stats). */
typedef struct {
    int64_t n_beads;
    int32_t n_systems;
    int32_t n_boxes;
    int32_t n_leaves;
    int32_t depth;              /* deepest level present */
    int32_t order_p;
    int32_t exp_nodes;          /* lambda nodes s */
    int32_t exp_terms;          /* sum_k M_k (plane waves per direction) */
    int32_t leaf_cap;
    int32_t digits;
    int32_t precision;
    int32_t max_leaf_count;     /* largest leaf (may exceed leaf_cap where the 2a rule stops refinement) */
    int32_t leaves_over_cap;
    int64_t u_pairs;            /* bead pairs summed directly (near field, incl. self) */
    int64_t n_ulist, n_wlist, n_xlist, n_vpairs;
    int64_t n_dlist;            /* (leaf, source box) pairs summed directly in place of W / X */
    int64_t d_pairs;            /* bead pairs summed directly in place of W / X */
    int64_t device_bytes;       /* device memory held by the handle */
    double build_ms;            /* host-measured wall time of the last build */
    int32_t quad;               /* plane-wave quadrature rule in use (3..6) */
} rpy_stats;

/*
 * Build an adaptive octree over N beads and all interaction lists: the tree of
 * the paper's evaluate(sources, targets, threshold, method, accuracy) call
 * (Sec. 4.2), with `threshold` the refinement limit (leaf_cap: a box splits
 * while it holds more beads) and `accuracy` the digit setting (Sec. 4.3).
 *   pos_dev   device, n x 3 FP64, caller order
 *   n         number of beads, >= 1
 *   a         bead radius, > 0 and finite
 *   digits    3, 6 or 9
 *   leaf_cap  refinement limit, 0 = default (40 for 3 digits, 100 for 6, 120 for 9)
 *   precision rpy_precision
 *   out       receives the handle (NULL on failure)
 * Boxes split while they hold more than leaf_cap beads and their children
 * would have side >= 2a, so every pair closer than 2a is summed directly.
 * Synchronises `stream`.  Non-finite positions give RPY_ERR_NONFINITE.
 */
int rpy_tree_build(const double *pos_dev, int64_t n, double a, int digits, int leaf_cap,
                   int precision, void *stream, rpy_tree *out);

/*
 * Build one tree over many independent systems (the batching form): system
 * k owns beads [sys_offsets[k], sys_offsets[k+1]) of pos_dev and has radius
 * a_host[k].  Systems do not interact.  Every later matvec treats all of
 * them in the same launches.
 *   pos_dev      device, sys_offsets[nsys] x 3 FP64
 *   sys_offsets  host, nsys + 1 non-decreasing int64, sys_offsets[0] = 0,
 *                every system non-empty
 *   a_host       host, nsys radii
 *   params       host, build parameters (digits required)
 */
int rpy_forest_build(const double *pos_dev, const int64_t *sys_offsets, int nsys, const double *a_host,
                     const rpy_build_params *params, void *stream, rpy_tree *out);

/*
 * Rebuild the tree of `t` for new positions of the same beads (same N, same
 * systems, same radii and parameters), reusing its device buffers where they
 * fit.  Used between Brownian-dynamics steps: the Ermak-McCammon update of
 * Sec. 1 moves every bead, and D of the next step is the tensor at the new
 * positions.  Synchronises `stream`.
 */
int rpy_tree_update_positions(rpy_tree t, const double *pos_dev, void *stream);

/*
 * u = D F for every bead of the tree (the hot path): D the RPY tensor of
 * Sec. 1 (self term, r >= 2a far branch, r < 2a overlap branch), pairs of
 * adjacent leaves summed directly and all others through the four Laplace
 * potentials of Sec. 2 combined by Eq. 2.8.  From the second call on
 * the same build, the body of the matvec (everything after the force gather
 * and before the final combine) is replayed as a CUDA graph captured once on
 * a stream owned by the tree (unless RPY_FLAG_NO_GRAPH or profiling is on).
 *   f_dev        device, N x 3 FP64 forces, caller order
 *   kT_over_eta  kT/eta, finite
 *   u_dev        device, N x 3 FP64 velocities, caller order (overwritten)
 * Asynchronous on `stream`; allocates nothing.  For a forest every system
 * uses the same kT_over_eta; see rpy_forest_matvec.
 */
int rpy_matvec(rpy_tree t, const double *f_dev, double kT_over_eta, double *u_dev, void *stream);

/* Forest matvec with a per-system kT/eta (host array of nsys values). */
int rpy_forest_matvec(rpy_tree t, const double *f_dev, const double *kT_over_eta_host, double *u_dev,
                      void *stream);

/*
 * Matvecs of several separately built trees, issued back to back on one stream
 * (each replays its own captured graph): tree k reads f_dev[k] and writes
 * u_dev[k] with kT_over_eta[k].  All arguments are checked before the first
 * launch.  For many small systems a forest (rpy_forest_build) is faster: it
 * runs every system in the same launches.  Asynchronous on `stream`.
 */
int rpy_matvec_batched(rpy_tree const *trees, int ntrees, const double *const *f_dev, const double *kT_over_eta,
                       double *const *u_dev, void *stream);

/*
 * Diagnostic split of rpy_matvec: parts = RPY_PART_NEAR (direct pairs of
 * adjacent leaves, self term included), RPY_PART_FAR (everything else, via
 * the FMM), or both.  u_dev receives the sum of the selected parts.
 */
enum { RPY_PART_NEAR = 1, RPY_PART_FAR = 2, RPY_PART_ALL = 3 };
int rpy_matvec_parts(rpy_tree t, const double *f_dev, double kT_over_eta, double *u_dev, int parts,
                     void *stream);

/*
 * The matvec of a resident tree with HOST buffers: the step of a Brownian-
 * dynamics loop or a serving request (Sec. 1: D F at the current positions).
 * When pos_host is non-NULL it is copied to the device and the tree is rebuilt
 * for it (as rpy_tree_update_positions), while f_host is copied on a stream of
 * the tree's own; then u = D F is applied (as rpy_forest_matvec, after both
 * copies) and u is copied back to u_host.  The work is ordered on `stream` and
 * synchronised before return.  Page-locked host buffers
 * (cudaHostAlloc, cudaHostRegister) copy at full bus speed; pageable ones work
 * and copy slower.  The tree allocates 9 N doubles of device buffers for the
 * copies on the first call and keeps them until rpy_tree_free.
 *   pos_host           host, N x 3 FP64 (caller order), or NULL: positions unchanged
 *   f_host             host, N x 3 FP64
 *   kT_over_eta_host   host, one value per system (finite)
 *   u_host             host, N x 3 FP64 (written)
 */
int rpy_tree_matvec_host(rpy_tree t, const double *pos_host, const double *f_host,
                         const double *kT_over_eta_host, double *u_host, void *stream);

/*
 * One-shot form with the paper's argument list (positions, radius, forces,
 * kT/eta, accuracy digits; the Bead / kparams interface of Sec. 4.2): u = D F
 * with D the tensor of Sec. 1 split as in Sec. 2; builds a tree, applies it
 * once, frees it.
 * All arrays are device arrays.  Synchronises `stream`.
 */
int rpy_matvec_oneshot(const double *pos_dev, int64_t n, double a, const double *f_dev,
                       double kT_over_eta, int digits, double *u_dev, void *stream);

/*
 * The same with HOST arrays: copies pos and f to the device, runs the
 * one-shot matvec and copies u back, all on `stream` (synchronised before
 * return).  Device scratch is allocated and freed inside.
 */
int rpy_matvec_host(const double *pos_host, int64_t n, double a, const double *f_host,
                    double kT_over_eta, int digits, int precision, double *u_host, void *stream);

/*
 * The paper's evaluate(sources, targets) form (Sec. 4.2): velocities at nt target
 * points from ns source beads of radius a with forces f,
 *   u_t = sum_j D(t, j) F_j,
 * D the same tensor as between two beads of radius a (the overlap branch for
 * r < 2a, the r -> 0 limit for a target on a source); targets exert no force and
 * have no self term.  One tree is built over the union of sources and targets
 * (targets as beads with zero force), applied once and freed.
 *   src_pos_dev, src_f_dev   device, ns x 3 FP64
 *   tgt_pos_dev              device, nt x 3 FP64
 *   params                   build parameters (digits, precision, ...)
 *   u_tgt_dev                device, nt x 3 FP64 (written)
 * Allocates and frees device scratch; synchronises `stream`.
 */
int rpy_evaluate(const double *src_pos_dev, const double *src_f_dev, int64_t ns, const double *tgt_pos_dev,
                 int64_t nt, double a, double kT_over_eta, const rpy_build_params *params, double *u_tgt_dev,
                 void *stream);

/*
 * Laplace far field of the tree (Sec. 2): for four charge sets q (device,
 * N x 4 FP64, caller order) returns, at every bead, the FMM part of the
 * potential, its gradient and its Hessian (device, N x 4 x 13 FP64:
 * [phi, dx, dy, dz, Hxx, Hxy, Hxz, Hyx, Hyy, Hyz, Hzx, Hzy, Hzz]), i.e. the
 * sum over all sources outside the bead's U list.  Used to test the
 * expansions operator by operator against direct sums.
 */
int rpy_laplace_far(rpy_tree t, const double *q_dev, double *out_dev, void *stream);

/*
 * Copy one array of the tree to host memory for inspection and tests.
 *   field      one of RPY_FIELD_*
 *   host_dst   host buffer, may be NULL to query the size
 *   capacity   bytes available at host_dst
 *   bytes_out  receives the size of the field in bytes
 * Synchronises `t`'s last stream.
 */
enum {
    RPY_FIELD_PERM = 1,        /* int32[N]: sorted position -> caller index */
    RPY_FIELD_KEYS = 2,        /* uint64[N]: Morton keys in sorted order */
    RPY_FIELD_BOX_LEVEL = 3,   /* int32[nbox] */
    RPY_FIELD_BOX_RANGE = 4,   /* int32[nbox][2]: sorted bead range [begin, end) */
    RPY_FIELD_BOX_PARENT = 5,  /* int32[nbox], -1 for roots */
    RPY_FIELD_BOX_CENTER = 6,  /* double[nbox][3] */
    RPY_FIELD_BOX_LEAF = 7,    /* int32[nbox]: 1 if the box is a leaf */
    RPY_FIELD_BOX_SYS = 8,     /* int32[nbox]: system of the box */
    RPY_FIELD_BOX_SIDE = 9,    /* double[nbox] */
    RPY_FIELD_LEAVES = 10,     /* int32[nleaf]: leaf box ids */
    RPY_FIELD_U_OFF = 11,      /* int32[nleaf + 1]: CSR offsets of U lists (per leaf) */
    RPY_FIELD_U_IDX = 12,      /* int32[]: source leaf boxes */
    RPY_FIELD_W_OFF = 13,      /* int32[nleaf + 1]: W lists (per leaf) */
    RPY_FIELD_W_IDX = 14,
    RPY_FIELD_X_OFF = 15,      /* int32[nbox + 1]: X lists (per box) */
    RPY_FIELD_X_IDX = 16,
    RPY_FIELD_V_OFF = 17,      /* int32[nbox + 1]: V lists (per box), built on request */
    RPY_FIELD_V_IDX = 18,
    RPY_FIELD_CUBE = 19,       /* double[nsys][4]: cube centre x, y, z, side */
    RPY_FIELD_D_OFF = 20,      /* int32[nleaf + 1]: direct substitutes of W / X (per leaf) */
    RPY_FIELD_D_IDX = 21
};
int rpy_tree_export(rpy_tree t, int field, void *host_dst, int64_t capacity, int64_t *bytes_out);

/* Fill *out with the statistics of t.  Synchronises t's last stream. */
int rpy_tree_stats(rpy_tree t, rpy_stats *out);

/* Wait for t's last stream and report any error recorded on the device. */
int rpy_tree_sync(rpy_tree t);

/*
 * Estimate the device bytes a tree over n beads would hold (upper bound
 * used for admission control by the serving loop).  Host only.
 */
int rpy_tree_footprint(int64_t n, int digits, int precision, int leaf_cap, int64_t *bytes);

/* Release the handle and all its device memory.  NULL is ignored. */
void rpy_tree_free(rpy_tree t);

/* Static description of a status code. */
const char *rpy_strerror(int status);

/* Text of the last CUDA error seen by this thread (empty if none). */
const char *rpy_last_cuda_error(void);

/*
 * Host-only inspection of the operator tables for expansion order p and a
 * plane-wave quadrature rule `digits` (3..6 or 9, as rpy_build_params.quad; no
 * device needed): which = 1 M2M, 2 L2L (transposed real
 * matrices per child octant), 3 / 4 frame rotations world->frame / frame->world,
 * 5 M2X coefficients, 6 X2L coefficients, 7 stored plane waves (k, cos, sin,
 * w/M), 8 shift factors, 9 merge-and-shift groups, 10 rotation block offsets,
 * 11 quadrature (s, then lambda, w, M per node), 12 / 13 child-octant rotations
 * world->frame / frame->world, 14 / 15 z-axis M2M / L2L shift coefficients, 16 / 17 / 18
 * per-axis shift factors e^{-lambda dz} [6][S], e^{i lambda dx cos a} and e^{i lambda dy sin a}
 * [6][S][2] (offset index - 2.5 along the axis).  dst (host, may be NULL to query) receives
 * *count doubles.
 */
int rpy_debug_table(int p, int digits, int which, double *dst, int64_t capacity, int64_t *count);

/*
 * Per-stage timing of later matvecs of t: when enabled, CUDA events are
 * recorded on the call's stream between the stages of rpy_matvec.
 * rpy_tree_stage_times writes the stage durations (ms) of the last matvec,
 * in the order of RPY_STAGE_*, after synchronising; n = slots in ms_host.
 */
enum {
    RPY_STAGE_GATHER = 0, RPY_STAGE_P2P, RPY_STAGE_P2M, RPY_STAGE_M2M, RPY_STAGE_M2X, RPY_STAGE_X2X,
    RPY_STAGE_X2L, RPY_STAGE_P2L, RPY_STAGE_L2L, RPY_STAGE_EVAL, RPY_STAGE_COMBINE, RPY_NUM_STAGES
};
int rpy_tree_set_profiling(rpy_tree t, int enable);
int rpy_tree_stage_times(rpy_tree t, double *ms_host, int n);

/* ------------------------------------------------------------------ Brownian dynamics
 * Consumers of repeated matvecs on a resident tree (Sec. 1: the drift D F and a
 * random displacement with covariance 2 dt D of the Ermak-McCammon step).
 *
 * rpy_lanczos_sqrt: y = D^{1/2} z approximated by the Lanczos process on D
 * (one matvec per step; Krylov basis kept on the device, m_max x 3N doubles):
 * y_m = |z| V_m T_m^{1/2} e_1 with T_m the m x m Lanczos tridiagonal matrix.
 * Stops when the relative change |y_m - y_(m-1)| / |y_m| <= tol or after m_max
 * steps.
 *   z_dev              device, N x 3 FP64 (caller order), e.g. N(0,1) samples
 *   kT_over_eta_host   host, one value per system
 *   m_max              1..1000; tol >= 0
 *   y_dev              device, N x 3 FP64 (written)
 *   iters, rel_change  host, may be NULL: steps taken, last relative change
 * Allocates and frees device scratch; synchronises `stream`.
 */
int rpy_lanczos_sqrt(rpy_tree t, const double *z_dev, const double *kT_over_eta_host, int m_max, double tol,
                     double *y_dev, int *iters, double *rel_change, void *stream);

/*
 * One Ermak-McCammon step (no divergence term: the RPY tensor is divergence
 * free): r <- r + (dt / kT) D F + sqrt(2 dt) D^{1/2} xi, with D evaluated at the
 * tree's current positions (kT/eta per system), D^{1/2} xi by rpy_lanczos_sqrt,
 * then the tree is rebuilt for the new positions (rpy_tree_update_positions).
 *   pos_dev    device, N x 3: on entry the positions the tree was built for,
 *              on return the new positions
 *   f_dev      device, N x 3 forces; xi_dev device, N x 3 N(0,1) samples
 *              (drawn by the caller)
 *   kT_host, eta_host   host, one value per system (> 0)
 *   dt         time step (>= 0)
 *   disp_dev   device, N x 3 displacement of the step (written), or NULL
 * Synchronises `stream`.
 */
int rpy_bd_step(rpy_tree t, double *pos_dev, const double *f_dev, const double *xi_dev, const double *kT_host,
                const double *eta_host, double dt, int m_max, double tol, double *disp_dev, int *iters,
                void *stream);

/* ------------------------------------------------------------------ tuning
 * FP64 direct sum of u_t = sum_j D_tj F_j at chosen targets t (caller
 * indices into the whole array), over all beads j of t's system (Sec. 1:
 * self term, r >= 2a branch, r < 2a overlap branch, coincident beads), on the
 * GPU.  The autotuner's accuracy reference; also a check for callers.
 *   pos_dev, f_dev        device, N x 3 FP64, caller order (N = sys_offsets[nsys])
 *   sys_offsets, a_host, kT_over_eta_host   host, as for rpy_forest_build /
 *                         rpy_forest_matvec (one system: {0, N})
 *   targets_host          host, nt indices in [0, N)
 *   u_host                host, nt x 3 FP64 (written)
 * Allocates and frees device scratch; synchronises `stream`.
 */
int rpy_direct_sampled(const double *pos_dev, const int64_t *sys_offsets, int nsys, const double *a_host,
                       const double *f_dev, const double *kT_over_eta_host, const int64_t *targets_host,
                       int64_t nt, double *u_host, void *stream);

typedef struct {
    int n_samples;       /* sampled targets of the error estimate; 0 = 256 */
    int timed_reps;      /* timed matvecs per candidate (median kept); 0 = 3 */
    double margin;       /* accept settings whose sampled relative L2 error is at most
                            margin x bound (bound 1e-3 at 3 digits, 1e-6 at 6, 1e-9 at 9);
                            0 = 0.3 */
    uint64_t seed;       /* sample seed; 0 = a fixed default */
} rpy_autotune_params;

typedef struct {
    int leaf_cap, order_p, direct_w, direct_x;   /* the candidate */
    int quad;                                    /* its plane-wave quadrature rule */
    int status;                                  /* RPY_OK, or why it was skipped */
    double est_rel_l2;                           /* sampled relative L2 error vs rpy_direct_sampled */
    double matvec_ms;                            /* median timed matvec; < 0 when not timed */
} rpy_autotune_trial;

typedef struct {
    rpy_build_params best;   /* chosen parameters (digits and precision as requested) */
    double est_rel_l2;       /* sampled error at the choice */
    double matvec_ms;        /* median matvec time at the choice */
    double goal;             /* margin x bound */
    double tune_ms;          /* host wall time of the search */
    int n_trials;            /* entries of trials[] filled (the search stops recording at 48) */
    rpy_autotune_trial trials[48];
    double verify_rel_l2;    /* error of the choice on the verification sample */
    int n_verify;            /* targets of the verification sample */
    int verify_ok;           /* 1 when verify_rel_l2 <= 0.5 x bound */
} rpy_autotune_result;

/*
 * Autotuner for one bead configuration (one system or a forest): picks the
 * expansion order, the leaf capacity and the direct-substitution thresholds
 * of small W / X interactions for the matvec at `digits` / `precision`.
 *   1. draws n_samples distinct targets and sums RPY there directly
 *      (rpy_direct_sampled, FP64);
 *   2. order p: for each plane-wave quadrature rule (6 digits: the rules of
 *      6, 5 and 4 digits; 3 and 9 digits: their own), the smallest p whose sampled
 *      relative L2 error (default leaf capacity) is at most margin x bound,
 *      then the (rule, p) pair with the fastest timed matvec; if no pair
 *      meets the goal, the one of least error;
 *   3. leaf capacity in {0.5, 0.7, 1, 1.4, 2} x default, then the thresholds
 *      {never, half, automatic, double}: the fastest median matvec (CUDA events
 *      on `stream`) among candidates that keep the error within the goal;
 *   4. verification: the choice against an independent FP64 direct sum on four
 *      times n_samples fresh targets, half uniform over all beads and half over
 *      the beads of the tree's two deepest leaf levels (where the translation
 *      chains are longest).  It must reach 0.5 x bound.  Otherwise, for RPY_FP32,
 *      the FP64 path at the same parameters is verified and taken when it passes
 *      (the excess was FP32 rounding, which a higher order cannot remove), and
 *      the order is raised by one while neither passes (at most four times).
 *      out->best.precision is then RPY_FP64 although RPY_FP32 was asked for; the
 *      caller sees the change there and in verify_rel_l2 / verify_ok.
 * Builds and frees one tree per candidate; allocates device scratch of
 * N x 3 doubles.  Synchronises `stream`.  Arguments as for rpy_forest_build and
 * rpy_forest_matvec; params may be NULL (all defaults).
 */
int rpy_autotune(const double *pos_dev, const int64_t *sys_offsets, int nsys, const double *a_host,
                 const double *f_dev, const double *kT_over_eta_host, int digits, int precision,
                 const rpy_autotune_params *params, rpy_autotune_result *out, void *stream);

/*
 * Measured FMA throughput of the current device (FLOP/s, 2 per FMA) for
 * RPY_FP64 or RPY_FP32: a short kernel of independent FMA chains on every
 * SM, best of three timed runs.  Used as the ALU roofline denominator.
 */
int rpy_alu_peak(int precision, double *flops_per_s, void *stream);

/*
 * Bounding cube of n beads without allocating device memory, for callers
 * that cannot call cudaMalloc (code that runs while their own memory pool is
 * locked, real-time step loops, allocation-free embeddings).  The paper has
 * no counterpart: it is the tree builder's first reduction exposed on its own.
 *   pos_dev   device, n x 3 FP64 positions (read)
 *   n         1 <= n <= 33,554,432 (beyond it: RPY_ERR_INVALID, message in
 *             rpy_last_cuda_error())
 *   cube_dev  device, 4 FP64 written: centre x, y, z and side, the same values
 *             rpy_tree_build uses (side NaN if a position is not finite)
 * Scratch is a fixed file-scope device array (about 230 KB) that every GPU
 * loading the library holds until exit.  The first call on a device looks up
 * that array's device address (cudaGetSymbolAddress, no allocation) and keeps
 * it for the life of the process; make the first call before any stream
 * capture, and do not call this entry point after a cudaDeviceReset of that
 * device in the same process (the kept address would be stale).  NULL
 * pointers and n < 1 give RPY_ERR_INVALID with a message in
 * rpy_last_cuda_error().  All calls share the array:
 * calls that overlap on the GPU (different streams, no ordering) race and
 * give wrong cubes.  Asynchronous on `stream`; allocates nothing.
 */
int rpy_bounding_cube_noalloc(const double *pos_dev, int64_t n, double *cube_dev, void *stream);

/*
 * Algorithmic work of one matvec on t, per stage (RPY_STAGE_*): flops_host[k]
 * floating-point operations (an FMA counts 2) and bytes_host[k] DRAM bytes that
 * stage k needs at this tree, order and plane-wave rule, counted from the tree
 * (near-list bead pairs, boxes per level, present merge-and-shift sources per
 * parent and direction, X- and W-list sizes): the numerators of the roofline
 * fractions reported beside measured stage times.  The paper has no
 * counterpart (it is instrumentation); the operation counts follow the
 * kernels' algorithms as listed in rpy_work.cu.  n = slots in each array
 * (entries beyond RPY_NUM_STAGES are zeroed).  Copies tree arrays to the host;
 * synchronises t's last stream.
 */
int rpy_tree_work(rpy_tree t, double *flops_host, double *bytes_host, int n);

/*
 * Self-test of the bounded device waits of the bulk-copy pipelines (the paper
 * has no counterpart): one thread waits on an mbarrier phase that nothing will
 * complete, gives up after limit_ms (0 < limit_ms <= 2000) and reports it in a
 * status word, as the pipelined kernels do when a copy never lands.  Returns
 * RPY_ERR_TIMEOUT when the wait gave up (the expected outcome), RPY_OK if it
 * did not.  No copy is issued, so nothing is left in flight; the context stays
 * usable.  Allocates and frees one word of device memory; synchronises `stream`.
 */
int rpy_debug_wait_timeout(double limit_ms, void *stream);

/* Number of kernels this library has launched in this process (all devices). */
int64_t rpy_launch_count(void);

/* ------------------------------------------------------------------ serving
 * A request loop for many resident Brownian-dynamics systems (the serving
 * form): every system keeps its tree, expansions and bead buffers on the
 * device between requests; requests (new positions and forces of one system)
 * are admitted as worker slots and device memory allow, and several
 * requests of different systems run at once on separate streams (continuous
 * batching).  Requests of one system run in submission order.  Systems that
 * do not fit the memory budget wait; idle resident systems are evicted
 * (least recently used) to make room.  Host-side C++, one worker thread per
 * slot.  All arrays here are HOST arrays owned by the caller; u_host must
 * stay valid until the request completes.
 */
typedef struct rpy_server_s *rpy_server;

typedef struct {
    int64_t device_budget_bytes;   /* admission limit on resident bytes; 0 = 85% of free memory */
    int slots;                     /* concurrent requests on the device; 0 = 4 */
    int device;                    /* CUDA device; the caller's current device if < 0 */
} rpy_server_params;

typedef struct {
    int64_t submitted, completed, failed, cancelled, evictions, rebuilds;
    int64_t beads_done;            /* beads of completed requests */
    int64_t resident_bytes, peak_resident_bytes;
    int32_t resident_systems, queued, running;
    double p50_ms, p99_ms, mean_ms;  /* latency submit -> completion of completed requests */
    double busy_s;                   /* wall time from first submit to last completion */
} rpy_server_stats;

int rpy_server_create(const rpy_server_params *params, rpy_server *out);
/* Register a system (host positions copied; the tree is built on first admission). */
int rpy_server_add_system(rpy_server s, const double *pos_host, int64_t n, double a,
                          const rpy_build_params *params, int *system_id);
/* Enqueue u = D(pos) f for a system.  pos_host may be NULL (keep the last positions).
 * pos_host and f_host are copied into page-locked buffers of the server before the
 * call returns (the caller may reuse them at once); returns a request id; the result
 * lands in u_host (page-locked memory there copies back fastest).  RPY_ERR_OOM when
 * no page-locked host memory is left for the copies. */
int rpy_server_submit(rpy_server s, int system_id, const double *pos_host, const double *f_host,
                      double kT_over_eta, double *u_host, int64_t *request_id);
/* Wait for a request; timeout_ms < 0 waits forever.  Returns the request's own
 * status (RPY_OK, an error of its computation, RPY_ERR_STATE if cancelled) or
 * RPY_ERR_TIMEOUT if it is still pending.  latency_ms may be NULL. */
int rpy_server_wait(rpy_server s, int64_t request_id, int timeout_ms, double *latency_ms);
/* Per-request timing, filled by rpy_server_wait_times: host wall time in the queue and
 * on a worker, and the device time of each phase on the worker's stream. */
typedef struct {
    double queue_ms;    /* submit -> start on a worker */
    double run_ms;      /* start -> completion */
    double h2d_ms;      /* host-to-device copies of positions (if new) and forces */
    double build_ms;    /* tree build or rebuild for new positions (0 when they were kept) */
    double matvec_ms;   /* the matvec */
    double d2h_ms;      /* device-to-host copy of the velocities */
} rpy_request_times;
/* rpy_server_wait, also returning the request's phase times (times may be NULL). */
int rpy_server_wait_times(rpy_server s, int64_t request_id, int timeout_ms, double *latency_ms,
                          rpy_request_times *times);
/* Cancel a request that has not started; RPY_ERR_STATE if it already started or finished. */
int rpy_server_cancel(rpy_server s, int64_t request_id);
/* Wait until every submitted request has finished. */
int rpy_server_drain(rpy_server s);
int rpy_server_stats_get(rpy_server s, rpy_server_stats *out);
/* Stop the workers (pending requests are cancelled) and free every resident system. */
void rpy_server_destroy(rpy_server s);

/* Library version (major * 10000 + minor * 100 + patch). */
int rpy_version(void);

#ifdef __cplusplus
}
#endif
#endif /* RPYFMM_H */
