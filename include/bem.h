/*
 * bem.h -- C ABI of the GB300 FMM-accelerated collocation boundary element
 * library (Carley, "BEM3D: a free adaptive fast multipole boundary element
 * library").
 *
 * The library computes, on one CUDA device, the two matrix-vector products of
 * the discrete exterior boundary integral equation (Section 2.1, Eq. 1-3)
 *
 *      A phi = B chi,   A = diag(C) - D,   B = -S,   C_i = 1 + sum_j D0_ij,
 *
 *      D_ij = sum_m int L_j dG/dn1 dS_m,   S_ij = sum_m int L_j G dS_m,
 *
 * with G = 1/(4 pi R) (Laplace, Eq. 1a) or exp(jkR)/(4 pi R) (Helmholtz, Eq.
 * 1b) and D0 the Laplace double layer, by the adaptive fast multipole method
 * of Section 3 (octree over vertices, Taylor expansions, convergence-radius
 * separation), and solves the system by restarted GMRES.  The sign of Eq. 1 is
 * read as the exterior problem, C phi = int (phi dG/dn1 - G dphi/dn1) dS.
 *
 * Conventions for every call:
 *   - Return value: BEM_OK (0) or a negative BEM_E* code; bem_last_error()
 *     then returns a message for the calling thread.
 *   - Host arrays passed in are copied; the caller keeps ownership.
 *   - Device arrays (x_dev, y_dev, chi_dev, phi_dev) are owned by the caller,
 *     must be allocated on the plan's device and stay alive until the given
 *     stream has passed the call.  Work is ordered on that stream
 *     (cudaStream_t passed as void*; NULL = the legacy default stream).
 *   - Handles belong to the library until the matching *_destroy call.
 *   - Real vectors are float64; Helmholtz vectors are complex float64 stored
 *     as interleaved (re, im) pairs.
 *   - Elements are counter-clockwise seen from outside (outward normal).
 *     6-node triangles list corners 0, 1, 2, then the mid-side nodes of
 *     edges 0-1, 1-2, 2-0.
 */
#ifndef BEM_H
#define BEM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define BEM_OK 0
#define BEM_EINVAL (-1)   /* bad argument (message says which) */
#define BEM_ENOMEM (-2)   /* device or host allocation failed */
#define BEM_ECUDA (-3)    /* a CUDA call failed (message has the CUDA error) */
#define BEM_ENOCONV (-4)  /* solver stopped before the tolerance; solution written */
#define BEM_ETIMEOUT (-5) /* a bounded device wait gave up */
#define BEM_EBUSY (-6)    /* resource in use */

#define BEM_TRI3 1        /* flat 3-node triangle (first order, Section 2.2) */
#define BEM_TRI6 2        /* curved 6-node triangle (second order, Section 2.2) */

#define BEM_LAPLACE 0     /* G = 1/(4 pi R), Eq. 1a */
#define BEM_HELMHOLTZ 1   /* G = exp(jkR)/(4 pi R), Eq. 1b, time factor exp(-j omega t) */

#define BEM_F64 0         /* every stage in float64 */
#define BEM_MIXED 1       /* near field and expansions in float32, Krylov in float64 */

#define BEM_OP_A 0        /* y = C x - D x  (x indexed by node) */
#define BEM_OP_B 1        /* y = -S x       (x indexed by chi index) */

typedef struct bem_ctx bem_ctx;
typedef struct bem_mesh bem_mesh;
typedef struct bem_plan bem_plan;

/* Fast multipole and quadrature parameters.
 *   p            expansion order: terms with total degree |alpha|+|beta| <= p
 *                are kept in the local expansion (Eq. 7); moments to degree p.
 *   leaf_size    B of Section 3.1: a box holding B or more vertices is split.
 *   eta          separation factor: two boxes interact through expansions iff
 *                |x_c1 - x_c2| > eta (r_C1 + r_C2); eta = 1 is Eq. 13.
 *   max_level    deepest tree level (<= 20).
 *   leaf_descend 1: a leaf keeps opening non-leaf near-list boxes until each
 *                entry is separated or a leaf; 0: the whole subtree is near.
 *   precision    BEM_F64 or BEM_MIXED.
 *   n_duffy      Gauss-Legendre order of the Duffy self-element rule.
 *   tau_near     near-singular threshold: |x_i - X_e(1/3,1/3)| < tau h_e.
 *   max_subdiv   depth limit of the near-singular 4-way subdivision.
 *   p_min        0: every box uses order p.  Otherwise the order depends on
 *                the level (Section 3.6, end): L_l = min(p, p_min + l_max - l),
 *                l_max the deepest level, so the smallest boxes use p_min and
 *                the order grows by one per level towards the root.  Moments
 *                and locals of a box stop at its level's order; a shift or a
 *                translation keeps the terms both sides hold (an M2L between
 *                boxes of orders p_s, p_t keeps |alpha| <= p_s, |beta| <= p_t,
 *                |alpha| + |beta| <= max(p_s, p_t)).  The tensor-core M2L
 *                needs a single order; with p_min the SIMT form runs. */
typedef struct {
    int p;
    int leaf_size;
    double eta;
    int max_level;
    int leaf_descend;
    int precision;
    int n_duffy;
    double tau_near;
    int max_subdiv;
    int p_min;
} bem_fmm_params;

typedef struct {
    int restart;      /* GMRES restart length (30) */
    double tol;       /* stop when ||b - A x|| / ||b|| <= tol */
    int max_iter;     /* total Arnoldi steps (GMRES) or iterations (BiCGStab) allowed */
    int method;       /* BEM_GMRES (default) or BEM_BICGSTAB (bem_solve only) */
} bem_solve_params;

#define BEM_GMRES 0
#define BEM_BICGSTAB 1   /* the paper's solver (Section 4): two products per iteration */

typedef struct {
    int iters;            /* Arnoldi steps taken */
    int restarts;         /* true-residual evaluations */
    double rel_residual;  /* last true relative residual */
    int status;           /* BEM_OK or BEM_ENOCONV */
} bem_solve_info;

/* Octree export for parity checks (Sections 3.1, 3.4, 3.6).  Call
 * bem_plan_tree_sizes() to fill the counts, allocate the arrays on the host,
 * then bem_plan_export_tree().  Boxes are numbered level by level. */
typedef struct {
    int64_t n_boxes, n_near, n_inter, n_nodes, n_elems;
    double lo[3], side;            /* root cube: lower corner and edge */
    int32_t *level;                /* [n_boxes] */
    int64_t *ijk;                  /* [n_boxes][3] integer box coordinates at its level */
    int32_t *parent;               /* [n_boxes], -1 for the root */
    int32_t *leaf;                 /* [n_boxes] 1 if leaf */
    double *centre;                /* [n_boxes][3] */
    double *radius;                /* [n_boxes] convergence radius r_C (Eq. 12 for parents) */
    int64_t *near_ptr, *near_idx;  /* CSR near-field lists */
    int64_t *inter_ptr, *inter_idx;/* CSR interaction lists */
    int64_t *leaf_of_node;         /* [n_nodes] leaf box of every vertex */
    int64_t *owner;                /* [n_elems] leaf owning each element (leaf of its node 0) */
} bem_tree_view;

/* Defaults: p 8, leaf_size 64, eta 2, max_level 20, leaf_descend 1, F64,
 * n_duffy 12, tau_near 2, max_subdiv 6. */
void bem_fmm_params_default(bem_fmm_params *params);
void bem_solve_params_default(bem_solve_params *params);

/* Context on one CUDA device.  Fails with BEM_ECUDA if the device is absent. */
int bem_ctx_create(int device, bem_ctx **out);
void bem_ctx_destroy(bem_ctx *ctx);

/* Message of the last failing call on this thread ("" if none). */
const char *bem_last_error(void);

/* Mesh of the surface S (Section 2.2), host side only (ctx may be NULL for a
 * mesh that is only inspected; bem_plan_create needs a context).
 * nodes: host float64 [n_nodes][3];
 * elems: host int32 [n_elems][3 or 6] node indices.  The Neumann data index
 * space is built here by the sharp-edge rule of Section 2.3: at every node,
 * element normals within edge_angle_deg of a cluster's first normal share one
 * chi index.  The potential phi keeps one index per node.
 * BEM_EINVAL on a bad element type, an out-of-range node index or a
 * degenerate element. */
int bem_mesh_create(bem_ctx *ctx, const double *nodes, int64_t n_nodes, const int32_t *elems,
                    int64_t n_elems, int elem_type, double edge_angle_deg, bem_mesh **out);
void bem_mesh_destroy(bem_mesh *mesh);

/* Keeps a device-resident copy of the mesh (nodes, elements, chi indices) on
 * the context's device, owned by the mesh, so that later bem_plan_create calls
 * read it from HBM instead of host memory.  Synchronises the stream. */
int bem_mesh_upload(bem_mesh *mesh, void *cuda_stream);

/* n_phi = number of nodes, n_chi = number of Neumann-data indices. */
int bem_mesh_sizes(const bem_mesh *mesh, int64_t *n_phi, int64_t *n_chi);

/* chi index of every (element, local node): host int32 [n_elems][npe]. */
int bem_mesh_chi_index(const bem_mesh *mesh, int32_t *elem_local_to_chi);

/* Builds on the device everything the matrix multiplication needs
 * (Section 3.6, set-up): quadrature geometry, the octree over vertices
 * (Morton codes, Section 3.1), element ownership, convergence radii
 * (Section 3.4, Eq. 12), near-field and interaction lists (Section 3.6),
 * the stored near-field correction for singular and near-singular pairs and
 * the diagonal C_i.  Blocks until done.  green: BEM_LAPLACE or
 * BEM_HELMHOLTZ with wavenumber k.  params NULL = defaults. */
int bem_plan_create(bem_mesh *mesh, int green, double k, const bem_fmm_params *params,
                    void *cuda_stream, bem_plan **out);
void bem_plan_destroy(bem_plan *plan);

/* One fast matrix multiplication (Section 3.6, steps 1-4) plus the stored
 * correction and the diagonal: op BEM_OP_A: y = C x - D x; BEM_OP_B: y = -S x.
 * x_dev: device [n_phi] (op A) or [n_chi] (op B); y_dev: device [n_phi].
 * Stream ordered; no host synchronisation. */
int bem_matvec(bem_plan *plan, int op, const void *x_dev, void *y_dev, void *cuda_stream);

/* The product of bem_matvec for callers that cannot allocate device memory at
 * the point of the call: real-time loops that must not synchronise the device
 * (which an allocation may do), or hosts whose device memory all belongs to
 * another allocator (a framework's pool) that forbids stray cudaMalloc calls.  The paper has no counterpart: this is an interface for
 * such callers.  Same arguments and result as bem_matvec; the kernels are
 * launched directly and their scratch (quadrature strengths, moments, local
 * expansions, regular sums) lives in one fixed 48 MiB device array of the
 * library instead of the plan's buffers.  Every GPU that loads the library
 * holds that array until the process exits.  The first call on a device looks
 * up the array's address, so make it before any stream capture.  BEM_EINVAL
 * (with the sizes in the message) if the plan needs more scratch than the
 * array holds.  All calls share the array: calls that overlap on the GPU race;
 * order them on one stream.  The result equals bem_matvec's bit for bit, and
 * the caller's current device is the same after the call as before. */
int bem_matvec_noalloc(bem_plan *plan, int op, const void *x_dev, void *y_dev, void *cuda_stream);

/* Solves A phi = B chi for nrhs right-hand sides: b = B chi by one
 * matrix multiplication, then restarted GMRES with float64 Arnoldi (CGS2),
 * Givens rotations and a true residual at every restart.  chi_dev: device
 * [nrhs][n_chi]; phi_dev: device [nrhs][n_phi] (written).  info: host array
 * of nrhs entries (may be NULL).  Returns BEM_ENOCONV if any right-hand side
 * stopped at max_iter; its best iterate is written.  Synchronises the stream
 * once per restart cycle.  A BEM_MIXED plan aims at max(tol, 1e-7), a little
 * above the float32 operator's residual floor (2-5e-8), and also stops when a whole
 * restart cycle fails to halve the true residual: that stop is BEM_OK when the
 * residual reached is at most max(tol, 1e-6) and BEM_ENOCONV above it
 * (bem_solve_stop_rule); info reports the residual reached. */
int bem_solve(bem_plan *plan, const void *chi_dev, void *phi_dev, int nrhs,
              const bem_solve_params *params, bem_solve_info *info, void *cuda_stream);

/* The decision bem_solve (GMRES and BiCGStab), bem_batch and bem_group take
 * after every true residual, as a host function without device work, so that
 * a caller or a test can check it.  precision: the plan's (BEM_F64 or
 * BEM_MIXED); tol, max_iter: the solve parameters; restarts: true residuals
 * evaluated so far, this one included; rel: this true relative residual
 * ||b - A x|| / ||b||; prev_rel: the previous one (any value above 2 rel on
 * the first); iters: Arnoldi steps (or iterations) taken.  Returns 1 when the
 * solve ends here and writes *status:
 *   rel <= tol (mixed: max(tol, 1e-7))                    -> BEM_OK;
 *   mixed, restarts > 1 and rel > prev_rel / 2 (a stall)  -> BEM_OK if
 *       rel <= max(tol, 1e-6), else BEM_ENOCONV;
 *   iters >= max_iter                                     -> BEM_ENOCONV.
 * Returns 0 (status untouched) when the solve goes on.  The paper's solver
 * (Section 4) stops on its tolerance alone; the stall rule is this library's
 * for float32 operators, whose rounding sets a residual floor. */
int bem_solve_stop_rule(int precision, double tol, int restarts, double rel, double prev_rel, int iters,
                        int max_iter, int *status);

/* Field of the surface data at points off the surface (Section 2.2,
 * accelerated field evaluation): u(x) = integral over S of
 * (phi dG/dn1 - G chi) dS, the representation of Eq. 1 with C(x) = 1 outside
 * the body (and 0 inside).  Tree descent from the root for every point: a box
 * whose centre is farther than eta r_C contributes its multipole expansion,
 * a nearer leaf is integrated directly (7-point rule, subdivided within
 * tau h_e of an element).  phi_dev [n_phi], chi_dev [n_chi] as for
 * bem_solve; pts_dev device f64 [npts][3]; u_dev device [npts] (complex
 * pairs for Helmholtz).  Points on the surface are not supported.  Stream
 * ordered; uses the plan's product work space (no product may run on the
 * plan at the same time).  A descent deeper than the kernel's stack sets
 * bem_plan_device_status to 2. */
int bem_field(bem_plan *plan, const void *phi_dev, const void *chi_dev, int64_t npts, const double *pts_dev,
              void *u_dev, void *cuda_stream);

/* Concurrent solves for request serving.  The paper solves one problem at a
 * time; a server keeps many plans resident and advances their solves together
 * so that the device work of small problems overlaps.  A batch owns
 * max_slots CUDA streams; each submitted solve (b = B chi, then the GMRES of
 * bem_solve) runs on its slot's stream as a sequence of device steps, and the
 * host only reads back a few scalars asynchronously.  Submissions may arrive
 * at any time while other solves are in flight (continuous batching).
 *   bem_batch_submit   starts a solve in a free slot; BEM_EBUSY if no slot is
 *                      free or the plan already has a solve in this batch (a
 *                      plan holds the work space of one solve).  chi_dev and
 *                      phi_dev must stay alive until the slot is released;
 *                      chi_dev must already hold its data (the slot streams
 *                      do not wait on other streams), and the plan takes no
 *                      other product or solve until the slot is released.
 *   bem_batch_progress non-blocking: advances every solve whose pending device
 *                      work has finished; *n_active = solves still running.
 *   bem_batch_poll     *done = 1 when the slot's solve ended (all its device
 *                      work, phi_dev included, is then complete); info as
 *                      bem_solve.
 *   bem_batch_wait     blocks until the slot ends or timeout_s passes
 *                      (BEM_ETIMEOUT; the solve keeps running).
 *   bem_batch_release  frees a finished slot (BEM_EBUSY while running).
 *   bem_batch_stream   the slot's stream (cudaStream_t), e.g. to build the
 *                      next request's plan without waiting for others. */
typedef struct bem_batch bem_batch;
int bem_batch_create(bem_ctx *ctx, int max_slots, bem_batch **out);
void bem_batch_destroy(bem_batch *batch);
int bem_batch_submit(bem_batch *batch, bem_plan *plan, const void *chi_dev, void *phi_dev,
                     const bem_solve_params *params, int *slot);
int bem_batch_progress(bem_batch *batch, int *n_active);
int bem_batch_poll(bem_batch *batch, int slot, int *done, bem_solve_info *info);
int bem_batch_wait(bem_batch *batch, int slot, double timeout_s);
int bem_batch_release(bem_batch *batch, int slot);
void *bem_batch_stream(bem_batch *batch, int slot);

/* Group solves: many plans -- meshes of uneven size, either Green's function,
 * either precision -- solved together in lock step.  Every member's restart
 * cycle (the Arnoldi steps with their fast products, the update and the true
 * residual) is captured once into one CUDA graph with the members as parallel
 * branches, so each cycle of the whole group is a single graph launch; a
 * member that has converged is halted and its branch returns at once.  The
 * iterations, stopping rules and results are those of bem_solve.
 *   bem_group_create  plans: host array of nplans distinct plans (the group
 *                     keeps the pointers; destroy the group before them).
 *   bem_group_solve   chis / phis: host arrays of nplans device pointers
 *                     (chi_dev / phi_dev of bem_solve; a NULL pair leaves the
 *                     member out of this solve); info: host [nplans];
 *                     launches (optional): kernels launched.  Blocks until
 *                     every member has ended; BEM_ENOCONV if one did not
 *                     converge.  The graphs are captured on the first call
 *                     and again whenever restart or tol change. */
typedef struct bem_group bem_group;
int bem_group_create(bem_ctx *ctx, bem_plan *const *plans, int nplans, bem_group **out);
void bem_group_destroy(bem_group *group);
int bem_group_solve(bem_group *group, const void *const *chis, void *const *phis, const bem_solve_params *params,
                    bem_solve_info *info, long long *launches);

/* Tree export (see bem_tree_view).  Blocks. */
int bem_plan_tree_sizes(const bem_plan *plan, bem_tree_view *view);
int bem_plan_export_tree(const bem_plan *plan, bem_tree_view *view);

/* Stored near-field correction (special-rule minus regular-rule integrals of
 * singular and near-singular pairs) as host COO triplets.  counts[0] = nnz of
 * the double-layer part (columns: node index), counts[1] = nnz of the
 * single-layer part (columns: chi index).  Call with NULL arrays to get the
 * counts.  Values are returned as float64 (complex pairs for Helmholtz); a
 * mixed-precision plan holds and returns them rounded to float32. */
int bem_plan_export_correction(const bem_plan *plan, int64_t *counts, int64_t *rowD, int64_t *colD,
                               double *valD, int64_t *rowS, int64_t *colS, double *valS);

/* Multipole moments and local expansions left by the last bem_matvec, per
 * box (level-by-level numbering) and multi-index, unscaled, float64 (complex
 * pairs for Helmholtz); mnk: host int32 [n_p][3] multi-indices.  Blocks.
 * The product forms moments only at levels at or below the coarsest level
 * holding an interaction-list source, and locals only at or below the
 * coarsest level holding an interaction-list target (coarser ones never
 * reach the result); the values exported for coarser boxes are unspecified. */
int bem_plan_export_expansions(const bem_plan *plan, int32_t *mnk, double *moments, double *locals);

/* Diagonal C_i = 1 + sum_j D0_ij (Eq. 2-3) as computed at set-up: host [n_phi]. */
int bem_plan_diagonal(const bem_plan *plan, double *c);

/* Device memory held by the plan, in bytes. */
int bem_plan_footprint(const bem_plan *plan, size_t *hbm_bytes);

/* Device-side status of the plan's kernels (blocks until the device is idle):
 * 0, or 1 when a kernel's bounded wait on the tensor cores gave up (that
 * kernel then stopped early and its product is incomplete), or 2 when a field
 * evaluation's descent stack was full (a branch was skipped). */
int bem_plan_device_status(const bem_plan *plan, int *status);

/* Most device memory the plan has held at any one time, in bytes: set-up
 * allocates temporaries (the diagonal's higher-order product) and the first
 * solve adds the Krylov basis, so this is what admission control must reserve. */
int bem_plan_peak_footprint(const bem_plan *plan, size_t *hbm_bytes);

/* Integer counters of the plan (host array of BEM_NSTATS): [0] n_boxes,
 * [1] n_leaves, [2] n_levels, [3] near-list entries, [4] interaction-list
 * entries, [5] near-field source-target pairs per matrix multiplication,
 * [6] correction nnz (D), [7] correction nnz (S), [8] quadrature points,
 * [9] n_p, [10] / [11] kernels in the captured op A / op B product graph (0
 * until the first product), [12] 1 when the M2L runs on the tensor cores
 * (tcgen05), 0 for the SIMT form, [13] canonical offset classes of the
 * interaction pairs. */
#define BEM_NSTATS 14
int bem_plan_stats(const bem_plan *plan, int64_t *stats);

/* Stages of one product, in launch order, for bem_plan_stage_times. */
#define BEM_NSTAGES 7   /* P2Q, P2M, M2M, M2L, L2L, near field + L2P, correction + diagonal */

/* Runs the product y = op x `reps` times outside its graph with CUDA events
 * between the stages on the given stream and returns the mean duration of each
 * stage in milliseconds (host array of BEM_NSTAGES).  Synchronises. */
int bem_plan_stage_times(bem_plan *plan, int op, const void *x_dev, void *y_dev, int reps, double *ms,
                         void *cuda_stream);

/* Stages of bem_plan_create, for bem_plan_setup_times. */
#define BEM_NSETUP 7   /* mesh upload, octree, geometry + radii + lists, special-pair correction,
                          offset classes, diagonal + translation tables, stats */

/* Milliseconds of every set-up stage of the plan (host array of BEM_NSETUP).
 * Upload, octree, geometry and stats are wall clock with the stream
 * synchronised at each boundary.  The correction and the diagonal are GPU
 * spans on two streams that overlap; the offset classes are host time spent
 * while the correction runs. */
int bem_plan_setup_times(const bem_plan *plan, double *ms);

/* Kernel launches issued by this library in this process so far (a graph
 * launch counts the kernels it holds). */
int bem_launch_count(long long *count);

/* Measured fused multiply-add throughput of the current device in TFLOP/s
 * (kind 0: float32, kind 1: float64; 2 flops per FMA), the denominator of
 * the arithmetic rooflines.  Measurement infrastructure: the paper has no
 * counterpart.  Synchronises. */
int bem_measure_peak(int kind, double *tflops, void *cuda_stream);

#ifdef __cplusplus
}
#endif
#endif /* BEM_H */
