/*
 * hdd.h -- C ABI of the GB300 HDD likelihood library (libhdd.so).
 *
 * Hierarchical domain decomposition (HDD) for -div(kappa grad u) = f on the unit
 * square, P1 elements on an N x N vertex grid, homogeneous Dirichlet data, with
 * kappa = exp(q(x, Z)) and q a KL expansion in the parameters Z (Sec. 1.1,
 * Eq. elliptic; notation table: kappa = e^q).  For a batch of parameter vectors Z
 * the library returns u at a few observation vertices and the Gaussian
 * log-likelihood of observed data y (Sec. 1.2), without forming the full solution:
 *
 *   hdd_plan         decomposition tree, index maps and launch schedule (Sec. 2.1)
 *   hdd_assemble     kappa per triangle for each sample            (Sec. 3.1)
 *   hdd_upsweep      "Leaves to Root": Schur maps of every node    (Sec. 2.4, 3.3, 3.4)
 *   hdd_point_solve  pruned "Root to Leaves" to the observation vertices (Sec. 3.4, 5.3)
 *   hdd_loglik       Gaussian data-misfit log-likelihood           (Sec. 1.2)
 * and, on the same factors:
 *   hdd_solve_loads      many load vectors at a fixed kappa         (Sec. 2)
 *   hdd_subdomain_means  mean of u over every subdomain of the tree (Sec. 5, 5.1)
 *
 * Conventions shared by every call
 *   - Vertex (i, j) of the grid sits at (i h, j h), h = 1/(N-1), flat id j*N + i.
 *     Cell (i, j) is split by its "/" diagonal into triangle 2*(j*(N-1)+i) (lower
 *     right, right angle at (i+1, j)) and triangle 2*(j*(N-1)+i)+1 (upper left,
 *     right angle at (i, j+1)).
 *   - "device" pointers are CUDA global memory of the plan's device; "host"
 *     pointers are ordinary (pageable or pinned) CPU memory.
 *   - The caller owns every buffer it passes.  The library owns the plan and the
 *     device copies it makes in hdd_plan, and allocates nothing else: all scratch
 *     lives in the caller's workspace (size from hdd_workspace_size).
 *   - Device work is enqueued on `stream` (a cudaStream_t; NULL = legacy default
 *     stream) and is asynchronous.  A return value covers argument and launch
 *     errors only; numerical failures are reported per sample by hdd_loglik.
 *   - No call throws, traps or aborts.  Calls on one plan may run concurrently
 *     from several threads if each uses its own workspace.
 *   - The workspace passed to hdd_upsweep / hdd_point_solve / hdd_loglik must be
 *     the one hdd_assemble filled, with the same batch.
 */
#ifndef HDD_H
#define HDD_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct hdd_plan_s* hdd_plan_t;

typedef enum {
  HDD_OK = 0,
  HDD_EINVAL = -1,    /* bad argument (size, pointer, observation on the boundary ...) */
  HDD_ENOMEM = -2,    /* host or device allocation inside hdd_plan failed */
  HDD_ECUDA = -3,     /* a CUDA call failed; hdd_last_error() has the text */
  HDD_ENOTSPD = -4,   /* per sample: a pivot of a Schur block was not positive */
  HDD_ENOCONV = -5,   /* per sample: iterative refinement did not reach ir_tol */
  HDD_ETIMEOUT = -6,  /* per sample: a bounded device wait gave up (hdd_set_wait_bound) */
  HDD_ESTATE = -7     /* call needs a device plan but the plan is host-only */
} hdd_status;

typedef enum {
  HDD_FP64 = 0,       /* every step in FP64 */
  HDD_MIXED_FP32 = 1  /* FP32 Schur factorisation + FP64-residual iterative refinement */
} hdd_precision;

typedef enum {
  HDD_OBS_VERTEX = 0,  /* observations are u at vertices (obs_vertex: flat vertex ids) */
  HDD_OBS_MEANS = 1    /* observations are the mean values of u over subdomains of the tree
                          (Sec. 5, Eq. mean); obs_vertex then holds tree node ids */
} hdd_obs_kind;

typedef struct {
  int32_t N;                  /* vertices per side, N >= 3 */
  int32_t leaf;               /* leaf size in cells per side, >= 1 */
  int32_t n_z;                /* KL terms, 1..256 */
  const double* kl_basis;     /* host, [n_t x n_z] row-major, n_t = 2 (N-1)^2, already scaled
                                 by sqrt(lambda_k); copied by hdd_plan (may be NULL for a
                                 host-only plan) */
  double f;                   /* constant right-hand side f */
  int32_t n_obs;              /* observation count, >= 1 */
  const int32_t* obs_vertex;  /* host, [n_obs] flat vertex ids j*N+i; every one must be an
                                 interior vertex (1 <= i, j <= N-2), else HDD_EINVAL */
  double sigma;               /* noise standard deviation, > 0 */
  int32_t precision;          /* hdd_precision */
  int32_t ir_max_iter;        /* mixed only: refinement steps after the first solve (0..64) */
  double ir_tol;              /* mixed only: target relative error at the observations, estimated
                                 after the last step as d_K min(1, d_K / d_{K-1}) / max_k |u_k|
                                 with d = max_k |du_k| over the observations */
  int32_t fp64_top_levels;    /* mixed only: tree depths 0..fp64_top_levels-1 are factorised in FP64 */
  int32_t fuse_height;        /* 0: off; else the largest height (<= 6) of bottom subtrees eliminated
                                 by one CTA each with their Schur complements kept on chip */
  int32_t device;             /* CUDA device ordinal, or -1 for a host-only plan that supports
                                 the hdd_plan_info / hdd_node_info queries and nothing else */
  int32_t obs_kind;           /* hdd_obs_kind.  HDD_OBS_MEANS: obs_vertex[k] is a node id of the
                                 decomposition tree (the numbering of hdd_node_info, which a
                                 host-only plan of the same N and leaf reports; node 0 = Omega),
                                 and observation k is the mean of u over that node's rectangle.
                                 The point solve then computes the mean functionals of Sec. 5.1
                                 (Lemma, Eq. prop1/prop2) and descends only to the observed
                                 nodes' ancestors (Sec. 5.2 Remark b): see hdd_point_solve. */
} hdd_plan_desc;

typedef struct {
  int32_t n_nodes;            /* nodes of the decomposition tree (node 0 = Omega) */
  int32_t n_leaves;
  int32_t depth;              /* max depth (root = 0) */
  int32_t height;             /* height of the root (leaves = 0) */
  int32_t n_visited;          /* nodes on the root-to-observation paths (Sec. 5.3) */
  int32_t max_front;          /* largest front m + b + 1 */
  double flops_upsweep;       /* algorithmic flops per sample of hdd_upsweep */
  double flops_point_solve;   /* algorithmic flops per sample of one pruned descent */
  double factor_bytes;        /* per sample, bytes of stored factors */
  double schur_bytes;         /* per sample, peak bytes of live Schur complements */
  int32_t launches_upsweep;   /* kernel launches of one hdd_upsweep */
  int32_t launches_evaluate;  /* kernel launches of assemble + upsweep + point solve + loglik */
  /* Algorithmic bytes per sample, each input read once and each output written
   * once: the roofline denominators of the stages.  Upsweep fronts read their
   * sons' lower Schur triangles (leaves: their triangles' kappa) and write the
   * factor columns, y_g and their own lower Schur triangle; they are split by
   * the kernel class that runs them: fronts of up to 32 rows (one warp each),
   * up to 128 rows in FP32 / 160 in FP64 (one CTA each in shared memory),
   * larger ones (global-memory path), fused subtrees. */
  double bytes_upsweep_tiny;
  double bytes_upsweep_small;
  double bytes_upsweep_large;
  double bytes_upsweep_fused;
  double bytes_forward;          /* one right-hand-side sweep over every node */
  double bytes_descent_all;      /* one descent over every node */
  double bytes_descent_visited;  /* one pruned descent (Sec. 5.3) */
  double bytes_residual;         /* one FP64 residual r = b - A u */
  double bytes_assemble;         /* kappa written (FP64, plus the FP32 copy of mixed plans) and Z read */
  double bytes_kl_basis;         /* the KL basis, read once per hdd_assemble call */
  double bytes_upsweep_leaf;     /* condensed leaves (at most 16 interior vertices): kappa in; K_gg^-1,
                                    the boundary couplings, y_g and the lower Schur triangle out */
  int32_t n_condensed_leaves;    /* leaves stored as K_gg^-1 and boundary couplings instead of factors */
  int32_t sweep_fuse_height;     /* height of the bottom subtrees whose full sweeps run fused (0: none;
                                    hdd_set_sweep_fusion) */
} hdd_plan_info_t;

typedef struct {
  int32_t x0, x1, y0, y1;     /* closed rectangle in vertex indices */
  int32_t parent, child0, child1;   /* -1 where absent */
  int32_t depth, height;
  int32_t m;                  /* eliminated vertices: |gamma| (interface), or leaf interior */
  int32_t b;                  /* boundary unknowns |I(d omega)| without Dirichlet vertices */
  int32_t visited;            /* 1 if the pruned descent computes this node's gamma */
} hdd_node_info_t;

/* Build a plan (Sec. 2.1: binary tree, longer side split at the cell-aligned
 * midpoint, x first on ties, leaves of at most `leaf` x `leaf` cells).  On
 * success *out owns host tables and, for device >= 0, device copies of the KL
 * basis, node tables and index maps.  Errors: HDD_EINVAL, HDD_ENOMEM, HDD_ECUDA. */
hdd_status hdd_plan(const hdd_plan_desc* desc, hdd_plan_t* out);

/* Release a plan and its device memory.  NULL is accepted.  The caller must make
 * sure no work that uses the plan is still in flight. */
hdd_status hdd_plan_destroy(hdd_plan_t plan);

/* Bytes of device workspace for `batch` samples (batch >= 1). */
hdd_status hdd_workspace_size(hdd_plan_t plan, int32_t batch, size_t* bytes);

/* Assembly (Sec. 3.1, Eq. coefA, Eq. coefc; kappa = e^q): for each sample s and
 * triangle t, q = sum_k Phi[t,k] Z[s,k] and kappa = exp(q), written to the
 * workspace -- in FP64 for FP64 plans, in double-float arithmetic (FP32 pairs,
 * ~1e-14 relative) for mixed plans, which also keep an FP32 copy; the per-triangle stiffness kappa_t |t| grad b_i . grad b_j is
 * formed from it by hdd_upsweep.  Z: device, [batch x n_z] row-major FP64.
 * workspace: device, >= hdd_workspace_size(plan, batch) bytes, 256-byte aligned. */
hdd_status hdd_assemble(hdd_plan_t plan, const double* Z, int32_t batch,
                        void* workspace, void* stream);

/* "Leaves to Root" (Sec. 3.4) with the Schur maps of Sec. 2.4 (Eq. SchurC1) and
 * the father system of Sec. 3.3 (Eq. block_equation4): at each leaf the interior
 * is eliminated; at each father the sons' boundary Schur complements are added
 * into the union of their boundaries, and the interface gamma is eliminated by a
 * partial Cholesky (L_gg L_gg^T = K_gg, L_Bg = K_Bg L_gg^-T,
 * S = K_BB - L_Bg L_Bg^T, right-hand side bordered as one more row).  The
 * factors (which represent Phi_omega) stay in the workspace. */
hdd_status hdd_upsweep(hdd_plan_t plan, int32_t batch, void* workspace, void* stream);

/* Pruned "Root to Leaves" (Sec. 3.4, Sec. 5.3): from the root down the nodes on
 * the paths to the observation vertices, u_gamma = L_gg^-T (y_g - L_Bg^T u_B);
 * then u at the observation vertices.  Mixed precision adds FP64-residual
 * iterative refinement (full descents).  u_obs: device, [batch x n_obs] FP64.
 * Plans that observe subdomain means (HDD_OBS_MEANS) descend only to the observed
 * nodes' ancestors, which gives u on each observed node's boundary, build the mean
 * functionals of the observed nodes and their subtrees leaves to root through the
 * stored factors (Sec. 5.1 Lemma with c_i = |omega_i| / |omega|: w = L_gg^-1 z_gamma,
 * lambda^g = z_B - L_Bg w, (lambda^f, c) = sum_i c_i (lambda^f_i, c) + w . y_g), and
 * return mean(omega) = (lambda^g, u on d omega) + (lambda^f, c) (Eq. prop1).  On refined
 * mixed plans the mean is Eq. mean of the refined iterate plus the functional of the
 * last correction; the refinement's convergence test runs on the observed nodes'
 * boundary unknowns.
 * Refinement reuses the stored y_gamma for its correction sweeps, so on mixed
 * plans call it once per hdd_upsweep (FP64 plans leave y_gamma unchanged). */
hdd_status hdd_point_solve(hdd_plan_t plan, int32_t batch, void* workspace, double* u_obs,
                           void* stream);

/* Likelihood of Sec. 1.2 with i.i.d. N(0, sigma^2) noise:
 * loglik[s] = -1/2 sum_k (y_k - u_k)^2 / sigma^2 - (n_obs/2) log(2 pi sigma^2).
 * u_obs: device [batch x n_obs] from hdd_point_solve.  y: device, [n_obs]
 * (y_per_sample = 0) or [batch x n_obs] (y_per_sample = 1).  loglik: device
 * [batch] FP64.  sample_status: device [batch] int32 or NULL; 0 = ok, otherwise
 * (-code) | (node << 8) with code a negative hdd_status (HDD_ENOTSPD, HDD_ENOCONV,
 * HDD_ETIMEOUT) and node the first failing tree node.  A failed sample gets
 * loglik = -inf. */
hdd_status hdd_loglik(hdd_plan_t plan, int32_t batch, void* workspace, const double* u_obs,
                      const double* y, int32_t y_per_sample, double* loglik,
                      int32_t* sample_status, void* stream);

/* End to end with HOST buffers: copies Z (host [batch x n_z]) and y (host) to the
 * workspace, runs assemble, upsweep, point solve and loglik on `stream`, copies
 * loglik (host [batch]), u_obs (host [batch x n_obs], may be NULL) and
 * sample_status (host [batch], may be NULL) back, and waits for the stream.
 * Blocking. */
hdd_status hdd_evaluate_host(hdd_plan_t plan, int32_t batch, void* workspace,
                             const double* Z, const double* y, int32_t y_per_sample,
                             double* loglik, double* u_obs, int32_t* sample_status,
                             void* stream);

/* Multiple loads at a fixed coefficient field (Sec. 2: the operators of every
 * node are computed once, by hdd_upsweep, and then applied to any number of
 * right-hand sides).  For each sample and each of its n_loads load vectors c,
 * solves K u = c over the unknowns through the stored factors: a right-hand-side
 * sweep ("Leaves to Root" with the stored L_gg, L_Bg: y_g = L_gg^-1 c_g,
 * condensed load c_B - L_Bg y_g), then "Root to Leaves" over every node.  Mixed
 * plans add ir_max_iter refinement steps (FP64 residual c - K u over all
 * unknowns, a correction solve through the same factors) and mark a sample
 * HDD_ENOCONV when the last correction, scaled by the observed contraction,
 * exceeds ir_tol * max |u| (the test hdd_point_solve applies at the
 * observation vertices).
 *   c: device [batch x n_loads x N^2] FP64, the assembled load per vertex
 *      c_i = sum_{t containing x_i} |t|/3 f(x_i) (Eq. coefc), i.e. h^2 f(x_i)
 *      at the interior vertices of this mesh; entries at boundary vertices are
 *      ignored.
 *   u: device [batch x n_loads x N^2] FP64, written at every vertex (0 on the
 *      boundary: Dirichlet data g = 0).
 *   sample_status: device [batch] int32 or NULL, as in hdd_loglik (it also
 *      carries the HDD_ENOTSPD flags of the upsweep).
 * Needs the workspace of hdd_assemble + hdd_upsweep with the same batch.  It
 * overwrites the stored y_gamma and the workspace's solution vectors: run
 * hdd_point_solve for the plan's own load before it, or hdd_upsweep again
 * after it. */
hdd_status hdd_solve_loads(hdd_plan_t plan, int32_t batch, void* workspace, const double* c, int32_t n_loads,
                           double* u, int32_t* sample_status, void* stream);

/* Many loads AND Dirichlet data at a fixed coefficient field, the load given on the
 * fine grid or on the coarse grid H = 2h (Sec. 2: the operators of every node are
 * computed once and applied to any number of right-hand sides and boundary data,
 * u|_gamma = Phi(u|_dOmega, f); Sec. 3.5: a smooth right-hand side discretised on a
 * coarser mesh, f in V_H, a subspace of V_h).  For each sample and each of its n_loads
 * data sets it solves A_II u_I = c_I - A_IB g_B and sets u_B = g_B, in correction form:
 * u = g on the boundary, 0 inside; r = c - A u (FP64 five-point residual, boundary
 * neighbours contributing g); d = the HDD solve of r through the stored factors (a
 * right-hand-side sweep "Leaves to Root", then "Root to Leaves" over every node);
 * u += d.  Mixed plans repeat the last three steps ir_max_iter more times (iterative
 * refinement) and flag HDD_ENOCONV as hdd_solve_loads does.  The loads of a sample go
 * through the sweeps in groups of four: each node's factors are read once per group and
 * applied to all four right-hand sides.
 *   c:        device [batch x n_loads x N^2] FP64 assembled loads c_i = sum_{t at x_i}
 *             |t|/3 f(x_i) (Eq. coefc; h^2 f(x_i) on this mesh), boundary entries ignored;
 *             or NULL when f_coarse is given.
 *   f_coarse: device [batch x n_loads x NH^2] FP64 nodal values of f on the coarse grid,
 *             NH = (N+1)/2 vertices per side (N odd), coarse vertex (a, b) at fine vertex
 *             (2a, 2b); the load is the vertex quadrature of its fine P1 interpolant; or
 *             NULL when c is given.  Exactly one of c and f_coarse.
 *   g:        device [batch x n_loads x N^2] FP64 Dirichlet data at the boundary vertices
 *             (interior entries ignored), or NULL for g = 0.
 *   u:        device [batch x n_loads x N^2] FP64, the solution at every vertex.
 *   scratch:  device, >= hdd_data_scratch_size(plan, batch) bytes, 256-byte aligned,
 *             caller-owned (the group's residuals and corrections).
 *   sample_status: device [batch] int32 or NULL, as in hdd_loglik.
 * Needs the workspace of hdd_assemble + hdd_upsweep with the same batch; it overwrites
 * the slots the right-hand-side sweep uses (not y_g, not the factors).
 * Errors: HDD_EINVAL (both or neither of c and f_coarse, f_coarse with an even N,
 * n_loads < 1, NULL or unaligned buffers). */
hdd_status hdd_data_scratch_size(hdd_plan_t plan, int32_t batch, size_t* bytes);
hdd_status hdd_solve_data(hdd_plan_t plan, int32_t batch, void* workspace, void* scratch, const double* c,
                          const double* f_coarse, const double* g, int32_t n_loads, double* u,
                          int32_t* sample_status, void* stream);

/* Mean of u over every subdomain omega of the tree (Sec. 5, Eq. mean):
 * mean(omega) = sum_{t in omega} |t|/3 (u_1 + u_2 + u_3) / |omega|, computed at
 * the leaves from u and at each father from its sons as in Sec. 5.1,
 * mean(omega) = c_1 mean(omega_1) + c_2 mean(omega_2), c_i = |omega_i| / |omega|.
 *   u: device FP64, sample s at u + s * u_stride, N^2 values (vertex j*N + i),
 *      e.g. from hdd_solve_loads; u_stride >= N^2.
 *   means: device [batch x n_nodes] FP64, in the node numbering of
 *      hdd_node_info (node 0 = the root, the whole domain).
 * Needs no workspace.  One launch per tree height. */
hdd_status hdd_subdomain_means(hdd_plan_t plan, int32_t batch, const double* u, int64_t u_stride, double* means,
                               void* stream);

/* Evaluation without any allocation and without a caller workspace.  The paper
 * has no counterpart: this entry point exists for callers that cannot allocate
 * device memory at evaluation time -- for example a host application whose whole
 * device memory is reserved at start-up by another framework's pool, a plug-in
 * that is given no allocator, or a latency-critical sampling loop that must not
 * call cudaMalloc/cudaFree (those calls can synchronize the device).
 *
 * It runs the same kernels as hdd_assemble + hdd_upsweep + hdd_point_solve +
 * hdd_loglik, with the workspace placed in one static device array of
 * HDD_STATIC_WORKSPACE_BYTES that every GPU which loads the library holds until
 * the process exits.  It calls no cudaMalloc, cudaFree or other allocating
 * routine.  Z: device [batch x n_z]; y: device [n_obs] or [batch x n_obs];
 * loglik: device [batch]; u_obs: device [batch x n_obs] or NULL; sample_status:
 * device [batch] or NULL.  Returns HDD_EINVAL if hdd_workspace_size(plan, batch)
 * exceeds HDD_STATIC_WORKSPACE_BYTES.
 *
 * The first call on a device looks up the array's device address (with that
 * device current); make that first call before any stream capture.  All calls
 * share the one array and each call overwrites it (the per-sample status words
 * are cleared at the start of every call): calls whose GPU work overlaps --
 * on different streams, or from several threads -- race with each other.  */
#define HDD_STATIC_WORKSPACE_BYTES ((size_t)32 << 20)
hdd_status hdd_evaluate_static(hdd_plan_t plan, int32_t batch, const double* Z, const double* y,
                               int32_t y_per_sample, double* loglik, double* u_obs, int32_t* sample_status,
                               void* stream);

/* The mean functionals of the observed nodes of a plan with obs_kind = HDD_OBS_MEANS
 * (Sec. 5.1 Lemma: mean(omega) = (lambda^g, u on the boundary unknowns of omega) +
 * (lambda^f, load inside omega), Eq. prop1), as the last hdd_point_solve on this
 * workspace left them:
 *   lambda_g: device [batch x sum_k b_k] FP64 or NULL: lambda^g of each observed node,
 *             nodes in observation order, b_k entries each in the order of
 *             hdd_node_indices(bnd);
 *   mu_f:     device [batch x n_nodes] FP64 or NULL: mu^f = (lambda^f, c) of every node
 *             whose functional was built (the observed nodes and their subtrees), with c
 *             the load the stored y_g carry: the plan's load on FP64 plans and on mixed
 *             plans without refinement, the last refinement residual otherwise (the
 *             functional of the last correction).
 * On mixed plans both come from the FP32 factors.  Errors: HDD_ESTATE for other plans. */
hdd_status hdd_mean_functionals(hdd_plan_t plan, int32_t batch, void* workspace, double* lambda_g, double* mu_f,
                                void* stream);

/* Uneven batches: several plans evaluated together, "Leaves to Root" as one launch
 * per tree height and front class over the nodes of all of them.  An uneven
 * workload mixes grids of 129^2 to 1025^2 with different KL bases and observation
 * sets; run one plan at a time, the upper tree levels of each leave most of the GPU
 * idle, while one launch per height over every plan fills it.  The paper has no
 * counterpart (its algorithms treat one problem): the arithmetic per sample is the
 * same as for the plan alone, so every result equals the plan's own.
 *
 * hdd_multi_create binds n_plans plans (same device, no fused subtrees), each with its
 * batch size and its workspace (>= hdd_workspace_size(plan, batch) bytes, 256-byte
 * aligned, caller-owned, used by later calls until hdd_multi_destroy).  It copies the
 * plans' node tables and maps into one device table; the plans must outlive it.
 * Errors: HDD_EINVAL, HDD_ENOMEM, HDD_ECUDA. */
typedef struct hdd_multi_s* hdd_multi_t;
hdd_status hdd_multi_create(const hdd_plan_t* plans, int32_t n_plans, const int32_t* batches,
                            void* const* workspaces, hdd_multi_t* out);
hdd_status hdd_multi_destroy(hdd_multi_t multi);
/* "Leaves to Root" of every bound plan on its workspace (after hdd_assemble of each):
 * the same factors and Schur complements as hdd_upsweep per plan. */
hdd_status hdd_multi_upsweep(hdd_multi_t multi, void* stream);
/* End to end on device buffers, arrays of n_plans pointers in binding order:
 * hdd_assemble per plan, hdd_multi_upsweep, then hdd_point_solve and hdd_loglik per
 * plan.  The per-plan phases run on streams that hdd_multi_create made (one per plan),
 * forked from `stream` and joined back to it by events, so the call is ordered on
 * `stream` like any other and the plans' small launches overlap on the device.  Z[q]: [batch_q x n_z_q]; y[q]: [n_obs_q] or [batch_q x n_obs_q] per
 * y_per_sample[q]; loglik[q]: [batch_q]; u_obs[q]: [batch_q x n_obs_q] (required);
 * sample_status: NULL or an array whose entries are NULL or [batch_q]. */
hdd_status hdd_multi_evaluate(hdd_multi_t multi, const double* const* Z, const double* const* y,
                              const int32_t* y_per_sample, double* const* loglik, double* const* u_obs,
                              int32_t* const* sample_status, void* stream);
/* The whole hdd_multi_evaluate of these buffers recorded once as a CUDA graph (stream
 * capture of the call: its assembly, one launch per height and front class of the
 * upsweep, the per-plan point solves and likelihoods, and the fork and join of the
 * plan streams) and instantiated, so that later evaluations of the same batch shape
 * replay it with one hdd_graph_launch instead of issuing each launch from the host.
 * The graph keeps the pointers it was captured with: new parameters are written into
 * the same Z[q] (and y[q]) buffers before a launch, and the results appear in the same
 * loglik[q], u_obs[q] and sample_status[q].  Arguments as for hdd_multi_evaluate; the
 * multi handle and its workspaces must outlive the graph, and no other work of the
 * multi handle may run while a launch of the graph is in flight.  Nothing runs during
 * the capture itself.  Errors: those of hdd_multi_evaluate, HDD_ENOMEM, HDD_ECUDA
 * (capture or instantiation refused). */
typedef struct hdd_graph_s* hdd_graph_t;
hdd_status hdd_multi_capture(hdd_multi_t multi, const double* const* Z, const double* const* y,
                             const int32_t* y_per_sample, double* const* loglik, double* const* u_obs,
                             int32_t* const* sample_status, hdd_graph_t* out);
/* One replay of a captured evaluation, ordered on `stream`.  Errors: HDD_EINVAL, HDD_ECUDA. */
hdd_status hdd_graph_launch(hdd_graph_t graph, void* stream);
hdd_status hdd_graph_destroy(hdd_graph_t graph);
/* Kernel launches of one hdd_multi_upsweep and of one hdd_multi_evaluate. */
hdd_status hdd_multi_info(hdd_multi_t multi, int32_t* launches_upsweep, int32_t* launches_evaluate);

/* Copy of the coefficient field of the last hdd_assemble on this workspace:
 * kappa: device [batch x n_t] FP64 (triangle order as above).  For inspection
 * and tests. */
hdd_status hdd_kappa(hdd_plan_t plan, int32_t batch, void* workspace, double* kappa, void* stream);

/* Bounded device waits.  The tensor-core Schur update (large FP32 fronts of mixed
 * plans) waits on shared-memory barriers for its operand copies and its MMAs; each
 * wait polls at most `polls` times (default 2^24, far above any real wait) and then
 * gives up: the kernel issues no further copies or MMAs, waits with the same bound
 * for what it already issued, skips its output tile and marks the sample
 * HDD_ETIMEOUT (loglik = -inf).  No call of the library waits without a bound and
 * none traps.
 *   polls:        >= 1.
 *   stall_node, stall_sample: test hook, -1 = off.  When set, the copies of the
 *                 second operand chunk of that (node, sample) are never issued, so
 *                 its wait is certain to run out: this is how the timeout path is
 *                 tested without any fault.  Leave it off in production.
 * Applies to the plan's later hdd_upsweep calls.  Errors: HDD_EINVAL. */
hdd_status hdd_set_wait_bound(hdd_plan_t plan, uint32_t polls, int32_t stall_node, int32_t stall_sample);

/* Fused bottom subtrees of the full sweeps (the right-hand-side sweeps and the full
 * descents of the refinement, hdd_solve_loads): "Leaves to Root" on a new load and
 * "Root to Leaves" (Sec. 3.4) over every subtree of height <= h, where a subtree is a
 * node of height <= h whose father is higher, with all its descendants, run as one
 * kernel with one warp per (subtree, sample) that keeps the values of the subtree's
 * rectangle on chip; the levels above run as before.  h is the largest height
 * <= max_height whose subtrees qualify (every front with at most 32 eliminated
 * vertices and 128 rows, or a condensed leaf; one precision; the shared memory of
 * eight samples per CTA within 75 KiB); 0 = none.  Plans start with max_height = 2.
 * The arithmetic per node is the same elimination in another order of operations, so
 * results agree with the level-by-level sweeps to rounding.  Replaces device tables:
 * call it when no work of the plan is in flight.  hdd_plan_info reports the height
 * in use.  Errors: HDD_EINVAL (max_height outside 0..6), HDD_ENOMEM, HDD_ECUDA (the
 * plan then runs its sweeps level by level). */
hdd_status hdd_set_sweep_fusion(hdd_plan_t plan, int32_t max_height);

/* Per-kernel timing, for benchmarks.  Between hdd_profile_begin and
 * hdd_profile_end every kernel the library launches for this plan is bracketed
 * by a pair of CUDA events on its stream (a few microseconds of overhead per
 * launch).  hdd_profile_end waits for those events and returns, per kernel
 * family, the launches, the summed event time and the summed algorithmic flops
 * (2 per multiply-add: Cholesky m^3/3, TRSM (b+1) m^2/2, SYRK b(b+1)m/2 and
 * (b+1)m for the bordered row, per node and sample).  Not thread-safe: profile
 * a plan from one thread.  stats: host array of max_stats entries. */
typedef struct {
  char name[24];
  int32_t launches;
  double ms;
  double flops;
} hdd_kernel_stat_t;
hdd_status hdd_profile_begin(hdd_plan_t plan);
hdd_status hdd_profile_end(hdd_plan_t plan, hdd_kernel_stat_t* stats, int32_t max_stats, int32_t* n_stats);

/* Plan queries (work on host-only plans too). */
hdd_status hdd_plan_info(hdd_plan_t plan, hdd_plan_info_t* info);
hdd_status hdd_node_info(hdd_plan_t plan, int32_t node, hdd_node_info_t* info);
/* gamma: [m] and bnd: [b] vertex ids in the order the fronts use (either may be NULL). */
hdd_status hdd_node_indices(hdd_plan_t plan, int32_t node, int32_t* gamma, int32_t* bnd);

/* Static text for a status code; thread-local text of the last CUDA error. */
const char* hdd_status_string(hdd_status status);
const char* hdd_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* HDD_H */
