/*
 * sft.h -- C ABI of libsft, a GB300 (sm_103a) implementation of the
 * stochastic conservative field transfer: the control-variate Monte Carlo
 * approximation of the Galerkin projection (paper Sec. 4), with the source
 * field queried pointwise as a black box (here: P1 point location in a
 * uniform-grid-bucketed source mesh, Sec. 5.3) and the target mass-matrix
 * system solved to an FP64 residual tolerance (sft_cg_mode).
 *
 * Conventions shared by every entry point
 *  - Plain pointers and sizes only. A pointer is device memory when the
 *    matching `device_ptrs` / `out_device` flag is 1, host memory otherwise.
 *  - Handles own every device buffer they allocate; the caller owns its
 *    input arrays, which are copied at create time, and its output arrays.
 *  - Work is ordered on the CUDA stream given in the descriptor/options
 *    (NULL = the legacy default stream). Calls that return results to the
 *    host (statistics, status of the solve) synchronise that stream.
 *  - Errors are returned as sft_status; sft_last_error() gives a message for
 *    the calling thread. No C++ exception crosses the ABI.
 *  - Index types: int32 connectivity and element ids, int64 sizes.
 */
#ifndef SFT_H
#define SFT_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct sft_source_s* sft_source;
typedef struct sft_target_s* sft_target;
typedef struct sft_batch_s* sft_batch;
typedef struct sft_mlp_s* sft_mlp;

typedef enum {
    SFT_OK = 0,
    SFT_ERR_ARG = 1,            /* invalid argument (null, size, enum) */
    SFT_ERR_MESH = 2,           /* invalid mesh: connectivity, orientation, non-finite value */
    SFT_ERR_CUDA = 3,           /* a CUDA runtime call failed */
    SFT_ERR_OOM = 4,            /* device allocation failed */
    SFT_ERR_NOT_CONVERGED = 5,  /* the solve reached cg_max_iter iterations (FP32 inner
                                   steps in MIXED mode) or stagnated; u is the last iterate */
    SFT_ERR_OUTSIDE = 6,        /* strict mode: a query fell in an empty grid cell */
    SFT_ERR_DEVICE_STATUS = 7,  /* a kernel reported an error (bounded wait expired, bad index) */
    SFT_ERR_UNSUPPORTED = 8     /* valid request this build does not implement */
} sft_status;

/* Arithmetic of the sampling / location / residual part of a transfer.
 * FP32: samples, containment predicate, source evaluation and residual in
 * FP32 with compensated (two-sum) per-element partials; load vector, CG and
 * global reductions in FP64. FP64: everything in FP64. */
typedef enum { SFT_PREC_FP64 = 0, SFT_PREC_FP32 = 1 } sft_precision;

/* How the FP64 system M u = b of step 7 is solved (both stop on the true
 * FP64 residual ||b - M u||_2 <= cg_tol ||b||_2, which is computed in FP64).
 * MIXED: iterative refinement -- FP64 residual and solution, each correction
 * by the Chebyshev iteration in FP32 on the symmetrically Jacobi-scaled
 * matrix diag(M)^-1/2 M diag(M)^-1/2, whose spectrum lies in [1/2, 2]
 * (triangles) or [1/2, 5/2] (tetrahedra) for any P1 mass matrix: the interval
 * fixes the step count for each cycle's target, and FP32 inner solves are
 * safe.
 * FP64: Jacobi-preconditioned CG in FP64 throughout. */
typedef enum { SFT_CG_MIXED = 0, SFT_CG_FP64 = 1 } sft_cg_mode;

/* Where the N samples of a target element are drawn (Sec. 4 step 3). UNIFORM:
 * N independent uniform points (the paper's scheme). STRATIFIED: the element
 * is cut into m^d equal-measure strata, m the largest integer with
 * m^d <= N (the images of the cells of an m^d grid on the unit square / cube
 * under the uniform-to-simplex map), one uniform point in each, plus N - m^d
 * uniform points; every sample keeps the weight |T| / N, so the estimator
 * stays unbiased (Eq. mc_element_integral_operator_general) and its error
 * falls like N^-1 instead of N^-1/2 for a Lipschitz residual in 2D.
 * IMPORTANCE: the samples follow the non-uniform density p_t = (1/4 +
 * sum_{a<b} pi_e (d+1)(d+2) lambda_a lambda_b) / |T| (pi_e = 1/4 in 2D, 1/8
 * in 3D), a mixture of the uniform density and the edge-bubble densities
 * that the control-variate residual of a smooth field follows, and every
 * sample is weighted by 1 / (|T| p_t) <= 4 (Eq.
 * mc_element_integral_operator_general). Philox counters (j, t, stream, 6)
 * and (j, t, stream, 7) per sample. sft_transfer only (plain mode). */
typedef enum {
    SFT_SAMPLING_UNIFORM = 0,
    SFT_SAMPLING_STRATIFIED = 1,
    SFT_SAMPLING_IMPORTANCE = 2
} sft_sampling;

/* element type of coordinate / value arrays */
typedef enum { SFT_F32 = 0, SFT_F64 = 1 } sft_dtype;

/* A P1 simplex mesh (Sec. 2: the target FE space V_t; the source P1 field
 * "interpolated onto the source mesh" of Sec. 5.1). */
typedef struct {
    int32_t dim;            /* 2 (triangles) or 3 (tetrahedra) */
    int32_t nfields;        /* source: nodal fields carried (1..8); target: 0 */
    int64_t nnodes;
    int64_t nelems;
    const void* coords;     /* [nnodes][dim] of `dtype`, row-major */
    const int32_t* conn;    /* [nelems][dim+1], positively oriented */
    const void* values;     /* source: [nfields][nnodes] of `dtype`; target: NULL */
    int32_t dtype;          /* sft_dtype of coords and values */
    int32_t device_ptrs;    /* 1: coords/conn/values are device pointers */
    double grid_scale_L;    /* source: grid cells per axis = int(L * nelems^(1/dim)); <= 0 means 1 */
    void* cuda_stream;      /* cudaStream_t for the setup work */
} sft_mesh_desc;

/* Options of one transfer (Sec. 4 steps 1-7). */
typedef struct {
    int32_t samples_per_elem;   /* N >= 1 samples per target element */
    int32_t precision;          /* sft_precision */
    uint64_t seed;              /* Philox key */
    uint32_t stream_id;         /* Philox counter word 2 (independent sample streams) */
    int32_t cg_max_iter;        /* >= 0; bound on the solve's iterations (in MIXED mode the
                                   FP32 inner steps summed over the cycles); 0 skips the
                                   solve (u = 0) */
    double alpha;               /* control-variate parameter (Eq. cv_centered_integrand); 1 recommended */
    double cg_tol;              /* stop when ||b - M u||_2 <= cg_tol ||b||_2 */
    int32_t strict_inside;      /* 1: SFT_ERR_OUTSIDE when a query lands in an empty grid cell */
    int32_t out_device;         /* 1: u_out, b_out, g_out, sample_elem_out are device pointers */
    void* cuda_stream;          /* cudaStream_t */
    int32_t* sample_elem_out;   /* optional [nelems][N]: source element located for every sample */
    int32_t field_count;        /* 0: every source field; k > 0: the first k fields only */
    int32_t cg_mode;            /* sft_cg_mode (0: mixed-precision refinement) */
    int32_t sampling;           /* sft_sampling (0: uniform) */
    int32_t cg_warm_start;      /* 1: the solve starts from the values u_out holds (the previous
                                   transfer's result, say) instead of 0; needs cg_mode MIXED.
                                   The stopping test is unchanged (true FP64 residual relative
                                   to ||b||), so the result meets the same tolerance. */
    double adapt_ref_measure;   /* > 0: per-element sample counts N_t = min(8 N, max(1,
                                   ceil(N D_t / D_ref))), D_t = d! |T| (the edge determinant of
                                   the element's vertices in the path precision, in FP64) and
                                   D_ref = d! adapt_ref_measure: samples in proportion to the
                                   element's measure, N per reference measure (for a residual of
                                   uniform variance per unit measure the global sum's variance
                                   is lowest so); weights |T| / N_t. 0: N for every element.
                                   sft_transfer only (uniform or importance sampling);
                                   sample_elem_out is then [nelems][8 N], -1 past N_t. */
} sft_options;

typedef struct {
    int32_t cg_iters;           /* largest iteration count over the fields (MIXED: FP32
                                   inner steps summed over the cycles) */
    int32_t reserved;
    double cg_rel_resid;        /* largest final ||r||/||b|| over the fields */
    int64_t queries;            /* source queries issued: nodes (control) + the samples
                                   (nelems * N, or sum_t N_t with adapt_ref_measure) */
    int64_t fallback_queries;   /* queries no candidate accepted (nearest candidate used) */
    int64_t empty_queries;      /* queries that landed in an empty cell (value 0) */
    float ms_setup;             /* lazily built source/target structures inside this call */
    float ms_control;           /* step 1: control values g at the target nodes */
    float ms_assembly;          /* steps 2-6: fused sample / query / control / scatter kernel */
    float ms_solve;             /* step 7: CG */
    float ms_total;
    float reserved2;
} sft_stats;

/* Copy a source mesh and its nodal fields to the device and build the
 * uniform-grid point-location structure (Sec. 5.3: nx = ny = int(L sqrt(#elements)),
 * extended to 3D with the cube root) for the precision matching `dtype`
 * (F32 -> FP32 location, F64 -> FP64 location); the other precision is built
 * on first use. The exact P1 integral int f^s of every field is computed on
 * the first sft_conservation_error call (and again after new values).
 * Errors: SFT_ERR_ARG (null/size/dim/nfields), SFT_ERR_MESH (index out of
 * range, non-positive element, non-finite coordinate), SFT_ERR_OOM, SFT_ERR_CUDA. */
sft_status sft_source_create(const sft_mesh_desc* desc, sft_source* out);

/* Copy a target P1 mesh to the device and assemble its FP64 mass matrix
 * M_ki = int psi_k psi_i (Eq. mass_matrix; exact P1 quadrature, Sec. 2) in
 * CSR form, its Jacobi diagonal and lumped masses m_i = sum_k M_ik.
 * Errors as for sft_source_create. */
sft_status sft_target_create(const sft_mesh_desc* desc, sft_target* out);

/* Replace the nodal values of every field of a source (same shape and dtype
 * as at create: [nfields][nnodes]; device pointer if device_ptrs) keeping its
 * mesh and location grid: the per-coupling-step update of a fixed mesh
 * (the paper's online cost, Sec. 5.3). Ordered on cuda_stream; does not
 * synchronise it. */
sft_status sft_source_set_values(sft_source src, const void* values, int32_t device_ptrs, void* cuda_stream);

void sft_source_destroy(sft_source src);
void sft_target_destroy(sft_target tgt);

/* One transfer, Sec. 4 steps 1-7 (Eqs. cv_load_expanded and cv_galerkin_system):
 *   g   = source evaluated at the target nodes (step 1);
 *   b_i = alpha int g psi_i  +  sum_t |T|/N sum_j (f^s - alpha g)(X_tj) psi_i(X_tj)
 *         with X_tj uniform in t from Philox4x32-10 (steps 2-6; stratified
 *         with opt->sampling = SFT_SAMPLING_STRATIFIED);
 *   M u = b by the sft_cg_mode of opt->cg_mode, from u = 0 or, with
 *         opt->cg_warm_start, from the values u_out holds (step 7).
 * nfields = opt->field_count if > 0, else the source's field count.
 * u_out [nfields][nnodes_target] FP64 (required); b_out, g_out same shape,
 * optional (NULL). u_out is written on SFT_OK and SFT_ERR_NOT_CONVERGED.
 * stats may be NULL. Synchronises opt->cuda_stream before returning. */
sft_status sft_transfer(sft_source src, sft_target tgt, const sft_options* opt,
                        double* u_out, double* b_out, double* g_out, sft_stats* stats);

/* ---- mesh intersection (2D): the exact judge ----
 * Sec. 3, Intersection-Based Galerkin Projection: every target triangle is
 * partitioned by the source triangles it overlaps (Eq. partition_ts); each
 * piece is clipped (Sutherland-Hodgman), split into a fan from its first
 * vertex and integrated with the edge-midpoint rule, exact for the products
 * of two functions linear on the piece; all arithmetic FP64. A target
 * triangle's pieces are found by a walk over source face neighbours from
 * the source triangle holding its centroid (at most 256 source triangles
 * visited per target triangle, else SFT_ERR_UNSUPPORTED).
 * sft_mi_load_vector: the exact P1 load vector b_i = int psi_i f^s of source
 * field `field` (Eq. galerkin_system's right-hand side), b_out [nnodes_target]
 * FP64, a device pointer if out_device. sft_mi_l2_error: the supermesh L2
 * error of a target field u [nnodes_target] (FP64, device pointer if
 * u_on_device) against source field `field` (Eq. relative_L2_error):
 * out2[0] = ||f^s - f^t||_L2, out2[1] = ||f^s||_L2 (host array of 2).
 * Both need 2D meshes (SFT_ERR_UNSUPPORTED otherwise), return
 * SFT_ERR_OUTSIDE if a target centroid lies in no source triangle, and
 * synchronise `cuda_stream`. */
sft_status sft_mi_load_vector(sft_source src, sft_target tgt, int32_t field, double* b_out,
                              int32_t out_device, void* cuda_stream);
sft_status sft_mi_l2_error(sft_source src, sft_target tgt, int32_t field, const double* u,
                           int32_t u_on_device, void* cuda_stream, double* out2);

/* Relative conservation error (Eq. relative_conservation_error) of a target
 * field u [nnodes_target] (FP64; device pointer if u_on_device):
 *   out3[0] = |int f^s - int f^t| / |int f^s|, out3[1] = int f^s (field `field`
 *   of the source, exact P1 integral), out3[2] = int f^t = sum_i m_i u_i.
 * out3 is a host array of 3 doubles. Synchronises `cuda_stream`. Computes the
 * source integrals when the values changed since they were last computed, so
 * it must not run concurrently with other calls on the same source. */
sft_status sft_conservation_error(sft_source src, sft_target tgt, const double* u,
                                  int32_t u_on_device, int32_t field, void* cuda_stream,
                                  double* out3);

/* Black-box source query at arbitrary points (the step-4 query on its own):
 * pts [n][dim] FP64 (rounded to FP32 first when precision = FP32);
 * elem_out [n] located source element (-1: empty cell), val_out [nfields][n]
 * FP64 P1 value (may be NULL). Pointers are device memory if device_ptrs. */
sft_status sft_locate(sft_source src, int32_t precision, int64_t n, const double* pts,
                      int32_t device_ptrs, int32_t* elem_out, double* val_out,
                      void* cuda_stream);

/* Solve M u = b on the target (step 7 alone) for nrhs right-hand sides
 * b [nrhs][nnodes] -> u [nrhs][nnodes] (FP64), from u = 0, by the sft_cg_mode
 * `cg_mode`. max_iter bounds the iterations (FP32 inner Chebyshev steps
 * summed over the refinement cycles in MIXED mode). iters_out / rel_resid_out (host,
 * may be NULL) get the worst field; rel_resid is the true FP64 residual of the
 * returned u in MIXED mode, the recurrence residual in FP64 mode. */
sft_status sft_mass_solve(sft_target tgt, int32_t nrhs, const double* b, double* u,
                          int32_t device_ptrs, double tol, int32_t max_iter, int32_t cg_mode,
                          void* cuda_stream, int32_t* iters_out, double* rel_resid_out);

/* Limit of every device wait in the solves on this target (the grid barriers
 * of the cooperative CG kernels of step 7, Eq. cv_galerkin_system, reached
 * through sft_transfer, sft_plan_transfer and sft_mass_solve): a wait that
 * runs past it sets the kernel's error word, every block of the launch
 * returns, and the call reports SFT_ERR_DEVICE_STATUS; the stream and the
 * context stay usable. Default 2 s; `seconds` in (0, 3600], else SFT_ERR_ARG.
 * The paper has no counterpart (failure detection of the device path). */
sft_status sft_target_set_wait_limit(sft_target tgt, double seconds);

/* ---- batched transfers ----
 * Many requests (source, target, options) of uneven size run together: the
 * paper's per-request method (Sec. 4 steps 1-7) is unchanged; batching has no
 * counterpart in the paper. The plan groups requests by dimension and field
 * count, and records one CUDA graph: control values of every request, a
 * persistent fused assembly per group (warps pull (request, element-tile)
 * work items from an atomic counter), and one cooperative solve over the
 * block-diagonal system of every (request, field) right-hand side: the
 * mixed-precision refinement when every request asks for SFT_CG_MIXED, else
 * the FP64 CG for all. */
typedef struct {
    int32_t nreq;
    int32_t graph;              /* 1: runs replay a captured CUDA graph; 0: direct launches */
    int32_t max_cg_iters;       /* over all (request, field) systems */
    int32_t nonconverged;       /* systems that reached their iteration cap */
    double max_rel_resid;
    int64_t queries;            /* all source queries of the batch */
    int64_t fallback_queries;
    int64_t empty_queries;
    float ms_control, ms_assembly, ms_solve, ms_total;  /* device time of the last run */
    int32_t tile[6];            /* work-item tile per group (2D, 3D) x (fields <= 2, <= 4, <= 8); 0: empty */
} sft_batch_stats;

/* Build a batch plan. srcs/tgts/opts are arrays of nreq (1..4096) entries;
 * every request must use precision SFT_PREC_FP32 (SFT_ERR_UNSUPPORTED
 * otherwise); field_count selects the first k source fields. The handles
 * must outlive the plan. autotune = 1 times trial launches of each group's
 * assembly (tiles 1..16 work items per pull) and keeps the fastest; results
 * are cached per process and, if the environment variable
 * SFT_AUTOTUNE_CACHE names a file, in that file. Synchronises cuda_stream. */
sft_status sft_batch_create(int32_t nreq, const sft_source* srcs, const sft_target* tgts,
                            const sft_options* opts, int32_t autotune, void* cuda_stream,
                            sft_batch* out);
/* Run every request of the plan (stream NULL: the plan's stream) and wait.
 * stats may be NULL. Returns SFT_ERR_NOT_CONVERGED if a system reached its
 * cap (its last iterate is kept). */
sft_status sft_batch_run(sft_batch b, void* cuda_stream, sft_batch_stats* stats);
/* Copy request req's solution (and optionally load vector) [nfields][nnodes]
 * of the last run to u_out / b_out (device pointers if out_device). */
sft_status sft_batch_result(sft_batch b, int32_t req, double* u_out, double* b_out, int32_t out_device,
                            void* cuda_stream);
/* The plan's request groups and their tuned launch shape: out [6][5] host
 * int32, per group (dimension 2 then 3; field-count classes <= 2, <= 4,
 * <= 8): request count, dimension, largest field count of the class, tile
 * (tasks a warp takes per atomic work claim) and lanes per element (a
 * warp holds 32 / lanes elements; each element's lanes share its samples),
 * as chosen by the autotuner (or the defaults without autotuning). */
sft_status sft_batch_groups(sft_batch plan, int32_t* out);
void sft_batch_destroy(sft_batch b);

/* ---- learned surrogate source (spec item 4; no counterpart in the
 * paper beyond its motivation: black-box sources "such as machine-learned
 * surrogates") ----
 * Network x in R^3 -> 256 -> 256 -> 256 -> 256 -> 1, SiLU after each hidden
 * layer, FP32 parameters with BF16 copies of the three 256x256 weight
 * matrices (run on the tensor cores), BF16 hidden activations, FP32
 * accumulation. Parameter vector (sft_mlp_nparam() floats): W1 [256][3],
 * c1 [256], W2 [256][256], c2, W3, c3, W4, c4, w5 [256], c5; weights [out][in]. */
int64_t sft_mlp_nparam(void);
/* params: host or device FP32 vector (copied). */
sft_status sft_mlp_create(const float* params, int32_t device_ptrs, void* cuda_stream, sft_mlp* out);
/* Current FP32 parameters to out (device pointer if out_device). */
sft_status sft_mlp_params(sft_mlp m, float* out, int32_t out_device, void* cuda_stream);
/* Surrogate query: out[i] = network(pts[i]) for pts [n][3] FP32. */
sft_status sft_mlp_forward(sft_mlp m, int64_t n, const float* pts, float* out, int32_t device_ptrs,
                           void* cuda_stream);
/* Gradient of the mean squared error 1/n sum (net(pts_i) - targets_i)^2 with
 * respect to every parameter (grad_out [nparam] FP32) and the loss value
 * (host double); all arrays device memory. Hand-written BF16 forward and
 * backward on the tensor cores (activations and activation gradients in
 * BF16, FP32 accumulation, FP32 gradient). */
sft_status sft_mlp_loss_grad(sft_mlp m, int64_t n, const float* pts, const float* targets, float* grad_out,
                             double* loss_out, int32_t device_ptrs, void* cuda_stream);
/* Adam training (beta 0.9 / 0.999, eps 1e-8) on device data: `epochs` passes
 * over the n points in minibatches of `batch` (rounded to 128), learning rate
 * decaying geometrically from lr to lr_final; loss_history [epochs] (host,
 * may be NULL) gets each epoch's mean loss. */
sft_status sft_mlp_train(sft_mlp m, int64_t n, const float* pts, const float* targets, int32_t epochs,
                         int32_t batch, float lr, float lr_final, double* loss_history, int32_t device_ptrs,
                         void* cuda_stream);
void sft_mlp_destroy(sft_mlp m);

/* ---- Transfer plans: initialization once, online transfers many times ----
 *
 * The paper's cost split (Sec. 5.3): the initialization, paid once per pair
 * of fixed meshes, localizes the target nodes and every sample point; the
 * online part, paid per coupling iteration, evaluates the integrals with the
 * source's current values and solves. sft_plan_create runs the transfer of
 * `opt` once, keeping for every target node and every sample the source
 * element and barycentric coordinates found (mu_1..d in the path precision;
 * plan memory (4 + d*sizeof(P)) bytes per node and per sample, see
 * sft_plan_bytes). The plan refers to src and tgt, which must outlive it;
 * opt->sample_elem_out is ignored. sft_plan_transfer evaluates steps 1-7
 * with the source's current nodal values (sft_source_set_values), the
 * samples' target weights regenerated from the same Philox counters, and
 * writes u_out, b_out, g_out as sft_transfer with opt would (host or device
 * per opt->out_device, on opt->cuda_stream). Its result equals that of
 * sft_transfer with the same options and values up to the order of the
 * floating-point sums. stats->fallback_queries and empty_queries are those
 * found at plan creation. */
typedef struct sft_plan_s* sft_plan;
sft_status sft_plan_create(sft_source src, sft_target tgt, const sft_options* opt, sft_plan* out);
sft_status sft_plan_transfer(sft_plan plan, double* u_out, double* b_out, double* g_out, sft_stats* stats);
int64_t sft_plan_bytes(sft_plan plan);
void sft_plan_destroy(sft_plan plan);

/* ---- Surrogate source: the network as the black-box query ----
 *
 * The transfer of Sec. 4 (steps 1-7) with the source queried through a
 * trained surrogate network (the learned black-box source the paper's
 * introduction motivates) instead of a mesh location. Network inputs are the
 * 3 coordinates of a sample point (z = 0 for a 2D target). An optional exact
 * source mesh, of dimension d_s <= the target's, backs it: an exact query
 * locates the point's first d_s coordinates. */
typedef struct {
    int32_t exact_field;   /* field of the exact source answering exact queries */
    int32_t subsample;     /* s in 0..min(N,128): the first s samples of every element are also
                              queried exactly; 0 disables the fallback */
    float tau;             /* >= 0: an element whose subsample has max |f_net - f_exact| > tau
                              (or a non-finite difference) uses exact queries for all N samples */
    int32_t exact_cost;    /* >= 0: stand-in cost of a costly black-box source: every exact
                              query (subsample, fallback and, without a network, control and
                              samples) runs this many dependent FP32 fused multiply-adds after
                              its mesh location, which leave its value unchanged; 0 = the mesh
                              query alone. It measures the query cost above which the surrogate
                              pays off (the paper's motivating case); the paper has no such
                              parameter. */
    int32_t* fallback_out; /* optional [nelems]: 1 where the element used exact queries */
    float* sample_f_out;   /* optional [nelems][N]: the source value used at every sample */
} sft_surrogate_opts;

typedef struct {
    int32_t cg_iters;
    int32_t reserved;
    double cg_rel_resid;
    int64_t net_queries;     /* network evaluations: target nodes + nelems * s (the subsample)
                                + N for every element that keeps the network */
    int64_t exact_queries;   /* exact mesh queries (subsample + fallback elements) */
    int64_t fallback_elems;  /* elements that used exact queries */
    int64_t empty_queries;   /* exact queries that landed in an empty grid cell (value 0) */
    float ms_control;        /* step 1: control values at the target nodes */
    float ms_assembly;       /* steps 2-6: fused sample / network / fallback / scatter kernel */
    float ms_solve;          /* step 7 */
    float ms_total;
} sft_surrogate_stats;

/* Transfer with the surrogate `net` (may be NULL: every query exact, the
 * plain mesh-query transfer of a d_s-dimensional source onto the target) and
 * the exact source `exact` (may be NULL: no fallback). opt->precision must be
 * SFT_PREC_FP32 (else SFT_ERR_UNSUPPORTED); opt->field_count and
 * sample_elem_out are ignored; one field. Control values g at the target
 * nodes come from the network (exact source without one). Outputs as
 * sft_transfer: u_out, b_out, g_out [nnodes] FP64, fallback_out and
 * sample_f_out host or device per opt->out_device. Samples are those of
 * sft_transfer with the same seed / stream_id / N (Philox counters of the
 * target dimension), so both paths see identical points. */
sft_status sft_transfer_surrogate(sft_mlp net, sft_source exact, sft_target tgt, const sft_options* opt,
                                  const sft_surrogate_opts* sopt, double* u_out, double* b_out, double* g_out,
                                  sft_surrogate_stats* stats);

/* Training set for the surrogate: n points in the box [box_lo, box_hi]
 * (host float[3] each), point j = lo + u * (hi - lo) per axis in FP32 (one
 * rounded product, one rounded sum), u = Philox4x32-10(key = seed, counter =
 * (j_lo32, j_hi32, stream_id, 1)) words 0..2 mapped as the FP32 sampler's
 * uniforms; f = the exact source's field `field` at the point's first d_s
 * coordinates (FP32 location; 0 in an empty cell). pts_out [n][3] and f_out
 * [n] are device memory; *max_abs_out (host, may be NULL) = max |f|. */
sft_status sft_surrogate_dataset(sft_source src, int32_t field, int64_t n, uint64_t seed, uint32_t stream_id,
                                 const float* box_lo, const float* box_hi, float* pts_out, float* f_out,
                                 float* max_abs_out, void* cuda_stream);

/* Allocation-free solve of M u = b for callers that cannot allocate device
 * memory at solve time (for example a coupled code whose memory pool owns
 * the device, or a time-stepping loop that must not call cudaMalloc/cudaFree,
 * which synchronise the device and can fail mid-run). The paper has no
 * counterpart; this is the FP64 Jacobi-PCG of sft_mass_solve (cg_mode
 * SFT_CG_FP64: it takes any SPD matrix) with the caller's CSR matrix and its work vectors kept in a fixed 32 MiB device array that
 * the library reserves on every device it is loaded on, until process exit.
 * All pointers are device memory: row_ptr [n+1], col / val [row_ptr[n]]
 * (FP64, symmetric positive definite, diagonal present), b and u
 * [nrhs][n]. Jacobi-PCG from u = 0 to ||b - M u|| <= tol ||b||.
 * Limits: 1 <= nrhs <= 8 and 8 n (1 + 4 nrhs) bytes plus small per-block
 * partials must fit in 32 MiB (n (1 + 4 nrhs) below about 4.1e6);
 * larger problems are rejected with SFT_ERR_ARG before any device work.
 * The first call on a device looks up the array's device address once and
 * keeps it, so resetting the device (cudaDeviceReset) while the library is
 * loaded is not supported.
 * A row without a positive diagonal entry gives SFT_ERR_ARG. Every call uses the same
 * array, so calls that overlap on the GPU (other streams, other threads)
 * race and must be serialised by the caller. Nothing is allocated or freed;
 * the stream is synchronised before returning. iters_out / rel_resid_out are
 * host pointers (may be NULL). */
sft_status sft_mass_solve_static(int64_t n, const int32_t* row_ptr, const int32_t* col, const double* val,
                                 int32_t nrhs, const double* b, double* u, double tol, int32_t max_iter,
                                 void* cuda_stream, int32_t* iters_out, double* rel_resid_out);

/* Inspection of the built structures (host copies; any output may be NULL).
 * Source grid for `precision`: cells per axis n[3], cell count, registration
 * count, CSR start [ncells+1] and items [nitems] (within a cell in no
 * particular order: no rule depends on it). */
sft_status sft_source_grid(sft_source src, int32_t precision, int32_t n_out[3],
                           int64_t* ncells_out, int64_t* nitems_out,
                           int64_t* start_out, int32_t* items_out);
/* Start element of the location walk in every cell of the source grid for
 * `precision` (Sec. 4, step 4; Sec. 5.3 grid): first_out [ncells] host or
 * device memory, the element of the cell's list deepest at the cell centre
 * (largest min barycentric coordinate there, ties to the lowest id), -1 for an
 * empty cell. SFT_ERR_ARG for a null source or output. */
sft_status sft_source_cell_first(sft_source src, int32_t precision, int32_t* first_out);
/* Face neighbours of the source mesh used by the location walk (Sec. 4,
 * step 4: localizing each sample in the source mesh): adj_out [nelems][dim+1]
 * host or device memory, adj_out[e][m] = the other element holding every
 * vertex of the face of e opposite its local vertex m (the smallest id if
 * several), -1 on the boundary. Built with the source's first location
 * structure (of either precision; `precision` selects which one to build if
 * none exists yet). SFT_ERR_ARG for a null source or output. */
sft_status sft_source_adjacency(sft_source src, int32_t precision, int32_t* adj_out);
/* Target mass matrix: nnz, row_ptr [nnodes+1] (int64), col [nnz], val [nnz],
 * lumped masses [nnodes]. */
sft_status sft_target_mass(sft_target tgt, int64_t* nnz_out, int64_t* row_ptr_out,
                           int32_t* col_out, double* val_out, double* lumped_out);

/* Device memory: every buffer of this library comes from its own
 * stream-ordered memory pool on each device, which keeps blocks freed by
 * *_destroy and by finished calls for later calls instead of returning them
 * to the driver at each synchronisation (creating and destroying meshes in a
 * loop then maps no new memory). This returns the pools' unused blocks to
 * the driver; memory in use is untouched. The paper has no counterpart. */
sft_status sft_trim_memory(void);

const char* sft_status_str(sft_status s);
/* Message of the last error on the calling thread (empty if none). */
const char* sft_last_error(void);
/* Number of CUDA kernels this library has launched in this process
 * (diagnostics; monotone, thread-safe). */
int64_t sft_kernel_launches(void);

#ifdef __cplusplus
}
#endif
#endif /* SFT_H */
