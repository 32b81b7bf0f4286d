/*
 * Oracle for the stochastic conservative field transfer (control-variate
 * Monte Carlo Galerkin projection, Sec. 4 of the paper).
 *
 * TEST INFRASTRUCTURE ONLY. This is a plain, slow, single-threaded FP64 CPU
 * restatement of the method, used to check the CUDA library. Only the test
 * suite, the smoke check and the benchmark's CPU-baseline leg may load it; the
 * product path never calls it. It shares no code, header, table or constant
 * generator with the CUDA library.
 *
 * Precision convention: every routine that draws samples or decides a point
 * location takes ``prec`` (0 = FP64 path, 1 = FP32 path). Sample coordinates
 * and the containment predicate are computed in that precision, because the
 * location decision is an integer that both implementations must take in the
 * same arithmetic. Everything downstream (source evaluation, control,
 * residual, accumulation, mass matrix, solve, integrals) is FP64.
 *
 * Array conventions: coordinates are double arrays [V][d] holding the stored
 * values (rounded to float first when prec = 1); connectivity int32 [E][d+1];
 * nodal values double [nf][V]; outputs [nf][V].
 */
#ifndef SFT_ORACLE_H
#define SFT_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- random numbers: Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11) ---- */
void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);
float orc_u01_f32(uint32_t x);
double orc_u01_f64(uint32_t x);

/* ---- Sec. 4 step 3: area/volume-uniform samples in one target element ----
 * node_xyz: the element's k = d+1 vertex coordinates [k][d];
 * lam_out [N][k] (barycentric weights), X_out [N][d]. */
void orc_sample_element(int prec, int dim, uint64_t seed, uint32_t stream, int64_t t,
                        int32_t nsamp, const double* node_xyz, double* lam_out, double* X_out);
/* The same with a sampling scheme: 0 uniform (as above), 1 stratified (the
 * uniforms of sample j < m^d, m = largest integer with m^d <= nsamp, are
 * confined to cell j of an m^d grid on the unit square / cube before the map;
 * see rng_sample.c). */
void orc_sample_element_s(int prec, int dim, uint64_t seed, uint32_t stream, int64_t t,
                          int32_t nsamp, int sampling, const double* node_xyz, double* lam_out,
                          double* X_out);
/* strata per axis for nsamp samples in dimension dim: largest m with m^dim <= nsamp */
int orc_strata_per_axis(int dim, int32_t nsamp);
/* The same with importance sampling (sampling 2, see rng_sample.c) as well:
 * w_out [N] gets each sample's weight 1 / (|T| p_t(X_j)) (1 for schemes 0, 1). */
void orc_sample_element_w(int prec, int dim, uint64_t seed, uint32_t stream, int64_t t,
                          int32_t nsamp, int sampling, const double* node_xyz, double* lam_out,
                          double* X_out, double* w_out);
/* weight 1 / (|T| p_t) of importance sampling at lambda [d+1]:
 * 1 / (1/4 + 3 sum_{a<b} lambda_a lambda_b) in 2D, 1 / (1/4 + 5/2 sum ...) in 3D */
double orc_importance_weight(int dim, const double* lam);
/* samples of an element under the adaptive count: min(8 N, max(1, ceil(N D / D_ref)))
 * with D = d! |T| the edge determinant of node_xyz and D_ref = d! ref_measure */
int32_t orc_adaptive_samples(int dim, const double* node_xyz, int32_t nsamp, double ref_measure);

/* ---- point location in a uniform-grid-bucketed source mesh ---- */
typedef struct orc_grid orc_grid;
orc_grid* orc_grid_build(int prec, int dim, int64_t nv, const double* coords,
                         int64_t ne, const int32_t* conn, double grid_scale_L);
void orc_grid_free(orc_grid* g);
/* cells per axis, number of cells, number of (cell, element) registrations */
void orc_grid_shape(const orc_grid* g, int32_t n_out[3], int64_t* ncells, int64_t* nitems);
/* CSR copy: start [ncells+1], items [nitems] */
void orc_grid_csr(const orc_grid* g, int64_t* start, int32_t* items);
/* depth of each cell's centre in each listed element (min barycentric), [nitems] */
void orc_grid_depths(const orc_grid* g, double* out);
/* face neighbours [ne][dim+1]: across the face opposite local vertex m, or -1 */
void orc_grid_adjacency(const orc_grid* g, int32_t* out);
/* elem_out: containing element (the walk through face neighbours from the
 * cell's first element, else the first accepting candidate in the cell
 * order), the best-scoring candidate when none accepts, or -1 for an empty
 * cell. status_out: 0 accepted, 1 fallback, 2 empty cell. */
void orc_grid_locate(const orc_grid* g, int64_t npts, const double* pts,
                     int32_t* elem_out, int32_t* status_out);
/* same predicate, scanning every element (no grid) */
void orc_brute_locate(int prec, int dim, int64_t nv, const double* coords, int64_t ne,
                      const int32_t* conn, int64_t npts, const double* pts,
                      int32_t* elem_out, int32_t* status_out);
/* P1 evaluation of nodal values (FP64) in element e at point X */
void orc_eval_p1(int dim, const double* coords, const int32_t* conn, int nf, int64_t nv,
                 const double* values, int32_t e, const double* X, double* f_out);

/* ---- mass matrix (Eq. mass_matrix) in CSR and the solve (Eq. galerkin_system) ---- */
int64_t orc_mass_nnz(int dim, int64_t nv, int64_t ne, const int32_t* conn);
void orc_mass_csr(int dim, int64_t nv, const double* coords, int64_t ne, const int32_t* conn,
                  int64_t* row_ptr, int32_t* col, double* val);
void orc_lumped_mass(int dim, int64_t nv, const double* coords, int64_t ne,
                     const int32_t* conn, double* m_out);
/* Jacobi-preconditioned CG, x0 = 0, stop at ||b - M x|| <= tol ||b||.
 * Returns iterations; rel_resid_out gets the final relative residual. */
int orc_pcg(int64_t nv, const int64_t* row_ptr, const int32_t* col, const double* val,
            const double* b, double* x, double tol, int max_iter, double* rel_resid_out);

/* ---- the full transfer (Sec. 4, steps 1-7) ---- */
typedef struct {
    int prec;             /* 0 fp64, 1 fp32 sampling/location */
    int samples_per_elem; /* N */
    uint64_t seed;
    uint32_t stream;
    double alpha;
    double grid_scale_L;
    double cg_tol;
    int cg_max_iter;
    int sampling;         /* 0 uniform, 1 stratified, 2 importance (orc_sample_element_w) */
    double adapt_ref_measure; /* > 0: N_t = orc_adaptive_samples(...) per element; 0: N */
} orc_params;

typedef struct {
    int cg_iters;
    double cg_rel_resid;
    int64_t fallback_queries;   /* queries no candidate accepted */
    int64_t empty_queries;      /* queries landing in an empty cell */
    int64_t samples;            /* sum over elements of the samples drawn */
} orc_stats;

/* g_out [nf][Vt]; bg_out, bres_out, b_out, u_out [nf][Vt]; sample_elem_out
 * [Et][Nmax] (may be NULL; Nmax = N, or 8 N with the adaptive count; -1 past
 * an element's count). */
void orc_transfer(int dim, const orc_params* p,
                  int64_t nvs, const double* src_coords, int64_t nes, const int32_t* src_conn,
                  int nf, const double* src_values,
                  int64_t nvt, const double* tgt_coords, int64_t net, const int32_t* tgt_conn,
                  double* g_out, double* bg_out, double* bres_out, double* b_out, double* u_out,
                  int32_t* sample_elem_out, orc_stats* stats);

/* ---- integrals and errors (Eqs. relative_conservation_error, relative_L2_error) ---- */
double orc_integral_p1(int dim, int64_t nv, const double* coords, int64_t ne,
                       const int32_t* conn, const double* values);
/* brute-force mesh intersection (Sec. 3): exact load vector of a P1 source on
 * a 2D target by clipping every target/source triangle pair. */
void orc_mi_load_vector_2d(int64_t nvs, const double* src_coords, int64_t nes,
                           const int32_t* src_conn, const double* src_values,
                           int64_t nvt, const double* tgt_coords, int64_t net,
                           const int32_t* tgt_conn, double* b_out);
/* exact ||f^s - f^t||_L2 and ||f^s||_L2 on the supermesh (2D) */
void orc_l2_error_2d(int64_t nvs, const double* src_coords, int64_t nes,
                     const int32_t* src_conn, const double* src_values,
                     int64_t nvt, const double* tgt_coords, int64_t net,
                     const int32_t* tgt_conn, const double* tgt_values,
                     double* err_out, double* norm_out);

/* ---- the surrogate network (see mlp.c for the parameter layout) ---- */
int64_t orc_mlp_nparam(void);
double orc_bf16_round(double x);
void orc_mlp_forward(const double* params, int64_t n, const double* X, int act_bf16, double* y_out);
double orc_mlp_loss_grad(const double* params, int64_t n, const double* X, const double* t, int act_bf16,
                         double* grad);
void orc_adam_step(int64_t np, double* params, const double* grad, double* m, double* v, int64_t t,
                   double lr, double beta1, double beta2, double eps);

#ifdef __cplusplus
}
#endif
#endif
