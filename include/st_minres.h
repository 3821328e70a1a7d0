/*
 * st_minres.h -- C ABI of the GB300 (sm_103a) sine-transform preconditioned MINRES solver for
 * all-at-once heat-equation systems.
 *
 * Method: Hon, Fung, Dong, Serra-Capizzano, "A sine transform based preconditioned MINRES method
 * for all-at-once systems from constant and variable-coefficient evolutionary PDEs"
 * (arXiv 2201.10062).  The heat equation u_t = div(a grad u) + f on (0,1)^dim x (0,T], u = 0 on
 * the boundary (Sec. 1, eq. heat), is discretised with finite differences in space (M = I, K the
 * 3-/5-/7-point stiffness matrix of eq. matrix_Km_va in 1D/2D/3D; 3D as in Sec. 5, Example 3)
 * and the theta-method (Sec. 1, eq. theta) or
 * BDF2 (Sec. 4, eq. matrix_gen) in time.  The all-at-once system T u = f_H is flipped to the
 * symmetric Y T u = Y f_H (eq. main_system) and solved by MINRES with the SPD preconditioner P_H
 * (eq. def:matrix_P), P-hat (eq. def:matrix_P_gen) or P_theta (eq. def:matrix_mod_P).
 *
 * Conventions shared by every entry point
 *   - Grid: interior nodes only; x_i = (i+1)/(mx+1), y_j = (j+1)/(my+1), z_l = (l+1)/(mz+1);
 *     dim 1 has my = 1; dim 1 and 2 have mz = 1 (0 is accepted as 1).
 *   - A space vector has m = mx*my*mz entries, index (l*my + j)*mx + i (x fastest).
 *   - A space-time vector has N = n*m entries, index k*m + j*mx + i, k = 0..n-1 for the time
 *     levels t_1..t_n (the stacked u = [u^(1); ...; u^(n)] of Sec. 1).
 *   - Pointers named *_dev are caller-owned device memory (float64, contiguous) on the device
 *     that was current at st_setup; *_host are caller-owned host memory (pinned memory makes the
 *     copies faster but is not required).  The library never frees caller memory.
 *   - Every call is asynchronous on the stream given in st_problem unless stated otherwise.
 *   - Every int-returning call returns ST_OK or one of the ST_ERR_* codes below.  Nothing
 *     prints, aborts or traps.  After ST_ERR_CUDA the handle should be destroyed.
 */
#ifndef ST_MINRES_H
#define ST_MINRES_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

/* status codes */
#define ST_OK 0
#define ST_ERR_ARG 1            /* invalid argument (null pointer, size out of range, ...)  */
#define ST_ERR_CUDA 2           /* a CUDA runtime call or kernel launch failed              */
#define ST_ERR_NOT_CONVERGED 3  /* maxit reached; the output holds the last iterate          */
#define ST_ERR_BREAKDOWN 4      /* <v, P^-1 v> <= 0 or a non-finite Lanczos/Givens scalar     */
#define ST_ERR_TIMEOUT 5        /* a device-side bounded wait gave up.  If a tensor-core    */
                                /* kernel then could not confirm that its matrix operations  */
                                /* had finished, it keeps its tensor memory rather than free */
                                /* it under a running operation, and every later call on     */
                                /* that device (st_setup included) returns ST_ERR_TIMEOUT.   */
#define ST_ERR_OOM 6            /* device or pinned-host allocation failed                  */

/* time discretisation */
#define ST_THETA 0  /* theta-method, Sec. 1 (theta = 1 backward Euler, 1/2 Crank-Nicolson)    */
#define ST_BDF2 1   /* two-step backward differentiation formula, Sec. 4 with l = 2          */

/* preconditioner */
#define ST_PREC_PH 0     /* P_H (theta) or P-hat (BDF2): DST in time and space, closed-form   */
                         /* spectral scaling; varying a uses the diagonal-averaged K (Sec.    */
                         /* 3.1.1, after eq. matrix_Km_va)                                    */
#define ST_PREC_PTHETA 1 /* P_theta = H (x) M + H_theta (x) tau K (eq. def:matrix_mod_P).     */
                         /* Constant a: spatial DST; 1D varying a: per-frequency tridiagonal  */
                         /* solves by parallel cyclic reduction; 2D/3D varying a: per-freq.   */
                         /* fixed-degree Chebyshev iteration (st_problem.inner_degree steps)  */
                         /* preconditioned by the sine solve with a = mean face value.  The   */
                         /* paper leaves this solver open (Sec. 3.1.4, step 2).  The result   */
                         /* is a fixed SPD map.  theta-method only.                           */

/* default number of Chebyshev steps of the 2D varying-a P_theta (st_problem.inner_degree = 0) */
#define ST_PTHETA_DEFAULT_DEGREE 2
#define ST_PTHETA_MAX_DEGREE 16

/* arithmetic */
#define ST_FP64 0  /* every step in float64                                                   */
#define ST_MIXED 1 /* preconditioner (both DSTs, scaling) in float32 inside float64 iterative */
                   /* refinement; stencil, Lanczos vectors, Givens rotations in float64       */

typedef struct st_problem {
  int dim;                /* 1, 2 or 3                                                       */
  int mx, my;             /* interior points per axis, mx+1 and my+1 powers of two in         */
                          /* [4, 1024] (the spatial DST is a radix-2 FFT); my = 1 if dim = 1  */
  int n;                  /* time steps, 1 <= n <= 1024                                      */
  double T;               /* final time, tau = T/n                                           */
  int scheme;             /* ST_THETA or ST_BDF2                                             */
  double theta;           /* in [0,1] for ST_THETA, ignored for ST_BDF2                       */
  const double *a_nodal;  /* host, nodal a on the (my+2) x (mx+2) grid incl. boundary nodes  */
                          /* ((mx+2) in 1D, (mz+2) x (my+2) x (mx+2) in 3D), finite, a >= 0, */
                          /* and every face value (the mean of the two nodes of a face on an  */
                          /* interior grid line) > 0, so a may vanish on the boundary (Sec. 5 */
                          /* Example 2); NULL means a = 1.  Copied by st_setup.               */
  int prec;               /* ST_PREC_PH or ST_PREC_PTHETA                                    */
  int precision;          /* ST_FP64 or ST_MIXED                                             */
  void *stream;           /* cudaStream_t; NULL = the legacy default stream                  */
  int inner_degree;       /* ST_PREC_PTHETA with 2D/3D a_nodal: Chebyshev steps per apply in  */
                          /* [1, ST_PTHETA_MAX_DEGREE]; 0 = ST_PTHETA_DEFAULT_DEGREE; must be  */
                          /* 0 otherwise.  The map is symmetric positive definite at any     */
                          /* degree (its error polynomial stays below one on the spectrum).    */
  int mz;                 /* dim 3: interior points along z, mz+1 a power of two in [4, 1024]; */
                          /* otherwise 0 or 1.  n*mx*my*mz must stay below 2^31, and in 3D    */
                          /* my*mz at most 524,280 (the stencil grid's row axis).             */
} st_problem;

typedef struct st_stats {
  int iterations;      /* MINRES iterations (all inner iterations for ST_MIXED)              */
  int outer_steps;     /* refinement steps (ST_MIXED), 1 for ST_FP64                         */
  int true_checks;     /* true-residual evaluations made by the stopping rule                */
  int status;          /* same code the call returned                                        */
  double est_rel_res;  /* last M^-1-norm relative residual estimate |eta|/beta_1             */
  double true_rel_res; /* ||Y f_H - Y T u||_2 / ||f_H||_2 at exit                            */
  double seconds;      /* wall time of the call (host clock, includes the final sync)        */
} st_stats;

typedef struct st_handle st_handle;

/* Validate *prob, allocate the device workspace (about 9 space-time vectors of float64; in
 * ST_MIXED about 12.5, of which 7 float32 vectors hold the preconditioned vectors of the MINRES
 * iterations whose direction/solution update is still pending: st_solve applies those updates 8
 * iterations at a time, ST_UPDATE_GROUP=1..8 sets the group and with it the vectors kept) and
 * precompute face coefficients, spectral tables and twiddles.  a_nodal is read during the call
 * only.  Synchronous.  Returns ST_ERR_ARG for unsupported sizes. */
int st_setup(const st_problem *prob, st_handle **out);

/* Free the workspace (synchronises the handle's stream first).  NULL is ignored. */
void st_destroy(st_handle *h);

/* Device bytes st_setup will allocate for *prob (no allocation, no GPU needed). */
int st_workspace_bytes(const st_problem *prob, size_t *bytes);

/* All-at-once right-hand side f_H (Sec. 1 for the theta-method; Sec. 4 for BDF2).
 * f_dev: (n+1) x m, f at t_0..t_n.  u0_dev: m.  uprev_dev: m, u^(-1) for the BDF2 start-up (the
 * history moves to blocks 1 and 2 of the rhs so that T stays Toeplitz); NULL means u^(-1) = u0;
 * ignored for theta.  extra_dev: n x m term added to f_H (e.g. a perturbation), or NULL.
 * fH_dev: n x m output, must not overlap the inputs. */
int st_assemble_rhs(st_handle *h, const double *f_dev, const double *u0_dev,
                    const double *uprev_dev, const double *extra_dev, double *fH_dev);

/* y = Y T v (eq. main_system / main_system_gem_sym): the flipped all-at-once operator, computed
 * as a fused space-time stencil.  v_dev, y_dev: N entries, must not overlap. */
int st_apply_op(st_handle *h, const double *v_dev, double *y_dev);

/* z = P^-1 v by the three steps of Sec. 3.1.1 (or Sec. 3.1.4 for P_theta): transform, scale,
 * transform back.  Always float64 here, whatever st_problem.precision says.  v_dev, z_dev: N
 * entries; z_dev may equal v_dev. */
int st_apply_prec(st_handle *h, const double *v_dev, double *z_dev);

/* z = P^-1 v with every preconditioner step in float32 (the preconditioner ST_MIXED uses);
 * v_dev float64, z_dev float32, N entries each, must not overlap. */
int st_apply_prec_f32(st_handle *h, const double *v_dev, float *z_dev);

/* Solve T u = f_H by preconditioned MINRES on Y T u = Y f_H, zero initial guess (Sec. 5).
 * Stopping rule: MINRES runs until its estimate |eta|/beta_1 <= target (first target = tol); the
 * true 2-norm relative residual rho is then computed and the solve stops if rho <= tol, else the
 * target becomes target*tol/rho and MINRES continues.  ST_MIXED instead runs MINRES with the
 * float32 preconditioner inside float64 iterative refinement on the true residual.
 * fH_dev, u_dev: N entries.  stats may be NULL.  Synchronises the stream before returning. */
int st_solve(st_handle *h, const double *fH_dev, double *u_dev, double tol, int maxit,
             st_stats *stats);

/* st_solve with host buffers: copies fH_host to the device, solves, copies u back to u_host. */
int st_solve_host(st_handle *h, const double *fH_host, double *u_host, double tol, int maxit,
                  st_stats *stats);

/* Solve T^T lam = g.  The blocks of T are symmetric, so T^T = Y T Y and the same preconditioned
 * MINRES solves (Y T) mu = g with lam = Y mu.  g_dev, lam_dev: N entries. */
int st_solve_transpose(st_handle *h, const double *g_dev, double *lam_dev, double tol, int maxit,
                       st_stats *stats);

/* Adjoint of st_assemble_rhs: given lam = dL/df_H (N entries, e.g. from st_solve_transpose),
 * writes dL/df (grad_f_dev, (n+1) x m), dL/du0 (grad_u0_dev, m, may be NULL) and, for BDF2,
 * dL/du^(-1) (grad_uprev_dev, m, may be NULL; zeros for theta).  From the rhs of Sec. 1:
 * theta: df^(k) = theta tau lam_k + (1-theta) tau lam_{k+1}, du0 = (I - (1-theta) tau K) lam_1;
 * BDF2: df^(k) = tau lam_k (k >= 1), du0 = 2 lam_1 - lam_2/2, du^(-1) = -lam_1/2. */
int st_grad_rhs(st_handle *h, const double *lam_dev, double *grad_f_dev, double *grad_u0_dev,
                double *grad_uprev_dev);

/* Gradient of L(a) through T(a) u = f_H(a) given the adjoint lam = T^-T dL/du: for theta,
 * dL/da = -tau sum_k lam_k^T (dK/da) (theta u_k + (1-theta) u_{k-1}) with u_0 = u0 (BDF2: u_k);
 * each face value is the mean of its two nodal values, so half of each face term goes to each
 * node.  lam_dev, u_dev: N; u0_dev: m; grad_dev: the nodal grid ((my+2)(mx+2), or mx+2 in 1D),
 * overwritten.  1D and 2D only: ST_ERR_ARG for a 3D handle. */
int st_grad_a(st_handle *h, const double *lam_dev, const double *u_dev, const double *u0_dev,
              double *grad_dev);

/* Autotuner: times the candidate launch shapes of this handle's kernels on its own buffers
 * (CUDA events, `reps` launches each, 1..100) -- blocks per stencil launch, sequences per
 * spatial-DST block, column tile of the FFMA time kernel -- and, in float32, the tensor-core
 * kernel of each stage (time DST with scaling, y and z passes) against its CUDA-core
 * counterpart.  It keeps the fastest of each and caches the choice per (dim, mx, my, mz, n,
 * precision, kernel path) for the process.  Synchronous; clobbers the handle's workspace (call
 * it between solves).  st_setup_batch runs it for every instance. */
int st_autotune(st_handle *h, int reps);

/* Batched solves: `count` independent instances (each its own st_problem, precision ST_MIXED;
 * sizes, theta/BDF2 and a(x) may all differ) solved concurrently, one stream per instance, by a
 * single CUDA graph that the call relaunches until every instance has converged.  The refinement
 * decisions (restart or stop) are taken on the device, so nothing inside the graph waits for the
 * host.  st_setup_batch allocates every instance's workspace (probs[i].stream is ignored; the
 * batch works on `stream`).  st_solve_batch: fH_devs[i], u_devs[i] as in st_solve; tol and maxit
 * apply to every instance; stats (count entries, may be NULL) per instance; returns ST_OK when
 * every instance converged, else the first failure code.  The graph is captured on the first
 * solve and again whenever the buffer pointers change.  Synchronises `stream` before returning. */
typedef struct st_batch st_batch;
int st_setup_batch(const st_problem *probs, int count, void *stream, st_batch **out);
int st_solve_batch(st_batch *b, const double *const *fH_devs, double *const *u_devs, double tol,
                   int maxit, st_stats *stats);
/* Handle of instance i (owned by the batch) for st_assemble_rhs, st_apply_op, ...; those calls
 * run on the batch's `stream`. */
int st_batch_instance(st_batch *b, int i, st_handle **out);
void st_destroy_batch(st_batch *b);

/* Residual check that allocates nothing (the paper has no counterpart; it is a deployment aid).
 * Some callers cannot allocate device memory at the moment they need a residual: code that is
 * recording a CUDA graph, latency-critical loops where cudaFree's implicit device synchronisation
 * is not acceptable, or hosts that give all device memory to their own arena up front.  This call
 * needs no handle and no cudaMalloc/cudaFree: its per-block partial sums live in a fixed static
 * __device__ array of 64 KB (room for 4096 blocks; every GPU that loads the library keeps it until
 * the process exits).  It covers 1D and 2D problems only (every 1D/2D size st_setup accepts
 * fits); a 3D problem, or a size beyond the array, returns ST_ERR_ARG.
 * prob: sizes, scheme, theta, T and stream (prob->a_nodal must be NULL); a_nodal_dev: device copy
 * of the nodal a grid (layout as st_problem.a_nodal) or NULL for a = 1.  It must meet the same
 * conditions as st_problem.a_nodal (finite, >= 0, every interior face value > 0) but, unlike
 * st_setup, this call does not check them (reading the array would need a copy to the host):
 * a field that breaks them gives a meaningless residual, not an error.  fH_dev, u_dev: N entries.
 * Outputs: r_dev (N entries, may be NULL) = Y f_H - Y T u; it must not overlap fH_dev or u_dev
 * (ST_ERR_ARG otherwise); sums_dev[0] = ||r||^2 and sums_dev[1] = ||f_H||^2 (two device doubles),
 * both written on prob->stream.
 * The first call on a device looks up the array's device address (cudaGetSymbolAddress) with
 * that device current; make that first call before any stream capture (a lookup that fails is
 * retried by the next call).  Every call shares the one array, so calls that overlap on the GPU
 * (other streams, other host threads) race. */
int st_residual_noalloc(const st_problem *prob, const double *a_nodal_dev, const double *fH_dev,
                        const double *u_dev, double *r_dev, double *sums_dev);

/* Kernel-class profiler.  st_profile_begin starts bracketing every kernel the handle launches
 * with CUDA events on the handle's stream (room for `capacity` launches; later launches are only
 * counted).  st_profile_end synchronises the stream, writes per-class totals for classes
 * 0..nclasses-1 (ST_KC_* below) and stops profiling. */
#define ST_KC_STENCIL 0  /* flipped space-time stencil                                        */
#define ST_KC_LANCZOS 1  /* Lanczos three-term update fused into the first spatial DST along */
                         /* x of the preconditioner pass (that whole launch)                  */
#define ST_KC_DSTX 2     /* spatial DST along x (the other launches)                          */
#define ST_KC_DSTY 3     /* spatial DST along y                                               */
#define ST_KC_TIME 4     /* time DST, spectral scaling, time DST                              */
#define ST_KC_UPDATE 5   /* MINRES direction / solution update                                */
#define ST_KC_RESID 6    /* true residual                                                     */
#define ST_KC_AUX 7      /* rhs assembly, flips, norms, gradient                              */
#define ST_KC_COUNT 8
typedef struct st_kernel_time {
  int launches; /* kernels launched in this class while profiling                          */
  int timed;    /* of those, how many were bracketed by events                              */
  double ms;    /* summed event time of the timed launches                                  */
} st_kernel_time;
int st_profile_begin(st_handle *h, int capacity);
int st_profile_end(st_handle *h, st_kernel_time *out, int nclasses);
const char *st_kernel_class_name(int kernel_class);

const char *st_strerror(int code);
int st_version(void);

#ifdef __cplusplus
}
#endif

#endif /* ST_MINRES_H */
