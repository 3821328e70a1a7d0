// Internal declarations shared by the translation units of the solver library.
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include "../../include/st_minres.h"
#include "st_dd.cuh"
#include "st_df.cuh"

namespace st {

// Geometry and coefficients of one problem, passed by value to kernels.  A space vector is
// u[z][y][x] (x fastest); "rows" are the my*mz lines of x, row r = jz*my + jy.
struct Geom {
  int dim, mx, my, n;
  long long m, N;       // m = mx*my*mz, N = n*m
  int scheme;           // ST_THETA / ST_BDF2
  double tau, theta;
  const double *cx;     // [mz*my][mx+1]  tau * a(x-face) / hx^2, faces i = 0..mx between nodes i-1, i
  const double *cy;     // [mz][my+1][mx] tau * a(y-face) / hy^2 (NULL in 1D)
  const df *cxd, *cyd;  // the same coefficients as double-float pairs (mixed-precision stencil)
  df th_d, omth_d;      // theta and 1 - theta as double-float pairs
  int th_exact;         // theta in {0, 1/2, 1}: products with theta, 1 - theta are exact scalings
  int st_target;        // stencil launch: target number of blocks (0: default), set by autotune
  int mz;               // interior points along z: 1 unless 3D
  const double *cz;     // [mz+1][my][mx] tau * a(z-face) / hz^2 (NULL unless 3D)
  const df *czd;
  int c_uniform;        // every face coefficient equals c_uni (constant a, equal spacing)
  df c_uni;             // that coefficient as a double-float pair
};

// The six face coefficients (tau a / h^2) around interior node (i, jy, jz): west/east along x,
// south/north along y, down/up along z; zero along axes the grid does not have.
template <class T>
struct Faces6 {
  T w, e, s, n, d, u;
};

__host__ __device__ inline Faces6<double> faces_at(const Geom &g, int i, int jy, int jz) {
  const long long row = (long long)jz * g.my + jy;
  Faces6<double> f{g.cx[row * (g.mx + 1) + i], g.cx[row * (g.mx + 1) + i + 1], 0.0, 0.0, 0.0, 0.0};
  if (g.dim >= 2) {
    const long long ys = ((long long)jz * (g.my + 1) + jy) * g.mx + i;
    f.s = g.cy[ys];
    f.n = g.cy[ys + g.mx];
  }
  if (g.dim == 3) {
    const long long zs = row * g.mx + i;
    f.d = g.cz[zs];
    f.u = g.cz[zs + (long long)g.mx * g.my];
  }
  return f;
}

__host__ __device__ inline Faces6<df> faces_df_at(const Geom &g, int i, int jy, int jz) {
  const long long row = (long long)jz * g.my + jy;
  const df zero{0.f, 0.f};
  Faces6<df> f{g.cxd[row * (g.mx + 1) + i], g.cxd[row * (g.mx + 1) + i + 1], zero, zero, zero,
               zero};
  if (g.dim >= 2) {
    const long long ys = ((long long)jz * (g.my + 1) + jy) * g.mx + i;
    f.s = g.cyd[ys];
    f.n = g.cyd[ys + g.mx];
  }
  if (g.dim == 3) {
    const long long zs = row * g.mx + i;
    f.d = g.czd[zs];
    f.u = g.czd[zs + (long long)g.mx * g.my];
  }
  return f;
}

// Spectral tables used by the preconditioner kernels.
template <class T>
struct Spec {
  const T *mux;    // [mx]  x-part of the (averaged) stiffness eigenvalue, times tau
  const T *muy;    // [mz*my] y- plus z-part, times tau, indexed by the row jz*my + jy (zeros in 1D)
  const T *hk;     // [n]   1 - cos(x_k), x_k = k pi/(n+1), k = 1..n (from 2 sin^2(x_k/2))
  const T *ck;     // [n]   cos(x_k)
  const T *sk;     // [n]   sin(x_k)
  const T *lh;     // [n]   eigenvalues of H = sqrt(tridiag(-1,2,-1)): 2 sin(x_k/2)
  const T *lht;    // [n]   eigenvalues of H_theta
  const T *sintab; // [2(n+1)] sqrt(2/(n+1)) sin(r pi/(n+1))
  int prec;        // ST_PREC_PH / ST_PREC_PTHETA
  int scheme;
  T theta;
};

// Device-resident MINRES scalars.  Written only by the last block of a kernel (the
// "last block" reduction pattern) or by the host between solves.
// Most iterations whose direction/solution updates one grouped update pass applies.
constexpr int kUpdRing = 8;

struct State {
  double alpha, beta, beta_prev, beta1, eta;
  double c1, s1, c2, s2;               // rotations k-1 and k-2
  double inv_beta;                     // 1/beta_k, scale of z_k in the stencil
  double lz_a, lz_b;                   // vhat_{k+1} = p - lz_a vhat_k - lz_b vhat_{k-1}
  double dz, d1, d2, xc;               // d_k = dz z_k + d1 d_{k-1} + d2 d_{k-2};  x += xc d_k
  double est, target;
  double rnorm2;                       // residual kernel output ||r||^2
  double bnorm2;                       // ||b||^2
  int k, maxit;
  int active, finish, status;
  int pad;
  unsigned int counter[8];             // completion counters of the last-block reductions
  // device-driven refinement (batched solves): after an inner run finishes, the residual
  // kernel decides between done and a restart of the inner run
  double tol_outer;                    // requested ||r||/||b||
  double inner_floor;                  // lowest target of an inner run (device-side restarts)
  double rho;                          // last true relative residual
  int done, restart, total, outer, maxit_total;
  int upd;                             // grouped update: iterations whose d/x update is applied
  // double-float copies of the per-iteration scalars, refreshed by whoever sets the float64
  // values, so that the double-float vector kernels read them without float64 instructions
  df dfs[8];
  // grouped update (mixed single solves): the direction/solution scalars of iteration j, in
  // slot (j - 1) % kUpdRing as {dz, d1, d2, xc}, kept until the pass that applies them
  df ucoef[kUpdRing][4];
  // Set (never cleared on the device) by a tensor-core kernel whose bounded waits ran out twice,
  // so that it exited without releasing its tensor memory (an MMA might still have been writing
  // it).  It is the last member: the host pushes the state up to it (kStatePushBytes) and so
  // never overwrites it; once the host reads it set, the device is closed to further calls.
  int tmem_held;
};

// bytes of State the host writes to the device: everything before tmem_held
constexpr size_t kStatePushBytes = offsetof(State, tmem_held);

enum { DFS_IB = 0, DFS_LA, DFS_LB, DFS_DZ, DFS_D1, DFS_D2, DFS_XC };

__host__ __device__ inline void refresh_df(State *S) {
  S->dfs[DFS_IB] = df_of_double(S->inv_beta);
  S->dfs[DFS_LA] = df_of_double(S->lz_a);
  S->dfs[DFS_LB] = df_of_double(S->lz_b);
  S->dfs[DFS_DZ] = df_of_double(S->dz);
  S->dfs[DFS_D1] = df_of_double(S->d1);
  S->dfs[DFS_D2] = df_of_double(S->d2);
  S->dfs[DFS_XC] = df_of_double(S->xc);
}

enum { CNT_STENCIL = 0, CNT_TIME = 1, CNT_RESID = 2, CNT_NORM = 3, CNT_UPD = 4 };

// Last-block completion: every block writes its partial, the last block to arrive sums all
// partials in a fixed order (deterministic) and returns the total to thread 0.
// Returns true in the (single) last block; *total is valid in its thread 0.
__device__ inline double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

template <int NT>
__device__ inline double block_sum(double v, double *red) {
  v = warp_sum(v);
  const int lane = threadIdx.x & 31, wid = (threadIdx.x + threadIdx.y * blockDim.x) >> 5;
  __syncthreads();
  if (lane == 0) red[wid] = v;
  __syncthreads();
  double t = 0.0;
  if (wid == 0) {
    t = (lane < NT / 32) ? red[lane] : 0.0;
    t = warp_sum(t);
  }
  return t;  // valid in warp 0
}

// Flat thread index within the block, for 1D/2D blocks.
__device__ inline int flat_tid() { return threadIdx.x + threadIdx.y * blockDim.x; }

template <int NT>
__device__ inline bool last_block_reduce(double part, double *partials, unsigned int *counter,
                                         int nblocks, int bid, double *red, double *total) {
  __shared__ bool is_last;
  const int tid = flat_tid();
  double s = block_sum<NT>(part, red);
  if (tid == 0) {
    partials[bid] = s;
    __threadfence();
    unsigned int prev = atomicAdd(counter, 1u);
    is_last = (prev == (unsigned int)(nblocks - 1));
  }
  __syncthreads();
  if (!is_last) return false;
  __threadfence();
  double acc = 0.0;
  for (int i = tid; i < nblocks; i += NT) acc += ((volatile double *)partials)[i];
  double tot = block_sum<NT>(acc, red);
  if (tid == 0) {
    *total = tot;
    *counter = 0u;
  }
  return true;
}

// ---------------------------------------------------------------- MINRES scalar steps
// Run by one thread of the last block of the kernel that completes <v, P^-1 v>.
// Start of a run: beta_1 = sqrt(<b, P^-1 b>).
__device__ inline void minres_init_scalars_dev(State *S, double E) {
  if (!(E >= 0.0) || !isfinite(E)) {
    S->status = ST_ERR_BREAKDOWN;
    S->finish = 1;
    refresh_df(S);
    return;
  }
  const double b1 = sqrt(E);
  S->beta1 = b1;
  S->beta = b1;
  S->beta_prev = 1.0;
  S->inv_beta = (b1 > 0.0) ? 1.0 / b1 : 0.0;
  S->eta = b1;
  S->c1 = 1.0;
  S->s1 = 0.0;
  S->c2 = 1.0;
  S->s2 = 0.0;
  S->k = 0;
  S->est = 1.0;
  S->active = 1;  // `restart` stays set until the run's first stencil: the inverse transforms of
                  // this preconditioner pass are still gated on it
  if (b1 == 0.0) S->finish = 1;
  refresh_df(S);
}

// One Givens step of MINRES (Paige-Saunders) once beta_{k+1}^2 = E is known.
__device__ inline void minres_givens_dev(State *S, double E) {
  if (!(E >= 0.0) || !isfinite(E)) {
    S->status = ST_ERR_BREAKDOWN;
    S->finish = 1;
    S->xc = 0.0;
    S->dz = S->d1 = S->d2 = 0.0;
    refresh_df(S);
    return;
  }
  const double bnext = sqrt(E);
  const int k = S->k + 1;
  const double off = (S->k > 0) ? S->beta : 0.0;
  const double eps = S->s2 * off;
  const double dbar = S->c2 * off;
  const double delta = S->c1 * dbar + S->s1 * S->alpha;
  const double gbar = -S->s1 * dbar + S->c1 * S->alpha;
  const double rho = hypot(gbar, bnext);
  if (!(rho > 0.0) || !isfinite(rho) || !isfinite(S->alpha)) {
    S->status = ST_ERR_BREAKDOWN;
    S->finish = 1;
    S->xc = 0.0;
    S->dz = S->d1 = S->d2 = 0.0;
    refresh_df(S);
    return;
  }
  const double c = gbar / rho, s = bnext / rho;
  S->dz = 1.0 / (S->beta * rho);
  S->d1 = -delta / rho;
  S->d2 = -eps / rho;
  S->xc = c * S->eta;
  S->eta = -s * S->eta;
  S->c2 = S->c1;
  S->s2 = S->s1;
  S->c1 = c;
  S->s1 = s;
  S->beta_prev = S->beta;
  S->beta = bnext;
  S->inv_beta = (bnext > 0.0) ? 1.0 / bnext : 0.0;
  S->k = k;
  S->est = fabs(S->eta) / S->beta1;
  if (S->est <= S->target || bnext == 0.0 || k >= S->maxit) S->finish = 1;
  refresh_df(S);
  df *uc = S->ucoef[(k - 1) % kUpdRing];
  uc[0] = S->dfs[DFS_DZ];
  uc[1] = S->dfs[DFS_D1];
  uc[2] = S->dfs[DFS_D2];
  uc[3] = S->dfs[DFS_XC];
}


// ---------------------------------------------------------------- kernel-class profiler
// While a handle's profiler is on, each kernel launch is bracketed by CUDA events recorded on
// the launching stream; the host sums the elapsed times per kernel class afterwards.
enum {
  KC_STENCIL = 0,  // flipped space-time stencil (MINRES and apply modes)
  KC_LANCZOS = 1,  // Lanczos three-term update fused into the first x-pass of the preconditioner
  KC_DSTX = 2,     // spatial DST along x (contiguous lines)
  KC_DSTY = 3,     // spatial DST along y (strided lines)
  KC_TIME = 4,     // time DST -> spectral scaling -> time DST (+ energy, Givens)
  KC_UPDATE = 5,   // direction and solution update
  KC_RESID = 6,    // true residual (stencil in residual mode)
  KC_AUX = 7,      // rhs assembly, flips, norms, gradient
  KC_COUNT = 8
};

struct Prof {
  int on;
  int cap, used;
  cudaEvent_t *ev;  // 2*cap events
  int *cls;         // class of each recorded pair
  long long launches[KC_COUNT];
};

// per-thread pointer to the profiler of the handle whose call is running (or null)
void prof_begin(int cls, cudaStream_t st);
void prof_end(cudaStream_t st);

// ---------------------------------------------------------------- launch-side declarations
// stencil modes
enum { SM_MINRES = 0, SM_APPLY = 1, SM_RESID = 2, SM_TRANSPOSE_APPLY = 3, SM_RESID_OUTER = 4 };

template <class Tz>
cudaError_t launch_stencil(const Geom &g, int mode, const Tz *z, double *out, const double *fH,
                           State *S, double *partials, int nblocks_hint, cudaStream_t st);
int stencil_blocks(const Geom &g);

cudaError_t launch_rhs(const Geom &g, const double *f, const double *u0, const double *uprev,
                       const double *extra, double *fH, cudaStream_t st);
cudaError_t launch_grad_rhs(const Geom &g, const double *lam, double *gf, double *gu0,
                            double *gup, cudaStream_t st);
cudaError_t launch_grad_a(const Geom &g, const double *lam, const double *u, const double *u0,
                          double *gface_x, double *gface_y, double *grad, cudaStream_t st);

// preconditioner pipeline: z = P^-1 v (v may be double, z double or float)
struct PrecPlan {
  int Lx, Ly, Lz;             // FFT lengths 2(mx+1), 2(my+1), 2(mz+1)
  const double *twx_d, *twy_d, *twz_d;  // e^{-2 pi i j/L}, j < L/2, interleaved (re, im)
  const float *twx_f, *twy_f, *twz_f;
  Spec<double> spec_d;
  Spec<float> spec_f;
  int time_J_d, time_J_f;     // spatial columns per FFMA time-kernel block (0: default)
  int dst_shift;              // spatial DST: sequences per block divided by 2^dst_shift
  int time_blocks_d, time_blocks_f;
  const double *pcr_diag;     // P_theta 1D varying a: tau*K diagonal [mx]
  const double *pcr_off;      // tau*K off-diagonal [mx] (entry i couples i and i+1)
  const unsigned short *sop;  // fp16 S_n operand image for the tensor-core time kernel, or null
  const unsigned short *sop_y;  // fp16 S_my image for the tensor-core y-DST (2D/3D mixed), or null
  const unsigned short *sop_z;  // fp16 S_mz image for the tensor-core z-DST (3D mixed), or null
  const unsigned short *sop_x;  // fp16 S_mx image for the tensor-core x-DST of the last spatial
                                // pass (mixed), or null
  const unsigned short *sop_long;  // streamed S_n chunks for the tensor-core time kernel when
                                   // 256 < n <= 512 (mixed), or null
  const unsigned char *sdig;  // integer-digit image of S_n for the float64-accurate tensor-core
                              // time kernel (float64 path, double-float engine), or null
  int sdig_e;                 // its scale: the digits are those of S_n 2^sdig_e
  dd *tscratch;               // N double-floats the tensor-core time stage writes between its
                              // two transforms (the handle's stencil-output vector, free
                              // during a preconditioner pass)
  int pcr;                    // P_theta with varying a in 1D: tridiagonal solves per frequency
  const unsigned short *sop_t1;  // fp16 S_n image for unscaled single time transforms on the
                                 // tensor cores (mixed P_theta with varying a), or null
  // P_theta with varying a in 2D/3D: Chebyshev steps per apply (0: not this path), the per-step,
  // per-frequency scalars [cheb][n] (a: carry-over of the previous direction, s: factor of
  // B_k^-1 r), and five N-vectors of float64 scratch (used as the transform type: residual,
  // transformed residual, iterate, two directions)
  int cheb;
  const double *cheb_a_d, *cheb_s_d;
  const float *cheb_a_f, *cheb_s_f;
  void *cheb_work;
  // float64 preconditioner (P_H / P-hat path): the transforms and the scaling in double-float
  // arithmetic on the float32 pipes (1) or in float64 (0); the intermediate vectors between the
  // passes are then stored as double-floats in the output buffer.  Tables in double-float:
  Spec<dd> spec_dd;
  const dd *twx_dd, *twy_dd, *twz_dd;
  int fp64_dd;
  int time_J_dd;  // spatial columns per double-float time-kernel block (0: default)
};

// Lowest relative target of an inner (float32-preconditioned) MINRES run of the mixed solve:
// 1e-7, where the float32 preconditioner still lets the estimate fall steadily (ST_INNER_FLOOR
// overrides it, for measurements).
double inner_floor();

// Iterations per grouped direction/solution update of a mixed single solve: kUpdRing unless
// ST_UPDATE_GROUP (1..kUpdRing) sets it, for measurements.
int update_group();

// st_setup with an explicit update group (the batched solve's instance handles take 1: their
// captured loop updates every iteration and keeps no extra z vectors)
int setup_handle(const st_problem *prob, st_handle **out, int ugroup);

// A device on which a tensor-core kernel kept its tensor memory after a timeout is closed: every
// later call there returns ST_ERR_TIMEOUT (the host learns it from State::tmem_held).
void close_device(int dev);
bool device_closed(int dev);

bool time_tc_supported(int n);
size_t time_tc_sop_halves(int n);
void time_tc_build_sop(int n, unsigned short *out);
cudaError_t launch_time_tc(float *data, const Geom &g, const Spec<float> &sp,
                           const unsigned short *sop, State *S, int tmode, double *partials,
                           int gk, cudaStream_t st);
bool dst_tc_supported(int len);
// float64-accurate time stage on the tensor cores (integer digits of S_n and of the double-float
// data, exact float32 accumulation per digit group; k_time_tcd)
bool time_tcd_supported(int n);
size_t time_tcd_bytes(int n);
int time_tcd_build(int n, unsigned char *out);  // returns the scale exponent of the digits
// scratch: an N-vector of double-floats that overlaps neither data nor anything the stage reads
cudaError_t launch_time_tcd(dd *data, dd *scratch, const Geom &g, const Spec<dd> &sp,
                            const unsigned char *img, int eS, State *S, int tmode,
                            double *partials, int gk, cudaStream_t st);
bool time_tc_long_supported(int n);
size_t time_tc_long_bytes(int n);
void time_tc_long_build(int n, unsigned short *out);
cudaError_t launch_time_tc_long(float *data, const Geom &g, const Spec<float> &sp,
                                const unsigned short *A, State *S, int tmode, double *partials,
                                int gk, cudaStream_t st);
cudaError_t launch_dst_tc_y(float *data, const Geom &g, const unsigned short *sop, State *S,
                            int gk, cudaStream_t st);
cudaError_t launch_dst_tc_z(float *data, const Geom &g, const unsigned short *sop, State *S,
                            int gk, cudaStream_t st);
cudaError_t launch_dst_tc_x(float *data, const Geom &g, const unsigned short *sop, State *S,
                            int gk, cudaStream_t st);
bool dst_tc_len_supported(int len);
cudaError_t launch_time_tc_single(const float *in, float *out, const Geom &g,
                                  const unsigned short *sop, State *S, int gk, cudaStream_t st);

// energy mode of the time kernel's last block
enum { TM_NONE = 0, TM_INIT = 1, TM_ITER = 2, TM_RESTART = 3 };

// Which state flag a preconditioner kernel waits for: none (standalone applies and the first
// start), `active` (inside a MINRES iteration) or `restart` (device-driven restart of an inner
// run in a batched solve).
enum { GK_NONE = 0, GK_ACTIVE = 1, GK_RESTART = 2 };
inline int gate_kind_of(int tmode) {
  return tmode == TM_ITER ? GK_ACTIVE : (tmode == TM_RESTART ? GK_RESTART : GK_NONE);
}
__device__ __forceinline__ bool gate_closed(const State *S, int gk) {
  if (gk == GK_ACTIVE) return !S->active;
  if (gk == GK_RESTART) return !S->restart;
  return false;
}

template <class Tc, class Tin, class Tout>
cudaError_t launch_prec_lanczos(const Geom &g, const PrecPlan &pp, const Tin *q, const Tin *vk,
                                Tin *vnext, Tout *z, State *S, double *partials, cudaStream_t st,
                                cudaEvent_t after_time = nullptr);
template <class Tc, class Tin, class Tout>
cudaError_t launch_prec(const Geom &g, const PrecPlan &pp, const Tin *v, Tout *z, State *S,
                        int tmode, double *partials, cudaStream_t st);
int time_blocks_for(const Geom &g, const PrecPlan &pp, bool fp32);
int time_J_default(int n, bool fp32);
// the spatial DST passes alone, ungated: float32 (fp32), else the float64 path's engine
// (double-float when pp.fp64_dd, float64 otherwise)
cudaError_t tune_run_dsts(const Geom &g, const PrecPlan &pp, bool fp32, void *data,
                          cudaStream_t st);
cudaError_t tune_run_time(const Geom &g, const PrecPlan &pp, bool fp32, void *data,
                          cudaStream_t st);
// the double-float time kernel alone (float64 preconditioner's double-float engine), ungated
cudaError_t tune_run_time_dd(const Geom &g, const PrecPlan &pp, void *data, cudaStream_t st);
bool time_J_fits(int n, int J, bool fp32);
// one spatial pass along y (axis 1) or z (axis 2), float32, in place and ungated: on the tensor
// cores with tc_img, by the shared-memory FFT when tc_img is null
cudaError_t tune_run_pass(const Geom &g, const PrecPlan &pp, int axis,
                          const unsigned short *tc_img, float *data, State *S, cudaStream_t st);

// mixed path: double-float (df) MINRES vectors, float32 preconditioned vectors
cudaError_t launch_stencil_df(const Geom &g, const float *z, df *q, State *S, double *partials,
                              cudaStream_t st);
cudaError_t launch_resid_df(const Geom &g, const double *x, df *r_out, const double *fH, State *S,
                            double *partials, cudaStream_t st);
// device-driven refinement step: runs only when the inner run has finished and the solve is not
// done; r = Y f_H - Y T x into r_out and, in the last block, the done/restart decision
cudaError_t launch_resid_outer(const Geom &g, const double *x, df *r_out, const double *fH,
                               State *S, double *partials, cudaStream_t st);
// every pending direction/solution update of a mixed solve (k_update_group_df), and the ring
// slot of a mixed handle's z vectors (slot s of Z[0], Z[1], Zx[0], ...)
cudaError_t launch_update_group(st_handle *h, cudaStream_t st);
float *zslot(st_handle *h, int s);
cudaError_t launch_flip_to_df(const Geom &g, const double *src, df *dst, cudaStream_t st);
cudaError_t launch_df_to_double(long long N, const df *src, double *dst, cudaStream_t st);

// real part used when a transform reads its input in the compute type
template <class Tc>
__device__ __forceinline__ Tc to_real(double v) { return (Tc)v; }
template <class Tc>
__device__ __forceinline__ Tc to_real(float v) { return (Tc)v; }
template <class Tc>
__device__ __forceinline__ Tc to_real(df v) { return (Tc)v.hi; }
// double-float storage of the float64 preconditioner's intermediate vectors, read by the
// double-float transforms
template <class Tc>
__device__ __forceinline__ Tc to_real(dd v) { return (Tc)v; }
template <>
__device__ __forceinline__ dd to_real<dd>(dd v) { return v; }

// Element sources for the first stage of a preconditioner pass.  prepare() runs once per thread
// after the gate; operator() returns element i in the transform type.
template <class Tc, class Tin>
struct SrcArray {
  const Tin *p;
  __device__ __forceinline__ void prepare(const State *) {}
  __device__ __forceinline__ Tc operator()(long long i) const { return to_real<Tc>(p[i]); }
};

// The Lanczos step fused into the load: v_{k+1} = q - lz_a v_k - lz_b v_{k-1}, written over
// v_{k-1} (every element is loaded exactly once) and returned for the transform.
template <class Tc, class Tv>
struct SrcLanczos;

template <class Tc>
struct SrcLanczos<Tc, double> {
  const double *q, *vk;
  double *vp;
  double a, b;
  __device__ __forceinline__ void prepare(const State *S) {
    a = S->lz_a;
    b = S->lz_b;
  }
  __device__ __forceinline__ Tc operator()(long long i) const {
    // q and v_k are read-only in this pass: read-only-cache loads, free to move ahead of the
    // stores to v_{k-1}
    const double v = __ldg(q + i) - a * __ldg(vk + i) - b * vp[i];
    vp[i] = v;
    return (Tc)v;
  }
};

// Double-float vectors: q holds Y T z_k without the 1/beta_k factor (the double-float stencil
// leaves that scaling to this pass), so v_{k+1} = q / beta_k - lz_a v_k - lz_b v_{k-1}.
template <class Tc>
struct SrcLanczos<Tc, df> {
  const df *q, *vk;
  df *vp;
  df a, b, sc;
  __device__ __forceinline__ void prepare(const State *S) {
    a = df_neg(S->dfs[DFS_LA]);
    b = df_neg(S->dfs[DFS_LB]);
    sc = S->dfs[DFS_IB];
  }
  // the three loads of element i, issued apart from the arithmetic and the store so that a
  // thread can have all of its elements' loads in flight before the first store (fetch, then
  // finish); operator() does both for one element
  struct Raw {
    float2 q, v, p;
  };
  __device__ __forceinline__ Raw fetch(long long i) const {
    // q and v_k are read-only in this pass (see the float64 source)
    Raw r;
    r.q = __ldg(reinterpret_cast<const float2 *>(q) + i);
    r.v = __ldg(reinterpret_cast<const float2 *>(vk) + i);
    r.p = *(reinterpret_cast<const float2 *>(vp) + i);
    return r;
  }
  __device__ __forceinline__ Tc finish(long long i, const Raw &r) const {
    // (s, t) = q / beta_k with the product's error kept (TwoProd)
    float s = sc.hi * r.q.x;
    float t = fmaf(sc.hi, r.q.x, -s);
    t = fmaf(sc.hi, r.q.y, fmaf(sc.lo, r.q.x, t));
    dacc_prod(s, t, a, df{r.v.x, r.v.y});
    dacc_prod(s, t, b, df{r.p.x, r.p.y});
    const df v = df_from_sum(s, t);
    vp[i] = v;
    return to_real<Tc>(v);
  }
  __device__ __forceinline__ Tc operator()(long long i) const { return finish(i, fetch(i)); }
};

// sources whose loads can be issued ahead of their stores (SrcLanczos over double-floats)
template <class Src>
struct has_fetch {
  static constexpr bool value = false;
};
template <class Tc>
struct has_fetch<SrcLanczos<Tc, df>> {
  static constexpr bool value = true;
};

// vector kernels
template <class Tz>
cudaError_t launch_update(long long N, const Tz *z, const double *d1, double *d2_out, double *x,
                          State *S, cudaStream_t st);
cudaError_t launch_flip(const Geom &g, const double *src, double *dst, cudaStream_t st);
cudaError_t launch_fill(long long N, double *p, double v, cudaStream_t st);
cudaError_t launch_norm2(long long N, const double *v, State *S, double *partials,
                         cudaStream_t st);

}  // namespace st

// ------------------------------------------------------------------ handle (C type of st_handle)
struct st_handle {
  st_problem prob;
  st::Geom g;
  st::PrecPlan pp;
  cudaStream_t stream;
  int device;
  bool mixed;
  // device memory
  void *tables;          // face coefficients, spectral tables, twiddles (one allocation)
  double *V[2];          // Lanczos vectors vhat
  void *Z[2];            // preconditioned vectors (double, or float in ST_MIXED)
  double *D[2];          // MINRES directions
  double *q;             // stencil output (a df array in ST_MIXED)
  st::df *Xdf;           // ST_MIXED: double-float solution accumulator
  double *partials;      // per-block partial sums
  st::State *S;          // device scalars
  double *hbuf_in, *hbuf_out;  // device staging for st_solve_host
  double *gfx, *gfy;     // face-gradient scratch for st_grad_a
  void *cheb;            // P_theta, 2D/3D varying a: Chebyshev scalars and scratch vectors
  // the tensor-core operand images the handle was built with (the autotuner may switch a stage
  // to its CUDA-core kernel by clearing the plan's pointer; these keep the originals)
  const unsigned short *tc_time_img, *tc_y_img, *tc_z_img, *tc_x_img;
  const unsigned char *tc_dig_img;  // the float64 path's digit image of S_n (see PrecPlan::sdig)
  int fp64_dd_ok;        // the float64 preconditioner may take the double-float engine
  st::State *hS;         // pinned host mirror of S
  int partials_len;
  st::Prof prof;         // kernel-class timing (off unless st_profile_begin was called)
  // ST_MIXED single solves: iterations per grouped direction/solution update (1..kUpdRing), and
  // the z vectors beyond Z[0], Z[1] that keep the pending iterations' z_j (ugroup - 1 of them):
  // z_j lives in slot (j - 1) % (ugroup + 1) of Z[0], Z[1], Zx[0], ...
  int ugroup;
  float *Zx[st::kUpdRing - 1];
};


