// Host driver and C ABI of the solver: setup (face coefficients, spectral tables, workspace),
// the preconditioned MINRES loop (Paige-Saunders recurrences with device-resident scalars) and
// the mixed-precision iterative refinement around it.
//
// One MINRES iteration k (1-based) is, on the handle's stream:
//   1. stencil:  p = Y T z_k / beta_k and alpha_k = <p, z_k/beta_k>            (st_stencil.cu)
//   2. prec:     vhat_{k+1} = p - (alpha_k/beta_k) vhat_k - (beta_k/beta_{k-1}) vhat_{k-1}
//                fused into the load of the first spatial DST, then z_{k+1} = P^-1 vhat_{k+1},
//                beta_{k+1}^2 = <vhat_{k+1}, z_{k+1}> and the Givens step (st_prec.cu,
//                st_time_tc.cu)
//   3. update:   d_k = (z_k/beta_k - delta d_{k-1} - eps d_{k-2})/rho,  x += c eta d_k; the
//                mixed single solve applies it for G iterations at once (k_update_group_df)
// Scalars never leave the device inside the loop; the host reads the state after each chunk of
// iterations to learn whether the device-side stopping test has fired, and sizes the next chunk
// from the observed convergence rate.  Kernels launched after that point return at entry.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <tuple>
#include <new>
#include <vector>

#include "st_internal.cuh"

using namespace st;

namespace st {
namespace {

constexpr int kNT = 256;
constexpr int kStreamBlocks = 152 * 8;

template <class Tz>
__global__ void __launch_bounds__(kNT)
    k_update(long long N, const Tz *__restrict__ z, const double *__restrict__ d1,
             double *__restrict__ d2, double *__restrict__ x, const State *S) {
  if (!S->active) return;
  const double cz = S->dz, c1 = S->d1, c2 = S->d2, cx = S->xc;
  for (long long i = blockIdx.x * (long long)kNT + threadIdx.x; i < N;
       i += (long long)gridDim.x * kNT) {
    const double d = cz * (double)z[i] + c1 * d1[i] + c2 * d2[i];
    d2[i] = d;
    x[i] += cx * d;
  }
}

// dst = Y src (block order reversed); in place when dst == src.
__global__ void k_flip(long long m, int n, const double *src, double *dst) {
  const long long total = (dst == src) ? (long long)(n / 2) * m : (long long)n * m;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const long long k = e / m, p = e - k * m;
    const long long a = k * m + p, b = (long long)(n - 1 - k) * m + p;
    if (dst == src) {
      const double t = dst[a];
      dst[a] = dst[b];
      dst[b] = t;
    } else {
      dst[b] = src[a];
    }
  }
}

__global__ void k_fill(long long N, double *p, double v) {
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < N;
       e += (long long)gridDim.x * blockDim.x)
    p[e] = v;
}

__global__ void __launch_bounds__(kNT)
    k_norm2(long long N, const double *__restrict__ v, State *S, double *__restrict__ partials) {
  __shared__ double red[32];
  double acc = 0.0;
  for (long long i = blockIdx.x * (long long)kNT + threadIdx.x; i < N;
       i += (long long)gridDim.x * kNT) {
    const double t = v[i];
    acc += t * t;
  }
  double tot;
  if (last_block_reduce<kNT>(acc, partials, &S->counter[CNT_NORM], gridDim.x, blockIdx.x, red,
                             &tot) &&
      threadIdx.x == 0)
    S->bnorm2 = tot;
}

}  // namespace

namespace {
// ------------------------------------------------------------------ double-float vectors
// Mixed path: vhat, d and x are double-floats (hi + lo float32 pairs, ~46 significant bits);
// the per-element arithmetic runs on the float32 pipes (see st_df.cuh).
//
// Grouped direction and solution update (mixed solves, single and batched).  The direction
// recurrence d_j = dz_j z_j + d1_j d_{j-1} + d2_j d_{j-2} and the solution update x += xc_j d_j
// consume the preconditioned vectors z_j but feed nothing back into the Lanczos recurrence, so
// the updates of up to kUpdRing iterations are applied in one pass: each element reads its
// pending z_j (one float32 vector per iteration), the two latest directions and x once, runs the
// recurrence in registers with every iteration's scalars (State::ucoef) and writes back the two
// latest directions and x.  With G iterations per pass the update moves 4 + 48/G bytes per unknown and
// iteration instead of 44, and every element goes through the same float32 operations in the
// same order, whatever G.
//
// The pending iterations are upd + 1 .. k of the device state: the pass reads both counters at
// entry and its last block to finish sets upd = k, so a pass with nothing pending returns at once
// and a pass never applies an iteration twice.  da holds d_upd and db d_{upd-1} on entry, d_k and
// d_{k-1} on exit; z_j is in zr.p[(j - 1) % zr.len].
struct ZRing {
  const float *p[kUpdRing + 1];
  int len;
};

// a shared-memory load the compiler may not hoist out of the element loop: holding every
// iteration's coefficients in registers (64 of them) would halve the resident warps
__device__ __forceinline__ float4 lds_f4(const float4 *p) {
  float4 v;
  asm volatile("ld.shared.v4.f32 {%0, %1, %2, %3}, [%4];"
               : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w)
               : "r"((unsigned)__cvta_generic_to_shared(p)));
  return v;
}

// The G steps of one element: d_j = dz_j z_j + d1_j d_{j-1} + d2_j d_{j-2}, x += xc_j d_j, with the
// scalars of each pending iteration read from shared memory.
__device__ __forceinline__ void upd_steps(const float (&zv)[kUpdRing], int np,
                                          const float4 (*sc)[2], df &d1, df &d2, float &xs,
                                          float &xt) {
#pragma unroll
  for (int j = 0; j < kUpdRing; ++j) {
    if (j < np) {
      const float4 a = lds_f4(&sc[j][0]), b = lds_f4(&sc[j][1]);
      const df cz{a.x, a.y}, c1{a.z, a.w}, c2{b.x, b.y}, cx{b.z, b.w};
      // the sum starts as the exact product cz.hi z plus its low-order terms
      float s, t;
      two_prod(cz.hi, zv[j], s, t);
      t = fmaf(cz.lo, zv[j], t);
      dacc_prod(s, t, c1, d1);
      dacc_prod(s, t, c2, d2);
      const df d = df_from_sum(s, t);
      dacc_prod(xs, xt, cx, d);
      const df xn = df_from_sum(xs, xt);
      xs = xn.hi;
      xt = xn.lo;
      d2 = d1;
      d1 = d;
    }
  }
}

// ILP elements per thread and trip (ILP = 2: two elements a grid stride apart, every load of
// both issued before the arithmetic of either; three blocks per SM instead of four)
template <int ILP>
__global__ void __launch_bounds__(kNT, ILP == 1 ? 4 : 3)
    k_update_group_df(long long N, ZRing zr, df *__restrict__ da, df *__restrict__ db,
                      df *__restrict__ x, State *S) {
  // per pending iteration: {dz.hi, dz.lo, d1.hi, d1.lo}, {d2.hi, d2.lo, xc.hi, xc.lo}
  __shared__ float4 sc[kUpdRing][2];
  __shared__ const float *sz[kUpdRing];
  const int kd = S->k, u = S->upd;
  const int np = kd - u;
  if (np <= 0 || np > kUpdRing) return;  // nothing pending (more than a ring never happens)
  if (threadIdx.x < 2 * np) {
    const int j = threadIdx.x >> 1, h = threadIdx.x & 1;
    const df *c = S->ucoef[(u + j) % kUpdRing] + 2 * h;
    sc[j][h] = make_float4(c[0].hi, c[0].lo, c[1].hi, c[1].lo);
  }
  if (threadIdx.x < np) sz[threadIdx.x] = zr.p[(u + threadIdx.x) % zr.len];
  __syncthreads();
  const long long stride = (long long)gridDim.x * kNT;
  for (long long i0 = blockIdx.x * (long long)kNT + threadIdx.x; i0 < N; i0 += ILP * stride) {
    float zv[ILP][kUpdRing];
    df d1[ILP], d2[ILP];
    float xs[ILP], xt[ILP];
    bool in[ILP];
#pragma unroll
    for (int e = 0; e < ILP; ++e) {
      const long long i = i0 + e * stride;
      in[e] = i < N;
      if (in[e]) {
#pragma unroll
        for (int j = 0; j < kUpdRing; ++j)
          if (j < np) zv[e][j] = sz[j][i];
        d1[e] = da[i];
        d2[e] = db[i];
        const df xo = x[i];
        xs[e] = xo.hi;
        xt[e] = xo.lo;
      }
    }
#pragma unroll
    for (int e = 0; e < ILP; ++e) {
      if (in[e]) {
        const long long i = i0 + e * stride;
        upd_steps(zv[e], np, sc, d1[e], d2[e], xs[e], xt[e]);
        da[i] = d1[e];
        db[i] = d2[e];
        x[i] = df{xs[e], xt[e]};
      }
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    const unsigned prev = atomicAdd(&S->counter[CNT_UPD], 1u);
    if (prev == gridDim.x - 1) {
      S->upd = kd;
      S->counter[CNT_UPD] = 0;
    }
  }
}

__global__ void k_flip_to_df(long long m, int n, const double *__restrict__ src,
                             df *__restrict__ dst) {
  const long long total = (long long)n * m;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const long long k = e / m, p = e - k * m;
    dst[(long long)(n - 1 - k) * m + p] = df_of_double(src[e]);
  }
}

__global__ void k_df_to_double(long long N, const df *__restrict__ src, double *__restrict__ dst) {
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < N;
       e += (long long)gridDim.x * blockDim.x)
    dst[e] = df_to_double(src[e]);
}
}  // namespace

// Devices on which a tensor-core kernel had to exit without releasing its tensor memory (see
// State::tmem_held): a later kernel that allocates tensor memory there could wait for it forever,
// so every call on such a device returns ST_ERR_TIMEOUT for the rest of the process.
namespace {
constexpr int kMaxDevices = 64;
std::atomic<int> g_device_closed[kMaxDevices];
}  // namespace

void close_device(int dev) {
  if (dev >= 0 && dev < kMaxDevices) g_device_closed[dev].store(1);
}

bool device_closed(int dev) {
  return dev >= 0 && dev < kMaxDevices && g_device_closed[dev].load() != 0;
}

double inner_floor() {
  static const double f = [] {
    const char *v = std::getenv("ST_INNER_FLOOR");
    const double x = v ? std::atof(v) : 0.0;
    return (x > 0.0 && x < 1.0) ? x : 1e-7;
  }();
  return f;
}

int update_group() {
  const char *v = std::getenv("ST_UPDATE_GROUP");
  const int x = v ? std::atoi(v) : 0;
  return (x >= 1 && x <= kUpdRing) ? x : kUpdRing;
}

thread_local Prof *t_prof = nullptr;

void prof_begin(int cls, cudaStream_t st) {
  Prof *p = t_prof;
  if (!p || !p->on) return;
  p->launches[cls] += 1;
  if (p->used < p->cap) {
    p->cls[p->used] = cls;
    cudaEventRecord(p->ev[2 * p->used], st);
  }
}

void prof_end(cudaStream_t st) {
  Prof *p = t_prof;
  if (!p || !p->on) return;
  if (p->used < p->cap) {
    cudaEventRecord(p->ev[2 * p->used + 1], st);
    p->used += 1;
  }
}

template <class Tz>
cudaError_t launch_update(long long N, const Tz *z, const double *d1, double *d2_out, double *x,
                          State *S, cudaStream_t st) {
  prof_begin(KC_UPDATE, st);
  k_update<Tz><<<kStreamBlocks, kNT, 0, st>>>(N, z, d1, d2_out, x, S);
  prof_end(st);
  return cudaGetLastError();
}

cudaError_t launch_flip(const Geom &g, const double *src, double *dst, cudaStream_t st) {
  prof_begin(KC_AUX, st);
  k_flip<<<kStreamBlocks, kNT, 0, st>>>(g.m, g.n, src, dst);
  prof_end(st);
  return cudaGetLastError();
}

cudaError_t launch_fill(long long N, double *p, double v, cudaStream_t st) {
  prof_begin(KC_AUX, st);
  k_fill<<<kStreamBlocks, kNT, 0, st>>>(N, p, v);
  prof_end(st);
  return cudaGetLastError();
}

// elements per thread and trip of the grouped update: two (220.7 against 244.6 us per 8-iteration
// pass at 255^2 x 256, the same iterates), or one with ST_UPDATE_ILP=1
int update_ilp() {
  static const int v = [] {
    const char *e = std::getenv("ST_UPDATE_ILP");
    return (e && e[0] == '1') ? 1 : 2;
  }();
  return v;
}

float *zslot(st_handle *h, int s) { return s < 2 ? (float *)h->Z[s] : h->Zx[s - 2]; }

// applies every pending direction/solution update of a mixed solve (see k_update_group_df); the
// device state decides how many
cudaError_t launch_update_group(st_handle *h, cudaStream_t st) {
  ZRing zr{};
  zr.len = h->ugroup + 1;
  for (int s = 0; s < zr.len; ++s) zr.p[s] = zslot(h, s);
  prof_begin(KC_UPDATE, st);
  if (update_ilp() == 2)
    k_update_group_df<2><<<kStreamBlocks, kNT, 0, st>>>(h->g.N, zr, (df *)h->D[0],
                                                        (df *)h->D[1], h->Xdf, h->S);
  else
    k_update_group_df<1><<<kStreamBlocks, kNT, 0, st>>>(h->g.N, zr, (df *)h->D[0],
                                                        (df *)h->D[1], h->Xdf, h->S);
  prof_end(st);
  return cudaGetLastError();
}

cudaError_t launch_flip_to_df(const Geom &g, const double *src, df *dst, cudaStream_t st) {
  prof_begin(KC_AUX, st);
  k_flip_to_df<<<kStreamBlocks, kNT, 0, st>>>(g.m, g.n, src, dst);
  prof_end(st);
  return cudaGetLastError();
}

cudaError_t launch_df_to_double(long long N, const df *src, double *dst, cudaStream_t st) {
  prof_begin(KC_AUX, st);
  k_df_to_double<<<kStreamBlocks, kNT, 0, st>>>(N, src, dst);
  prof_end(st);
  return cudaGetLastError();
}

cudaError_t launch_norm2(long long N, const double *v, State *S, double *partials,
                         cudaStream_t st) {
  prof_begin(KC_AUX, st);
  k_norm2<<<kStreamBlocks, kNT, 0, st>>>(N, v, S, partials);
  prof_end(st);
  return cudaGetLastError();
}

}  // namespace st

namespace {
// Makes the handle's profiler the current one for the duration of a C-ABI call.
struct ProfScope {
  Prof *saved;
  explicit ProfScope(st_handle *h) : saved(t_prof) { t_prof = h ? &h->prof : nullptr; }
  ~ProfScope() { t_prof = saved; }
};

void prof_free(Prof &p) {
  if (p.ev) {
    for (int i = 0; i < 2 * p.cap; ++i) cudaEventDestroy(p.ev[i]);
    delete[] p.ev;
    delete[] p.cls;
  }
  p.ev = nullptr;
  p.cls = nullptr;
  p.cap = p.used = 0;
  p.on = 0;
}
}  // namespace

namespace {

bool pow2(int v) { return v > 0 && (v & (v - 1)) == 0; }

int check_problem(const st_problem *p) {
  if (!p) return ST_ERR_ARG;
  if (p->dim < 1 || p->dim > 3) return ST_ERR_ARG;
  if (p->mx < 3 || p->mx > 1023 || !pow2(p->mx + 1)) return ST_ERR_ARG;
  if (p->dim == 1 && p->my != 1) return ST_ERR_ARG;
  if (p->dim >= 2 && (p->my < 3 || p->my > 1023 || !pow2(p->my + 1))) return ST_ERR_ARG;
  if (p->dim == 3 && (p->mz < 3 || p->mz > 1023 || !pow2(p->mz + 1))) return ST_ERR_ARG;
  if (p->dim < 3 && p->mz != 0 && p->mz != 1) return ST_ERR_ARG;
  if (p->n < 1 || p->n > 1024) return ST_ERR_ARG;
  {
    // element indices of a space-time vector stay below 2^31 (32-bit index arithmetic)
    const long long mz = (p->dim == 3) ? p->mz : 1;
    if ((long long)p->n * p->mx * p->my * mz > 2147483647LL) return ST_ERR_ARG;
    // the stencil kernels put the my*mz rows, 8 per block, on the grid's second axis
    if (p->dim == 3 && (long long)p->my * mz > 65535LL * 8) return ST_ERR_ARG;
  }
  if (!(p->T > 0.0) || !std::isfinite(p->T)) return ST_ERR_ARG;
  if (p->scheme != ST_THETA && p->scheme != ST_BDF2) return ST_ERR_ARG;
  if (p->scheme == ST_THETA && !(p->theta >= 0.0 && p->theta <= 1.0)) return ST_ERR_ARG;
  if (p->prec != ST_PREC_PH && p->prec != ST_PREC_PTHETA) return ST_ERR_ARG;
  if (p->precision != ST_FP64 && p->precision != ST_MIXED) return ST_ERR_ARG;
  if (p->prec == ST_PREC_PTHETA && p->scheme != ST_THETA) return ST_ERR_ARG;
  {
    const bool cheb = p->prec == ST_PREC_PTHETA && p->a_nodal != nullptr && p->dim >= 2;
    if (p->inner_degree < 0 || p->inner_degree > ST_PTHETA_MAX_DEGREE) return ST_ERR_ARG;
    if (!cheb && p->inner_degree != 0) return ST_ERR_ARG;
  }
  if (p->a_nodal) {
    const long long cnt = (p->dim == 1)   ? (p->mx + 2)
                          : (p->dim == 2) ? (long long)(p->mx + 2) * (p->my + 2)
                                          : (long long)(p->mx + 2) * (p->my + 2) * (p->mz + 2);
    for (long long i = 0; i < cnt; ++i)
      if (!(p->a_nodal[i] >= 0.0) || !std::isfinite(p->a_nodal[i])) return ST_ERR_ARG;
    // every face on an interior grid line (the mean of its two nodes) must be positive, so that
    // K is symmetric positive definite; nodes may be zero (a can vanish on the boundary)
    const int mx = p->mx, my = (p->dim >= 2) ? p->my : 1, mz = (p->dim == 3) ? p->mz : 1;
    const long long sy = mx + 2, sz = (long long)(mx + 2) * (my + 2);
    auto at = [&](int K, int J, int I) -> double {
      if (p->dim == 1) return p->a_nodal[I];
      if (p->dim == 2) return p->a_nodal[(long long)J * sy + I];
      return p->a_nodal[(long long)K * sz + (long long)J * sy + I];
    };
    const int k0 = (p->dim == 3) ? 1 : 0, j0 = (p->dim >= 2) ? 1 : 0;
    for (int k = k0; k < k0 + mz; ++k)
      for (int j = j0; j < j0 + my; ++j)
        for (int i = 0; i <= mx; ++i)
          if (!(at(k, j, i) + at(k, j, i + 1) > 0.0)) return ST_ERR_ARG;  // x faces
    if (p->dim >= 2)
      for (int k = k0; k < k0 + mz; ++k)
        for (int j = 0; j <= my; ++j)
          for (int i = 1; i <= mx; ++i)
            if (!(at(k, j, i) + at(k, j + 1, i) > 0.0)) return ST_ERR_ARG;  // y faces
    if (p->dim == 3)
      for (int k = 0; k <= mz; ++k)
        for (int j = 1; j <= my; ++j)
          for (int i = 1; i <= mx; ++i)
            if (!(at(k, j, i) + at(k + 1, j, i) > 0.0)) return ST_ERR_ARG;  // z faces
  }
  return ST_OK;
}

int map_cuda(cudaError_t e) {
  if (e == cudaSuccess) return ST_OK;
  if (e == cudaErrorMemoryAllocation) return ST_ERR_OOM;
  return ST_ERR_CUDA;
}

#define ST_TRY(expr)                      \
  do {                                    \
    cudaError_t _e = (expr);              \
    if (_e != cudaSuccess) return map_cuda(_e); \
  } while (0)

// start of a call on handle h: its device current, and not closed (see close_device)
#define ST_ENTER(h)                                         \
  do {                                                      \
    ST_TRY(cudaSetDevice((h)->device));                     \
    if (device_closed((h)->device)) return ST_ERR_TIMEOUT;  \
  } while (0)

// Enough per-block partial sums for every launch shape the autotuner may pick: the stencil with
// its largest block target and the time kernel with its narrowest column tile (16).
int partials_needed(const Geom &g) {
  Geom gt = g;
  gt.st_target = 4864;
  int r = stencil_blocks(gt);
  const int a = stencil_blocks(g);
  if (a > r) r = a;
  const int b = time_blocks_for(g, PrecPlan{}, false);
  const int c = time_blocks_for(g, PrecPlan{}, true);
  const int d = (int)((g.m + 15) / 16);
  if (b > r) r = b;
  if (c > r) r = c;
  if (d > r) r = d;
  if (r < kStreamBlocks) r = kStreamBlocks;
  return r;
}

Geom geom_of(const st_problem *p) {
  Geom g{};
  g.dim = p->dim;
  g.mx = p->mx;
  g.my = (p->dim == 1) ? 1 : p->my;
  g.mz = (p->dim == 3) ? p->mz : 1;
  g.n = p->n;
  g.m = (long long)g.mx * g.my * g.mz;
  g.N = g.m * g.n;
  g.scheme = p->scheme;
  g.tau = p->T / p->n;
  g.theta = (p->scheme == ST_THETA) ? p->theta : 1.0;
  return g;
}

// face coefficients along x, y and z (the last two zero-length where the axis is absent)
size_t faces_x(const Geom &g) { return (size_t)g.mz * g.my * (g.mx + 1); }
size_t faces_y(const Geom &g) { return g.dim >= 2 ? (size_t)g.mz * (g.my + 1) * g.mx : 0; }
size_t faces_z(const Geom &g) { return g.dim == 3 ? (size_t)(g.mz + 1) * g.my * g.mx : 0; }

size_t table_doubles(const Geom &g) {
  const size_t faces = faces_x(g) + faces_y(g) + faces_z(g);
  const size_t spec = (size_t)g.mx + (size_t)g.my * g.mz + 5 * (size_t)g.n + 2 * (size_t)(g.n + 1);
  const size_t tw = (size_t)(g.mx + 1) * 2 + (size_t)(g.my + 1) * 2 +
                    (g.dim == 3 ? (size_t)(g.mz + 1) * 2 : 0);  // L/2 complex per axis
  return faces + spec + tw;
}
size_t table_floats(const Geom &g) {
  const size_t spec = (size_t)g.mx + (size_t)g.my * g.mz + 5 * (size_t)g.n + 2 * (size_t)(g.n + 1);
  const size_t tw = (size_t)(g.mx + 1) * 2 + (size_t)(g.my + 1) * 2 +
                    (g.dim == 3 ? (size_t)(g.mz + 1) * 2 : 0);
  return spec + tw;
}

// Chebyshev steps of the 2D/3D varying-a P_theta, 0 for every other preconditioner
int cheb_degree(const st_problem *p) {
  if (p->prec != ST_PREC_PTHETA || p->a_nodal == nullptr || p->dim < 2) return 0;
  return p->inner_degree > 0 ? p->inner_degree : ST_PTHETA_DEFAULT_DEGREE;
}

size_t cheb_coef_bytes(const Geom &g, int deg) {
  return ((size_t)deg * g.n * 2 * (sizeof(double) + sizeof(float)) + 255) / 256 * 256;
}

size_t workspace_bytes(const Geom &g, bool mixed, int cheb, int ugroup) {
  const size_t N = (size_t)g.N;
  size_t b = 0;
  if (mixed) b += (size_t)(ugroup - 1) * N * sizeof(float);  // grouped update: pending z_j
  if (cheb) b += cheb_coef_bytes(g, cheb) + 5 * N * sizeof(double);
  b += 2 * N * sizeof(double);                             // V
  b += 2 * N * (mixed ? sizeof(float) : sizeof(double));   // Z
  b += 2 * N * sizeof(double);                             // D
  b += N * sizeof(double);                                 // q
  if (mixed) b += N * sizeof(df);                          // x accumulator
  b += 2 * N * sizeof(double);                             // host staging
  b += (size_t)partials_needed(g) * sizeof(double);
  b += sizeof(State);
  b += ((size_t)g.my * (g.mx + 1) + (size_t)(g.my + 1) * g.mx) * sizeof(double);  // grad faces
  b += table_doubles(g) * sizeof(double) + table_floats(g) * sizeof(float) + 256;
  b += table_floats(g) * sizeof(dd) + 256;  // double-float copies of the spectral tables
  b += (faces_x(g) + faces_y(g) + faces_z(g)) * sizeof(df) + 256;  // df faces
  if (mixed && time_tc_supported(g.n)) b += time_tc_sop_halves(g.n) * 2;
  if (mixed && !time_tc_supported(g.n) && time_tc_long_supported(g.n))
    b += time_tc_long_bytes(g.n) + 256;
  if (mixed && g.dim >= 2 && dst_tc_supported(g.my)) b += time_tc_sop_halves(g.my) * 2 + 256;
  if (mixed && g.dim == 3 && dst_tc_supported(g.mz)) b += time_tc_sop_halves(g.mz) * 2 + 256;
  if (mixed && dst_tc_supported(g.mx)) b += time_tc_sop_halves(g.mx) * 2 + 256;
  if (!mixed && time_tcd_supported(g.n)) b += time_tcd_bytes(g.n) + 256;  // digits of S_n
  b += 256;  // alignment of the z image
  return b;
}

// Build every table on the host (float64 with float32 copies) and upload them in one go.
int build_tables(st_handle *h) {
  const Geom &g = h->g;
  const st_problem &p = h->prob;
  const int mx = g.mx, my = g.my, mz = g.mz, n = g.n;
  const double tau = g.tau;
  const double hx = 1.0 / (mx + 1), hy = (g.dim >= 2) ? 1.0 / (my + 1) : 1.0;
  const double hz = (g.dim == 3) ? 1.0 / (mz + 1) : 1.0;
  const double *A = p.a_nodal;
  // nodal a at node (K, J, I) of the grid with boundary nodes (K ignored below 3D, J in 1D)
  auto anode = [&](int K, int J, int I) -> double {
    if (!A) return 1.0;
    if (g.dim == 1) return A[I];
    if (g.dim == 2) return A[(long long)J * (mx + 2) + I];
    return A[((long long)K * (my + 2) + J) * (mx + 2) + I];
  };
  std::vector<double> cx(faces_x(g)), cy(faces_y(g)), cz(faces_z(g));
  for (int jz = 0; jz < mz; ++jz)
    for (int j = 0; j < my; ++j)
      for (int i = 0; i <= mx; ++i)
        cx[((size_t)jz * my + j) * (mx + 1) + i] =
            tau * 0.5 * (anode(jz + 1, j + 1, i) + anode(jz + 1, j + 1, i + 1)) / (hx * hx);
  if (g.dim >= 2)
    for (int jz = 0; jz < mz; ++jz)
      for (int j = 0; j <= my; ++j)
        for (int i = 0; i < mx; ++i)
          cy[((size_t)jz * (my + 1) + j) * mx + i] =
              tau * 0.5 * (anode(jz + 1, j, i + 1) + anode(jz + 1, j + 1, i + 1)) / (hy * hy);
  if (g.dim == 3)
    for (int k = 0; k <= mz; ++k)
      for (int j = 0; j < my; ++j)
        for (int i = 0; i < mx; ++i)
          cz[((size_t)k * my + j) * mx + i] =
              tau * 0.5 * (anode(k, j + 1, i + 1) + anode(k + 1, j + 1, i + 1)) / (hz * hz);
  // diagonal-averaged stiffness matrix (times tau): mean diagonal, mean x-, y- and z-couplings.
  // The small eigenvalues d - 2 e_x cos - 2 e_y cos - 2 e_z cos cancel strongly, so the sums are
  // compensated (Neumaier) to keep their own rounding at the level of one ulp.
  struct CSum {
    double s = 0.0, c = 0.0;
    void add(double x) {
      const double t = s + x;
      c += (std::fabs(s) >= std::fabs(x)) ? (s - t) + x : (x - t) + s;
      s = t;
    }
    double get() const { return s + c; }
  };
  CSum dsum;
  for (int jz = 0; jz < mz; ++jz)
    for (int j = 0; j < my; ++j)
      for (int i = 0; i < mx; ++i) {
        const size_t row = (size_t)jz * my + j;
        dsum.add(cx[row * (mx + 1) + i]);
        dsum.add(cx[row * (mx + 1) + i + 1]);
        if (g.dim >= 2) {
          const size_t ys = ((size_t)jz * (my + 1) + j) * mx + i;
          dsum.add(cy[ys]);
          dsum.add(cy[ys + mx]);
        }
        if (g.dim == 3) {
          dsum.add(cz[row * mx + i]);
          dsum.add(cz[row * mx + i + (size_t)mx * my]);
        }
      }
  const double dbar = dsum.get() / (double)g.m;
  double ex = 0.0, ey = 0.0, ez = 0.0;
  if (mx > 1) {
    CSum sx;
    for (int r = 0; r < my * mz; ++r)
      for (int i = 1; i < mx; ++i) sx.add(cx[(size_t)r * (mx + 1) + i]);
    ex = sx.get() / ((double)my * mz * (mx - 1));
  }
  if (g.dim >= 2 && my > 1) {
    CSum sy;
    for (int jz = 0; jz < mz; ++jz)
      for (int j = 1; j < my; ++j)
        for (int i = 0; i < mx; ++i) sy.add(cy[((size_t)jz * (my + 1) + j) * mx + i]);
    ey = sy.get() / ((double)mz * (my - 1) * mx);
  }
  if (g.dim == 3 && mz > 1) {
    CSum sz;
    for (int k = 1; k < mz; ++k)
      for (int j = 0; j < my; ++j)
        for (int i = 0; i < mx; ++i) sz.add(cz[((size_t)k * my + j) * mx + i]);
    ez = sz.get() / ((double)(mz - 1) * my * mx);
  }
  const double PI = 3.14159265358979323846;
  // muy holds the y- and z-parts together, indexed by the row jz*my + jy
  std::vector<double> mux(mx), muy((size_t)my * mz), hk(n), ck(n), sk(n), lh(n), lht(n),
      sintab(2 * (n + 1));
  for (int i = 0; i < mx; ++i) mux[i] = dbar - 2.0 * ex * std::cos((i + 1) * PI / (mx + 1));
  for (int jz = 0; jz < mz; ++jz)
    for (int j = 0; j < my; ++j) {
      double v = (g.dim >= 2) ? -2.0 * ey * std::cos((j + 1) * PI / (my + 1)) : 0.0;
      if (g.dim == 3) v += -2.0 * ez * std::cos((jz + 1) * PI / (mz + 1));
      muy[(size_t)jz * my + j] = v;
    }
  // P_theta with a varying 2D/3D coefficient: the Chebyshev inner map is preconditioned by the
  // a = abar operator, so the spatial tables hold tau abar times the eigenvalues of K0 (a = 1),
  // 4 sin^2(i pi / (2(mx+1))) / hx^2 per axis, instead of the averaged K
  const int cheb = cheb_degree(&p);
  double f_min = 0.0, f_max = 0.0, f_bar = 0.0, mu0_max = 0.0;
  if (cheb) {
    CSum fs;
    f_min = INFINITY;
    f_max = 0.0;
    auto face = [&](double a) {
      fs.add(a);
      f_min = std::min(f_min, a);
      f_max = std::max(f_max, a);
    };
    for (int jz = 0; jz < mz; ++jz)
      for (int j = 0; j < my; ++j)
        for (int i = 0; i <= mx; ++i)
          face(0.5 * (anode(jz + 1, j + 1, i) + anode(jz + 1, j + 1, i + 1)));
    for (int jz = 0; jz < mz; ++jz)
      for (int j = 0; j <= my; ++j)
        for (int i = 0; i < mx; ++i)
          face(0.5 * (anode(jz + 1, j, i + 1) + anode(jz + 1, j + 1, i + 1)));
    if (g.dim == 3)
      for (int k = 0; k <= mz; ++k)
        for (int j = 0; j < my; ++j)
          for (int i = 0; i < mx; ++i)
            face(0.5 * (anode(k, j + 1, i + 1) + anode(k + 1, j + 1, i + 1)));
    f_bar = fs.get() / (double)(faces_x(g) + faces_y(g) + faces_z(g));
    auto mu0 = [&](int i, int len, double h2) {
      const double sv = std::sin((i + 1) * PI / (2.0 * (len + 1)));
      return 4.0 * sv * sv / h2;
    };
    for (int i = 0; i < mx; ++i) mux[i] = tau * f_bar * mu0(i, mx, hx * hx);
    for (int jz = 0; jz < mz; ++jz)
      for (int j = 0; j < my; ++j) {
        double mu = mu0(j, my, hy * hy);
        if (g.dim == 3) mu += mu0(jz, mz, hz * hz);
        muy[(size_t)jz * my + j] = tau * f_bar * mu;
      }
    mu0_max = mu0(mx - 1, mx, hx * hx) + mu0(my - 1, my, hy * hy);
    if (g.dim == 3) mu0_max += mu0(mz - 1, mz, hz * hz);
  }
  const double th = g.theta;
  for (int k = 1; k <= n; ++k) {
    const double x = k * PI / (n + 1);
    const double sh = std::sin(0.5 * x);
    hk[k - 1] = 2.0 * sh * sh;
    ck[k - 1] = std::cos(x);
    sk[k - 1] = std::sin(x);
    lh[k - 1] = 2.0 * sh;
    lht[k - 1] = std::sqrt(th * th + (1 - th) * (1 - th) + 2.0 * th * (1 - th) * std::cos(x));
  }
  const double sn = std::sqrt(2.0 / (n + 1));
  for (int r = 0; r < 2 * (n + 1); ++r) sintab[r] = sn * std::sin(r * PI / (n + 1));
  // Chebyshev scalars per step j and frequency k.  a_min K0 <= K <= a_max K0 over the faces, and
  // (lam + c a mu)/(lam + c abar mu) is monotone in mu and 1 at mu = 0, so the spectrum of
  // B_k^-1 A_k lies in [alpha, beta] = (lam + c {a_min, a_max} mu0_max)/(lam + c abar mu0_max),
  // c = lam_Htheta,k tau.  With centre and half-width of that interval (Saad, Alg. 12.1):
  // s_0 = 1/centre, rho_0 = half/centre; rho_j = 1/(2 centre/half - rho_{j-1}),
  // a_j = rho_j rho_{j-1}, s_j = 2 rho_j/half.  A zero-width interval (B_k = A_k) is solved by the
  // first step: the later scalars are zero.
  std::vector<double> cheb_a((size_t)cheb * n), cheb_s((size_t)cheb * n);
  bool cheb_all_exact = true;
  for (int k = 0; k < n && cheb; ++k) {
    const double c = lht[k] * tau;
    const double den = lh[k] + c * f_bar * mu0_max;
    const double alpha = (lh[k] + c * std::min(f_min, f_bar) * mu0_max) / den;
    const double beta = (lh[k] + c * std::max(f_max, f_bar) * mu0_max) / den;
    const double centre = 0.5 * (beta + alpha), half = 0.5 * (beta - alpha);
    cheb_a[k] = 0.0;
    cheb_s[k] = 1.0 / centre;
    const bool exact = !(half > 1e-14 * centre);
    cheb_all_exact = cheb_all_exact && exact;
    const double sigma1 = exact ? 0.0 : centre / half;
    double rho = exact ? 0.0 : 1.0 / sigma1;
    for (int j = 1; j < cheb; ++j) {
      double aj = 0.0, sj = 0.0;
      if (!exact) {
        const double rn = 1.0 / (2.0 * sigma1 - rho);
        aj = rn * rho;
        sj = 2.0 * rn / half;
        rho = rn;
      }
      cheb_a[(size_t)j * n + k] = aj;
      cheb_s[(size_t)j * n + k] = sj;
    }
  }
  const int Lx = 2 * (mx + 1), Ly = 2 * (my + 1), Lz = 2 * (mz + 1);
  std::vector<double> twx(Lx), twy(Ly), twz(g.dim == 3 ? Lz : 0);
  for (int j = 0; j < Lx / 2; ++j) {
    twx[2 * j] = std::cos(2.0 * PI * j / Lx);
    twx[2 * j + 1] = -std::sin(2.0 * PI * j / Lx);
  }
  for (int j = 0; j < Ly / 2; ++j) {
    twy[2 * j] = std::cos(2.0 * PI * j / Ly);
    twy[2 * j + 1] = -std::sin(2.0 * PI * j / Ly);
  }
  for (size_t j = 0; j < twz.size() / 2; ++j) {
    twz[2 * j] = std::cos(2.0 * PI * (double)j / Lz);
    twz[2 * j + 1] = -std::sin(2.0 * PI * (double)j / Lz);
  }
  // layout: doubles [cx cy cz mux muy hk ck sk lh lht sintab twx twy twz] then floats
  // [mux ... twz]
  std::vector<double> hd;
  hd.reserve(table_doubles(g));
  auto app = [&](const std::vector<double> &v) {
    size_t off = hd.size();
    hd.insert(hd.end(), v.begin(), v.end());
    return off;
  };
  const size_t o_cx = app(cx), o_cy = app(cy), o_cz = app(cz);
  const size_t o_mux = app(mux), o_muy = app(muy), o_hk = app(hk), o_ck = app(ck), o_sk = app(sk),
               o_lh = app(lh), o_lht = app(lht), o_sin = app(sintab), o_twx = app(twx),
               o_twy = app(twy), o_twz = app(twz);
  const size_t nd = hd.size();
  std::vector<float> hf(nd - o_mux);
  for (size_t i = o_mux; i < nd; ++i) hf[i - o_mux] = (float)hd[i];
  const size_t bytes_d = nd * sizeof(double);
  const size_t bytes_f = hf.size() * sizeof(float);
  // fp16 S_n image for the tensor-core time kernel (mixed precision, supported n)
  std::vector<unsigned short> sop;
  const char *no_tc = std::getenv("ST_DISABLE_TENSOR_CORES");
  const bool use_tc = p.precision == ST_MIXED && !(no_tc && no_tc[0] == '1');
  bool long_tc = false;
  if (use_tc && time_tc_supported(n)) {
    sop.resize(time_tc_sop_halves(n));
    time_tc_build_sop(n, sop.data());
  } else if (use_tc && time_tc_long_supported(n)) {
    // streamed chunks for 256 < n <= 512, in the same slot of the table allocation
    sop.resize(time_tc_long_bytes(n) / 2);
    time_tc_long_build(n, sop.data());
    long_tc = true;
  }
  const size_t o_sop = (bytes_d + bytes_f + 255) / 256 * 256;
  // double-float copies of the face coefficients
  std::vector<df> cdf(cx.size() + cy.size() + cz.size());
  for (size_t i = 0; i < cx.size(); ++i) cdf[i] = df_of_double(cx[i]);
  for (size_t i = 0; i < cy.size(); ++i) cdf[cx.size() + i] = df_of_double(cy[i]);
  for (size_t i = 0; i < cz.size(); ++i) cdf[cx.size() + cy.size() + i] = df_of_double(cz[i]);
  const size_t o_cdf = (o_sop + sop.size() * sizeof(unsigned short) + 255) / 256 * 256;
  // fp16 S_my / S_mz images for the tensor-core y- and z-DSTs (mixed precision, supported lengths)
  std::vector<unsigned short> sopy, sopz, sopx;
  if (p.precision == ST_MIXED && g.dim >= 2 && dst_tc_supported(g.my) &&
      !(no_tc && no_tc[0] == '1')) {
    sopy.resize(time_tc_sop_halves(g.my));
    time_tc_build_sop(g.my, sopy.data());
  }
  if (p.precision == ST_MIXED && g.dim == 3 && dst_tc_supported(g.mz) &&
      !(no_tc && no_tc[0] == '1')) {
    sopz.resize(time_tc_sop_halves(g.mz));
    time_tc_build_sop(g.mz, sopz.data());
  }
  // and S_mx for the tensor-core x-DST of the last spatial pass
  if (p.precision == ST_MIXED && dst_tc_supported(g.mx) && !(no_tc && no_tc[0] == '1')) {
    sopx.resize(time_tc_sop_halves(g.mx));
    time_tc_build_sop(g.mx, sopx.data());
  }
  const size_t o_sopy = (o_cdf + cdf.size() * sizeof(df) + 255) / 256 * 256;
  const size_t o_sopz = (o_sopy + sopy.size() * sizeof(unsigned short) + 255) / 256 * 256;
  const size_t o_sopx = (o_sopz + sopz.size() * sizeof(unsigned short) + 255) / 256 * 256;
  // double-float copies of the spectral tables and twiddles for the float64 preconditioner's
  // double-float engine (each value split exactly: hi the nearest float, lo the rest)
  std::vector<dd> hdd(nd - o_mux);
  for (size_t i = o_mux; i < nd; ++i) hdd[i - o_mux] = dd(hd[i]);
  const size_t o_dd = (o_sopx + sopx.size() * sizeof(unsigned short) + 255) / 256 * 256;
  // integer-digit image of S_n for the float64 path's tensor-core time stage (double-float
  // engine, P_H / P-hat and constant-coefficient P_theta)
  std::vector<unsigned char> sdig;
  int sdig_e = 0;
  if (p.precision == ST_FP64 && time_tcd_supported(n) && !(no_tc && no_tc[0] == '1')) {
    sdig.resize(time_tcd_bytes(n));
    sdig_e = time_tcd_build(n, sdig.data());
  }
  const size_t o_dig = (o_dd + hdd.size() * sizeof(dd) + 255) / 256 * 256;
  const size_t bytes = o_dig + sdig.size();
  ST_TRY(cudaMalloc(&h->tables, bytes));
  ST_TRY(cudaMemcpy(h->tables, hd.data(), bytes_d, cudaMemcpyHostToDevice));
  ST_TRY(cudaMemcpy((char *)h->tables + bytes_d, hf.data(), bytes_f, cudaMemcpyHostToDevice));
  if (!sop.empty())
    ST_TRY(cudaMemcpy((char *)h->tables + o_sop, sop.data(), sop.size() * sizeof(unsigned short),
                      cudaMemcpyHostToDevice));
  ST_TRY(cudaMemcpy((char *)h->tables + o_cdf, cdf.data(), cdf.size() * sizeof(df),
                    cudaMemcpyHostToDevice));
  if (!sopy.empty())
    ST_TRY(cudaMemcpy((char *)h->tables + o_sopy, sopy.data(),
                      sopy.size() * sizeof(unsigned short), cudaMemcpyHostToDevice));
  if (!sopz.empty())
    ST_TRY(cudaMemcpy((char *)h->tables + o_sopz, sopz.data(),
                      sopz.size() * sizeof(unsigned short), cudaMemcpyHostToDevice));
  if (!sopx.empty())
    ST_TRY(cudaMemcpy((char *)h->tables + o_sopx, sopx.data(),
                      sopx.size() * sizeof(unsigned short), cudaMemcpyHostToDevice));
  ST_TRY(cudaMemcpy((char *)h->tables + o_dd, hdd.data(), hdd.size() * sizeof(dd),
                    cudaMemcpyHostToDevice));
  if (!sdig.empty())
    ST_TRY(cudaMemcpy((char *)h->tables + o_dig, sdig.data(), sdig.size(),
                      cudaMemcpyHostToDevice));
  const double *D = (const double *)h->tables;
  const float *F = (const float *)((const char *)h->tables + bytes_d) - o_mux;
  h->g.cx = D + o_cx;
  h->g.cy = (g.dim >= 2) ? D + o_cy : nullptr;
  h->g.cz = (g.dim == 3) ? D + o_cz : nullptr;
  const df *CD = reinterpret_cast<const df *>((const char *)h->tables + o_cdf);
  h->g.cxd = CD;
  h->g.cyd = (g.dim >= 2) ? CD + cx.size() : nullptr;
  h->g.czd = (g.dim == 3) ? CD + cx.size() + cy.size() : nullptr;
  {
    // one face coefficient for the whole grid: the double-float stencil's uniform form
    const double c0 = cx.empty() ? 0.0 : cx[0];
    bool uni = !cx.empty() && !(std::getenv("ST_STENCIL_GENERAL") != nullptr);
    for (double v : cx) uni = uni && (v == c0);
    for (double v : cy) uni = uni && (v == c0);
    for (double v : cz) uni = uni && (v == c0);
    h->g.c_uniform = uni ? 1 : 0;
    h->g.c_uni = df_of_double(c0);
  }
  h->g.th_d = df_of_double(h->g.theta);
  h->g.omth_d = df_of_double(1.0 - h->g.theta);
  h->g.th_exact = (h->g.theta == 0.0 || h->g.theta == 0.5 || h->g.theta == 1.0) ? 1 : 0;
  PrecPlan &pp = h->pp;
  pp.pcr = (p.prec == ST_PREC_PTHETA && p.a_nodal != nullptr && g.dim == 1) ? 1 : 0;
  // every interval of zero width (a constant field): the steps after the first add exact zeros,
  // so one step gives the same map
  pp.cheb = (cheb > 1 && cheb_all_exact) ? 1 : cheb;
  if (cheb) {
    const size_t cb = cheb_coef_bytes(g, cheb);
    ST_TRY(cudaMalloc(&h->cheb, cb + 5 * (size_t)g.N * sizeof(double)));
    const size_t cnt = (size_t)cheb * n;
    std::vector<float> af(cnt), sf(cnt);
    for (size_t i = 0; i < cnt; ++i) {
      af[i] = (float)cheb_a[i];
      sf[i] = (float)cheb_s[i];
    }
    char *cbase = (char *)h->cheb;
    ST_TRY(cudaMemcpy(cbase, cheb_a.data(), cnt * sizeof(double), cudaMemcpyHostToDevice));
    ST_TRY(cudaMemcpy(cbase + cnt * sizeof(double), cheb_s.data(), cnt * sizeof(double),
                      cudaMemcpyHostToDevice));
    ST_TRY(cudaMemcpy(cbase + 2 * cnt * sizeof(double), af.data(), cnt * sizeof(float),
                      cudaMemcpyHostToDevice));
    ST_TRY(cudaMemcpy(cbase + 2 * cnt * sizeof(double) + cnt * sizeof(float), sf.data(),
                      cnt * sizeof(float), cudaMemcpyHostToDevice));
    pp.cheb_a_d = (const double *)cbase;
    pp.cheb_s_d = pp.cheb_a_d + cnt;
    pp.cheb_a_f = (const float *)(cbase + 2 * cnt * sizeof(double));
    pp.cheb_s_f = pp.cheb_a_f + cnt;
    pp.cheb_work = cbase + cb;
  }
  const unsigned short *sop_img =
      (sop.empty() || pp.pcr || pp.cheb) ? nullptr
                              : reinterpret_cast<const unsigned short *>((const char *)h->tables + o_sop);
  // the P_theta paths with varying a transform time alone (no scaling) on the tensor cores
  pp.sop_t1 = (!sop.empty() && !long_tc && (pp.pcr || pp.cheb) && dst_tc_len_supported(n))
                  ? reinterpret_cast<const unsigned short *>((const char *)h->tables + o_sop)
                  : nullptr;
  pp.sop = long_tc ? nullptr : sop_img;
  pp.sop_long = long_tc ? sop_img : nullptr;
  pp.sop_y = sopy.empty() ? nullptr
                          : reinterpret_cast<const unsigned short *>((const char *)h->tables + o_sopy);
  pp.sop_z = sopz.empty() ? nullptr
                          : reinterpret_cast<const unsigned short *>((const char *)h->tables + o_sopz);
  h->tc_time_img = pp.sop;
  h->tc_y_img = pp.sop_y;
  h->tc_z_img = pp.sop_z;
  // The last x pass runs on the tensor cores where mx + 1 allows (41.8 against 61.1 us per pass
  // for the FFT at 255^2 x 256); st_autotune times both, and ST_X_TENSOR_CORES=0 starts a handle
  // with the FFT.  The P_theta paths with varying a run their x passes through the Chebyshev and
  // PCR kernels.
  h->tc_x_img = (sopx.empty() || pp.pcr || pp.cheb)
                    ? nullptr
                    : reinterpret_cast<const unsigned short *>((const char *)h->tables + o_sopx);
  {
    const char *xtc = std::getenv("ST_X_TENSOR_CORES");
    pp.sop_x = (xtc && xtc[0] == '0') ? nullptr : h->tc_x_img;
  }
  pp.Lx = Lx;
  pp.Ly = Ly;
  pp.Lz = Lz;
  pp.twx_d = D + o_twx;
  pp.twy_d = D + o_twy;
  pp.twz_d = D + o_twz;
  pp.twx_f = F + o_twx;
  pp.twy_f = F + o_twy;
  pp.twz_f = F + o_twz;
  pp.spec_d = Spec<double>{D + o_mux, D + o_muy, D + o_hk, D + o_ck, D + o_sk, D + o_lh, D + o_lht,
                           D + o_sin, p.prec, p.scheme, th};
  pp.spec_f = Spec<float>{F + o_mux, F + o_muy, F + o_hk, F + o_ck, F + o_sk, F + o_lh, F + o_lht,
                          F + o_sin, p.prec, p.scheme, (float)th};
  const dd *DD = reinterpret_cast<const dd *>((const char *)h->tables + o_dd) - o_mux;
  pp.spec_dd = Spec<dd>{DD + o_mux, DD + o_muy, DD + o_hk, DD + o_ck, DD + o_sk, DD + o_lh,
                        DD + o_lht, DD + o_sin, p.prec, p.scheme, dd(th)};
  pp.twx_dd = DD + o_twx;
  pp.twy_dd = DD + o_twy;
  pp.twz_dd = DD + o_twz;
  pp.sdig = sdig.empty() ? nullptr : (const unsigned char *)h->tables + o_dig;
  pp.sdig_e = sdig_e;
  h->tc_dig_img = pp.sdig;
  // the float64 P_H / P-hat preconditioner runs its transforms in double-float unless
  // ST_FP64_ENGINE=dfma asks for float64 arithmetic; st_autotune times both and keeps the faster
  const char *eng = std::getenv("ST_FP64_ENGINE");
  pp.fp64_dd = (p.precision == ST_FP64 && !pp.pcr && !pp.cheb &&
                !(eng && std::strcmp(eng, "dfma") == 0))
                   ? 1
                   : 0;
  h->fp64_dd_ok = (p.precision == ST_FP64 && !pp.pcr && !pp.cheb) ? 1 : 0;
  return ST_OK;
}

void free_handle(st_handle *h) {
  if (!h) return;
  cudaFree(h->tables);
  for (int i = 0; i < 2; ++i) {
    cudaFree(h->V[i]);
    cudaFree(h->Z[i]);
    cudaFree(h->D[i]);
  }
  cudaFree(h->q);
  cudaFree(h->Xdf);
  cudaFree(h->partials);
  cudaFree(h->S);
  cudaFree(h->hbuf_in);
  cudaFree(h->hbuf_out);
  cudaFree(h->gfx);
  cudaFree(h->gfy);
  cudaFree(h->cheb);
  if (h->hS) cudaFreeHost(h->hS);
  for (int i = 0; i < kUpdRing - 1; ++i) cudaFree(h->Zx[i]);
  prof_free(h->prof);
  delete h;
}

// ---------------------------------------------------------------- MINRES driver
template <class Tz, class Tc>
cudaError_t launch_iteration(st_handle *h, int k, double *x) {
  const int c = (k - 1) & 1, o = k & 1;
  const Geom &g = h->g;
  cudaStream_t st = h->stream;
  Tz *zc = (Tz *)h->Z[c];
  Tz *zn = (Tz *)h->Z[o];
  cudaError_t e;
  e = launch_stencil<Tz>(g, SM_MINRES, zc, h->q, nullptr, h->S, h->partials, 0, st);
  if (e != cudaSuccess) return e;
  // Lanczos step (v_{k+1} over v_{k-1}) fused into the first transform of z_{k+1} = P^-1 v_{k+1}
  e = launch_prec_lanczos<Tc, double, Tz>(g, h->pp, h->q, h->V[c], h->V[o], zn, h->S, h->partials,
                                          st);
  if (e != cudaSuccess) return e;
  return launch_update<Tz>(g.N, zc, h->D[c], h->D[o], x, h->S, st);
}

// Mixed path iteration k: df vectors in V, D, q; float32 z_k in ring slot (k - 1) % (G + 1).
// The direction/solution update runs after every G-th iteration (G = ugroup) and applies the
// updates of the G iterations since the previous one; solve_mixed flushes the rest at the end
// of each inner run.
cudaError_t launch_iteration_mixed(st_handle *h, int k) {
  const int c = (k - 1) & 1, o = k & 1;
  const int R = h->ugroup + 1;
  const Geom &g = h->g;
  cudaStream_t st = h->stream;
  const float *zc = zslot(h, (k - 1) % R);
  float *zn = zslot(h, k % R);
  df *V0 = (df *)h->V[c], *V1 = (df *)h->V[o];
  df *q = (df *)h->q;
  cudaError_t e;
  e = launch_stencil_df(g, zc, q, h->S, h->partials, st);
  if (e != cudaSuccess) return e;
  e = launch_prec_lanczos<float, df, float>(g, h->pp, q, V0, V1, zn, h->S, h->partials, st);
  if (e != cudaSuccess) return e;
  if (k % h->ugroup == 0) return launch_update_group(h, st);
  return cudaSuccess;
}

int sync_state(st_handle *h) {
  ST_TRY(cudaMemcpyAsync(h->hS, h->S, sizeof(State), cudaMemcpyDeviceToHost, h->stream));
  ST_TRY(cudaStreamSynchronize(h->stream));
  if (h->hS->tmem_held) {
    close_device(h->device);
    return ST_ERR_TIMEOUT;
  }
  return ST_OK;
}

// the device keeps tmem_held: only the members before it are written
int push_state(st_handle *h) {
  refresh_df(h->hS);
  ST_TRY(cudaMemcpyAsync(h->S, h->hS, kStatePushBytes, cudaMemcpyHostToDevice, h->stream));
  return ST_OK;
}

// Start a MINRES run whose right-hand side b is already in V[0]; x keeps its content.
template <class Tz, class Tc>
int minres_start(st_handle *h, double target, int maxit) {
  const Geom &g = h->g;
  ST_TRY(cudaMemsetAsync(h->D[0], 0, g.N * sizeof(double), h->stream));
  ST_TRY(cudaMemsetAsync(h->D[1], 0, g.N * sizeof(double), h->stream));
  ST_TRY(cudaMemsetAsync(h->V[1], 0, g.N * sizeof(double), h->stream));
  State &s = *h->hS;
  const double bn = s.bnorm2;
  std::memset(&s, 0, sizeof(State));
  s.bnorm2 = bn;
  s.active = 1;
  s.finish = 0;
  s.target = target;
  s.maxit = maxit;
  int r = push_state(h);
  if (r) return r;
  ST_TRY((launch_prec<Tc, double, Tz>(g, h->pp, h->V[0], (Tz *)h->Z[0], h->S, TM_INIT,
                                      h->partials, h->stream)));
  return ST_OK;
}

// Run iterations until the device sets finish (or deactivates); returns with hS current.
// Iterations to enqueue before the next host check.  Iterations enqueued past convergence are
// gated no-ops on the device but still cost their launches, so once a chunk has shown the
// convergence rate of the estimate, the next chunk is the count that rate needs to reach the
// target, plus one (between 2 and 16); until then the schedule doubles from 4.
int next_chunk(int chunk, int dk, double est0, double est1, double target) {
  if (dk > 0 && est0 > 0.0 && est1 > 0.0 && est1 < est0 && target > 0.0) {
    if (est1 <= target) return 2;
    const double rate = std::log(est1 / est0) / dk;  // log decrease per iteration (< 0)
    const double need = std::log(target / est1) / rate;
    const int c = (int)std::ceil(need) + 1;
    return c < 2 ? 2 : (c > 16 ? 16 : c);
  }
  return chunk < 16 ? 2 * chunk : 16;
}

template <class Tz, class Tc>
int minres_iterate(st_handle *h, double *x) {
  int chunk = 4;
  bool known = false;  // hS holds the state of the last check (k, est)
  for (;;) {
    const int k0 = h->hS->k;
    const double est0 = known ? h->hS->est : 0.0;
    for (int i = 1; i <= chunk; ++i) ST_TRY((launch_iteration<Tz, Tc>(h, k0 + i, x)));
    int r = sync_state(h);
    if (r) return r;
    const State &s = *h->hS;
    if (s.status != 0 || s.finish || !s.active) return ST_OK;
    chunk = next_chunk(chunk, s.k - k0, est0, s.est, s.target);
    known = true;
  }
}

int true_residual(st_handle *h, const double *fH, const double *x, double *r_out, double *rho) {
  ST_TRY(launch_stencil<double>(h->g, SM_RESID, x, r_out, fH, h->S, h->partials, 0, h->stream));
  int e = sync_state(h);
  if (e) return e;
  const double bn = h->hS->bnorm2;
  *rho = (bn > 0.0) ? std::sqrt(h->hS->rnorm2 / bn) : 0.0;
  return ST_OK;
}

// b = Y f_H into V[0] and ||b||^2 into the device state (state otherwise cleared).
int prepare_rhs(st_handle *h, const double *fH) {
  cudaStream_t st = h->stream;
  std::memset(h->hS, 0, sizeof(State));
  int r = push_state(h);
  if (r) return r;
  ST_TRY(launch_flip(h->g, fH, h->V[0], st));
  ST_TRY(launch_norm2(h->g.N, fH, h->S, h->partials, st));
  return sync_state(h);
}

int finish_status(const State &s, bool converged) {
  if (s.status != 0) return s.status;
  return converged ? ST_OK : ST_ERR_NOT_CONVERGED;
}

// Plain float64 MINRES with the true-residual stopping rule.
int solve_fp64(st_handle *h, const double *fH, double *x, double tol, int maxit, st_stats *stats) {
  const Geom &g = h->g;
  ST_TRY(cudaMemsetAsync(x, 0, g.N * sizeof(double), h->stream));
  int r = prepare_rhs(h, fH);
  if (r) return r;
  if (h->hS->bnorm2 == 0.0) {
    if (stats) stats->iterations = 0;
    return ST_OK;
  }
  r = minres_start<double, double>(h, tol, maxit);
  if (r) return r;
  int checks = 0;
  double rho = 1.0;
  bool converged = false;
  for (;;) {
    r = minres_iterate<double, double>(h, x);
    if (r) return r;
    State s = *h->hS;
    r = true_residual(h, fH, x, nullptr, &rho);
    if (r) return r;
    ++checks;
    *h->hS = s;  // the residual kernel changed only rnorm2 / counters
    if (s.status != 0) break;
    if (rho <= tol || s.beta == 0.0) {
      converged = true;
      break;
    }
    if (s.k >= maxit) break;
    // continue MINRES with a tighter estimate target
    State &w = *h->hS;
    w.target = w.target * tol / rho;
    w.finish = 0;
    w.active = 1;
    w.rnorm2 = 0.0;
    r = push_state(h);
    if (r) return r;
  }
  if (stats) {
    stats->iterations = h->hS->k;
    stats->outer_steps = 1;
    stats->true_checks = checks;
    stats->est_rel_res = h->hS->est;
    stats->true_rel_res = rho;
  }
  return finish_status(*h->hS, converged);
}

// Mixed precision: MINRES with the float32 preconditioner and double-float vectors solves
// (Y T) d = r for the current residual r = Y f_H - Y T x, accumulating d into the double-float
// x; at the end of each refinement step x is converted to float64 and the residual is
// recomputed in float64 (iterative refinement) until ||r||/||b|| <= tol.
int mixed_start(st_handle *h, double target, int maxit) {
  const Geom &g = h->g;
  ST_TRY(cudaMemsetAsync(h->D[0], 0, g.N * sizeof(df), h->stream));
  ST_TRY(cudaMemsetAsync(h->D[1], 0, g.N * sizeof(df), h->stream));
  ST_TRY(cudaMemsetAsync(h->V[1], 0, g.N * sizeof(df), h->stream));
  State &s = *h->hS;
  const double bn = s.bnorm2;
  std::memset(&s, 0, sizeof(State));
  s.bnorm2 = bn;
  s.active = 1;
  s.target = target;
  s.maxit = maxit;
  int r = push_state(h);
  if (r) return r;
  ST_TRY((launch_prec<float, df, float>(g, h->pp, (const df *)h->V[0], (float *)h->Z[0], h->S,
                                        TM_INIT, h->partials, h->stream)));
  return ST_OK;
}

int mixed_iterate(st_handle *h) {
  int chunk = 4;
  bool known = false;
  for (;;) {
    const int k0 = h->hS->k;
    const double est0 = known ? h->hS->est : 0.0;
    for (int i = 1; i <= chunk; ++i) ST_TRY(launch_iteration_mixed(h, k0 + i));
    int r = sync_state(h);
    if (r) return r;
    const State &s = *h->hS;
    if (s.status != 0 || s.finish || !s.active) return ST_OK;
    chunk = next_chunk(chunk, s.k - k0, est0, s.est, s.target);
    known = true;
  }
}

int solve_mixed(st_handle *h, const double *fH, double *x, double tol, int maxit,
                st_stats *stats) {
  const Geom &g = h->g;
  cudaStream_t st = h->stream;
  ST_TRY(cudaMemsetAsync(h->Xdf, 0, g.N * sizeof(df), st));
  ST_TRY(cudaMemsetAsync(x, 0, g.N * sizeof(double), st));
  std::memset(h->hS, 0, sizeof(State));
  int r = push_state(h);
  if (r) return r;
  ST_TRY(launch_flip_to_df(g, fH, (df *)h->V[0], st));
  ST_TRY(launch_norm2(g.N, fH, h->S, h->partials, st));
  r = sync_state(h);
  if (r) return r;
  if (h->hS->bnorm2 == 0.0) return ST_OK;
  const double bn2 = h->hS->bnorm2;
  double rho = 1.0;
  int total = 0, outer = 0, checks = 0;
  bool converged = false;
  double last_est = 1.0;
  int status = 0;
  while (total < maxit) {
    ++outer;
    const double target = std::max(0.5 * tol / rho, inner_floor());
    h->hS->bnorm2 = bn2;
    r = mixed_start(h, target, maxit - total);
    if (r) return r;
    r = mixed_iterate(h);
    if (r) return r;
    const State s = *h->hS;
    total += s.k;
    last_est = s.est;
    status = s.status;
    ST_TRY(launch_update_group(h, st));  // the inner run's pending updates
    ST_TRY(launch_df_to_double(g.N, h->Xdf, x, st));
    // r = Y f_H - Y T x (float64), stored as the next step's double-float right-hand side
    ST_TRY(launch_resid_df(g, x, (df *)h->V[0], fH, h->S, h->partials, st));
    r = sync_state(h);
    if (r) return r;
    rho = (bn2 > 0.0) ? std::sqrt(h->hS->rnorm2 / bn2) : 0.0;
    ++checks;
    if (rho <= tol) {
      converged = true;
      break;
    }
    if (status != 0 || s.k == 0) break;
  }
  if (stats) {
    stats->iterations = total;
    stats->outer_steps = outer;
    stats->true_checks = checks;
    stats->est_rel_res = last_est;
    stats->true_rel_res = rho;
  }
  if (status != 0) return status;
  return converged ? ST_OK : ST_ERR_NOT_CONVERGED;
}

double now_s() {
  return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch())
      .count();
}

}  // namespace

// ------------------------------------------------------------------------------------ C ABI
int st::setup_handle(const st_problem *prob, st_handle **out, int ugroup) {
  if (!out) return ST_ERR_ARG;
  *out = nullptr;
  int r = check_problem(prob);
  if (r) return r;
  if (ugroup < 1 || ugroup > kUpdRing) return ST_ERR_ARG;
  st_handle *h = new (std::nothrow) st_handle();
  if (!h) return ST_ERR_OOM;
  std::memset(h, 0, sizeof(st_handle));
  h->prob = *prob;
  h->stream = (cudaStream_t)prob->stream;
  h->mixed = (prob->precision == ST_MIXED);
  h->g = geom_of(prob);
  if (cudaGetDevice(&h->device) != cudaSuccess) {
    delete h;
    return ST_ERR_CUDA;
  }
  if (device_closed(h->device)) {
    delete h;
    return ST_ERR_TIMEOUT;
  }
  const Geom g = h->g;
  const size_t N = (size_t)g.N;
  auto fail = [&](int code) {
    h->prob.a_nodal = nullptr;
    free_handle(h);
    return code;
  };
  r = build_tables(h);
  if (r) return fail(r);
  const size_t zsz = h->mixed ? sizeof(float) : sizeof(double);
  cudaError_t e = cudaSuccess;
  for (int i = 0; i < 2 && e == cudaSuccess; ++i) {
    e = cudaMalloc(&h->V[i], N * sizeof(double));
    if (e == cudaSuccess) e = cudaMalloc(&h->Z[i], N * zsz);
    if (e == cudaSuccess) e = cudaMalloc(&h->D[i], N * sizeof(double));
  }
  if (e == cudaSuccess) e = cudaMalloc(&h->q, N * sizeof(double));
  h->pp.tscratch = reinterpret_cast<dd *>(h->q);  // free during a preconditioner pass
  if (e == cudaSuccess && h->mixed) e = cudaMalloc(&h->Xdf, N * sizeof(df));
  h->partials_len = partials_needed(g);
  if (e == cudaSuccess) e = cudaMalloc(&h->partials, (size_t)h->partials_len * sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc(&h->S, sizeof(State));
  if (e == cudaSuccess) e = cudaMalloc(&h->hbuf_in, N * sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc(&h->hbuf_out, N * sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc(&h->gfx, (size_t)g.my * (g.mx + 1) * sizeof(double));
  if (e == cudaSuccess)
    e = cudaMalloc(&h->gfy, ((size_t)g.my + 1) * g.mx * sizeof(double));
  if (e == cudaSuccess) e = cudaMallocHost(&h->hS, sizeof(State));
  // z vectors of the iterations a grouped update keeps pending (mixed single solves)
  h->ugroup = h->mixed ? ugroup : 1;
  for (int i = 0; i < h->ugroup - 1 && e == cudaSuccess; ++i)
    e = cudaMalloc(&h->Zx[i], N * sizeof(float));
  if (e == cudaSuccess) e = cudaMemset(h->S, 0, sizeof(State));
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  if (e != cudaSuccess) return fail(map_cuda(e));
  std::memset(h->hS, 0, sizeof(State));
  h->prob.a_nodal = nullptr;
  *out = h;
  return ST_OK;
}

extern "C" {

int st_version(void) { return 1; }

int st_profile_begin(st_handle *h, int capacity) {
  if (!h || capacity < 1 || capacity > (1 << 20)) return ST_ERR_ARG;
  ST_ENTER(h);
  prof_free(h->prof);
  Prof &p = h->prof;
  std::memset(p.launches, 0, sizeof(p.launches));
  p.ev = new (std::nothrow) cudaEvent_t[2 * (size_t)capacity];
  p.cls = new (std::nothrow) int[capacity];
  if (!p.ev || !p.cls) {
    delete[] p.ev;
    delete[] p.cls;
    p.ev = nullptr;
    p.cls = nullptr;
    return ST_ERR_OOM;
  }
  for (int i = 0; i < 2 * capacity; ++i) {
    cudaError_t e = cudaEventCreate(&p.ev[i]);
    if (e != cudaSuccess) {
      p.cap = i / 2;
      prof_free(p);
      return map_cuda(e);
    }
  }
  p.cap = capacity;
  p.used = 0;
  p.on = 1;
  return ST_OK;
}

int st_profile_end(st_handle *h, st_kernel_time *out, int nclasses) {
  if (!h || !out || nclasses < 1) return ST_ERR_ARG;
  ST_ENTER(h);
  Prof &p = h->prof;
  if (!p.ev) return ST_ERR_ARG;
  ST_TRY(cudaStreamSynchronize(h->stream));
  for (int c = 0; c < nclasses; ++c) out[c] = st_kernel_time{0, 0, 0.0};
  for (int i = 0; i < p.used; ++i) {
    float ms = 0.f;
    cudaError_t e = cudaEventElapsedTime(&ms, p.ev[2 * i], p.ev[2 * i + 1]);
    if (e != cudaSuccess) return map_cuda(e);
    const int c = p.cls[i];
    if (c < nclasses) {
      out[c].timed += 1;
      out[c].ms += ms;
    }
  }
  for (int c = 0; c < nclasses && c < KC_COUNT; ++c) out[c].launches = (int)p.launches[c];
  prof_free(p);
  return ST_OK;
}

// ------------------------------------------------------------------ autotuner
namespace {
struct Knobs {
  int st_target, dst_shift, jd, jf;
  int tc_time, tc_y, tc_z;  // 1: the stage runs on the tensor cores (when the handle has them)
  int tc_x;                 // 1: the last x pass runs on the tensor cores
  int fp64_dd, jdd;         // float64 preconditioner: double-float engine, its time-kernel tile
  int tc_dd;                // 1: the double-float engine's time stage runs on the tensor cores
};
std::mutex g_tune_mu;
std::map<std::tuple<int, int, int, int, int, int, int>, Knobs> g_tune_cache;
}  // namespace

int st_autotune(st_handle *h, int reps) {
  if (!h || reps < 1 || reps > 100) return ST_ERR_ARG;
  ST_ENTER(h);
  const bool fp32 = h->mixed;
  const auto key = std::make_tuple(h->g.dim, h->g.mx, h->g.my, h->g.mz, h->g.n, (int)fp32,
                                   (h->tc_time_img ? 1 : 0) + (h->pp.pcr ? 2 : 0) +
                                       (h->pp.cheb ? 4 : 0) + (h->tc_y_img ? 8 : 0) +
                                       (h->tc_z_img ? 16 : 0) + (h->tc_dig_img ? 32 : 0) +
                                       (h->tc_x_img ? 64 : 0));
  auto apply_engines = [&](const Knobs &k) {
    h->pp.sop = k.tc_time ? h->tc_time_img : nullptr;
    h->pp.sop_y = k.tc_y ? h->tc_y_img : nullptr;
    h->pp.sop_z = k.tc_z ? h->tc_z_img : nullptr;
    h->pp.sop_x = k.tc_x ? h->tc_x_img : nullptr;
    h->pp.fp64_dd = h->fp64_dd_ok ? k.fp64_dd : 0;
    h->pp.time_J_dd = k.jdd;
    h->pp.sdig = k.tc_dd ? h->tc_dig_img : nullptr;
  };
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    auto it = g_tune_cache.find(key);
    if (it != g_tune_cache.end()) {
      h->g.st_target = it->second.st_target;
      h->pp.dst_shift = it->second.dst_shift;
      h->pp.time_J_d = it->second.jd;
      h->pp.time_J_f = it->second.jf;
      apply_engines(it->second);
      return ST_OK;
    }
  }
  // tune from the tensor-core configuration the handle was built with
  apply_engines(Knobs{0, 0, 0, 0, 1, 1, 1, 1, 1, 0, 1});
  cudaStream_t st = h->stream;
  const Geom &g = h->g;
  cudaEvent_t e0, e1;
  ST_TRY(cudaEventCreate(&e0));
  ST_TRY(cudaEventCreate(&e1));
  int rc = ST_OK;
  // best of two timed runs of `reps` launches each, after one warm-up launch
  auto timed = [&](auto &&launch) -> float {
    if (launch() != cudaSuccess) return 1e30f;
    float best = 1e30f;
    for (int trial = 0; trial < 2; ++trial) {
      cudaEventRecord(e0, st);
      for (int r = 0; r < reps; ++r)
        if (launch() != cudaSuccess) return 1e30f;
      cudaEventRecord(e1, st);
      if (cudaEventSynchronize(e1) != cudaSuccess) return 1e30f;
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0, e1);
      if (ms < best) best = ms;
    }
    return best;
  };
  cudaMemsetAsync(h->V[0], 0, g.N * sizeof(double), st);
  cudaMemsetAsync(h->Z[0], 0, g.N * (fp32 ? sizeof(float) : sizeof(double)), st);
  // 1. stencil: blocks per launch (time-chunk length)
  {
    const int cand[] = {608, 1216, 2432, 4864};
    State s{};
    s.active = 1;
    s.beta = 1.0;
    s.inv_beta = 1.0;
    refresh_df(&s);
    *h->hS = s;
    cudaMemcpyAsync(h->S, h->hS, kStatePushBytes, cudaMemcpyHostToDevice, st);
    float best = 1e30f;
    int bt = 0;
    for (int t : cand) {
      h->g.st_target = t;
      const float ms = timed([&]() -> cudaError_t {
        if (fp32)
          return launch_stencil_df(h->g, (const float *)h->Z[0], (df *)h->q, h->S, h->partials, st);
        return launch_stencil<double>(h->g, SM_APPLY, h->V[0], h->q, nullptr, h->S, h->partials, 0,
                                      st);
      });
      if (ms < best) {
        best = ms;
        bt = t;
      }
    }
    h->g.st_target = bt;
  }
  // 2. spatial DST: sequences per block
  if (!h->pp.pcr) {
    float best = 1e30f;
    int bs = 0;
    for (int sh = 0; sh <= 2; ++sh) {
      h->pp.dst_shift = sh;
      const float ms = timed([&]() { return tune_run_dsts(h->g, h->pp, fp32, h->Z[0], st); });
      if (ms < best) {
        best = ms;
        bs = sh;
      }
    }
    h->pp.dst_shift = bs;
  }
  // 3. float32/float64 FFMA time kernel (the tensor-core kernel has a fixed tile): column tile;
  // then, where the tensor-core kernel exists, the faster of the two engines (short time axes
  // give the tensor-core kernel little work per tile)
  int tc_time = h->tc_time_img ? 1 : 0, tc_y = h->tc_y_img ? 1 : 0, tc_z = h->tc_z_img ? 1 : 0;
  int tc_x = h->tc_x_img ? 1 : 0;
  if (!h->pp.sop_long) {
    const int cand[] = {16, 32, 48, 64};
    float best = 1e30f;
    int bj = 0;
    for (int J : cand) {
      if (!time_J_fits(g.n, J, fp32)) continue;
      if (fp32) h->pp.time_J_f = J; else h->pp.time_J_d = J;
      const float ms = timed([&]() { return tune_run_time(h->g, h->pp, fp32, h->Z[0], st); });
      if (ms < best) {
        best = ms;
        bj = J;
      }
    }
    if (fp32) h->pp.time_J_f = bj; else h->pp.time_J_d = bj;
    if (fp32 && h->tc_time_img && !h->pp.pcr && !h->pp.cheb) {
      const float ms_tc = timed([&]() {
        return launch_time_tc((float *)h->Z[0], h->g, h->pp.spec_f, h->tc_time_img, h->S,
                              TM_NONE, h->partials, GK_NONE, st);
      });
      tc_time = (ms_tc <= best) ? 1 : 0;
    }
  }
  // 4. spatial passes (float32): the last x pass, y and z, tensor cores against the
  // shared-memory FFT
  if (fp32) {
    const unsigned short *img[3] = {h->tc_x_img, h->tc_y_img, h->tc_z_img};
    int *use[3] = {&tc_x, &tc_y, &tc_z};
    for (int axis = 0; axis <= 2; ++axis) {
      if (!img[axis]) continue;
      const float ms_tc = timed([&]() {
        return tune_run_pass(h->g, h->pp, axis, img[axis], (float *)h->Z[0], h->S, st);
      });
      const float ms_fft = timed([&]() {
        return tune_run_pass(h->g, h->pp, axis, nullptr, (float *)h->Z[0], h->S, st);
      });
      *use[axis] = (ms_tc <= ms_fft) ? 1 : 0;
    }
  }
  // 5. float64 preconditioner: double-float engine (the tile of its CUDA-core time kernel first,
  // then that kernel against the tensor-core digit kernel) against the float64 one, the whole
  // P_H pass each
  int fp64_dd = 0, jdd = 0, tc_dd = 0;
  if (!fp32 && h->fp64_dd_ok) {
    const int cand[] = {16, 32, 48, 64};
    float best = 1e30f;
    h->pp.fp64_dd = 1;
    for (int J : cand) {
      if (!time_J_fits(g.n, J, false)) continue;
      h->pp.time_J_dd = J;
      const float ms = timed([&]() { return tune_run_time_dd(h->g, h->pp, h->Z[0], st); });
      if (ms < best) {
        best = ms;
        jdd = J;
      }
    }
    h->pp.time_J_dd = jdd;
    if (h->tc_dig_img) {
      const float ms_tc = timed([&]() {
        return launch_time_tcd((dd *)h->Z[0], (dd *)h->q, h->g, h->pp.spec_dd, h->tc_dig_img,
                               h->pp.sdig_e, h->S, TM_NONE, h->partials, GK_NONE, st);
      });
      tc_dd = (ms_tc <= best) ? 1 : 0;
    }
    h->pp.sdig = tc_dd ? h->tc_dig_img : nullptr;
    const float ms_dd = timed([&]() {
      return launch_prec<double, double, double>(h->g, h->pp, h->V[0], (double *)h->Z[0], h->S,
                                                 TM_NONE, h->partials, st);
    });
    h->pp.fp64_dd = 0;
    const float ms_d = timed([&]() {
      return launch_prec<double, double, double>(h->g, h->pp, h->V[0], (double *)h->Z[0], h->S,
                                                 TM_NONE, h->partials, st);
    });
    fp64_dd = (ms_dd <= ms_d) ? 1 : 0;
  }
  const Knobs chosen{h->g.st_target, h->pp.dst_shift, h->pp.time_J_d, h->pp.time_J_f, tc_time,
                     tc_y, tc_z, tc_x, fp64_dd, jdd, tc_dd};
  apply_engines(chosen);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaError_t le = cudaGetLastError();
  if (le != cudaSuccess) rc = map_cuda(le);
  if (rc == ST_OK) {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tune_cache[key] = chosen;
  }
  return rc;
}

const char *st_kernel_class_name(int c) {
  static const char *names[KC_COUNT] = {"stencil", "lanczos_dst_x", "dst_x", "dst_y",
                                        "time_dst_scale", "update", "residual", "aux"};
  return (c >= 0 && c < KC_COUNT) ? names[c] : "unknown";
}

const char *st_strerror(int code) {
  switch (code) {
    case ST_OK: return "ok";
    case ST_ERR_ARG: return "invalid argument";
    case ST_ERR_CUDA: return "CUDA error";
    case ST_ERR_NOT_CONVERGED: return "not converged within maxit";
    case ST_ERR_BREAKDOWN: return "breakdown (non-positive <v, P^-1 v> or non-finite scalar)";
    case ST_ERR_TIMEOUT: return "device wait timed out";
    case ST_ERR_OOM: return "out of memory";
    default: return "unknown status";
  }
}

int st_workspace_bytes(const st_problem *prob, size_t *bytes) {
  if (!bytes) return ST_ERR_ARG;
  int r = check_problem(prob);
  if (r) return r;
  Geom g = geom_of(prob);
  *bytes = workspace_bytes(g, prob->precision == ST_MIXED, cheb_degree(prob), update_group());
  return ST_OK;
}

int st_setup(const st_problem *prob, st_handle **out) {
  return setup_handle(prob, out, update_group());
}

void st_destroy(st_handle *h) {
  if (!h) return;
  cudaSetDevice(h->device);
  cudaStreamSynchronize(h->stream);
  free_handle(h);
}

int st_assemble_rhs(st_handle *h, const double *f_dev, const double *u0_dev,
                    const double *uprev_dev, const double *extra_dev, double *fH_dev) {
  if (!h || !f_dev || !u0_dev || !fH_dev) return ST_ERR_ARG;
  ProfScope prof_scope(h);
  ST_ENTER(h);
  ST_TRY(launch_rhs(h->g, f_dev, u0_dev, uprev_dev, extra_dev, fH_dev, h->stream));
  return ST_OK;
}

int st_apply_op(st_handle *h, const double *v_dev, double *y_dev) {
  if (!h || !v_dev || !y_dev || v_dev == y_dev) return ST_ERR_ARG;
  ProfScope prof_scope(h);
  ST_ENTER(h);
  ST_TRY(launch_stencil<double>(h->g, SM_APPLY, v_dev, y_dev, nullptr, h->S, h->partials, 0,
                                h->stream));
  return ST_OK;
}

int st_apply_prec(st_handle *h, const double *v_dev, double *z_dev) {
  if (!h || !v_dev || !z_dev) return ST_ERR_ARG;
  ProfScope prof_scope(h);
  ST_ENTER(h);
  ST_TRY((launch_prec<double, double, double>(h->g, h->pp, v_dev, z_dev, h->S, TM_NONE,
                                              h->partials, h->stream)));
  return ST_OK;
}

int st_apply_prec_f32(st_handle *h, const double *v_dev, float *z_dev) {
  if (!h || !v_dev || !z_dev) return ST_ERR_ARG;
  ProfScope prof_scope(h);
  ST_ENTER(h);
  ST_TRY((launch_prec<float, double, float>(h->g, h->pp, v_dev, z_dev, h->S, TM_NONE,
                                            h->partials, h->stream)));
  return ST_OK;
}

int st_solve(st_handle *h, const double *fH_dev, double *u_dev, double tol, int maxit,
             st_stats *stats) {
  if (!h || !fH_dev || !u_dev || fH_dev == u_dev || !(tol >= 0.0) || maxit < 1) return ST_ERR_ARG;
  ProfScope prof_scope(h);
  ST_ENTER(h);
  const double t0 = now_s();
  st_stats local{};
  int r = h->mixed ? solve_mixed(h, fH_dev, u_dev, tol, maxit, &local)
                   : solve_fp64(h, fH_dev, u_dev, tol, maxit, &local);
  if (r != ST_ERR_CUDA && r != ST_ERR_OOM) {
    cudaError_t e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) r = map_cuda(e);
  }
  local.status = r;
  local.seconds = now_s() - t0;
  if (stats) *stats = local;
  return r;
}

int st_solve_host(st_handle *h, const double *fH_host, double *u_host, double tol, int maxit,
                  st_stats *stats) {
  if (!h || !fH_host || !u_host) return ST_ERR_ARG;
  ProfScope prof_scope(h);
  ST_ENTER(h);
  const double t0 = now_s();
  const size_t bytes = (size_t)h->g.N * sizeof(double);
  ST_TRY(cudaMemcpyAsync(h->hbuf_in, fH_host, bytes, cudaMemcpyHostToDevice, h->stream));
  st_stats local{};
  int r = st_solve(h, h->hbuf_in, h->hbuf_out, tol, maxit, &local);
  if (r == ST_ERR_CUDA || r == ST_ERR_OOM) return r;
  cudaError_t e = cudaMemcpyAsync(u_host, h->hbuf_out, bytes, cudaMemcpyDeviceToHost, h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) r = map_cuda(e);
  local.status = r;
  local.seconds = now_s() - t0;
  if (stats) *stats = local;
  return r;
}

int st_solve_transpose(st_handle *h, const double *g_dev, double *lam_dev, double tol, int maxit,
                       st_stats *stats) {
  if (!h || !g_dev || !lam_dev || g_dev == lam_dev) return ST_ERR_ARG;
  ProfScope prof_scope(h);
  ST_ENTER(h);
  // (Y T) mu = g is st_solve with f_H = Y g; then lam = Y mu.
  ST_TRY(launch_flip(h->g, g_dev, h->hbuf_in, h->stream));
  int r = st_solve(h, h->hbuf_in, lam_dev, tol, maxit, stats);
  if (r == ST_ERR_CUDA || r == ST_ERR_OOM) return r;
  cudaError_t e = launch_flip(h->g, lam_dev, lam_dev, h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) return map_cuda(e);
  return r;
}

int st_grad_rhs(st_handle *h, const double *lam_dev, double *grad_f_dev, double *grad_u0_dev,
                double *grad_uprev_dev) {
  if (!h || !lam_dev || !grad_f_dev) return ST_ERR_ARG;
  ProfScope prof_scope(h);
  ST_ENTER(h);
  ST_TRY(launch_grad_rhs(h->g, lam_dev, grad_f_dev, grad_u0_dev, grad_uprev_dev, h->stream));
  return ST_OK;
}

int st_grad_a(st_handle *h, const double *lam_dev, const double *u_dev, const double *u0_dev,
              double *grad_dev) {
  if (!h || !lam_dev || !u_dev || !u0_dev || !grad_dev) return ST_ERR_ARG;
  if (h->g.dim == 3) return ST_ERR_ARG;  // the face gradient is written for 1D and 2D grids
  ProfScope prof_scope(h);
  ST_ENTER(h);
  ST_TRY(launch_grad_a(h->g, lam_dev, u_dev, u0_dev, h->gfx, h->gfy, grad_dev, h->stream));
  return ST_OK;
}

}  // extern "C"
