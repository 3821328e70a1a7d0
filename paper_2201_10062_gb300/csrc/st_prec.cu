// Preconditioner kernels: z = P^-1 v by the three steps of Sec. 3.1.1,
//   1. v~ = (S_n (x) U_m^T) v,  2. z~ = diag(1/p) v~,  3. z = (S_n (x) U_m) z~,
// with U_m = S_my (x) S_mx (uniform grid, x fastest) and S the orthonormal DST-I, which is
// symmetric and involutory, so the forward and inverse transforms are the same kernels.
//
// Spatial DST-I (lengths mx, my with mx+1, my+1 powers of two): two real lines a, b are packed
// into one complex sequence, odd-extended to length L = 2(len+1) and transformed by a radix-2
// FFT in shared memory.  The DFT of the odd extension of a real line x is -2i sum_j x_j
// sin(pi j k/(len+1)), so for z = a + i b: DST(a)_k = -Im Z_k / sqrt(L), DST(b)_k = Re Z_k /
// sqrt(L) (orthonormal scaling sqrt(2/(len+1)) folded in).
//
// Time DST-I (any n): a dense contraction with S_n over the time axis for a tile of spatial
// columns held in shared memory, halved by the symmetry S_{k,n+1-t} = (-1)^{k+1} S_{k,t}:
// odd k use U_t = x_t + x_{n+1-t}, even k use D_t = x_t - x_{n+1-t}.  Between the forward and
// inverse time transforms each entry is scaled by 1/p_kj, the eigenvalue of P in the transformed
// basis (Sec. 3.1.1 for theta, Sec. 4 for BDF2, Sec. 3.1.4 for P_theta), and the kernel
// accumulates <v, P^-1 v> = sum v~^2 / p for MINRES.
#include <math.h>

#include "st_fft.cuh"
#include "st_internal.cuh"
#include "st_symbol.cuh"

namespace st {

namespace {

constexpr int kNT = 256;


// Inside a MINRES iteration only the first kernel (the stencil) looks at `finish`; it clears
// `active` so that the rest of that iteration is skipped.  The preconditioner kernels check
// `active` alone (gate_closed, GK_ACTIVE), so an iteration whose time kernel raises `finish`
// still completes z_{k+1} (needed if the stopping rule later decides to continue).

// ------------------------------------------------------------------------------ spatial DST
// XL = true: lines are rows (contiguous, line l starts at l*len).
// XL = false: lines are columns of the (my x mx) planes: line l = k*mx + i starts at k*m + i and
// its elements are mx apart.  A block owns 2*PB consecutive lines (PB complex sequences, line
// 2p in the real part and line 2p+1 in the imaginary part), loads them coalesced into shared
// memory as odd extensions, runs in-place Stockham passes and writes the sine coefficients.
constexpr int kNTD = 512;  // threads per spatial-DST block

// Stockham passes for a compile-time length 2^LOGL: radix 8 while at least three stages remain,
// then one radix-4 or radix-2 pass.
template <class Tc, int LOGL, int LOGNS>
struct StockhamPasses {
  __device__ __forceinline__ static void run(cpx<Tc> *buf, const cpx<Tc> *tws, int PB, int Ls,
                                             int tid) {
    constexpr int REM = LOGL - LOGNS;
    if constexpr (REM > 0) {
      constexpr int LR = REM >= 3 ? 3 : REM;
      stockham_pass_inplace<Tc, (1 << LR), LOGL, LOGNS>(buf, tws, PB, Ls, tid, kNTD);
      StockhamPasses<Tc, LOGL, LOGNS + LR>::run(buf, tws, PB, Ls, tid);
    }
  }
};

// float32 transforms: three 512-thread blocks per SM (at most 40 registers); float64, double-float
// and the fused Lanczos source (its loads held in registers ahead of the stores): two
template <class Tc, class Src, class Tout, bool XL, int LOGL>
__global__ void __launch_bounds__(kNTD, (sizeof(Tc) == 4 && !has_fetch<Src>::value) ? 3 : 2)
    k_dst_space(Src src, Tout *out, int len, long long nlines, int mx, long long m,
                const Tc *tw, int PB, const State *S, int gk) {
  if (gate_closed(S, gk)) return;
  src.prepare(S);
  constexpr int logL = LOGL;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int L = 1 << logL;
  const int half = L >> 1;
  const int Ls = fft_seq_stride<Tc>(L);
  cpx<Tc> *tws = reinterpret_cast<cpx<Tc> *>(smem_raw);
  cpx<Tc> *buf = tws + half;
  const int tid = threadIdx.x;
  for (int e = tid; e < half; e += kNTD) tws[e] = cpx<Tc>{tw[2 * e], tw[2 * e + 1]};
  const long long line0 = (long long)blockIdx.x * 2 * PB;
  const int nl = (int)min((long long)2 * PB, nlines - line0);  // lines present in this block
  const int logH = logL - 1;
  const int logPB = 31 - __clz(PB);
  // slots 0 and len+1 of every sequence are zero
  for (int pp = tid; pp < PB; pp += kNTD) {
    buf[pp * Ls + fft_pad<Tc>(0)] = cpx<Tc>{Tc(0), Tc(0)};
    buf[pp * Ls + fft_pad<Tc>(len + 1)] = cpx<Tc>{Tc(0), Tc(0)};
  }
  // one work item per (sequence, element): both lines of the pair, stored as one complex value
  // at e+1 and its negative at L-1-e (odd extension).  Index maps avoid divisions: len + 1 =
  // L/2 and PB are powers of two.
  if constexpr (XL && has_fetch<Src>::value) {
    // the fused Lanczos source: every load of the thread's elements first (at most four work
    // items of two lines each: PB * L <= 8 * kNTD), then the arithmetic, the v_{k+1} stores and
    // the shared-memory writes, so that the loads are not held behind the stores
    constexpr int kItems = 4;
    typename Src::Raw ra[kItems], rb[kItems];
#pragma unroll
    for (int u = 0; u < kItems; ++u) {
      const int idx = tid + u * kNTD;
      const int pp = idx >> logH, e = idx & (half - 1);
      const int la = 2 * pp, lb = la + 1;
      const long long i0 = (line0 + la) * len + e;
      if (idx < (PB << logH) && e < len) {
        if (la < nl) ra[u] = src.fetch(i0);
        if (lb < nl) rb[u] = src.fetch(i0 + len);
      }
    }
#pragma unroll
    for (int u = 0; u < kItems; ++u) {
      const int idx = tid + u * kNTD;
      const int pp = idx >> logH, e = idx & (half - 1);
      if (idx >= (PB << logH) || e >= len) continue;
      const int la = 2 * pp, lb = la + 1;
      const long long i0 = (line0 + la) * len + e;
      const Tc a = (la < nl) ? src.finish(i0, ra[u]) : Tc(0);
      const Tc b = (lb < nl) ? src.finish(i0 + len, rb[u]) : Tc(0);
      cpx<Tc> *bq = buf + pp * Ls;
      bq[fft_pad<Tc>(e + 1)] = cpx<Tc>{a, b};
      bq[fft_pad<Tc>(L - 1 - e)] = cpx<Tc>{-a, -b};
    }
  } else if (XL) {
    // lines 2pp and 2pp+1 are consecutive rows: one base pointer serves both
    for (int idx = tid; idx < (PB << logH); idx += kNTD) {
      const int pp = idx >> logH, e = idx & (half - 1);
      if (e >= len) continue;
      const int la = 2 * pp, lb = la + 1;
      const long long i0 = (line0 + la) * len + e;
      const Tc a = (la < nl) ? src(i0) : Tc(0);
      const Tc b = (lb < nl) ? src(i0 + len) : Tc(0);
      cpx<Tc> *bq = buf + pp * Ls;
      bq[fft_pad<Tc>(e + 1)] = cpx<Tc>{a, b};
      bq[fft_pad<Tc>(L - 1 - e)] = cpx<Tc>{-a, -b};
    }
  } else {
    // PB divides the block size, so every thread keeps one sequence (pair of columns) and walks
    // its elements: the column decomposition (plane k, column i) is done once per thread.
    const int pp = tid & (PB - 1), estep = kNTD >> logPB;
    const int la = 2 * pp, lb = la + 1;
    long long ia = -1, ib = -1;  // first element of each column line (-1: line absent)
    if (la < nl) {
      const int l = (int)line0 + la;
      const int k = l / mx, i = l - k * mx;
      ia = (long long)k * m + i;
    }
    if (lb < nl) {
      const int l = (int)line0 + lb;
      const int k = l / mx, i = l - k * mx;
      ib = (long long)k * m + i;
    }
    cpx<Tc> *bq = buf + pp * Ls;
    for (int e = tid >> logPB; e < len; e += estep) {
      const long long off = (long long)e * mx;
      const Tc a = (ia >= 0) ? src(ia + off) : Tc(0);
      const Tc b = (ib >= 0) ? src(ib + off) : Tc(0);
      bq[fft_pad<Tc>(e + 1)] = cpx<Tc>{a, b};
      bq[fft_pad<Tc>(L - 1 - e)] = cpx<Tc>{-a, -b};
    }
  }
  __syncthreads();
  StockhamPasses<Tc, LOGL, 0>::run(buf, tws, PB, Ls, tid);
  const Tc sc = (Tc)(1.0 / sqrt((double)L));
  if (XL) {
    for (int idx = tid; idx < (PB << logH); idx += kNTD) {
      const int pp = idx >> logH, e = idx & (half - 1);
      if (e >= len) continue;
      const cpx<Tc> Z = buf[pp * Ls + fft_pad<Tc>(e + 1)];
      const int la = 2 * pp, lb = la + 1;
      Tout *p = out + (line0 + la) * len + e;
      if (la < nl) p[0] = (Tout)(-Z.y * sc);
      if (lb < nl) p[len] = (Tout)(Z.x * sc);
    }
  } else {
    const int pp = tid & (PB - 1), estep = kNTD >> logPB;
    const int la = 2 * pp, lb = la + 1;
    Tout *pa = nullptr, *pb = nullptr;
    if (la < nl) {
      const int l = (int)line0 + la;
      const int k = l / mx, i = l - k * mx;
      pa = out + (long long)k * m + i;
    }
    if (lb < nl) {
      const int l = (int)line0 + lb;
      const int k = l / mx, i = l - k * mx;
      pb = out + (long long)k * m + i;
    }
    const cpx<Tc> *bq = buf + pp * Ls;
    for (int e = tid >> logPB; e < len; e += estep) {
      const cpx<Tc> Z = bq[fft_pad<Tc>(e + 1)];
      const long long off = (long long)e * mx;
      if (pa) pa[off] = (Tout)(-Z.y * sc);
      if (pb) pb[off] = (Tout)(Z.x * sc);
    }
  }
}

// ------------------------------------------------------------------------------ time DST
// Dense folded S_n contraction on a tile X[n][J] in shared memory: Y = S_n X.
// X is folded in place first (rows t-1 <- U_t, n-t <- D_t).  Thread tiles of KT output rows of
// one parity class by JT columns.
template <class Tc, int KT, int JT>
__device__ void time_dst_tile(Tc *X, Tc *Y, const Tc *sintab, int n, int J) {
  const int tid = threadIdx.x;
  const int h = n >> 1;
  for (int idx = tid; idx < h * J; idx += kNT) {
    const int t = idx / J, c = idx - t * J;
    const Tc a = X[t * J + c], b = X[(n - 1 - t) * J + c];
    X[t * J + c] = a + b;
    X[(n - 1 - t) * J + c] = a - b;
  }
  __syncthreads();
  const int P2 = 2 * (n + 1);
  const int nodd = (n + 1) >> 1, neven = n >> 1;
  const int JG = J / JT;
  const int todd = ((nodd + KT - 1) / KT) * JG;
  const int tall = todd + ((neven + KT - 1) / KT) * JG;
  const bool nodd_mid = (n & 1);
  const int tm = (n + 1) >> 1;  // middle index (1-based) when n is odd
  for (int tile = tid; tile < tall; tile += kNT) {
    const bool odd = tile < todd;
    const int tt = odd ? tile : tile - todd;
    const int rg = tt / JG, jg = tt - rg * JG;
    const int cnt = odd ? nodd : neven;
    int kk[KT], ix[KT];
#pragma unroll
    for (int i = 0; i < KT; ++i) {
      int r = rg * KT + i;
      if (r >= cnt) r = cnt - 1;  // duplicate a valid row; its result is not stored
      kk[i] = odd ? 2 * r + 1 : 2 * r + 2;
      ix[i] = 0;
    }
    MacAcc<Tc> acc[KT][JT];
#pragma unroll
    for (int i = 0; i < KT; ++i)
#pragma unroll
      for (int c = 0; c < JT; ++c) acc[i][c].zero();
    const Tc *Fb = X + jg * JT;
    for (int t = 1; t <= h; ++t) {
      const Tc *F = Fb + (odd ? (t - 1) : (n - t)) * J;
      Tc f[JT];
#pragma unroll
      for (int c = 0; c < JT; ++c) f[c] = F[c];
#pragma unroll
      for (int i = 0; i < KT; ++i) {
        int q = ix[i] + kk[i];
        q = (q >= P2) ? q - P2 : q;
        ix[i] = q;
        const Tc sv = sintab[q];
#pragma unroll
        for (int c = 0; c < JT; ++c) acc[i][c].add(sv, f[c]);
      }
    }
    if (odd && nodd_mid) {
      const Tc *F = Fb + (tm - 1) * J;
#pragma unroll
      for (int i = 0; i < KT; ++i) {
        const Tc sv = sintab[(int)(((long long)kk[i] * tm) % P2)];
#pragma unroll
        for (int c = 0; c < JT; ++c) acc[i][c].add(sv, F[c]);
      }
    }
#pragma unroll
    for (int i = 0; i < KT; ++i) {
      if (rg * KT + i < cnt) {
        Tc *Yr = Y + (kk[i] - 1) * J + jg * JT;
#pragma unroll
        for (int c = 0; c < JT; ++c) Yr[c] = acc[i][c].get();
      }
    }
  }
  __syncthreads();
}


template <class Tc, int KT, int JT>
__global__ void __launch_bounds__(kNT)
    k_time(const Tc *data, Tc *out, int n, long long m, int mx, int J, Spec<Tc> sp, State *S,
           int tmode, int tkind, double *__restrict__ partials, int gk) {
  __shared__ double red[32];
  if (gate_closed(S, gk)) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  Tc *X = reinterpret_cast<Tc *>(smem_raw);
  Tc *Y = X + (size_t)n * J;
  Tc *sintab = Y + (size_t)n * J;
  Tc *tmu = sintab + 2 * (n + 1);
  const int tid = threadIdx.x;
  const long long j0 = (long long)blockIdx.x * J;
  const int Je = (int)min((long long)J, m - j0);
  for (int r = tid; r < 2 * (n + 1); r += kNT) sintab[r] = sp.sintab[r];
  for (int c = tid; c < J; c += kNT) {
    Tc v = Tc(0);
    if (c < Je) {
      const long long j = j0 + c;
      const long long jy = j / mx, jx = j - jy * mx;
      v = sp.mux[jx] + sp.muy[jy];
    }
    tmu[c] = v;
  }
  for (int idx = tid; idx < n * J; idx += kNT) {
    const int t = idx / J, c = idx - t * J;
    X[idx] = (c < Je) ? data[(long long)t * m + j0 + c] : Tc(0);
  }
  __syncthreads();
  time_dst_tile<Tc, KT, JT>(X, Y, sintab, n, J);
  // <v, P^-1 v> partial: compensated (Kahan) sum in the tile's type, float64 across threads
  Tc esum = Tc(0), ecomp = Tc(0);
  if (tkind == 0) {
    // scale by 1/p and accumulate <v, P^-1 v>
    for (int idx = tid; idx < n * J; idx += kNT) {
      const int kr = idx / J, c = idx - kr * J;
      const Tc ip = inv_symbol(sp, kr + 1, tmu[c]);
      const Tc y = Y[idx];
      if (c < Je) {
        const Tc term = y * y * ip - ecomp;
        const Tc t = esum + term;
        ecomp = (t - esum) - term;
        esum = t;
      }
      Y[idx] = y * ip;
    }
    __syncthreads();
    time_dst_tile<Tc, KT, JT>(Y, X, sintab, n, J);
    for (int idx = tid; idx < n * J; idx += kNT) {
      const int t = idx / J, c = idx - t * J;
      if (c < Je) out[(long long)t * m + j0 + c] = X[idx];
    }
  } else {
    for (int idx = tid; idx < n * J; idx += kNT) {
      const int t = idx / J, c = idx - t * J;
      if (c < Je) out[(long long)t * m + j0 + c] = Y[idx];
    }
  }
  if (tmode != TM_NONE) {
    const double e = (double)esum - (double)ecomp;
    double tot;
    if (last_block_reduce<kNT>(e, partials, &S->counter[CNT_TIME], gridDim.x, blockIdx.x, red,
                               &tot) &&
        tid == 0) {
      if (tmode == TM_INIT || tmode == TM_RESTART)
        minres_init_scalars_dev(S, tot);
      else
        minres_givens_dev(S, tot);
    }
  }
}

// ------------------------------------------------------------------------------ P_theta, 1D a(x)
// Step 2 of the P_theta apply (Sec. 3.1.4) when K has no fast diagonalisation: for every time
// frequency k solve (lam_H,k I + lam_Htheta,k tau K) z_k = v_k, a tridiagonal SPD system of size
// mx, by parallel cyclic reduction in shared memory (one block per k).  Each of the
// ceil(log2 mx) steps eliminates the couplings at distance s = 1, 2, 4, ... from every equation
// at once; at the end every equation is decoupled and z_i = d_i / b_i.  The block also forms
// <v_k, z_k>, whose sum over k is <v, P_theta^-1 v> (the time DST is orthogonal).
template <class Tc>
__global__ void __launch_bounds__(kNT)
    k_pcr_ptheta(Tc *data, int n, int mx, const double *__restrict__ cx, Spec<Tc> sp, State *S,
                 int tmode, double *__restrict__ partials, int gk) {
  __shared__ double red[32];
  if (gate_closed(S, gk)) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  Tc *a = reinterpret_cast<Tc *>(smem_raw);
  Tc *b = a + mx, *c = b + mx, *d = c + mx;
  Tc *a2 = d + mx, *b2 = a2 + mx, *c2 = b2 + mx, *d2 = c2 + mx;
  const int k = blockIdx.x;  // 0-based frequency
  const int tid = threadIdx.x;
  const Tc lh = sp.lh[k], lt = sp.lht[k];
  Tc *row = data + (long long)k * mx;
  for (int i = tid; i < mx; i += kNT) {
    const Tc w = (Tc)cx[i], e = (Tc)cx[i + 1];  // tau a/h^2 at the faces of node i
    b[i] = lh + lt * (w + e);
    a[i] = (i > 0) ? -lt * w : Tc(0);
    c[i] = (i < mx - 1) ? -lt * e : Tc(0);
    d[i] = row[i];
  }
  __syncthreads();
  for (int s = 1; s < mx; s <<= 1) {
    for (int i = tid; i < mx; i += kNT) {
      Tc na = Tc(0), nb = b[i], nc = Tc(0), nd = d[i];
      if (i - s >= 0) {
        const Tc k1 = a[i] / b[i - s];
        na = -a[i - s] * k1;
        nb -= c[i - s] * k1;
        nd -= d[i - s] * k1;
      }
      if (i + s < mx) {
        const Tc k2 = c[i] / b[i + s];
        nc = -c[i + s] * k2;
        nb -= a[i + s] * k2;
        nd -= d[i + s] * k2;
      }
      a2[i] = na;
      b2[i] = nb;
      c2[i] = nc;
      d2[i] = nd;
    }
    __syncthreads();
    Tc *t;
    t = a; a = a2; a2 = t;
    t = b; b = b2; b2 = t;
    t = c; c = c2; c2 = t;
    t = d; d = d2; d2 = t;
  }
  double e = 0.0;
  for (int i = tid; i < mx; i += kNT) {
    const Tc z = d[i] / b[i];
    e += (double)row[i] * (double)z;
    row[i] = z;
  }
  if (tmode != TM_NONE) {
    double tot;
    if (last_block_reduce<kNT>(e, partials, &S->counter[CNT_TIME], gridDim.x, blockIdx.x, red,
                               &tot) &&
        tid == 0) {
      if (tmode == TM_INIT || tmode == TM_RESTART)
        minres_init_scalars_dev(S, tot);
      else
        minres_givens_dev(S, tot);
    }
  }
}

// ---------------------------------------------------------------- P_theta, 2D/3D a(x, y[, z])
// Step 2 of the P_theta apply (Sec. 3.1.4) when K is not sine-diagonalisable (2D, 3D).  The paper
// leaves the solver of the shifted systems A_k = lam_H,k I + lam_Htheta,k tau K open; here each
// one gets a fixed number of preconditioned Chebyshev steps (Saad, Iterative Methods for Sparse
// Linear Systems, Alg. 12.1) with B_k = lam_H,k I + lam_Htheta,k tau abar K0 (K0 the a = 1
// stiffness matrix, abar the mean face value), which the spatial DST diagonalises.  All n
// frequencies advance together.  Step j:
//   w = s_j,k B_k^-1 r_j           four spatial DST passes, the diagonal fused into the third
//   d_j = a_j,k d_{j-1} + w        (d_{-1} = 0)
//   x_{j+1} = x_j + d_j,  r_{j+1} = r_j - A_k d_j    (k_cheb_resid; the last step: k_cheb_final)
// The scalars come from the Chebyshev interval of B_k^-1 A_k, set up on the host.

// The B_k^-1 diagonal times the step scalar, applied as the third transform loads its input.
template <class Tc>
struct SrcChebScale {
  const Tc *w;
  const Tc *s;  // [n] step scalar per frequency
  const Tc *lh, *lht, *mux, *muy;
  unsigned m, mx;
  __device__ __forceinline__ void prepare(const State *) {}
  __device__ __forceinline__ Tc operator()(long long i) const {
    const unsigned e = (unsigned)i;  // N < 2^31 for every accepted size
    const unsigned k = e / m, r = e - k * m;
    const unsigned jy = r / mx, ix = r - jy * mx;
    return w[i] * s[k] / (lh[k] + lht[k] * (mux[ix] + muy[jy]));
  }
};

// Face coefficient tau a / h^2 in the transform type: float64 tables for float64, the leading
// float of the double-float copy for float32 (no float64 conversion per element).
template <class Tc>
__device__ __forceinline__ Tc face_c(const double *c, const df *cd, long long i);
template <>
__device__ __forceinline__ double face_c<double>(const double *c, const df *, long long i) {
  return c[i];
}
template <>
__device__ __forceinline__ float face_c<float>(const double *, const df *cd, long long i) {
  return cd[i].hi;
}

// d_j = a_k d_{j-1} + w into dnext (its own buffer: the stencil reads neighbours of d_{j-1}),
// x = x + d_j (x = d_j when first), r = rsrc - A_k d_j with tau K the 5-point (2D) or 7-point
// (3D) stencil of the face coefficients cx, cy, cz (tau a / h^2).  r may alias rsrc.
// Blocks of 32 x 8 nodes: x by threadIdx.x and blockIdx.y, the my*mz rows by threadIdx.y and
// blockIdx.x, the frequency k by blockIdx.z, so no index is recovered by division.
constexpr int kChebBX = 32, kChebBY = 8;

template <class Tc>
__global__ void __launch_bounds__(kChebBX * kChebBY)
    k_cheb_resid(Geom g, const Tc *__restrict__ dprev, const Tc *__restrict__ w,
                 Tc *__restrict__ dnext, const Tc *rsrc, Tc *r, Tc *__restrict__ x,
                 const Tc *__restrict__ acoef, const Tc *__restrict__ lh,
                 const Tc *__restrict__ lht, int first, const State *S, int gk) {
  if (gate_closed(S, gk)) return;
  const int mx = g.mx, my = g.my, mz = g.mz;
  const int ix = blockIdx.y * kChebBX + threadIdx.x;
  const int row = blockIdx.x * kChebBY + threadIdx.y;
  const int k = blockIdx.z;
  if (ix >= mx || row >= my * mz) return;
  const long long pl = (long long)mx * my;
  {
    const long long e = (long long)k * g.m + (long long)row * mx + ix;
    const int jz = row / my, jy = row - jz * my;
    const Tc ak = first ? Tc(0) : acoef[k];
    auto dv = [&](long long q) -> Tc { return first ? w[q] : ak * dprev[q] + w[q]; };
    const Tc dc = dv(e);
    const long long fx = (long long)row * (mx + 1) + ix;
    const long long fy = ((long long)jz * (my + 1) + jy) * mx + ix;
    const Tc cw = face_c<Tc>(g.cx, g.cxd, fx), ce = face_c<Tc>(g.cx, g.cxd, fx + 1);
    const Tc cs = face_c<Tc>(g.cy, g.cyd, fy), cn = face_c<Tc>(g.cy, g.cyd, fy + mx);
    Tc cd = Tc(0), cu = Tc(0);
    if (g.dim == 3) {
      cd = face_c<Tc>(g.cz, g.czd, (long long)row * mx + ix);
      cu = face_c<Tc>(g.cz, g.czd, (long long)row * mx + ix + pl);
    }
    Tc kd = (cw + ce + cs + cn + cd + cu) * dc;
    if (ix > 0) kd -= cw * dv(e - 1);
    if (ix < mx - 1) kd -= ce * dv(e + 1);
    if (jy > 0) kd -= cs * dv(e - mx);
    if (jy < my - 1) kd -= cn * dv(e + mx);
    if (jz > 0) kd -= cd * dv(e - pl);
    if (jz < mz - 1) kd -= cu * dv(e + pl);
    r[e] = rsrc[e] - (lh[k] * dc + lht[k] * kd);
    x[e] = first ? dc : x[e] + dc;
    dnext[e] = dc;
  }
}

// Last step: d = a_k d_{j-1} + w (w alone when first), o = x + d (d alone when first); z holds
// the time-transformed v, and <v, P^-1 v> = sum z * o (the time DST is orthogonal) completes in
// the last block, which also runs the MINRES scalar step.  The per-thread sum is compensated in
// the transform type (float64 arithmetic per element would bind a float32 pass to the slow
// float64 pipe) and combined across threads in float64.  o is a separate array: rewriting z in
// place inside this accumulating loop measured five times slower (213 against 43 us per
// 255^2 x 128 float pass).
template <class Tc>
__global__ void __launch_bounds__(kNT)
    k_cheb_final(long long N, long long m, const Tc *__restrict__ dprev,
                 const Tc *__restrict__ w, const Tc *__restrict__ x, const Tc *__restrict__ z,
                 Tc *__restrict__ o, const Tc *__restrict__ acoef, int first, State *S, int tmode,
                 double *__restrict__ partials, int gk) {
  __shared__ double red[32];
  if (gate_closed(S, gk)) return;
  Tc esum = Tc(0), ecomp = Tc(0);
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < N;
       e += (long long)gridDim.x * blockDim.x) {
    const unsigned k = (unsigned)e / (unsigned)m;
    const Tc d = first ? w[e] : acoef[k] * dprev[e] + w[e];
    const Tc xv = first ? d : x[e] + d;
    const Tc term = z[e] * xv - ecomp;
    const Tc t = esum + term;
    ecomp = (t - esum) - term;
    esum = t;
    o[e] = xv;
  }
  if (tmode != TM_NONE) {
    const double en = (double)esum - (double)ecomp;
    double tot;
    if (last_block_reduce<kNT>(en, partials, &S->counter[CNT_TIME], gridDim.x, blockIdx.x, red,
                               &tot) &&
        threadIdx.x == 0) {
      if (tmode == TM_INIT || tmode == TM_RESTART)
        minres_init_scalars_dev(S, tot);
      else
        minres_givens_dev(S, tot);
    }
  }
}

// z = source elements in the transform type (a conversion, or the fused Lanczos step)
template <class Tc, class Src>
__global__ void k_copy_to(long long N, Src src, Tc *z, const State *S, int gk) {
  if (gate_closed(S, gk)) return;
  src.prepare(S);
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < N;
       e += (long long)gridDim.x * blockDim.x)
    z[e] = src(e);
}

// the x pass that carries the fused Lanczos step is timed as its own kernel class
template <class Src>
struct is_lanczos_src {
  static constexpr bool value = false;
};
template <class Tc, class Tv>
struct is_lanczos_src<SrcLanczos<Tc, Tv>> {
  static constexpr bool value = true;
};

template <class Tc>
size_t dst_smem(int L, int PB) {
  return (size_t)(L / 2) * sizeof(cpx<Tc>) + (size_t)PB * fft_seq_stride<Tc>(L) * sizeof(cpx<Tc>);
}

template <class Tc>
int dst_pairs(int L) {
  // PB sequences per block: a power of two, at most 16, with PB * L <= 8 * kNTD so that every
  // pass holds at most eight complex values per thread in registers
  int PB = 16;
  while (PB > 1 && PB * L > 8 * kNTD) PB /= 2;
  return PB;
}

template <class Tc>
size_t time_smem(int n, int J) {
  return ((size_t)2 * n * J + 2 * (n + 1) + J) * sizeof(Tc);
}

template <class Tc, class Src, class Tout, bool XL, int LOGL>
cudaError_t launch_dst_l(Src in, Tout *out, int len, long long nlines, int mx, long long m,
                         const Tc *tw, const State *S, int gk, int pbshift, cudaStream_t st) {
  constexpr int L = 1 << LOGL;
  int PB = dst_pairs<Tc>(L) >> pbshift;
  if (PB < 1) PB = 1;
  const size_t sm = dst_smem<Tc>(L, PB);
  const long long blocks = (nlines + 2 * PB - 1) / (2 * PB);
  auto kern = k_dst_space<Tc, Src, Tout, XL, LOGL>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  if (e != cudaSuccess) return e;
  prof_begin(XL ? (is_lanczos_src<Src>::value ? KC_LANCZOS : KC_DSTX) : KC_DSTY, st);
  kern<<<(unsigned)blocks, kNTD, sm, st>>>(in, out, len, nlines, mx, m, tw, PB, S, gk);
  prof_end(st);
  return cudaGetLastError();
}

template <class Tc, class Src, class Tout, bool XL>
cudaError_t launch_dst(Src in, Tout *out, int len, int L, long long nlines, int mx,
                       long long m, const Tc *tw, const State *S, int gk, int pbshift,
                       cudaStream_t st) {
  switch (L) {
    case 8: return launch_dst_l<Tc, Src, Tout, XL, 3>(in, out, len, nlines, mx, m, tw, S, gk, pbshift, st);
    case 16: return launch_dst_l<Tc, Src, Tout, XL, 4>(in, out, len, nlines, mx, m, tw, S, gk, pbshift, st);
    case 32: return launch_dst_l<Tc, Src, Tout, XL, 5>(in, out, len, nlines, mx, m, tw, S, gk, pbshift, st);
    case 64: return launch_dst_l<Tc, Src, Tout, XL, 6>(in, out, len, nlines, mx, m, tw, S, gk, pbshift, st);
    case 128: return launch_dst_l<Tc, Src, Tout, XL, 7>(in, out, len, nlines, mx, m, tw, S, gk, pbshift, st);
    case 256: return launch_dst_l<Tc, Src, Tout, XL, 8>(in, out, len, nlines, mx, m, tw, S, gk, pbshift, st);
    case 512: return launch_dst_l<Tc, Src, Tout, XL, 9>(in, out, len, nlines, mx, m, tw, S, gk, pbshift, st);
    case 1024: return launch_dst_l<Tc, Src, Tout, XL, 10>(in, out, len, nlines, mx, m, tw, S, gk, pbshift, st);
    case 2048: return launch_dst_l<Tc, Src, Tout, XL, 11>(in, out, len, nlines, mx, m, tw, S, gk, pbshift, st);
    default: return cudaErrorInvalidValue;
  }
}

template <class Tc>
struct TimeTile;
template <>
struct TimeTile<double> {
  static constexpr int KT = 4, JT = 2;
};
template <>
struct TimeTile<float> {
  static constexpr int KT = 8, JT = 4;
};
template <>
struct TimeTile<dd> {
  static constexpr int KT = 4, JT = 4;
};

template <class Tc>
int time_J(int n) {
  // columns per block: two n x J tiles within ~128 KB (at most ~200 KB for long time axes),
  // J a multiple of the thread-tile width, preferably of 16 for full 128-byte rows
  const int JT = TimeTile<Tc>::JT;
  const size_t per_col = (2 * (size_t)n + 1) * sizeof(Tc);
  int J = (int)((128 * 1024) / per_col);
  if (J >= 16) {
    J = (J / 16) * 16;
    if (J > 64) J = 64;
  } else {
    J = (int)((200 * 1024 - 2 * (size_t)(n + 1) * sizeof(Tc)) / per_col);
    if (J > 16) J = 16;
  }
  J = (J / JT) * JT;
  if (J < JT) J = JT;
  return J;
}

// out: null for in place, else an array that does not overlap data
template <class Tc>
cudaError_t launch_time(Tc *data, const Geom &g, const Spec<Tc> &sp, State *S, int tmode,
                        int tkind, double *partials, int gk, int Jover, cudaStream_t st,
                        Tc *out = nullptr) {
  const int J = Jover > 0 ? Jover : time_J<Tc>(g.n);
  const size_t sm = time_smem<Tc>(g.n, J);
  const long long blocks = (g.m + J - 1) / J;
  constexpr int KT = TimeTile<Tc>::KT, JT = TimeTile<Tc>::JT;
  auto kern = k_time<Tc, KT, JT>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  if (e != cudaSuccess) return e;
  prof_begin(KC_TIME, st);
  kern<<<(unsigned)blocks, kNT, sm, st>>>(data, out ? out : data, g.n, g.m, g.mx, J, sp, S, tmode,
                                          tkind, partials, gk);
  prof_end(st);
  return cudaGetLastError();
}

}  // namespace

int time_blocks_for(const Geom &g, const PrecPlan &pp, bool fp32) {
  int J = fp32 ? pp.time_J_f : pp.time_J_d;
  if (J <= 0) J = fp32 ? time_J<float>(g.n) : time_J<double>(g.n);
  return (int)((g.m + J - 1) / J);
}

int time_J_default(int n, bool fp32) { return fp32 ? time_J<float>(n) : time_J<double>(n); }

bool time_J_fits(int n, int J, bool fp32) {
  const int JT = fp32 ? TimeTile<float>::JT : TimeTile<double>::JT;
  if (J < JT || J % JT) return false;
  const size_t sm = fp32 ? time_smem<float>(n, J) : time_smem<double>(n, J);
  return sm <= 200 * 1024;
}

template <class Tc>
static const Tc *tw_of(const PrecPlan &pp, bool x);
template <>
const double *tw_of<double>(const PrecPlan &pp, bool x) {
  return x ? pp.twx_d : pp.twy_d;
}
template <>
const float *tw_of<float>(const PrecPlan &pp, bool x) {
  return x ? pp.twx_f : pp.twy_f;
}
template <>
const dd *tw_of<dd>(const PrecPlan &pp, bool x) {
  return x ? pp.twx_dd : pp.twy_dd;
}
template <class Tc>
static const Spec<Tc> &spec_of(const PrecPlan &pp);
template <>
const Spec<double> &spec_of<double>(const PrecPlan &pp) {
  return pp.spec_d;
}
template <>
const Spec<float> &spec_of<float>(const PrecPlan &pp) {
  return pp.spec_f;
}
template <>
const Spec<dd> &spec_of<dd>(const PrecPlan &pp) {
  return pp.spec_dd;
}

template <class Tc>
static const Tc *cheb_a_of(const PrecPlan &pp);
template <>
const double *cheb_a_of<double>(const PrecPlan &pp) {
  return pp.cheb_a_d;
}
template <>
const float *cheb_a_of<float>(const PrecPlan &pp) {
  return pp.cheb_a_f;
}
template <class Tc>
static const Tc *cheb_s_of(const PrecPlan &pp);
template <>
const double *cheb_s_of<double>(const PrecPlan &pp) {
  return pp.cheb_s_d;
}
template <>
const float *cheb_s_of<float>(const PrecPlan &pp) {
  return pp.cheb_s_f;
}

constexpr int kChebBlocks = 152 * 8;

// Spatial DST-I along y (lines mx apart, planes of mx*my, n*mz of them) or z (lines mx*my apart,
// planes of m, n of them), from src into out: the tensor cores in float32 when the plan has the
// S_len image, else the shared-memory FFT.  Tensor-core passes work in place (src must be out).
template <class Tc, class Src>
cudaError_t dst_y_pass(Src src, Tc *out, const Geom &g, const PrecPlan &pp, State *S, int gk,
                       cudaStream_t st) {
  if (sizeof(Tc) == sizeof(float) && pp.sop_y != nullptr)
    return launch_dst_tc_y(reinterpret_cast<float *>(out), g, pp.sop_y, S, gk, st);
  const long long ny = (long long)g.n * g.mz * g.mx;
  return launch_dst<Tc, Src, Tc, false>(src, out, g.my, pp.Ly, ny, g.mx, (long long)g.mx * g.my,
                                        tw_of<Tc>(pp, false), S, gk, pp.dst_shift, st);
}

// The last spatial pass, DST-I along x in place: the tensor cores in float32 when the plan has
// the S_mx image, else the shared-memory FFT.
template <class Tc, class Tout>
cudaError_t dst_x_last_pass(Tout *z, const Geom &g, const PrecPlan &pp, State *S, int gk,
                            cudaStream_t st) {
  if (sizeof(Tc) == sizeof(float) && pp.sop_x != nullptr)
    return launch_dst_tc_x(reinterpret_cast<float *>(z), g, pp.sop_x, S, gk, st);
  const long long nx = (long long)g.n * g.my * g.mz;
  return launch_dst<Tc, SrcArray<Tc, Tout>, Tout, true>(SrcArray<Tc, Tout>{z}, z, g.mx, pp.Lx,
                                                        nx, g.mx, g.m, tw_of<Tc>(pp, true), S,
                                                        gk, pp.dst_shift, st);
}

template <class Tc>
static const Tc *twz_of(const PrecPlan &pp);
template <>
const double *twz_of<double>(const PrecPlan &pp) {
  return pp.twz_d;
}
template <>
const float *twz_of<float>(const PrecPlan &pp) {
  return pp.twz_f;
}
template <>
const dd *twz_of<dd>(const PrecPlan &pp) {
  return pp.twz_dd;
}

template <class Tc, class Src>
cudaError_t dst_z_pass(Src src, Tc *out, const Geom &g, const PrecPlan &pp, State *S, int gk,
                       cudaStream_t st) {
  if (sizeof(Tc) == sizeof(float) && pp.sop_z != nullptr)
    return launch_dst_tc_z(reinterpret_cast<float *>(out), g, pp.sop_z, S, gk, st);
  const long long nz = (long long)g.n * g.mx * g.my;
  return launch_dst<Tc, Src, Tc, false>(src, out, g.mz, pp.Lz, nz, g.mx * g.my, g.m,
                                        twz_of<Tc>(pp), S, gk, pp.dst_shift, st);
}

// The time DST alone (the P_theta paths with varying a): tensor cores in float32 when the plan has
// the S_n image, else the FFMA/DFMA kernel.
// in -> out (the same array, or one that does not overlap).
template <class Tc>
cudaError_t time_single(Tc *in, Tc *out, const Geom &g, const PrecPlan &pp, State *S,
                        double *partials, int gk, int Jo, cudaStream_t st) {
  if (sizeof(Tc) == sizeof(float) && pp.sop_t1 != nullptr)
    return launch_time_tc_single(reinterpret_cast<const float *>(in),
                                 reinterpret_cast<float *>(out), g, pp.sop_t1, S, gk, st);
  return launch_time<Tc>(in, g, spec_of<Tc>(pp), S, TM_NONE, 1, partials, gk, Jo, st, out);
}

// P_theta with a varying 2D/3D coefficient: time DST, pp.cheb Chebyshev steps per frequency, time
// DST (see k_cheb_resid).  zc receives the source, then the transformed v, then the result (the
// last step leaves its iterate in R, from which the inverse time DST writes zc).
template <class Tc, class Src>
cudaError_t cheb_stages(const Geom &g, const PrecPlan &pp, Src src, Tc *zc, State *S, int tmode,
                        double *partials, cudaStream_t st, cudaEvent_t after_time) {
  using Arr = SrcArray<Tc, Tc>;
  const int gk = gate_kind_of(tmode);
  const Spec<Tc> &sp = spec_of<Tc>(pp);
  const long long N = g.N;
  Tc *R = reinterpret_cast<Tc *>(pp.cheb_work);
  Tc *W = R + N, *X = R + 2 * N;
  Tc *Dd[2] = {R + 3 * N, R + 4 * N};
  const Tc *acoef = cheb_a_of<Tc>(pp), *scoef = cheb_s_of<Tc>(pp);
  const int Jo = sizeof(Tc) == sizeof(float) ? pp.time_J_f : pp.time_J_d;
  const long long nx = (long long)g.n * g.my * g.mz;
  const Tc *twx = tw_of<Tc>(pp, true);
  cudaError_t e;
  // the y (and z) passes of one half of the spatial transform, in place
  auto yz_pass = [&](Tc *a) -> cudaError_t {
    cudaError_t r = dst_y_pass<Tc>(Arr{a}, a, g, pp, S, gk, st);
    if (r == cudaSuccess && g.dim == 3) r = dst_z_pass<Tc>(Arr{a}, a, g, pp, S, gk, st);
    return r;
  };
  prof_begin(KC_AUX, st);
  k_copy_to<Tc, Src><<<kChebBlocks, kNT, 0, st>>>(N, src, zc, S, gk);
  prof_end(st);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  e = time_single<Tc>(zc, zc, g, pp, S, partials, gk, Jo, st);
  if (e != cudaSuccess) return e;
  int cur = 0;
  for (int j = 0; j < pp.cheb; ++j) {
    // the axes commute: x, y (z), then x with the scaling fused into its loads, then y (z); the
    // y and z passes take the tensor cores in float32 when the plan has the S_my / S_mz image
    e = launch_dst<Tc, Arr, Tc, true>(Arr{j == 0 ? zc : R}, W, g.mx, pp.Lx, nx, g.mx, g.m, twx, S,
                                      gk, pp.dst_shift, st);
    if (e != cudaSuccess) return e;
    if ((e = yz_pass(W)) != cudaSuccess) return e;
    const SrcChebScale<Tc> sc{W, scoef + (size_t)j * g.n, sp.lh, sp.lht, sp.mux, sp.muy,
                              (unsigned)g.m, (unsigned)g.mx};
    e = launch_dst<Tc, SrcChebScale<Tc>, Tc, true>(sc, W, g.mx, pp.Lx, nx, g.mx, g.m, twx, S, gk,
                                                   pp.dst_shift, st);
    if (e != cudaSuccess) return e;
    if ((e = yz_pass(W)) != cudaSuccess) return e;
    const Tc *aj = acoef + (size_t)j * g.n;
    if (j + 1 < pp.cheb) {
      const dim3 rb(kChebBX, kChebBY);
      const dim3 rg((unsigned)((g.my * g.mz + kChebBY - 1) / kChebBY),
                    (unsigned)((g.mx + kChebBX - 1) / kChebBX), (unsigned)g.n);
      prof_begin(KC_TIME, st);
      k_cheb_resid<Tc><<<rg, rb, 0, st>>>(g, Dd[cur], W, Dd[cur ^ 1], j == 0 ? zc : R, R, X, aj,
                                          sp.lh, sp.lht, j == 0 ? 1 : 0, S, gk);
      prof_end(st);
      cur ^= 1;
    } else {
      prof_begin(KC_TIME, st);
      k_cheb_final<Tc><<<kChebBlocks, kNT, 0, st>>>(N, g.m, Dd[cur], W, X, zc, R, aj,
                                                    j == 0 ? 1 : 0, S, tmode, partials, gk);
      prof_end(st);
    }
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  if (after_time && (e = cudaEventRecord(after_time, st)) != cudaSuccess) return e;
  return time_single<Tc>(R, zc, g, pp, S, partials, gk, Jo, st);
}

// The same source with double-float as its transform type.
template <class Src>
struct AsDd;
template <class Tin>
struct AsDd<SrcArray<double, Tin>> {
  static SrcArray<dd, Tin> of(const SrcArray<double, Tin> &s) { return SrcArray<dd, Tin>{s.p}; }
};
template <>
struct AsDd<SrcLanczos<double, double>> {
  static SrcLanczos<dd, double> of(const SrcLanczos<double, double> &s) {
    SrcLanczos<dd, double> r{};
    r.q = s.q;
    r.vk = s.vk;
    r.vp = s.vp;
    return r;
  }
};

// The float64 preconditioner's P_H / P-hat pass with every transform and the scaling in
// double-float arithmetic: the first x pass reads the float64 source and stores double-floats in
// z; the y (z) passes and the time kernel work on that double-float copy in place; the last x pass
// reads it and writes float64 back into z.  Same stages and order as the float64 pass.
template <class Src>
cudaError_t prec_stages_dd(const Geom &g, const PrecPlan &pp, Src src, double *z, State *S,
                           int tmode, double *partials, cudaStream_t st, cudaEvent_t after_time) {
  using Inner = SrcArray<dd, dd>;
  const int gk = gate_kind_of(tmode);
  dd *zd = reinterpret_cast<dd *>(z);
  const long long nx = (long long)g.n * g.my * g.mz;
  cudaError_t e;
  e = launch_dst<dd, decltype(AsDd<Src>::of(src)), dd, true>(AsDd<Src>::of(src), zd, g.mx, pp.Lx,
                                                             nx, g.mx, g.m, pp.twx_dd, S, gk,
                                                             pp.dst_shift, st);
  if (e != cudaSuccess) return e;
  if (g.dim >= 2 && (e = dst_y_pass<dd>(Inner{zd}, zd, g, pp, S, gk, st)) != cudaSuccess) return e;
  if (g.dim == 3 && (e = dst_z_pass<dd>(Inner{zd}, zd, g, pp, S, gk, st)) != cudaSuccess) return e;
  if (pp.sdig && pp.tscratch)
    e = launch_time_tcd(zd, pp.tscratch, g, pp.spec_dd, pp.sdig, pp.sdig_e, S, tmode, partials,
                        gk, st);
  else
    e = launch_time<dd>(zd, g, pp.spec_dd, S, tmode, 0, partials, gk, pp.time_J_dd, st);
  if (e != cudaSuccess) return e;
  if (after_time && (e = cudaEventRecord(after_time, st)) != cudaSuccess) return e;
  if (g.dim == 3 && (e = dst_z_pass<dd>(Inner{zd}, zd, g, pp, S, gk, st)) != cudaSuccess) return e;
  if (g.dim >= 2 && (e = dst_y_pass<dd>(Inner{zd}, zd, g, pp, S, gk, st)) != cudaSuccess) return e;
  return launch_dst<dd, Inner, double, true>(Inner{zd}, z, g.mx, pp.Lx, nx, g.mx, g.m, pp.twx_dd,
                                             S, gk, pp.dst_shift, st);
}

// The stages of one preconditioner pass; `src` feeds the first one.
// after_time (optional) is recorded once the time kernel (which performs the MINRES scalar step)
// has been enqueued.
template <class Tc, class Src, class Tout>
cudaError_t prec_stages(const Geom &g, const PrecPlan &pp, Src src, Tout *z, State *S, int tmode,
                        double *partials, cudaStream_t st, cudaEvent_t after_time = nullptr) {
  static_assert(sizeof(Tc) == sizeof(Tout), "in-place stages need Tout == Tc");
  using Inner = SrcArray<Tc, Tout>;
  const int gk = gate_kind_of(tmode);
  cudaError_t e;
  if constexpr (sizeof(Tc) == sizeof(double)) {
    if (pp.fp64_dd && !pp.cheb && !pp.pcr)
      return prec_stages_dd(g, pp, src, reinterpret_cast<double *>(z), S, tmode, partials, st,
                            after_time);
  }
  if (pp.cheb)
    return cheb_stages<Tc>(g, pp, src, reinterpret_cast<Tc *>(z), S, tmode, partials, st,
                           after_time);
  if (pp.pcr) {
    // P_theta with a varying 1D coefficient: time DST, tridiagonal solves, time DST
    Tc *zc = reinterpret_cast<Tc *>(z);
    prof_begin(KC_AUX, st);
    k_copy_to<Tc, Src><<<152 * 8, kNT, 0, st>>>(g.N, src, zc, S, gk);
    prof_end(st);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    const int Jo = sizeof(Tc) == sizeof(float) ? pp.time_J_f : pp.time_J_d;
    e = time_single<Tc>(zc, zc, g, pp, S, partials, gk, Jo, st);
    if (e != cudaSuccess) return e;
    const size_t sm = (size_t)8 * g.mx * sizeof(Tc);
    auto kern = k_pcr_ptheta<Tc>;
    e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    prof_begin(KC_TIME, st);
    kern<<<g.n, kNT, sm, st>>>(zc, g.n, g.mx, g.cx, spec_of<Tc>(pp), S, tmode, partials, gk);
    prof_end(st);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if (after_time && (e = cudaEventRecord(after_time, st)) != cudaSuccess) return e;
    return time_single<Tc>(zc, zc, g, pp, S, partials, gk, Jo, st);
  }
  const long long nx = (long long)g.n * g.my * g.mz;
  Tc *zt = reinterpret_cast<Tc *>(z);
  e = launch_dst<Tc, Src, Tout, true>(src, z, g.mx, pp.Lx, nx, g.mx, g.m, tw_of<Tc>(pp, true), S,
                                      gk, pp.dst_shift, st);
  if (e != cudaSuccess) return e;
  if (g.dim >= 2 && (e = dst_y_pass<Tc>(Inner{z}, zt, g, pp, S, gk, st)) != cudaSuccess) return e;
  if (g.dim == 3 && (e = dst_z_pass<Tc>(Inner{z}, zt, g, pp, S, gk, st)) != cudaSuccess) return e;
  if (sizeof(Tc) == sizeof(float) && pp.sop != nullptr)
    e = launch_time_tc(reinterpret_cast<float *>(z), g, pp.spec_f, pp.sop, S, tmode, partials, gk,
                       st);
  else if (sizeof(Tc) == sizeof(float) && pp.sop_long != nullptr)
    e = launch_time_tc_long(reinterpret_cast<float *>(z), g, pp.spec_f, pp.sop_long, S, tmode,
                            partials, gk, st);
  else
    e = launch_time<Tc>(reinterpret_cast<Tc *>(z), g, spec_of<Tc>(pp), S, tmode, 0, partials, gk,
                        sizeof(Tc) == sizeof(float) ? pp.time_J_f : pp.time_J_d, st);
  if (e != cudaSuccess) return e;
  if (after_time && (e = cudaEventRecord(after_time, st)) != cudaSuccess) return e;
  if (g.dim == 3 && (e = dst_z_pass<Tc>(Inner{z}, zt, g, pp, S, gk, st)) != cudaSuccess) return e;
  if (g.dim >= 2 && (e = dst_y_pass<Tc>(Inner{z}, zt, g, pp, S, gk, st)) != cudaSuccess) return e;
  return dst_x_last_pass<Tc>(z, g, pp, S, gk, st);
}

template <class Tc, class Tin, class Tout>
cudaError_t launch_prec(const Geom &g, const PrecPlan &pp, const Tin *v, Tout *z, State *S,
                        int tmode, double *partials, cudaStream_t st) {
  return prec_stages<Tc>(g, pp, SrcArray<Tc, Tin>{v}, z, S, tmode, partials, st);
}

// One MINRES iteration's preconditioner pass with the Lanczos step fused into its first stage:
// vnext <- q - lz_a vk - lz_b vnext, z <- P^-1 vnext.
template <class Tc, class Tin, class Tout>
cudaError_t launch_prec_lanczos(const Geom &g, const PrecPlan &pp, const Tin *q, const Tin *vk,
                                Tin *vnext, Tout *z, State *S, double *partials, cudaStream_t st,
                                cudaEvent_t after_time) {
  SrcLanczos<Tc, Tin> src{};
  src.q = q;
  src.vk = vk;
  src.vp = vnext;
  return prec_stages<Tc>(g, pp, src, z, S, TM_ITER, partials, st, after_time);
}

// Autotuning helpers: the spatial DSTs (x then y, in place) and the FFMA time kernel alone,
// ungated, with the knobs currently in pp.
cudaError_t tune_run_dsts(const Geom &g, const PrecPlan &pp, bool fp32, void *data,
                          cudaStream_t st) {
  const long long nx = (long long)g.n * g.my * g.mz, ny = (long long)g.n * g.mz * g.mx;
  const long long nz = (long long)g.n * g.mx * g.my;
  cudaError_t e;
  if (fp32) {
    float *z = (float *)data;
    using A = SrcArray<float, float>;
    e = launch_dst<float, A, float, true>(A{z}, z, g.mx, pp.Lx, nx, g.mx, g.m, pp.twx_f, nullptr,
                                          GK_NONE, pp.dst_shift, st);
    if (e == cudaSuccess && g.dim >= 2)
      e = launch_dst<float, A, float, false>(A{z}, z, g.my, pp.Ly, ny, g.mx,
                                             (long long)g.mx * g.my, pp.twy_f, nullptr, GK_NONE,
                                             pp.dst_shift, st);
    if (e == cudaSuccess && g.dim == 3)
      e = launch_dst<float, A, float, false>(A{z}, z, g.mz, pp.Lz, nz, g.mx * g.my, g.m,
                                             pp.twz_f, nullptr, GK_NONE, pp.dst_shift, st);
  } else if (pp.fp64_dd) {
    // the float64 path's double-float engine: its own FFT kernels (double-float data in place)
    dd *z = (dd *)data;
    using A = SrcArray<dd, dd>;
    e = launch_dst<dd, A, dd, true>(A{z}, z, g.mx, pp.Lx, nx, g.mx, g.m, pp.twx_dd, nullptr,
                                    GK_NONE, pp.dst_shift, st);
    if (e == cudaSuccess && g.dim >= 2)
      e = launch_dst<dd, A, dd, false>(A{z}, z, g.my, pp.Ly, ny, g.mx, (long long)g.mx * g.my,
                                       pp.twy_dd, nullptr, GK_NONE, pp.dst_shift, st);
    if (e == cudaSuccess && g.dim == 3)
      e = launch_dst<dd, A, dd, false>(A{z}, z, g.mz, pp.Lz, nz, g.mx * g.my, g.m, pp.twz_dd,
                                       nullptr, GK_NONE, pp.dst_shift, st);
  } else {
    double *z = (double *)data;
    using A = SrcArray<double, double>;
    e = launch_dst<double, A, double, true>(A{z}, z, g.mx, pp.Lx, nx, g.mx, g.m, pp.twx_d,
                                            nullptr, GK_NONE, pp.dst_shift, st);
    if (e == cudaSuccess && g.dim >= 2)
      e = launch_dst<double, A, double, false>(A{z}, z, g.my, pp.Ly, ny, g.mx,
                                               (long long)g.mx * g.my, pp.twy_d, nullptr,
                                               GK_NONE, pp.dst_shift, st);
    if (e == cudaSuccess && g.dim == 3)
      e = launch_dst<double, A, double, false>(A{z}, z, g.mz, pp.Lz, nz, g.mx * g.my, g.m,
                                               pp.twz_d, nullptr, GK_NONE, pp.dst_shift, st);
  }
  return e;
}

cudaError_t tune_run_pass(const Geom &g, const PrecPlan &pp, int axis,
                          const unsigned short *tc_img, float *data, State *S, cudaStream_t st) {
  PrecPlan q = pp;
  using A = SrcArray<float, float>;
  if (axis == 0) {
    q.sop_x = tc_img;
    return dst_x_last_pass<float>(data, g, q, S, GK_NONE, st);
  }
  if (axis == 1) {
    q.sop_y = tc_img;
    return dst_y_pass<float>(A{data}, data, g, q, S, GK_NONE, st);
  }
  q.sop_z = tc_img;
  return dst_z_pass<float>(A{data}, data, g, q, S, GK_NONE, st);
}

cudaError_t tune_run_time_dd(const Geom &g, const PrecPlan &pp, void *data, cudaStream_t st) {
  return launch_time<dd>((dd *)data, g, pp.spec_dd, nullptr, TM_NONE, 0, nullptr, GK_NONE,
                         pp.time_J_dd, st);
}

cudaError_t tune_run_time(const Geom &g, const PrecPlan &pp, bool fp32, void *data,
                          cudaStream_t st) {
  if (fp32)
    return launch_time<float>((float *)data, g, pp.spec_f, nullptr, TM_NONE, 0, nullptr, GK_NONE,
                              pp.time_J_f, st);
  return launch_time<double>((double *)data, g, pp.spec_d, nullptr, TM_NONE, 0, nullptr, GK_NONE,
                             pp.time_J_d, st);
}

template cudaError_t launch_prec<double, double, double>(const Geom &, const PrecPlan &,
                                                         const double *, double *, State *, int,
                                                         double *, cudaStream_t);
template cudaError_t launch_prec<float, double, float>(const Geom &, const PrecPlan &,
                                                       const double *, float *, State *, int,
                                                       double *, cudaStream_t);
template cudaError_t launch_prec<float, df, float>(const Geom &, const PrecPlan &, const df *,
                                                   float *, State *, int, double *, cudaStream_t);
template cudaError_t launch_prec_lanczos<double, double, double>(const Geom &, const PrecPlan &,
                                                                 const double *, const double *,
                                                                 double *, double *, State *,
                                                                 double *, cudaStream_t,
                                                                 cudaEvent_t);
template cudaError_t launch_prec_lanczos<float, double, float>(const Geom &, const PrecPlan &,
                                                               const double *, const double *,
                                                               double *, float *, State *,
                                                               double *, cudaStream_t,
                                                               cudaEvent_t);
template cudaError_t launch_prec_lanczos<float, df, float>(const Geom &, const PrecPlan &,
                                                           const df *, const df *, df *, float *,
                                                           State *, double *, cudaStream_t,
                                                           cudaEvent_t);

}  // namespace st
