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

namespace st {

namespace {

constexpr int kNT = 256;

__device__ __forceinline__ double rsq(double x) { return rsqrt(x); }
__device__ __forceinline__ float rsq(float x) { return rsqrtf(x); }

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

// float32 transforms: three 512-thread blocks per SM (at most 40 registers); float64: two
template <class Tc, class Src, class Tout, bool XL, int LOGL>
__global__ void __launch_bounds__(kNTD, sizeof(Tc) == 4 ? 3 : 2)
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
  if (XL) {
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
    Tc acc[KT][JT];
#pragma unroll
    for (int i = 0; i < KT; ++i)
#pragma unroll
      for (int c = 0; c < JT; ++c) acc[i][c] = Tc(0);
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
        for (int c = 0; c < JT; ++c) acc[i][c] = fma(sv, f[c], acc[i][c]);
      }
    }
    if (odd && nodd_mid) {
      const Tc *F = Fb + (tm - 1) * J;
#pragma unroll
      for (int i = 0; i < KT; ++i) {
        const Tc sv = sintab[(int)(((long long)kk[i] * tm) % P2)];
#pragma unroll
        for (int c = 0; c < JT; ++c) acc[i][c] = fma(sv, F[c], acc[i][c]);
      }
    }
#pragma unroll
    for (int i = 0; i < KT; ++i) {
      if (rg * KT + i < cnt) {
        Tc *Yr = Y + (kk[i] - 1) * J + jg * JT;
#pragma unroll
        for (int c = 0; c < JT; ++c) Yr[c] = acc[i][c];
      }
    }
  }
  __syncthreads();
}

// 1/p for the eigenvalue of the preconditioner at time frequency k (1-based) and tau*mu.
template <class T>
__device__ __forceinline__ T inv_symbol(const Spec<T> &sp, int k, T tmu) {
  const T hk = sp.hk[k - 1], ck = sp.ck[k - 1], sk = sp.sk[k - 1];
  if (sp.prec == ST_PREC_PTHETA) {
    // lam_H = sqrt(2 - 2cos x) = 2 sin(x/2), lam_Htheta = sqrt(th^2 + (1-th)^2 + 2 th(1-th) cos x)
    return T(1) / (sp.lh[k - 1] + sp.lht[k - 1] * tmu);
  }
  T re, im;
  if (sp.scheme == ST_THETA) {
    // |a0 + a1 e^{ix}|, a0 = 1 + th tmu, a1 = -1 + (1-th) tmu;  a0 + a1 cos x = (1 - cos x) +
    // tmu (th + (1-th) cos x)
    re = hk + tmu * (sp.theta + (T(1) - sp.theta) * ck);
    im = (T(-1) + (T(1) - sp.theta) * tmu) * sk;
  } else {
    // |a0 + a1 e^{ix} + a2 e^{2ix}|, a0 = 3/2 + tmu, a1 = -2, a2 = 1/2:
    // re = (1 - cos x)^2 + tmu, im = -sin x (2 - cos x)
    re = hk * hk + tmu;
    im = -sk * (T(1) + hk);
  }
  return rsq(re * re + im * im);
}

template <class Tc, int KT, int JT>
__global__ void __launch_bounds__(kNT)
    k_time(Tc *data, int n, long long m, int mx, int J, Spec<Tc> sp, State *S,
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
      if (c < Je) data[(long long)t * m + j0 + c] = X[idx];
    }
  } else {
    for (int idx = tid; idx < n * J; idx += kNT) {
      const int t = idx / J, c = idx - t * J;
      if (c < Je) data[(long long)t * m + j0 + c] = Y[idx];
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

// z = source elements in the transform type (a conversion, or the fused Lanczos step)
template <class Tc, class Src>
__global__ void k_copy_to(long long N, Src src, Tc *z, const State *S, int gk) {
  if (gate_closed(S, gk)) return;
  src.prepare(S);
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < N;
       e += (long long)gridDim.x * blockDim.x)
    z[e] = src(e);
}

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
  prof_begin(XL ? KC_DSTX : KC_DSTY, st);
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

template <class Tc>
cudaError_t launch_time(Tc *data, const Geom &g, const Spec<Tc> &sp, State *S, int tmode,
                        int tkind, double *partials, int gk, int Jover, cudaStream_t st) {
  const int J = Jover > 0 ? Jover : time_J<Tc>(g.n);
  const size_t sm = time_smem<Tc>(g.n, J);
  const long long blocks = (g.m + J - 1) / J;
  constexpr int KT = TimeTile<Tc>::KT, JT = TimeTile<Tc>::JT;
  auto kern = k_time<Tc, KT, JT>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  if (e != cudaSuccess) return e;
  prof_begin(KC_TIME, st);
  kern<<<(unsigned)blocks, kNT, sm, st>>>(data, g.n, g.m, g.mx, J, sp, S, tmode, tkind, partials,
                                          gk);
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
  if (pp.pcr) {
    // P_theta with a varying 1D coefficient: time DST, tridiagonal solves, time DST
    Tc *zc = reinterpret_cast<Tc *>(z);
    prof_begin(KC_AUX, st);
    k_copy_to<Tc, Src><<<152 * 8, kNT, 0, st>>>(g.N, src, zc, S, gk);
    prof_end(st);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    const int Jo = sizeof(Tc) == sizeof(float) ? pp.time_J_f : pp.time_J_d;
    e = launch_time<Tc>(zc, g, spec_of<Tc>(pp), S, TM_NONE, 1, partials, gk, Jo, st);
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
    return launch_time<Tc>(zc, g, spec_of<Tc>(pp), S, TM_NONE, 1, partials, gk, Jo, st);
  }
  const long long nx = (long long)g.n * g.my, ny = (long long)g.n * g.mx;
  e = launch_dst<Tc, Src, Tout, true>(src, z, g.mx, pp.Lx, nx, g.mx, g.m, tw_of<Tc>(pp, true), S,
                                      gk, pp.dst_shift, st);
  if (e != cudaSuccess) return e;
  if (g.dim == 2) {
    if (sizeof(Tc) == sizeof(float) && pp.sop_y != nullptr)
      e = launch_dst_tc_y(reinterpret_cast<float *>(z), g, pp.sop_y, S, gk, st);
    else
      e = launch_dst<Tc, Inner, Tout, false>(Inner{z}, z, g.my, pp.Ly, ny, g.mx, g.m,
                                             tw_of<Tc>(pp, false), S, gk, pp.dst_shift, st);
    if (e != cudaSuccess) return e;
  }
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
  if (g.dim == 2) {
    if (sizeof(Tc) == sizeof(float) && pp.sop_y != nullptr)
      e = launch_dst_tc_y(reinterpret_cast<float *>(z), g, pp.sop_y, S, gk, st);
    else
      e = launch_dst<Tc, Inner, Tout, false>(Inner{z}, z, g.my, pp.Ly, ny, g.mx, g.m,
                                             tw_of<Tc>(pp, false), S, gk, pp.dst_shift, st);
    if (e != cudaSuccess) return e;
  }
  return launch_dst<Tc, Inner, Tout, true>(Inner{z}, z, g.mx, pp.Lx, nx, g.mx, g.m,
                                           tw_of<Tc>(pp, true), S, gk, pp.dst_shift, st);
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
  const long long nx = (long long)g.n * g.my, ny = (long long)g.n * g.mx;
  cudaError_t e;
  if (fp32) {
    float *z = (float *)data;
    using A = SrcArray<float, float>;
    e = launch_dst<float, A, float, true>(A{z}, z, g.mx, pp.Lx, nx, g.mx, g.m, pp.twx_f, nullptr,
                                          GK_NONE, pp.dst_shift, st);
    if (e == cudaSuccess && g.dim == 2)
      e = launch_dst<float, A, float, false>(A{z}, z, g.my, pp.Ly, ny, g.mx, g.m, pp.twy_f,
                                             nullptr, GK_NONE, pp.dst_shift, st);
  } else {
    double *z = (double *)data;
    using A = SrcArray<double, double>;
    e = launch_dst<double, A, double, true>(A{z}, z, g.mx, pp.Lx, nx, g.mx, g.m, pp.twx_d,
                                            nullptr, GK_NONE, pp.dst_shift, st);
    if (e == cudaSuccess && g.dim == 2)
      e = launch_dst<double, A, double, false>(A{z}, z, g.my, pp.Ly, ny, g.mx, g.m, pp.twy_d,
                                               nullptr, GK_NONE, pp.dst_shift, st);
  }
  return e;
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
