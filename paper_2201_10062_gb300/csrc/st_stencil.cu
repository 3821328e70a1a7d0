// Space-time stencil kernels: the flipped all-at-once operator Y T (Sec. 1, eq. theta and
// eq. main_system; Sec. 4, eq. matrix_gen / main_system_gem_sym), the all-at-once right-hand side
// and the face-coefficient gradient used by the adjoint.
//
// T is never stored.  Block row k of T v is A0 v_k + A1 v_{k-1} (+ A2 v_{k-2} for BDF2) with
//   theta: A0 = I + theta tau K, A1 = -I + (1-theta) tau K,
//   BDF2:  A0 = 3/2 I + tau K,   A1 = -2 I,  A2 = 1/2 I,
// and Y only reverses the block order, so row k of T v is written to block n-1-k.
// One thread owns one spatial node and walks a chunk of consecutive time levels (and their
// mirror images), carrying neighbouring planes in registers so that each plane of v is read once.
#include "st_internal.cuh"

namespace st {

namespace {

constexpr int kBX2 = 32, kBY2 = 8;   // 2D block: 32 x 8 nodes
constexpr int kBX1 = 256;            // 1D block: 256 nodes (all block reductions assume 256 threads)
constexpr int kNT = 256;

struct Tile {
  int kc, nchunk, gx, gy;
};

Tile tile_for(const Geom &g) {
  Tile t;
  if (g.dim == 1) {
    t.gx = (g.mx + kBX1 - 1) / kBX1;
    t.gy = 1;
  } else {
    // 2D blocks over x and the rows (y, and z in 3D)
    t.gx = (g.mx + kBX2 - 1) / kBX2;
    t.gy = (g.my * g.mz + kBY2 - 1) / kBY2;
  }
  // chunks cover the first ceil(n/2) planes (each thread also does their mirror images)
  const int half = (g.n + 1) / 2;
  const long long tiles = (long long)t.gx * t.gy;
  // default: 8 resident 256-thread blocks on each of 152 SMs; the autotuner may change it
  const long long target = g.st_target > 0 ? g.st_target : 152LL * 8;
  long long nchunk = (target + tiles - 1) / tiles;
  if (nchunk < 1) nchunk = 1;
  if (nchunk > half) nchunk = half;
  t.kc = (int)((half + nchunk - 1) / nchunk);
  t.nchunk = (half + t.kc - 1) / t.kc;
  return t;
}

template <class Tz>
__device__ __forceinline__ double ld(const Tz *p) {
  return (double)__ldg(p);
}

// tau*K applied at node p = (i, jy, jz) of plane base (zero Dirichlet values outside the grid);
// f holds the node's face coefficients (zero along absent axes, so 1D and 2D add exact zeros).
template <class Tz>
__device__ __forceinline__ double tauK(const Tz *__restrict__ base, long long p, int i, int jy,
                                       int jz, const Geom &g, const Faces6<double> &f, double c) {
  double r = (f.w + f.e + f.s + f.n + f.d + f.u) * c;
  if (i > 0) r -= f.w * ld(base + p - 1);
  if (i < g.mx - 1) r -= f.e * ld(base + p + 1);
  if (g.dim >= 2) {
    if (jy > 0) r -= f.s * ld(base + p - g.mx);
    if (jy < g.my - 1) r -= f.n * ld(base + p + g.mx);
  }
  if (g.dim == 3) {
    const long long pl = (long long)g.mx * g.my;
    if (jz > 0) r -= f.d * ld(base + p - pl);
    if (jz < g.mz - 1) r -= f.u * ld(base + p + pl);
  }
  return r;
}

// The dot products MINRES needs pair the two halves of the time axis: row k of T z lands in
// block n-1-k of Y T z, so <Y T z, z> = sum_k <(T z)_k, z_{n-1-k}>.  Each thread therefore walks
// a chunk of planes k upwards (side A) and the mirrored planes n-1-k downwards (side B) in lock
// step; the centre value of each side is exactly the z the other side's output is paired with,
// so the dot costs no extra loads.  Chunks cover the first ceil(n/2) planes; for odd n the middle
// plane is its own mirror and is done once.
__device__ __forceinline__ void put(double *p, double v) { *p = v; }
__device__ __forceinline__ void put(df *p, double v) { *p = df_of_double(v); }

template <class Tz, int MODE, class TO = double>
__global__ void __launch_bounds__(kNT) k_stencil(Geom g, const Tz *__restrict__ z,
                                                 TO *__restrict__ out,
                                                 const double *__restrict__ fH, State *S,
                                                 double *__restrict__ partials, int kc) {
  __shared__ double red[32];
  if (MODE == SM_MINRES) {
    if (!S->active) return;
    if (S->finish) {
      if (blockIdx.x == 0 && blockIdx.y == 0 && blockIdx.z == 0 && flat_tid() == 0) S->active = 0;
      return;
    }
  }
  if (MODE == SM_RESID_OUTER && !(S->finish && !S->done)) return;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y * blockDim.y + threadIdx.y;  // row jz*my + jy
  const int mx = g.mx, n = g.n;
  const long long m = g.m;
  const bool valid = (i < mx) && (j < g.my * g.mz);
  const int half = (n + 1) >> 1;
  const int k0 = blockIdx.z * kc;
  const int k1 = min(half, k0 + kc);
  const double s = (MODE == SM_MINRES) ? S->inv_beta : 1.0;
  double acc = 0.0;
  if (valid) {
    const int jz = j / g.my, jy = j - jz * g.my;
    const long long p = (long long)j * mx + i;
    const Faces6<double> fc = faces_at(g, i, jy, jz);
    const double th = g.theta, omth = 1.0 - g.theta;
    auto center = [&](int k) -> double { return ld(z + (long long)k * m + p); };
    auto stiff = [&](int k, double c) -> double {
      return tauK(z + (long long)k * m, p, i, jy, jz, g, fc, c);
    };
    // side A (ascending) carries plane kA-1 (and kA-2); side B (descending) carries plane kB and
    // the planes below it
    double a1 = 0.0, aK1 = 0.0, a2 = 0.0;
    double b0 = 0.0, bK0 = 0.0, b1 = 0.0;
    const bool theta = (g.scheme == ST_THETA);
    if (k0 > 0) {
      a1 = center(k0 - 1);
      if (theta) aK1 = stiff(k0 - 1, a1);
    }
    if (!theta && k0 > 1) a2 = center(k0 - 2);
    {
      const int kb = n - 1 - k0;
      b0 = center(kb);
      if (theta) bK0 = stiff(kb, b0);
      else if (kb > 0) b1 = center(kb - 1);
    }
    for (int kA = k0; kA < k1; ++kA) {
      const int kB = n - 1 - kA;
      const double cA = center(kA);
      const double KA = stiff(kA, cA);
      double yA;
      if (theta) {
        yA = (cA - a1) + th * KA + omth * aK1;
        a1 = cA;
        aK1 = KA;
      } else {
        yA = 1.5 * cA - 2.0 * a1 + 0.5 * a2 + KA;
        a2 = a1;
        a1 = cA;
      }
      const bool twin = (kB != kA);
      double yB = 0.0;
      const double zB = twin ? b0 : cA;  // z in plane kB, partner of yA
      if (twin) {
        if (theta) {
          double nb = 0.0, nK = 0.0;
          if (kB > 0) {
            nb = center(kB - 1);
            nK = stiff(kB - 1, nb);
          }
          yB = (b0 - nb) + th * bK0 + omth * nK;
          b0 = nb;
          bK0 = nK;
        } else {
          const double KB = stiff(kB, b0);
          const double nb2 = (kB > 1) ? center(kB - 2) : 0.0;
          yB = 1.5 * b0 - 2.0 * b1 + 0.5 * nb2 + KB;
          b0 = b1;
          b1 = nb2;
        }
      }
      const long long oA = (long long)kB * m + p;  // block n-1-kA receives row kA
      const long long oB = (long long)kA * m + p;  // block n-1-kB = kA receives row kB
      if (MODE == SM_MINRES) {
        yA *= s;
        put(out + oA, yA);
        acc += yA * (zB * s);
        if (twin) {
          yB *= s;
          put(out + oB, yB);
          acc += yB * (cA * s);
        }
      } else if (MODE == SM_APPLY) {
        put(out + oA, yA);
        if (twin) put(out + oB, yB);
      } else {  // SM_RESID(_OUTER): r = Y f_H - Y T x; block n-1-k of Y f_H is f_H block k
        const double rA = fH[(long long)kA * m + p] - yA;
        if (out) put(out + oA, rA);
        acc += rA * rA;
        if (twin) {
          const double rB = fH[(long long)kB * m + p] - yB;
          if (out) put(out + oB, rB);
          acc += rB * rB;
        }
      }
    }
  }
  if (MODE == SM_MINRES || MODE == SM_RESID || MODE == SM_RESID_OUTER) {
    const int nb = gridDim.x * gridDim.y * gridDim.z;
    const int bid = blockIdx.x + gridDim.x * (blockIdx.y + gridDim.y * blockIdx.z);
    double tot;
    unsigned int *cnt = &S->counter[MODE == SM_MINRES ? CNT_STENCIL : CNT_RESID];
    if (last_block_reduce<kNT>(acc, partials, cnt, nb, bid, red, &tot) && flat_tid() == 0) {
      if (MODE == SM_MINRES) {
        S->alpha = tot;
        S->lz_a = tot / S->beta;
        S->lz_b = (S->k > 0) ? S->beta / S->beta_prev : 0.0;
        refresh_df(S);
      } else {
        S->rnorm2 = tot;
        if (MODE == SM_RESID_OUTER) {
          // refinement decision (mirrors the host-driven mixed solve)
          const double rho = (S->bnorm2 > 0.0) ? sqrt(tot / S->bnorm2) : 0.0;
          S->rho = rho;
          S->total += S->k;
          S->outer += 1;
          if (rho <= S->tol_outer) {
            S->done = 1;
          } else if (S->status != 0 || S->total >= S->maxit_total || S->k == 0) {
            S->done = 1;
            if (S->status == 0) S->status = ST_ERR_NOT_CONVERGED;
          } else {
            const double t = 0.5 * S->tol_outer / rho;
            S->target = t > S->inner_floor ? t : S->inner_floor;
            S->maxit = S->maxit_total - S->total;
            S->k = 0;
            S->upd = 0;  // the grouped update of the new inner run starts from iteration 1
            S->finish = 0;
            S->active = 0;
            S->restart = 1;
          }
        }
      }
    }
  }
}

// ------------------------------------------------------------------ double-float stencil
// Mixed-precision MINRES: z_k is float32, the output Y T z_k is a double-float; the 1/beta_k
// of p = Y T z_k / beta_k is applied by the pass that reads it (SrcLanczos over double-floats).
// Every face term a_f (z_c - z_f) uses the exact float difference (TwoSum) and a TwoProd
// product with the double-float coefficient, and the terms are summed with the high parts
// added error-free, so the result carries ~46 significant bits with no float64 instruction per
// element (GB300 runs float64 at 1/64 of the float32 rate).  Same mirrored-plane walk as the
// float64 kernel; the dot <Y T z, z> is accumulated unscaled and scaled by 1/beta^2 at the end.
struct acc_df {
  float s, t;
  __device__ __forceinline__ void add(float p, float e) {
    float ss, err;
    two_sum(s, p, ss, err);
    s = ss;
    t += err + e;
  }
  __device__ __forceinline__ void add(df a) { add(a.hi, a.lo); }
  // add a float (no low-order part)
  __device__ __forceinline__ void add1(float p) {
    float ss, err;
    two_sum(s, p, ss, err);
    s = ss;
    t += err;
  }
  __device__ __forceinline__ void add_prod(df a, df b) {
    float p, e;
    two_prod(a.hi, b.hi, p, e);
    e = fmaf(a.hi, b.lo, fmaf(a.lo, b.hi, e));
    add(p, e);
  }
  __device__ __forceinline__ void add_prod(df a, float b) {
    float p, e;
    two_prod(a.hi, b, p, e);
    e = fmaf(a.lo, b, e);
    add(p, e);
  }
  __device__ __forceinline__ df get() const { return df_from_sum(s, t); }
};

__device__ __forceinline__ void face_term(acc_df &A, df c, float a, float b) {
  float dh, dl;
  two_sum(a, -b, dh, dl);
  float p, e;
  two_prod(c.hi, dh, p, e);
  e = fmaf(c.hi, dl, fmaf(c.lo, dh, e));
  A.add(p, e);
}

// D3: the 3D grid (7-point stencil; planes mx*my apart), at three resident blocks per SM so that
// its two extra planes stay in registers.  The 1D/2D instantiation carries no z terms.
// UNI: every face coefficient has the same value c (a constant coefficient on a grid with equal
// spacing along every axis, g.c_uniform): tau K z = c (f z_c - sum_f z_f) over the f faces of the
// node, so the face terms reduce to one exactly summed difference (TwoSum chain over floats) and
// one double-float product, in place of one product per face.
template <bool D3, bool UNI>
__global__ void __launch_bounds__(kNT, D3 ? 3 : 4) k_stencil_df(Geom g, const float *__restrict__ z,
                                                    df *__restrict__ out, State *S,
                                                    double *__restrict__ partials, int kc) {
  __shared__ double red[32];
  if (!S->active) return;
  const bool lead = blockIdx.x == 0 && blockIdx.y == 0 && blockIdx.z == 0 && flat_tid() == 0;
  if (S->finish) {
    if (lead) S->active = 0;
    return;
  }
  // first iteration after a device-side restart: the restart pass is complete
  if (lead && S->restart) S->restart = 0;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y * blockDim.y + threadIdx.y;  // row jz*my + jy
  const int mx = g.mx, my = g.my, dim = g.dim, n = g.n;
  const long long m = g.m, pl = (long long)mx * my;
  const bool valid = (i < mx) && (j < my * g.mz);
  const int half = (n + 1) >> 1;
  const int k0 = blockIdx.z * kc;
  const int k1 = min(half, k0 + kc);
  acc_df D{0.f, 0.f};
  if (valid) {
    const int jz = D3 ? j / my : 0, jy = j - jz * my;
    const long long p = (long long)j * mx + i;
    const df zero_f{0.f, 0.f};
    const Faces6<df> fc = UNI ? Faces6<df>{zero_f, zero_f, zero_f, zero_f, zero_f, zero_f}
                              : faces_df_at(g, i, jy, jz);
    const df cw = fc.w, ce = fc.e, cs = fc.s, cn = fc.n, cd = fc.d, cu = fc.u;
    const df th = g.th_d, omth = g.omth_d;
    const bool theta = (g.scheme == ST_THETA);
    auto center = [&](int k) -> float { return __ldg(z + (long long)k * m + p); };
    auto combine = [&](float c, float c1, float c2, df Kc, df K1) -> df {
      acc_df A{0.f, 0.f};
      if (theta) {
        // the exact difference c - c1 starts the sum
        two_sum(c, -c1, A.s, A.t);
        if (g.th_exact) {
          // theta and 1 - theta are 0, 1/2 or 1: the products are exact scalings (the same
          // values add_prod gives), and a zero weight adds nothing
          A.add(th.hi * Kc.hi, th.hi * Kc.lo);
          if (omth.hi != 0.f) A.add(omth.hi * K1.hi, omth.hi * K1.lo);
        } else {
          A.add_prod(th, Kc);
          A.add_prod(omth, K1);
        }
      } else {
        float pp, e;
        two_prod(1.5f, c, pp, e);
        A.add(pp, e);
        A.add1(-2.0f * c1);
        A.add1(0.5f * c2);
        A.add(Kc);
      }
      return A.get();
    };
    // The loads of iteration kA + 1 (stencil points of both walks) are issued before the
    // arithmetic of iteration kA, so their latency overlaps it.
    struct P5 {
      float c, w, e, s, n, d, u;
    };
    auto load5 = [&](int k) -> P5 {
      const float *b = z + (long long)k * m + p;
      P5 r;
      r.c = __ldg(b);
      r.w = i > 0 ? __ldg(b - 1) : 0.f;
      r.e = i < mx - 1 ? __ldg(b + 1) : 0.f;
      r.s = (dim >= 2 && jy > 0) ? __ldg(b - mx) : 0.f;
      r.n = (dim >= 2 && jy < my - 1) ? __ldg(b + mx) : 0.f;
      r.d = (D3 && jz > 0) ? __ldg(b - pl) : 0.f;
      r.u = (D3 && jz < g.mz - 1) ? __ldg(b + pl) : 0.f;
      return r;
    };
    // tau K at a plane: the face terms in a fixed order
    auto stiff5 = [&](const P5 &q, float c) -> df {
      if (UNI) {
        // c_uni (f z_c - z_w - z_e - ...): f z_c is exact (f = 2, 4, or 4 + 2 in 3D)
        acc_df A{(dim >= 2) ? 4.f * c : 2.f * c, 0.f};
        if (D3) A.add1(2.f * c);
        A.add1(-q.w);
        A.add1(-q.e);
        if (dim >= 2) {
          A.add1(-q.s);
          A.add1(-q.n);
        }
        if (D3) {
          A.add1(-q.d);
          A.add1(-q.u);
        }
        return df_mul(g.c_uni, A.get());
      }
      acc_df A{0.f, 0.f};
      face_term(A, cw, c, q.w);
      face_term(A, ce, c, q.e);
      if (dim >= 2) {
        face_term(A, cs, c, q.s);
        face_term(A, cn, c, q.n);
      }
      if (D3) {
        face_term(A, cd, c, q.d);
        face_term(A, cu, c, q.u);
      }
      return A.get();
    };
    auto stiff = [&](int k, float c) -> df { return stiff5(load5(k), c); };
    const df zero{0.f, 0.f};
    float a1 = 0.f, a2 = 0.f;
    df aK1 = zero;
    float b0 = 0.f, b1 = 0.f;
    df bK0 = zero;
    if (k0 > 0) {
      a1 = center(k0 - 1);
      if (theta) aK1 = stiff(k0 - 1, a1);
    }
    if (!theta && k0 > 1) a2 = center(k0 - 2);
    {
      const int kb = n - 1 - k0;
      b0 = center(kb);
      if (theta) bK0 = stiff(kb, b0);
      else if (kb > 0) b1 = center(kb - 1);
    }
    // planes read by iteration kA: A-walk plane kA; mirrored walk plane kB - 1 (theta) or kB
    // plus the centre of kB - 2 (BDF2)
    auto planes = [&](int kA, P5 &A, P5 &B, float &C) {
      const int kB = n - 1 - kA;
      A = load5(kA);
      B = P5{0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
      C = 0.f;
      if (kB != kA) {
        if (theta) {
          if (kB > 0) B = load5(kB - 1);
        } else {
          B = load5(kB);
          if (kB > 1) C = __ldg(z + (long long)(kB - 2) * m + p);
        }
      }
    };
    P5 pA{0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f}, pB = pA;
    float pC = 0.f;
    if (k0 < k1) planes(k0, pA, pB, pC);
    for (int kA = k0; kA < k1; ++kA) {
      P5 nA{0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f}, nB = nA;
      float nC = 0.f;
      if (kA + 1 < k1) planes(kA + 1, nA, nB, nC);
      const int kB = n - 1 - kA;
      const float cA = pA.c;
      const df KA = stiff5(pA, cA);
      const df yA = combine(cA, a1, a2, KA, aK1);
      if (theta) {
        aK1 = KA;
      } else {
        a2 = a1;
      }
      a1 = cA;
      const bool twin = (kB != kA);
      const float zB = twin ? b0 : cA;
      df yB = zero;
      if (twin) {
        if (theta) {
          float nb = 0.f;
          df nK = zero;
          if (kB > 0) {
            nb = pB.c;
            nK = stiff5(pB, nb);
          }
          yB = combine(b0, nb, 0.f, bK0, nK);
          b0 = nb;
          bK0 = nK;
        } else {
          const df KB = stiff5(pB, b0);
          const float nb2 = (kB > 1) ? pC : 0.f;
          yB = combine(b0, b1, nb2, KB, zero);
          b0 = b1;
          b1 = nb2;
        }
      }
      out[(long long)kB * m + p] = yA;
      D.add_prod(yA, zB);
      if (twin) {
        out[(long long)kA * m + p] = yB;
        D.add_prod(yB, cA);
      }
      pA = nA;
      pB = nB;
      pC = nC;
    }
  }
  const double acc = (double)D.s + (double)D.t;
  const int nb = gridDim.x * gridDim.y * gridDim.z;
  const int bid = blockIdx.x + gridDim.x * (blockIdx.y + gridDim.y * blockIdx.z);
  double tot;
  if (last_block_reduce<kNT>(acc, partials, &S->counter[CNT_STENCIL], nb, bid, red, &tot) &&
      flat_tid() == 0) {
    const double sd = S->inv_beta;
    const double alpha = tot * sd * sd;
    S->alpha = alpha;
    S->lz_a = alpha / S->beta;
    S->lz_b = (S->k > 0) ? S->beta / S->beta_prev : 0.0;
    refresh_df(S);
  }
}

// f_H (Sec. 1 for theta, Sec. 4 with the start-up history moved into blocks 1-2 for BDF2).
__global__ void k_rhs(Geom g, const double *__restrict__ f, const double *__restrict__ u0,
                      const double *__restrict__ uprev, const double *__restrict__ extra,
                      double *__restrict__ fH) {
  const long long N = g.N, m = g.m;
  const double tau = g.tau;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < N;
       e += (long long)gridDim.x * blockDim.x) {
    const long long k = e / m, p = e - k * m;
    double r;
    if (g.scheme == ST_THETA) {
      r = g.theta * tau * f[(k + 1) * m + p] + (1.0 - g.theta) * tau * f[k * m + p];
      if (k == 0) {
        const int i = (int)(p % g.mx), row = (int)(p / g.mx);
        const int jz = row / g.my, jy = row - jz * g.my;
        const double c = u0[p];
        const double Kc = tauK(u0, p, i, jy, jz, g, faces_at(g, i, jy, jz), c);
        r += c - (1.0 - g.theta) * Kc;
      }
    } else {
      r = tau * f[(k + 1) * m + p];
      if (k == 0) r += 2.0 * u0[p] - 0.5 * (uprev ? uprev[p] : u0[p]);
      if (k == 1) r -= 0.5 * u0[p];
    }
    if (extra) r += extra[e];
    fH[e] = r;
  }
}

// Adjoint of the right-hand-side assembly: given lam = dL/df_H, the gradients with respect to
// f (at t_0..t_n), u0 and (BDF2) u^(-1).
//   theta: f_H block k = theta tau f^(k) + (1-theta) tau f^(k-1), block 1 += (I - (1-theta) tau K) u0
//   BDF2:  f_H block k = tau f^(k), block 1 += 2 u0 - u^(-1)/2, block 2 += -u0/2
__global__ void k_grad_rhs(Geom g, const double *__restrict__ lam, double *__restrict__ gf,
                           double *__restrict__ gu0, double *__restrict__ gup) {
  const long long m = g.m, total = (long long)(g.n + 1) * m;
  const int n = g.n;
  const double tau = g.tau;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const long long k = e / m, p = e - k * m;  // f^(k), k = 0..n
    double r = 0.0;
    if (g.scheme == ST_THETA) {
      if (k >= 1) r += g.theta * tau * lam[(k - 1) * m + p];
      if (k <= n - 1) r += (1.0 - g.theta) * tau * lam[k * m + p];
    } else {
      if (k >= 1) r = tau * lam[(k - 1) * m + p];
    }
    gf[e] = r;
    if (k == 0) {
      const double l1 = lam[p];
      if (g.scheme == ST_THETA) {
        if (gu0) {
          const int i = (int)(p % g.mx), row = (int)(p / g.mx);
          const int jz = row / g.my, jy = row - jz * g.my;
          const double Kl = tauK(lam, p, i, jy, jz, g, faces_at(g, i, jy, jz), l1);
          gu0[p] = l1 - (1.0 - g.theta) * Kl;
        }
        if (gup) gup[p] = 0.0;
      } else {
        const double l2 = (n > 1) ? lam[m + p] : 0.0;
        if (gu0) gu0[p] = 2.0 * l1 - 0.5 * l2;
        if (gup) gup[p] = -0.5 * l1;
      }
    }
  }
}

// Face terms of dL/da: g_face = -(tau/h^2) sum_k (lam_p - lam_q)(w_p - w_q), with
// w_k = theta u_k + (1-theta) u_{k-1} (u_{-1} = u0) for theta and w_k = u_k for BDF2.
// Thread (j, i) of the (my+1) x (mx+1) face grid owns x-face (j, i) [between nodes (j,i-1) and
// (j,i)] when j < my and y-face (j, i) [between (j-1,i) and (j,i)] when i < mx.
// cx/cy already hold tau*a/h^2; a_face enters linearly, so tau/h^2 = c/a_face is recovered from
// the unit-coefficient spacing passed in sx, sy.
__global__ void k_grad_faces(Geom g, const double *__restrict__ lam, const double *__restrict__ u,
                             const double *__restrict__ u0, double sx, double sy,
                             double *__restrict__ gx, double *__restrict__ gy) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y * blockDim.y + threadIdx.y;
  const int mx = g.mx, my = g.my;
  if (i > mx || j > my) return;
  const long long m = g.m;
  const bool doX = (j < my);
  const bool doY = (g.dim == 2) && (i < mx);
  if (!doX && !doY) return;
  const double th = (g.scheme == ST_THETA) ? g.theta : 1.0;
  // node indices (or -1 for a boundary node)
  const long long pc = (i < mx && j < my) ? (long long)j * mx + i : -1;
  const long long pl = (i > 0 && j < my) ? (long long)j * mx + i - 1 : -1;
  const long long pd = (j > 0 && i < mx) ? (long long)(j - 1) * mx + i : -1;
  double ax = 0.0, ay = 0.0;
  double uc_prev = pc >= 0 ? u0[pc] : 0.0, ul_prev = pl >= 0 ? u0[pl] : 0.0,
         ud_prev = pd >= 0 ? u0[pd] : 0.0;
  for (int k = 0; k < g.n; ++k) {
    const double *L = lam + (long long)k * m;
    const double *U = u + (long long)k * m;
    const double uc = pc >= 0 ? U[pc] : 0.0;
    const double ul = pl >= 0 ? U[pl] : 0.0;
    const double ud = pd >= 0 ? U[pd] : 0.0;
    const double wc = th * uc + (1.0 - th) * uc_prev;
    const double wl = th * ul + (1.0 - th) * ul_prev;
    const double wd = th * ud + (1.0 - th) * ud_prev;
    const double lc = pc >= 0 ? L[pc] : 0.0;
    if (doX) {
      const double ll = pl >= 0 ? L[pl] : 0.0;
      ax += (lc - ll) * (wc - wl);
    }
    if (doY) {
      const double ld_ = pd >= 0 ? L[pd] : 0.0;
      ay += (lc - ld_) * (wc - wd);
    }
    uc_prev = uc;
    ul_prev = ul;
    ud_prev = ud;
  }
  if (doX) gx[(long long)j * (mx + 1) + i] = -sx * ax;
  if (doY) gy[(long long)j * mx + i] = -sy * ay;
}

// Nodal gradient: each face gradient is split half/half between its two nodes.
__global__ void k_grad_nodes(int dim, int mx, int my, const double *__restrict__ gx,
                             const double *__restrict__ gy, double *__restrict__ grad) {
  const int I = blockIdx.x * blockDim.x + threadIdx.x;  // 0..mx+1
  const int J = blockIdx.y * blockDim.y + threadIdx.y;  // 0..my+1 (0 in 1D)
  if (dim == 1) {
    if (I > mx + 1 || J > 0) return;
    double s = 0.0;
    if (I <= mx) s += 0.5 * gx[I];      // face I: between nodes I and I+1
    if (I >= 1) s += 0.5 * gx[I - 1];   // face I-1: between nodes I-1 and I
    grad[I] = s;
    return;
  }
  if (I > mx + 1 || J > my + 1) return;
  double s = 0.0;
  // x-faces lie on interior rows j = J-1; face (j, i) joins nodal columns i and i+1
  if (J >= 1 && J <= my) {
    const int j = J - 1;
    if (I <= mx) s += 0.5 * gx[(long long)j * (mx + 1) + I];
    if (I >= 1) s += 0.5 * gx[(long long)j * (mx + 1) + I - 1];
  }
  // y-faces lie on interior columns i = I-1; face (j, i) joins nodal rows j and j+1
  if (I >= 1 && I <= mx) {
    const int i = I - 1;
    if (J <= my) s += 0.5 * gy[(long long)J * mx + i];
    if (J >= 1) s += 0.5 * gy[(long long)(J - 1) * mx + i];
  }
  grad[(long long)J * (mx + 2) + I] = s;
}

}  // namespace

int stencil_blocks(const Geom &g) {
  Tile t = tile_for(g);
  return t.gx * t.gy * t.nchunk;
}

template <class Tz>
cudaError_t launch_stencil(const Geom &g, int mode, const Tz *z, double *out, const double *fH,
                           State *S, double *partials, int, cudaStream_t st) {
  Tile t = tile_for(g);
  dim3 block = (g.dim == 1) ? dim3(kBX1, 1) : dim3(kBX2, kBY2);
  dim3 grid(t.gx, t.gy, t.nchunk);
  prof_begin(mode == SM_RESID ? KC_RESID : KC_STENCIL, st);
  switch (mode) {
    case SM_MINRES:
      k_stencil<Tz, SM_MINRES><<<grid, block, 0, st>>>(g, z, out, fH, S, partials, t.kc);
      break;
    case SM_APPLY:
      k_stencil<Tz, SM_APPLY><<<grid, block, 0, st>>>(g, z, out, fH, S, partials, t.kc);
      break;
    case SM_RESID:
      k_stencil<Tz, SM_RESID><<<grid, block, 0, st>>>(g, z, out, fH, S, partials, t.kc);
      break;
    default:
      return cudaErrorInvalidValue;
  }
  prof_end(st);
  return cudaGetLastError();
}

cudaError_t launch_stencil_df(const Geom &g, const float *z, df *q, State *S, double *partials,
                              cudaStream_t st) {
  Tile t = tile_for(g);
  dim3 block = (g.dim == 1) ? dim3(kBX1, 1) : dim3(kBX2, kBY2);
  dim3 grid(t.gx, t.gy, t.nchunk);
  prof_begin(KC_STENCIL, st);
  if (g.dim == 3) {
    if (g.c_uniform)
      k_stencil_df<true, true><<<grid, block, 0, st>>>(g, z, q, S, partials, t.kc);
    else
      k_stencil_df<true, false><<<grid, block, 0, st>>>(g, z, q, S, partials, t.kc);
  } else {
    if (g.c_uniform)
      k_stencil_df<false, true><<<grid, block, 0, st>>>(g, z, q, S, partials, t.kc);
    else
      k_stencil_df<false, false><<<grid, block, 0, st>>>(g, z, q, S, partials, t.kc);
  }
  prof_end(st);
  return cudaGetLastError();
}

cudaError_t launch_resid_outer(const Geom &g, const double *x, df *r_out, const double *fH,
                               State *S, double *partials, cudaStream_t st) {
  Tile t = tile_for(g);
  dim3 block = (g.dim == 1) ? dim3(kBX1, 1) : dim3(kBX2, kBY2);
  dim3 grid(t.gx, t.gy, t.nchunk);
  prof_begin(KC_RESID, st);
  k_stencil<double, SM_RESID_OUTER, df><<<grid, block, 0, st>>>(g, x, r_out, fH, S, partials, t.kc);
  prof_end(st);
  return cudaGetLastError();
}

cudaError_t launch_resid_df(const Geom &g, const double *x, df *r_out, const double *fH, State *S,
                            double *partials, cudaStream_t st) {
  Tile t = tile_for(g);
  dim3 block = (g.dim == 1) ? dim3(kBX1, 1) : dim3(kBX2, kBY2);
  dim3 grid(t.gx, t.gy, t.nchunk);
  prof_begin(KC_RESID, st);
  k_stencil<double, SM_RESID, df><<<grid, block, 0, st>>>(g, x, r_out, fH, S, partials, t.kc);
  prof_end(st);
  return cudaGetLastError();
}

template cudaError_t launch_stencil<double>(const Geom &, int, const double *, double *,
                                            const double *, State *, double *, int, cudaStream_t);
template cudaError_t launch_stencil<float>(const Geom &, int, const float *, double *,
                                           const double *, State *, double *, int, cudaStream_t);

cudaError_t launch_rhs(const Geom &g, const double *f, const double *u0, const double *uprev,
                       const double *extra, double *fH, cudaStream_t st) {
  long long blocks = (g.N + 255) / 256;
  if (blocks > 152LL * 16) blocks = 152LL * 16;
  prof_begin(KC_AUX, st);
  k_rhs<<<(unsigned)blocks, 256, 0, st>>>(g, f, u0, uprev, extra, fH);
  prof_end(st);
  return cudaGetLastError();
}

cudaError_t launch_grad_rhs(const Geom &g, const double *lam, double *gf, double *gu0,
                            double *gup, cudaStream_t st) {
  long long blocks = ((long long)(g.n + 1) * g.m + 255) / 256;
  if (blocks > 152LL * 16) blocks = 152LL * 16;
  prof_begin(KC_AUX, st);
  k_grad_rhs<<<(unsigned)blocks, 256, 0, st>>>(g, lam, gf, gu0, gup);
  prof_end(st);
  return cudaGetLastError();
}

cudaError_t launch_grad_a(const Geom &g, const double *lam, const double *u, const double *u0,
                          double *gface_x, double *gface_y, double *grad, cudaStream_t st) {
  const double hx = 1.0 / (g.mx + 1), hy = 1.0 / (g.my + 1);
  const double sx = g.tau / (hx * hx), sy = g.tau / (hy * hy);
  dim3 b(32, 8);
  const int fy = (g.dim == 2) ? g.my + 1 : 1;
  dim3 gr((g.mx + 1 + 31) / 32, (fy + 7) / 8);
  prof_begin(KC_AUX, st);
  k_grad_faces<<<gr, b, 0, st>>>(g, lam, u, u0, sx, sy, gface_x, gface_y);
  prof_end(st);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const int ny = (g.dim == 2) ? g.my + 2 : 1;
  dim3 gn((g.mx + 2 + 31) / 32, (ny + 7) / 8);
  prof_begin(KC_AUX, st);
  k_grad_nodes<<<gn, b, 0, st>>>(g.dim, g.mx, g.my, gface_x, gface_y, grad);
  prof_end(st);
  return cudaGetLastError();
}

}  // namespace st
