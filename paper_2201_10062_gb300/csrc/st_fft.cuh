// Radix-8/4/2 Stockham FFT (self-sorting, forward e^{-2 pi i jk/L}) for a batch of complex
// sequences of length L = 2^p held in shared memory, used by the spatial DST kernels.
//
// Pass with radix R and span Ns (Ns = 1, R1, R1 R2, ...): work item j (0..L/R-1) loads the R
// values j + r L/R, multiplies value r by W_{Ns R}^{r (j mod Ns)}, takes an R-point DFT in
// registers and stores output q at (j div Ns) Ns R + (j mod Ns) + q Ns.  After the last pass
// the sequence is in natural order.  Shared-memory slots are padded (one slot every 2^PADSHIFT
// elements) so that the strided stores of the early passes hit at most two-way bank conflicts.
// tw[t] = W_L^t for t < L/2.
#pragma once

#include "st_dd.cuh"

namespace st {

template <class T>
struct cpx {
  T x, y;
};

template <class T>
__host__ __device__ __forceinline__ cpx<T> cadd(cpx<T> a, cpx<T> b) {
  return cpx<T>{a.x + b.x, a.y + b.y};
}
template <class T>
__host__ __device__ __forceinline__ cpx<T> csub(cpx<T> a, cpx<T> b) {
  return cpx<T>{a.x - b.x, a.y - b.y};
}
template <class T>
__host__ __device__ __forceinline__ cpx<T> cmulc(cpx<T> a, cpx<T> b) {
  return cpx<T>{a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x};
}
// a * (-i)
template <class T>
__host__ __device__ __forceinline__ cpx<T> mul_mi(cpx<T> a) {
  return cpx<T>{a.y, -a.x};
}

template <class T>
struct PadShift;
template <>
struct PadShift<float> {
  static constexpr int v = 4;  // 16 complex floats per 128-byte bank row
};
template <>
struct PadShift<double> {
  static constexpr int v = 3;  // 8 complex doubles per 128-byte bank row
};
template <>
struct PadShift<dd> {
  static constexpr int v = 3;  // 8 complex double-floats (16 bytes each) per 128-byte bank row
};

template <class T>
__host__ __device__ __forceinline__ int fft_pad(int e) {
  return e + (e >> PadShift<T>::v);
}

template <class T>
__host__ __device__ __forceinline__ int fft_padded_len(int L) {
  return L + (L >> PadShift<T>::v);
}

// Distance between consecutive sequences in shared memory: at least the padded length and one
// more than a multiple of a bank row, so that the same element of neighbouring sequences falls
// in different banks.
template <class T>
__host__ __device__ __forceinline__ int fft_seq_stride(int L) {
  const int row = 1 << PadShift<T>::v;
  const int p = fft_padded_len<T>(L);
  return ((p + row - 1) / row) * row + 1;
}

// In-register R-point DFT, natural order in and out.
template <class T, int R>
struct Dft;

template <class T>
struct Dft<T, 2> {
  __host__ __device__ __forceinline__ static void run(cpx<T> *v) {
    const cpx<T> a = v[0], b = v[1];
    v[0] = cadd(a, b);
    v[1] = csub(a, b);
  }
};

template <class T>
struct Dft<T, 4> {
  __host__ __device__ __forceinline__ static void run(cpx<T> *v) {
    const cpx<T> s0 = cadd(v[0], v[2]), d0 = csub(v[0], v[2]);
    const cpx<T> s1 = cadd(v[1], v[3]), d1 = mul_mi(csub(v[1], v[3]));
    v[0] = cadd(s0, s1);
    v[2] = csub(s0, s1);
    v[1] = cadd(d0, d1);
    v[3] = csub(d0, d1);
  }
};

template <class T>
struct Dft<T, 8> {
  __host__ __device__ __forceinline__ static void run(cpx<T> *v) {
    const T h = T(0.70710678118654752440084436210485);
    // split into even and odd samples: X_q = E_q + W8^q O_q, X_{q+4} = E_q - W8^q O_q
    cpx<T> e[4] = {v[0], v[2], v[4], v[6]};
    cpx<T> o[4] = {v[1], v[3], v[5], v[7]};
    Dft<T, 4>::run(e);
    Dft<T, 4>::run(o);
    // W8^1 = (1 - i)/sqrt2, W8^2 = -i, W8^3 = -(1 + i)/sqrt2
    const cpx<T> o1 = cpx<T>{h * (o[1].x + o[1].y), h * (o[1].y - o[1].x)};
    const cpx<T> o2 = mul_mi(o[2]);
    const cpx<T> o3 = cpx<T>{h * (o[3].y - o[3].x), -h * (o[3].x + o[3].y)};
    v[0] = cadd(e[0], o[0]);
    v[4] = csub(e[0], o[0]);
    v[1] = cadd(e[1], o1);
    v[5] = csub(e[1], o1);
    v[2] = cadd(e[2], o2);
    v[6] = csub(e[2], o2);
    v[3] = cadd(e[3], o3);
    v[7] = csub(e[3], o3);
  }
};

// In-place Stockham pass over `count` sequences `stride` slots apart, with the length L = 2^LOGL,
// the radix R and the span Ns = 2^LOGNS known at compile time: every thread first loads the R
// values of each of its 8/R work items (eight complex values per thread for every radix), the
// block synchronises, then every thread transforms and stores.  Requires count * L <= 8 *
// nthreads.  The padded slot of element x is x + (x >> s) (s = PadShift); for every access of
// a pass, pad(base + r * step) = pad(base) + r * step + ((r * step) >> s) holds (step = L/R for
// loads, Ns for stores, base < step or a multiple of step * R), so each access is a base
// register plus a compile-time offset.
template <class T, int R, int LOGL, int LOGNS>
__device__ __forceinline__ void stockham_pass_inplace(cpx<T> *buf, const cpx<T> *tw, int count,
                                                      int stride, int tid, int nthreads) {
  constexpr int LOGR = (R == 8) ? 3 : (R == 4) ? 2 : 1;
  constexpr int TASKS = 8 / R;
  constexpr int L = 1 << LOGL;
  constexpr int LR = L / R;
  constexpr int LOGLR = LOGL - LOGR;
  constexpr int NS = 1 << LOGNS;
  constexpr int TWSTEP = L >> (LOGNS + LOGR);
  constexpr int S = PadShift<T>::v;
  const int ntask = count * LR;
  cpx<T> v[TASKS][R];
#pragma unroll
  for (int u = 0; u < TASKS; ++u) {
    const int task = tid + u * nthreads;
    if (task < ntask) {
      const int pp = task >> LOGLR;
      const int j = task & (LR - 1);
      const cpx<T> *s = buf + pp * stride + (j + (j >> S));
#pragma unroll
      for (int r = 0; r < R; ++r) v[u][r] = s[r * LR + ((r * LR) >> S)];
    }
  }
  __syncthreads();
#pragma unroll
  for (int u = 0; u < TASKS; ++u) {
    const int task = tid + u * nthreads;
    if (task < ntask) {
      const int pp = task >> LOGLR;
      const int j = task & (LR - 1);
      const int k = j & (NS - 1);
      if (NS > 1) {
        const cpx<T> w1 = tw[k * TWSTEP];
        cpx<T> w = w1;
#pragma unroll
        for (int r = 1; r < R; ++r) {
          v[u][r] = cmulc(v[u][r], w);
          if (r + 1 < R) w = cmulc(w, w1);
        }
      }
      Dft<T, R>::run(v[u]);
      const int idxD = ((j >> LOGNS) << (LOGNS + LOGR)) + k;
      cpx<T> *d = buf + pp * stride + (idxD + (idxD >> S));
#pragma unroll
      for (int r = 0; r < R; ++r) d[r * NS + ((r * NS) >> S)] = v[u][r];
    }
  }
  __syncthreads();
}

}  // namespace st
