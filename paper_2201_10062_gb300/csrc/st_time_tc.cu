// Time-axis DST-I -> spectral scaling -> DST-I on the 5th-generation tensor cores (tcgen05),
// float32-accurate, for the mixed-precision preconditioner (Sec. 3.1.1, steps 1-3 along time).
//
// The folded transform is two dense products per parity of the output index k:
//   odd  k = 2r+1:  Y_k = sum_{t=1..h} S_{k,t} (x_t + x_{n+1-t})
//   even k = 2r+2:  Y_k = sum_{t=1..h} S_{k,t} (x_t - x_{n+1-t}),     h = n/2,
// i.e. D_P[r][j] = sum_t A_P[r][t] B_P[t][j] with A_P (h x h) fixed and B_P the folded data of a
// tile of 32 spatial columns.  Both operands are split into two fp16 pieces (hi + lo, 22 bits);
// hi*hi + hi*lo + lo*hi accumulate in float32 in tensor memory.  Columns of B are scaled by a
// power of two so that fp16 keeps its range; S is scaled by 8.
//
// One persistent block per SM keeps A (both parities, both pieces, 128 KB for n = 256) in shared
// memory and walks the column tiles.  One thread issues tcgen05.mma (M = 128, N = 32, K = 16,
// A and B from shared-memory descriptors, no swizzle, K-major core matrices of 8 rows x 16
// bytes), tcgen05.commit signals an mbarrier, and all warps read the accumulators with
// tcgen05.ld.  Every wait on the mbarrier is bounded; on timeout the block records
// ST_ERR_TIMEOUT in the MINRES state and stops issuing work.
#include <cuda_fp16.h>

#include <cmath>

#include "st_internal.cuh"

namespace st {
namespace {

constexpr int kNT = 256;
constexpr int kTN = 32;          // spatial columns per tile (MMA N)
constexpr int kM = 128;          // MMA M (rows of S of one parity, zero padded)
constexpr float kSScale = 8.0f;  // S is stored times 8
constexpr long long kSpinLimit = 1LL << 20;  // bounded mbarrier wait

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

// byte offset of element (row, k) in a K-major, no-swizzle canonical operand with K columns
__host__ __device__ __forceinline__ uint32_t canon_off(int row, int k, int K) {
  return (uint32_t)((((row >> 3) * (K >> 3) + (k >> 3)) << 7) + ((row & 7) << 4) + ((k & 7) << 1));
}

// shared-memory matrix descriptor: start address, leading-dimension byte offset (between
// core matrices along K) = 128, stride byte offset (between 8-row groups) = 16 K bytes,
// descriptor version 1, no swizzle
__device__ __forceinline__ uint64_t make_desc(uint32_t saddr, int K) {
  const uint64_t lbo = 128, sbo = (uint64_t)K * 16;
  uint64_t d = 0;
  d |= (uint64_t)((saddr >> 4) & 0x3FFF);
  d |= (uint64_t)((lbo >> 4) & 0x3FFF) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFF) << 32;
  d |= (uint64_t)1 << 46;
  return d;
}

// instruction descriptor, kind::f16: D f32, A f16, B f16, both K-major, N = 32, M = 128
constexpr uint32_t kIdesc = (1u << 4) | ((uint32_t)(kTN >> 3) << 17) | ((uint32_t)(kM >> 4) << 24);

__device__ __forceinline__ void mma_f16(uint32_t dtmem, uint64_t ad, uint64_t bd, uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(dtmem),
      "l"(ad), "l"(bd), "r"(kIdesc), "r"(acc));
}

__device__ __forceinline__ void mma_commit(uint32_t mbar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                   mbar)
               : "memory");
}

__device__ __forceinline__ bool mbar_wait(uint32_t mbar, uint32_t phase) {
  for (long long it = 0; it < kSpinLimit; ++it) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(done)
        : "r"(mbar), "r"(phase)
        : "memory");
    if (done) return true;
  }
  return false;
}

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float *v) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,"
      "%15,%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]),
        "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]),
        "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ void fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void fence_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// split v into fp16 hi + lo
__device__ __forceinline__ void split_h(float v, __half &hi, __half &lo) {
  hi = __float2half_rn(v);
  lo = __float2half_rn(v - __half2float(hi));
}

// 1/p for time frequency k (1-based) and tau*mu (same closed forms as the float kernel)
__device__ __forceinline__ float inv_symbol_f(const Spec<float> &sp, int k, float tmu) {
  const float hk = sp.hk[k - 1], ck = sp.ck[k - 1], sk = sp.sk[k - 1];
  if (sp.prec == ST_PREC_PTHETA) return 1.0f / (sp.lh[k - 1] + sp.lht[k - 1] * tmu);
  float re, im;
  if (sp.scheme == ST_THETA) {
    re = hk + tmu * (sp.theta + (1.0f - sp.theta) * ck);
    im = (-1.0f + (1.0f - sp.theta) * tmu) * sk;
  } else {
    re = hk * hk + tmu;
    im = -sk * (1.0f + hk);
  }
  return rsqrtf(re * re + im * im);
}

struct TcSmem {
  // offsets in bytes from the dynamic shared-memory base
  uint32_t sop, bop, ytile, colscale, colmax, tmu, mbar, tmem;
  uint32_t total;
};

__host__ __device__ inline TcSmem tc_layout(int n) {
  const int h = n / 2;
  TcSmem L;
  uint32_t o = 0;
  L.sop = o;
  o += 2u * 2u * kM * h * 2u;  // [parity][piece][128][h] fp16
  L.bop = o;
  o += 2u * 2u * kTN * h * 2u;  // [parity][piece][32][h] fp16
  L.ytile = o;
  o += (uint32_t)n * kTN * 4u;  // float [n][32]
  L.colscale = o;
  o += kTN * 4u;
  L.colmax = o;
  o += kTN * 4u;
  L.tmu = o;
  o += kTN * 4u;
  L.mbar = o;
  o += 16;
  L.tmem = o;
  o += 16;
  L.total = o;
  return L;
}

// Fold rows t and n-1-t of a float tile column, scale by a power of two per column and write the
// fp16 pieces of both parities in canonical layout.  src(t, c) gives the value.
template <class Src>
__device__ __forceinline__ void build_b(unsigned char *smem, const TcSmem &L, int n, Src src,
                                        int tid) {
  const int h = n >> 1;
  unsigned int *colmax = reinterpret_cast<unsigned int *>(smem + L.colmax);
  float *colscale = reinterpret_cast<float *>(smem + L.colscale);
  const int c = tid & (kTN - 1), rg = tid >> 5;  // 8 row groups
  for (int i = tid; i < kTN; i += kNT) colmax[i] = 0u;
  __syncthreads();
  float mx = 0.f;
  for (int t = rg; t < h; t += kNT / kTN) {
    const float a = src(t, c), b = src(n - 1 - t, c);
    mx = fmaxf(mx, fmaxf(fabsf(a + b), fabsf(a - b)));
  }
  atomicMax(&colmax[c], __float_as_uint(mx));
  __syncthreads();
  if (tid < kTN) {
    const float m = __uint_as_float(colmax[tid]);
    float s = 1.0f;
    if (m > 0.f && isfinite(m)) {
      int e;
      frexpf(m, &e);           // m in [2^(e-1), 2^e)
      s = ldexpf(1.0f, 14 - e);  // scaled maximum below 2^14
    }
    colscale[tid] = s;
  }
  __syncthreads();
  const float s = colscale[c];
  unsigned char *bop = smem + L.bop;
  const uint32_t piece = (uint32_t)kTN * h * 2u;
  for (int t = rg; t < h; t += kNT / kTN) {
    const float a = src(t, c), b = src(n - 1 - t, c);
    __half uh, ul, dh, dl;
    split_h((a + b) * s, uh, ul);
    split_h((a - b) * s, dh, dl);
    const uint32_t off = canon_off(c, t, h);
    *reinterpret_cast<__half *>(bop + 0 * piece + off) = uh;  // parity 0 (odd k), hi
    *reinterpret_cast<__half *>(bop + 1 * piece + off) = ul;  // parity 0, lo
    *reinterpret_cast<__half *>(bop + 2 * piece + off) = dh;  // parity 1 (even k), hi
    *reinterpret_cast<__half *>(bop + 3 * piece + off) = dl;  // parity 1, lo
  }
}

// Issue the 2 parities x (h/16) K-steps x 3 piece products and commit to the mbarrier.
__device__ __forceinline__ void issue_mmas(unsigned char *smem, const TcSmem &L, int h,
                                           uint32_t tmem) {
  const uint32_t sbase = smem_u32(smem + L.sop), bbase = smem_u32(smem + L.bop);
  const uint32_t apiece = (uint32_t)kM * h * 2u, bpiece = (uint32_t)kTN * h * 2u;
  for (int P = 0; P < 2; ++P) {
    const uint32_t d = tmem + (uint32_t)(P * kTN);
    const uint32_t a_hi = sbase + (2 * P) * apiece, a_lo = a_hi + apiece;
    const uint32_t b_hi = bbase + (2 * P) * bpiece, b_lo = b_hi + bpiece;
    for (int ks = 0; ks < h / 16; ++ks) {
      const uint32_t koff = (uint32_t)ks * 256u;  // two core matrices along K
      mma_f16(d, make_desc(a_hi + koff, h), make_desc(b_hi + koff, h), ks > 0 ? 1u : 0u);
      mma_f16(d, make_desc(a_hi + koff, h), make_desc(b_lo + koff, h), 1u);
      mma_f16(d, make_desc(a_lo + koff, h), make_desc(b_hi + koff, h), 1u);
    }
  }
  mma_commit(smem_u32(smem + L.mbar));
}

__global__ void __launch_bounds__(kNT, 1)
    k_time_tc(float *data, int n, long long m, int mx, Spec<float> sp, const __half *sop_g,
              State *S, int tmode, double *__restrict__ partials, int gk) {
  __shared__ double red[32];
  if (gate_closed(S, gk)) return;
  extern __shared__ __align__(1024) unsigned char smem[];
  const int h = n >> 1;
  const TcSmem L = tc_layout(n);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  uint64_t *mbar = reinterpret_cast<uint64_t *>(smem + L.mbar);
  uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(smem + L.tmem);
  const float *colscale = reinterpret_cast<const float *>(smem + L.colscale);
  float *ytile = reinterpret_cast<float *>(smem + L.ytile);
  // A operands: straight copy of the precomputed canonical image
  {
    const uint4 *src = reinterpret_cast<const uint4 *>(sop_g);
    uint4 *dst = reinterpret_cast<uint4 *>(smem + L.sop);
    const int cnt = (int)((2u * 2u * kM * h * 2u) / 16u);
    for (int i = tid; i < cnt; i += kNT) dst[i] = src[i];
  }
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(mbar)) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 64;" ::"r"(
                     smem_u32(tmem_slot))
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tmem = *tmem_slot;
  uint32_t phase = 0;
  bool ok = true;
  float esum = 0.f, ecomp = 0.f;
  const long long ntiles = (m + kTN - 1) / kTN;
  const int P = warp >> 2;                      // parity block this warp reads
  const int r = ((warp & 3) << 5) + lane;       // accumulator row = TMEM lane
  const int krow = (P == 0) ? 2 * r + 1 : 2 * r + 2;  // 1-based time frequency of that row
  const uint32_t tl = tmem + ((uint32_t)((warp & 3) * 32) << 16) + (uint32_t)(P * kTN);
  for (long long tile = blockIdx.x; tile < ntiles && ok; tile += gridDim.x) {
    const long long j0 = tile * kTN;
    const int je = (int)min((long long)kTN, m - j0);
    float *tmus = reinterpret_cast<float *>(smem + L.tmu);
    if (tid < kTN) {
      float t = 0.f;
      if (tid < je) {
        const long long j = j0 + tid;
        const long long jy = j / mx, jx = j - jy * mx;
        t = sp.mux[jx] + sp.muy[jy];
      }
      tmus[tid] = t;
    }
    // ---- first transform: B from global data
    build_b(smem, L, n,
            [&](int t, int c) -> float {
              return (c < je) ? data[(long long)t * m + j0 + c] : 0.f;
            },
            tid);
    fence_async_smem();
    __syncthreads();
    fence_after();
    if (tid == 0) issue_mmas(smem, L, h, tmem);
    ok = __syncthreads_and(mbar_wait(smem_u32(mbar), phase) ? 1 : 0) != 0;
    phase ^= 1u;
    fence_after();
    float v[32];
    tmem_ld32(tl, v);
    // unscale, spectral scaling, energy; scaled Y into the float tile
    if (r < h) {
#pragma unroll
      for (int c = 0; c < kTN; ++c) {
        const float y = v[c] / (colscale[c] * kSScale);
        const float ip = inv_symbol_f(sp, krow, tmus[c]);
        if (c < je) {
          const float term = y * y * ip - ecomp;
          const float t = esum + term;
          ecomp = (t - esum) - term;
          esum = t;
        }
        ytile[(krow - 1) * kTN + c] = y * ip;
      }
    }
    fence_before();
    __syncthreads();
    fence_after();
    // ---- second transform: B from the scaled tile
    build_b(smem, L, n, [&](int t, int c) -> float { return ytile[t * kTN + c]; }, tid);
    fence_async_smem();
    __syncthreads();
    fence_after();
    if (tid == 0 && ok) issue_mmas(smem, L, h, tmem);
    ok = __syncthreads_and((ok && mbar_wait(smem_u32(mbar), phase)) ? 1 : 0) != 0;
    phase ^= 1u;
    fence_after();
    tmem_ld32(tl, v);
    if (r < h) {
      float *row = data + (long long)(krow - 1) * m + j0;
#pragma unroll
      for (int c = 0; c < kTN; ++c)
        if (c < je) row[c] = v[c] / (colscale[c] * kSScale);
    }
    fence_before();
    __syncthreads();
    fence_after();
  }
  if (!ok && tid == 0) S->status = ST_ERR_TIMEOUT;
  fence_before();
  __syncthreads();
  if (warp == 0) {
    fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 64;" ::"r"(tmem) : "memory");
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

}  // namespace

bool time_tc_supported(int n) { return n >= 32 && n <= 256 && (n % 32) == 0; }

size_t time_tc_sop_halves(int n) { return (size_t)2 * 2 * kM * (n / 2); }

// Host: canonical fp16 image of 8 S_P (hi, lo) for both parities.
void time_tc_build_sop(int n, unsigned short *out) {
  const int h = n / 2;
  const double PI = 3.14159265358979323846;
  const double sn = std::sqrt(2.0 / (n + 1));
  const size_t piece = (size_t)kM * h;  // halves per piece
  for (size_t i = 0; i < 4 * piece; ++i) out[i] = 0;
  for (int P = 0; P < 2; ++P)
    for (int r = 0; r < h; ++r) {
      const int k = (P == 0) ? 2 * r + 1 : 2 * r + 2;
      for (int t = 0; t < h; ++t) {
        const double v = kSScale * sn * std::sin(PI * (double)k * (t + 1) / (n + 1));
        const __half hi = __float2half_rn((float)v);
        const __half lo = __float2half_rn((float)(v - (double)__half2float(hi)));
        const uint32_t off = canon_off(r, t, h) / 2;  // in halves
        __half_raw rh = hi, rl = lo;
        out[(2 * P) * piece + off] = rh.x;
        out[(2 * P + 1) * piece + off] = rl.x;
      }
    }
}

int time_tc_grid() {
  static int sms = 0;
  if (!sms) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (sms <= 0) sms = 152;
  }
  return sms;
}

cudaError_t launch_time_tc(float *data, const Geom &g, const Spec<float> &sp,
                           const unsigned short *sop, State *S, int tmode, double *partials,
                           int gk, cudaStream_t st) {
  const TcSmem L = tc_layout(g.n);
  cudaError_t e = cudaFuncSetAttribute(k_time_tc, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)L.total);
  if (e != cudaSuccess) return e;
  const long long ntiles = (g.m + kTN - 1) / kTN;
  int grid = time_tc_grid();
  if (ntiles < grid) grid = (int)ntiles;
  prof_begin(KC_TIME, st);
  k_time_tc<<<grid, kNT, L.total, st>>>(data, g.n, g.m, g.mx, sp,
                                        reinterpret_cast<const __half *>(sop), S, tmode, partials,
                                        gk);
  prof_end(st);
  return cudaGetLastError();
}

}  // namespace st
