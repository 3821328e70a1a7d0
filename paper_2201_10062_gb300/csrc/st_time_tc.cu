// Time-axis DST-I -> spectral scaling -> DST-I on the 5th-generation tensor cores (tcgen05):
// float32-accurate for the mixed-precision preconditioner (Sec. 3.1.1, steps 1-3 along time),
// and, at the end of this file, float64-accurate with integer digits for the float64 path.
//
// The folded transform is two dense products per parity of the output index k:
//   odd  k = 2r+1:  Y_k = sum_{t=1..h} S_{k,t} (x_t + x_{n+1-t})
//   even k = 2r+2:  Y_k = sum_{t=1..h} S_{k,t} (x_t - x_{n+1-t}),     h = n/2,
// i.e. D_P[r][j] = sum_t A_P[r][t] B_P[t][j] with A_P (h x h) fixed and B_P the folded data of a
// tile of 32 spatial columns.  Both operands are split into two fp16 pieces (hi + lo, 22 bits);
// hi*hi + hi*lo + lo*hi accumulate in float32 in tensor memory.  Columns of B are scaled by a
// power of two so that fp16 keeps its range; S is scaled by 8.
//
// S (both parities, both pieces: 128 KB for n = 256) lives in tensor memory as the A operand of
// tcgen05.mma; one block per SM walks tiles of 32 columns: the time kernel (k_time_tc3) runs three
// independent 8-warp tile pipelines, the spatial one (k_dst_tc_yw: strided y and z lines, or
// contiguous x lines) splits build, MMA issue and epilogue over separate warps.
// One thread per pipeline issues tcgen05.mma (M = 128, N = 32, K = 16; B from a shared-memory
// descriptor, no swizzle, K-major core matrices of 8 rows x 16 bytes), tcgen05.commit signals the
// pipeline's mbarrier, and its warps read the accumulators with tcgen05.ld.  For 256 < n <= 512
// (k_time_tc_long) S is streamed from global memory through a shared-memory ring instead.  Every
// wait on an mbarrier is bounded; on timeout the block records ST_ERR_TIMEOUT in the MINRES
// state and stops.  Before it releases its tensor memory it gives every MMA batch whose commit
// it has not seen complete one more bounded wait: MMAs still in flight may be writing that
// memory.  If that wait runs out as well, the block keeps the memory (it is never handed to
// another block while an MMA may write it) and sets State::tmem_held, which closes the device to
// further calls on the host side.
#include <cuda_fp16.h>

#include <cmath>
#include <cstdlib>

#include "st_internal.cuh"
#include "st_symbol.cuh"

namespace st {
namespace {

constexpr int kNT = 512;         // 16 warps
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

__device__ __forceinline__ void mbar_arrive(uint32_t mbar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(mbar) : "memory");
}

// 16 columns of this warp's 32 lanes into registers; the values are valid only after
// tmem_wait_ld (several loads may be in flight)
__device__ __forceinline__ void tmem_ld16_async(uint32_t taddr, uint32_t (&r)[16]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,"
      "%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
}
__device__ __forceinline__ void tmem_wait_ld() {
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float *v) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,"
      "%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
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


// End of a tensor-core block: after a timeout (ok false), one more bounded wait on each commit
// barrier whose last wait ran out (pendN, waited with phase phN).  Tensor memory is released only
// when every MMA batch has completed and no other asynchronous copy is left in flight
// (copies_done, uniform); otherwise the block records that it keeps it.  The decision is uniform
// across the block (one __syncthreads_and); warp 0 releases COLS columns at tmem.
template <int COLS>
__device__ __forceinline__ void tc_release_cols(bool ok, bool pend1, uint32_t mbar1, uint32_t ph1,
                                                bool pend2, uint32_t mbar2, uint32_t ph2,
                                                uint32_t tmem, State *S, bool copies_done = true) {
  // every thread that saw a timeout waits (bounded) on the barriers that still owe a completion;
  // the results are combined over the whole block (ok may differ between the tile pipelines of
  // one block), so that every thread takes the same decision
  bool d = true;
  if (!ok) {
    d = copies_done;
    if (pend1) d = mbar_wait(mbar1, ph1) && d;
    if (pend2) d = mbar_wait(mbar2, ph2) && d;
  }
  const bool drained = __syncthreads_and(d ? 1 : 0) != 0;
  const bool failed = __syncthreads_or(ok ? 0 : 1) != 0;
  if (failed && threadIdx.x == 0) {
    S->status = ST_ERR_TIMEOUT;
    if (!drained) atomicExch(&S->tmem_held, 1);
  }
  fence_before();
  __syncthreads();
  if (drained && (threadIdx.x >> 5) == 0) {
    fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "n"(COLS)
                 : "memory");
  }
}

constexpr int kYS = kTN + 1;  // padded row of the parity-split Y tile (conflict-free row writes)

__device__ __forceinline__ void cp_async4(uint32_t saddr, const float *g) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(saddr), "l"(g) : "memory");
}
__device__ __forceinline__ void cp_async16(uint32_t saddr, const float *g) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(saddr), "l"(g) : "memory");
}
__device__ __forceinline__ void cp_async_commit() {
  asm volatile("cp.async.commit_group;" ::: "memory");
}
__device__ __forceinline__ void cp_async_wait_all() {
  asm volatile("cp.async.wait_group 0;" ::: "memory");
}
// all but the `N` most recent commit groups of this thread are complete
template <int N>
__device__ __forceinline__ void cp_async_wait_pending() {
  asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

// fp16 (hi, lo) pieces of two floats, packed as half2 words
__device__ __forceinline__ void split_h2(float a, float b, uint32_t &hi, uint32_t &lo) {
  const __half2 h = __floats2half2_rn(a, b);
  const float2 f = __half22float2(h);
  const __half2 l = __floats2half2_rn(a - f.x, b - f.y);
  hi = *reinterpret_cast<const uint32_t *>(&h);
  lo = *reinterpret_cast<const uint32_t *>(&l);
}

// Per-row (time frequency k) constants of 1/p(k, tau mu), hoisted out of the column loop.
struct SymRow {
  float a, b, c;
};

__device__ __forceinline__ SymRow sym_row(const Spec<float> &sp, int k) {
  SymRow r;
  const float hk = sp.hk[k - 1], ck = sp.ck[k - 1], sk = sp.sk[k - 1];
  if (sp.prec == ST_PREC_PTHETA) {
    r.a = sp.lh[k - 1];
    r.b = sp.lht[k - 1];
    r.c = 0.f;
  } else if (sp.scheme == ST_THETA) {
    r.a = hk;
    r.b = sp.theta + (1.0f - sp.theta) * ck;
    r.c = sk;
  } else {
    r.a = hk * hk;
    r.b = 1.0f;
    r.c = -sk * (1.0f + hk);
  }
  return r;
}

// 1/p: theta:  re = (1 - cos x) + tmu (th + (1-th) cos x), im = (-1 + (1-th) tmu) sin x;
// BDF2: re = (1 - cos x)^2 + tmu, im = -sin x (2 - cos x);  P_theta: 1/(lam_H + lam_Htheta tmu)
__device__ __forceinline__ float inv_sym(const Spec<float> &sp, const SymRow &r, float tmu) {
  if (sp.prec == ST_PREC_PTHETA) return 1.0f / (r.a + r.b * tmu);
  float re, im;
  if (sp.scheme == ST_THETA) {
    re = r.a + tmu * r.b;
    im = (-1.0f + (1.0f - sp.theta) * tmu) * r.c;
  } else {
    re = r.a + tmu;
    im = r.c;
  }
  return rsqrtf(re * re + im * im);
}

// ------------------------------------------------------------------ tile pipelines per block
// S (both parities, hi and lo) lives in tensor memory as the A operand of tcgen05.mma (256 of
// the 512 columns), which leaves shared memory for independent tile pipelines of 8 warps each.
// Each group has its own B operands, tiles, accumulators, mbarriers and named barrier, so one
// group's fold/split/scale phases run while the others wait on their barriers or their MMAs; the
// MMAs read only B from shared memory.  The time kernel runs three such groups per block; group
// g of block b takes the tiles 3 b + g, 3 b + g + 3 gridDim.x, ...
constexpr int kGT = 256;  // threads per group

__device__ __forceinline__ void mma_f16_ta(uint32_t dtmem, uint32_t atmem, uint64_t bd,
                                           uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], [%1], %2, %3, p;\n\t}\n" ::"r"(dtmem),
      "r"(atmem), "l"(bd), "r"(kIdesc), "r"(acc));
}

__device__ __forceinline__ void tmem_st8(uint32_t taddr, const uint32_t (&r)[8]) {
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8};" ::"r"(taddr),
      "r"(r[0]), "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]), "r"(r[7])
      : "memory");
}

// barrier of the `nthreads` threads of named barrier `id`
__device__ __forceinline__ void group_sync(int id, int nthreads) {
  asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(nthreads) : "memory");
}

// barrier that also returns whether v holds in every participating thread
__device__ __forceinline__ bool group_sync_and(bool v, int id, int nthreads) {
  uint32_t out;
  asm volatile(
      "{\n\t.reg .pred p, q;\n\t"
      "setp.ne.b32 q, %1, 0;\n\t"
      "bar.red.and.pred p, %2, %3, q;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(out)
      : "r"((uint32_t)v), "r"(id), "r"(nthreads)
      : "memory");
  return out != 0;
}


// Fold, scale and split of one tile for a group of 256 threads: thread (column c = gt % 32,
// t-blocks tb = gt / 32 and gt / 32 + 8 of 8 rows; h/8 <= 16 t-blocks).  A warp reads or writes
// whole rows of 32 columns, so the staged loads are coalesced and the 16-byte operand stores of
// a quarter-warp cover eight distinct rows.  The column maximum is reduced in one step: each warp
// leaves its 32 per-column partial maxima in `part` (8 x 32 floats), the group passes one
// barrier, and every thread combines the eight partials of its own column.
template <class Src>
__device__ __forceinline__ void load_b_g_src(int n, int gt, Src src, float (&a)[2][8],
                                             float (&b)[2][8]) {
  const int h = (n + 1) >> 1, hb = h >> 3;
  const int c = gt & (kTN - 1);
#pragma unroll
  for (int it = 0; it < 2; ++it) {
    const int tb = (gt >> 5) + 8 * it;
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const int t = tb * 8 + q;
      a[it][q] = (tb < hb) ? src(t, c) : 0.f;
      b[it][q] = (tb < hb && n - 1 - t != t) ? src(n - 1 - t, c) : 0.f;  // odd middle row once
    }
  }
}

// Fold (u = a + b, d = a - b), scale each column by a power of two so that its largest folded
// value lies in [2^13, 2^14), and write the fp16 (hi, lo) pieces of both parities in canonical
// layout at `bop`, with 1/(scale * 8) in `colinv` (written by warp 0; read after the caller's next
// barrier).  `part` is the group's 8 x 32 partial-maximum array; one group barrier inside.
__device__ __forceinline__ void build_b_g(unsigned char *bop, float *colinv, float *part, int n,
                                          const float (&a)[2][8], const float (&b)[2][8], int gt,
                                          int bar) {
  const int h = (n + 1) >> 1, hb = h >> 3;
  const int c = gt & (kTN - 1), w = gt >> 5;
  float u[2][8], d[2][8];
  float mx = 0.f;
#pragma unroll
  for (int it = 0; it < 2; ++it) {
    const int tb = w + 8 * it;
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      u[it][q] = a[it][q] + b[it][q];
      d[it][q] = a[it][q] - b[it][q];
      if (tb < hb) mx = fmaxf(mx, fmaxf(fabsf(u[it][q]), fabsf(d[it][q])));
    }
  }
  part[w * kTN + c] = mx;
  group_sync(bar, kGT);
#pragma unroll
  for (int k = 0; k < 8; ++k) mx = fmaxf(mx, part[k * kTN + c]);
  float sc = 1.0f;
  if (mx > 0.f && isfinite(mx)) {
    int e;
    frexpf(mx, &e);
    sc = ldexpf(1.0f, 14 - e);
  }
  if (w == 0) colinv[c] = 1.0f / (sc * kSScale);
  const uint32_t piece = (uint32_t)kTN * h * 2u;
#pragma unroll
  for (int it = 0; it < 2; ++it) {
    const int tb = w + 8 * it;
    if (tb < hb) {
      uint32_t uh[4], ul[4], dh[4], dl[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        split_h2(u[it][2 * q] * sc, u[it][2 * q + 1] * sc, uh[q], ul[q]);
        split_h2(d[it][2 * q] * sc, d[it][2 * q + 1] * sc, dh[q], dl[q]);
      }
      const uint32_t off = canon_off(c, tb * 8, h);
      *reinterpret_cast<uint4 *>(bop + 0 * piece + off) = make_uint4(uh[0], uh[1], uh[2], uh[3]);
      *reinterpret_cast<uint4 *>(bop + 1 * piece + off) = make_uint4(ul[0], ul[1], ul[2], ul[3]);
      *reinterpret_cast<uint4 *>(bop + 2 * piece + off) = make_uint4(dh[0], dh[1], dh[2], dh[3]);
      *reinterpret_cast<uint4 *>(bop + 3 * piece + off) = make_uint4(dl[0], dl[1], dl[2], dl[3]);
    }
  }
}

// 2 parities x (h/16) K steps x 3 piece products: A pieces from tensor memory (piece 2P + hi/lo at
// column a_base + 64 (2P + lo) + 8 ks), B from shared memory; commit to mbar.
__device__ __forceinline__ void issue_mmas_ta(uint32_t a_base, uint32_t bbase, int h,
                                              uint32_t dcol, uint32_t mbar) {
  const uint32_t bpiece = (uint32_t)kTN * h * 2u;
  for (int P = 0; P < 2; ++P) {
    const uint32_t d = dcol + (uint32_t)(P * kTN);
    const uint32_t a_hi = a_base + (uint32_t)(2 * P) * 64u, a_lo = a_hi + 64u;
    const uint32_t b_hi = bbase + (2 * P) * bpiece, b_lo = b_hi + bpiece;
    for (int ks = 0; ks < h / 16; ++ks) {
      const uint32_t koff = (uint32_t)ks * 256u;  // two core matrices along K in B
      const uint32_t acol = (uint32_t)ks * 8u;    // 16 fp16 values of A per lane
      mma_f16_ta(d, a_hi + acol, make_desc(b_hi + koff, h), ks > 0 ? 1u : 0u);
      mma_f16_ta(d, a_hi + acol, make_desc(b_lo + koff, h), 1u);
      mma_f16_ta(d, a_lo + acol, make_desc(b_hi + koff, h), 1u);
    }
  }
  mma_commit(mbar);
}

// ------------------------------------------------------------------ y-DST: warp-specialised
// One DST-I of length len along lines (y, z, or a single time transform) of 32-line tiles, with
// S_len (both parities, hi and lo) in tensor memory as the A operand and the phases of a tile in
// separate warps that work on different tiles at once, handing off through mbarriers (every wait
// bounded):
//   - eight build warps keep the loads of the next two tiles in flight (cp.async into a ring of
//     three staging buffers) while they fold, scale and split the current one into one of two B
//     buffers (with its column factors);
//   - one thread issues the tile's MMAs into one of two 64-column accumulators and frees the B
//     buffer when they complete;
//   - four epilogue warps (one per lane quadrant, both parities of a row) take the accumulator
//     out, unscale it into the Y tile and write the tile back row by row.
// A B buffer is free again once its MMAs are done and every epilogue warp has applied its column
// factors (1 + 4 arrivals), so the build may run a tile ahead of the epilogue.
constexpr int kEpiW = 4;                              // warps 0..3: epilogue
constexpr int kBldW = 8;                              // warps 4..11: build
constexpr int kNTW = (kEpiW + kBldW + 1) * 32;        // and warp 12: the MMA thread (416)
constexpr int kBarE = 1, kBarBl = 2;                  // named barriers of the two groups
constexpr int kYwStages = 3;                          // staging ring: the tile built + 2 loading

struct TcYwSmem {
  uint32_t bop, ytile, stage, colinv, colmax, mbar, tmem, total;
};

// x lines write a tile back element by element along each line, so consecutive threads read
// rows e/2 of alternating parity: the odd-parity rows are shifted by this many floats so that the
// two parities fall 16 banks apart (h is 16, 32, 64 or 128)
__host__ __device__ inline int yw_odd_off(int h) { return (16 - h) & 31; }

__host__ __device__ inline TcYwSmem tcyw_layout(int len) {
  const int h = (len + 1) / 2;
  TcYwSmem L{};
  uint32_t o = 0;
  L.bop = o;  // two B buffers, each [parity][piece][32][h] fp16
  o += 2u * 2u * 2u * kTN * h * 2u;
  L.ytile = o;  // (x lines: the odd-parity rows start 16 banks over, see yw_odd_off)
  o += 2u * h * kYS * 4u + 64u;
  L.stage = o;  // kYwStages staged input tiles, each [len][32] floats
  o += (uint32_t)kYwStages * len * kTN * 4u;
  L.colinv = o;  // per B buffer: 1/(scale 8) of each column
  o += 2u * kTN * 4u;
  L.colmax = o;  // 8 build warps x 32 per-column partial maxima
  o += 8u * kTN * 4u;
  L.mbar = o;  // bfull[2], bempty[2], afull[2], aempty[2], done
  o += 9u * 8u;
  L.tmem = o;
  o += 8u;
  L.total = o;
  return L;
}

// XL: the lines are contiguous x-lines instead (line R holds elements R len .. R len + len - 1;
// `nplanes` is then the number of lines and mx, m are unused).  A tile is 32 consecutive lines,
// one contiguous block of 32 len floats, staged with 16-byte copies when the block is whole and
// 16-byte aligned; its transformed lines are written back from the Y tile line by line.
template <bool XL>
__global__ void __launch_bounds__(kNTW, 1)
    k_dst_tc_yw(const float *data, float *out, int len, int mx, long long m, long long nplanes,
                const __half *sop_g, State *S, int gk) {
  if (gate_closed(S, gk)) return;
  extern __shared__ __align__(1024) unsigned char smem[];
  const int h = (len + 1) >> 1;
  const TcYwSmem L = tcyw_layout(len);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(smem + L.tmem);
  float *stage = reinterpret_cast<float *>(smem + L.stage);
  float *ytile = reinterpret_cast<float *>(smem + L.ytile);
  float *colinv = reinterpret_cast<float *>(smem + L.colinv);
  const uint32_t bbuf = 2u * 2u * kTN * h * 2u;  // one B buffer
  const uint32_t mb = smem_u32(smem + L.mbar);
  const uint32_t bfull = mb, bempty = mb + 16u, afull = mb + 32u, aempty = mb + 48u,
                 done = mb + 64u;
  const int tpp = XL ? 1 : (mx + kTN - 1) / kTN;  // tiles per plane
  const long long ntiles = XL ? (nplanes + kTN - 1) / kTN : nplanes * tpp;
  auto tile_at = [&](long long tile, long long &base, int &je) {
    if (XL) {
      const long long r0 = tile * kTN;
      base = r0 * len;
      je = (int)min((long long)kTN, nplanes - r0);
    } else {
      const long long t = tile / tpp;
      const int x0 = (int)(tile - t * tpp) * kTN;
      base = t * m + x0;
      je = min(kTN, mx - x0);
    }
  };
  if (tid == 0) {
    for (int i = 0; i < 9; ++i) {
      uint32_t cnt = 1u;
      if (i == 2 || i == 3) cnt = 1u + kEpiW;              // bempty: MMA commit + epilogue warps
      if (i == 6 || i == 7) cnt = (uint32_t)kEpiW;         // aempty: every epilogue warp
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(mb + 8u * i), "r"(cnt)
                   : "memory");
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 512;" ::"r"(
                     smem_u32(tmem_slot))
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  fence_before();
  __syncthreads();
  fence_after();
  if (tid == 0) {  // both B buffers and both accumulators start free
    for (int k = 0; k < 1 + kEpiW; ++k) {
      mbar_arrive(bempty);
      mbar_arrive(bempty + 8u);
    }
    for (int k = 0; k < kEpiW; ++k) {
      mbar_arrive(aempty);
      mbar_arrive(aempty + 8u);
    }
  }
  const uint32_t tmem = *tmem_slot;
  const uint32_t a_base = tmem;
  const uint32_t dcol = tmem + 256u;  // the two 64-column accumulators follow S
  // S_len (four fp16 pieces) into tensor memory: warp w writes lanes 32 (w % 4).., the pieces
  // split among the warps of that quadrant
  {
    const int q = warp & 3, nq = (kNTW / 32 - q + 3) / 4, r = q * 32 + lane;
    const uint32_t lanes = (uint32_t)(q * 32) << 16;
    for (int piece = warp >> 2; piece < 4; piece += nq) {
      const unsigned char *img = reinterpret_cast<const unsigned char *>(sop_g) +
                                 (size_t)piece * kM * h * 2u;
      for (int ks = 0; ks < h / 16; ++ks) {
        uint32_t w[8];
        const uint4 c0 = *reinterpret_cast<const uint4 *>(img + canon_off(r, ks * 16, h));
        const uint4 c1 = *reinterpret_cast<const uint4 *>(img + canon_off(r, ks * 16 + 8, h));
        w[0] = c0.x; w[1] = c0.y; w[2] = c0.z; w[3] = c0.w;
        w[4] = c1.x; w[5] = c1.y; w[6] = c1.z; w[7] = c1.w;
        tmem_st8(a_base + lanes + (uint32_t)piece * 64u + (uint32_t)ks * 8u, w);
      }
    }
    asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
  }
  fence_before();
  __syncthreads();
  fence_after();
  bool ok = true;
  // mbarrier phases, one bit per buffer (registers; an indexed array would live in local memory)
  uint32_t pbf = 0u, pbe = 0u, paf = 0u, pae = 0u;
  if (warp == kEpiW + kBldW) {
    // ------------------------------------------------------------------ MMA thread
    if (lane == 0) {
      int u = 0;
      for (long long tile = blockIdx.x; tile < ntiles; tile += gridDim.x, ++u) {
        const int b = u & 1;
        if (!mbar_wait(bfull + 8u * b, ((pbf >> b) & 1u)) || !mbar_wait(aempty + 8u * b, ((pae >> b) & 1u))) {
          ok = false;
          break;
        }
        pbf ^= 1u << b;
        pae ^= 1u << b;
        fence_after();
        issue_mmas_ta(a_base, smem_u32(smem + L.bop) + (uint32_t)b * bbuf, h,
                      dcol + 64u * (uint32_t)b, afull + 8u * b);
        mma_commit(bempty + 8u * b);
      }
      mma_commit(done);
    }
    __syncwarp();
  } else if (warp >= kEpiW) {
    // ------------------------------------------------------------------ build warps
    const int gt = tid - kEpiW * 32;  // 0..255
    // the loads of `tile` into staging buffer s; one commit group per call, empty past the end
    auto prefetch = [&](long long tile, int s) {
      if (tile < ntiles) {
        long long base;
        int je;
        tile_at(tile, base, je);
        float *sp = stage + (size_t)s * len * kTN;
        if (XL) {
          // the tile is one contiguous block of je lines; rows past je are never read
          const float *gp = data + base;
          const uint32_t sa0 = smem_u32(sp);
          const int total = je * len;
          if (je == kTN && (reinterpret_cast<uintptr_t>(gp) & 15u) == 0) {
            for (int i = gt; i < total / 4; i += kGT) cp_async16(sa0 + 16u * (uint32_t)i, gp + 4 * i);
          } else {
            for (int i = gt; i < total; i += kGT) cp_async4(sa0 + 4u * (uint32_t)i, gp + i);
          }
        } else {
          const int c = gt & (kTN - 1), e0 = gt >> 5;
          const float *gp = data + base + (long long)e0 * mx + c;
          const long long gstep = (long long)(kGT / kTN) * mx;
          uint32_t sa = smem_u32(sp) + 4u * (uint32_t)gt;
          for (int e = e0; e < len; e += kGT / kTN, gp += gstep, sa += 4u * kGT) {
            if (c < je)
              cp_async4(sa, gp);
            else
              sp[e * kTN + c] = 0.f;
          }
        }
      }
      cp_async_commit();
    };
    prefetch(blockIdx.x, 0);
    prefetch((long long)blockIdx.x + gridDim.x, 1);
    int u = 0, s = 0;
    for (long long tile = blockIdx.x; tile < ntiles; tile += gridDim.x, ++u) {
      const int b = u & 1;
      // buffer s + 2 (mod 3) held the tile built last trip, which every build thread has read
      // (the barriers of that trip): the tile two ahead goes there
      prefetch(tile + 2LL * gridDim.x, s == 0 ? 2 : s - 1);
      ok = group_sync_and(mbar_wait(bempty + 8u * b, ((pbe >> b) & 1u)), kBarBl, kBldW * 32);
      if (!ok) break;
      pbe ^= 1u << b;
      cp_async_wait_pending<2>();  // this tile's group is complete; the next two may load
      group_sync(kBarBl, kBldW * 32);  // the tile is staged
      {
        const float *sp = stage + (size_t)s * len * kTN;
        float a[2][8], bb[2][8];
        if (XL) {
          // line c of the tile at sp + c len (len odd: the lanes' rows fall in distinct banks)
          long long base;
          int je;
          tile_at(tile, base, je);
          load_b_g_src(len, gt,
                       [&](int t, int c) -> float { return c < je ? sp[c * len + t] : 0.f; }, a,
                       bb);
        } else {
          load_b_g_src(len, gt, [&](int t, int c) -> float { return sp[t * kTN + c]; }, a, bb);
        }
        build_b_g(smem + L.bop + (uint32_t)b * bbuf, colinv + b * kTN,
                  reinterpret_cast<float *>(smem + L.colmax), len, a, bb, gt, kBarBl);
      }
      s = (s == kYwStages - 1) ? 0 : s + 1;
      fence_async_smem();
      group_sync(kBarBl, kBldW * 32);  // the B buffer and its column factors are written
      if (gt == 0) mbar_arrive(bfull + 8u * b);
    }
    cp_async_wait_all();
  } else {
    // ------------------------------------------------------------------ epilogue warps
    const int q = warp, r = (q << 5) + lane;
    const uint32_t lanes = (uint32_t)(q * 32) << 16;
    const bool ok0 = r < h && 2 * r + 1 <= len, ok1 = r < h && 2 * r + 2 <= len;
    const int odd = XL ? yw_odd_off(h) : 0;  // shift of the odd-parity rows in the Y tile
    // x lines: thread tid writes elements tid and tid + 128 of every line (len <= 255); their
    // places in the parity-split Y tile
    const int xo0 = (tid >> 1) * kYS + (tid & 1) * (h * kYS + odd), xo1 = xo0 + 64 * kYS;
    const bool xw0 = tid < len, xw1 = tid + 128 < len;
    int u = 0;
    for (long long tile = blockIdx.x; tile < ntiles; tile += gridDim.x, ++u) {
      const int b = u & 1;
      long long base;
      int je;
      tile_at(tile, base, je);
      ok = __all_sync(0xffffffffu, mbar_wait(bfull + 8u * b, ((pbf >> b) & 1u)) ? 1 : 0) != 0;
      if (ok) {
        pbf ^= 1u << b;
        ok = __all_sync(0xffffffffu, mbar_wait(afull + 8u * b, ((paf >> b) & 1u)) ? 1 : 0) != 0;
      }
      uint32_t v0[2][16], v1[2][16];
      if (ok) {
        paf ^= 1u << b;
        fence_after();
        const uint32_t tl = dcol + 64u * (uint32_t)b + lanes;
        tmem_ld16_async(tl, v0[0]);
        tmem_ld16_async(tl + 16u, v0[1]);
        tmem_ld16_async(tl + 32u, v1[0]);
        tmem_ld16_async(tl + 48u, v1[1]);
        tmem_wait_ld();
        fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(aempty + 8u * b);  // the accumulator is free
      }
      ok = group_sync_and(ok, kBarE, kEpiW * 32);
      if (!ok) break;
      {
        // unscale by the column factors of B buffer b, read here from shared memory (the buffer
        // is released only after this loop)
        const float *ci = colinv + b * kTN;
        float *y0 = ytile + r * kYS, *y1 = ytile + (h + r) * kYS + odd;
#pragma unroll
        for (int c = 0; c < kTN; ++c) {
          const float f = ci[c];
          if (ok0) y0[c] = __uint_as_float(v0[c >> 4][c & 15]) * f;
          if (ok1) y1[c] = __uint_as_float(v1[c >> 4][c & 15]) * f;
        }
        __syncwarp();
        if (lane == 0) mbar_arrive(bempty + 8u * b);  // the column factors are read
      }
      group_sync(kBarE, kEpiW * 32);
      if (XL) {
        // line c of the tile: consecutive threads write consecutive elements
        float *op = out + base;
        const float *yc = ytile;
        for (int c = 0; c < je; ++c, op += len, ++yc) {
          if (xw0) op[tid] = yc[xo0];
          if (xw1) op[tid + 128] = yc[xo1];
        }
      } else {
        // column c of rows et / 32, + 4, ...: rows of one parity, 2 rows apart in the Y tile
        const int et = tid, c = et & (kTN - 1), e0 = et >> 5;
        if (c < je) {
          float *op = out + base + (long long)e0 * mx + c;
          const float *yp = ytile + ((e0 & 1) * h + (e0 >> 1)) * kYS + c;
          const long long ostep = (long long)(kEpiW * 32 / kTN) * mx;
          for (int e = e0; e < len; e += kEpiW * 32 / kTN, op += ostep,
                   yp += (kEpiW * 32 / kTN / 2) * kYS)
            *op = *yp;
        }
      }
      group_sync(kBarE, kEpiW * 32);  // the Y tile is free again
    }
  }
  fence_before();
  ok = __syncthreads_and(ok ? 1 : 0) != 0;
  fence_after();
  // after a timeout `done` tracks every MMA issued: tc_release_cols waits for it (bounded)
  tc_release_cols<512>(ok, true, done, 0u, false, 0u, 0u, tmem, S, true);
}

// ------------------------------------------------------------------ time kernel: three pipelines
// Time DST, 1/p scaling, <v, P^-1 v> and time DST of 32-column tiles.  Two pipelines (16 warps
// per SM, 4 per scheduler) cannot hide the latency of the ALU phases between the MMAs; three
// 8-warp pipelines (24 warps) with one B buffer and one 64-column accumulator each run both
// transforms of a tile in sequence while the other two pipelines fill the gaps (103 against
// 110 us per 255^2 x 256 launch); each pipeline stages its next tile with cp.async while the
// current one is transformed.  Registers are capped at 80 per thread (768 threads); tensor
// memory holds S in 256 columns and the three accumulators in 192.  The same organisation for
// the spatial kernel was slower (79 against 54 us): its transformed rows, written from the
// accumulator registers without a staged Y tile, left the stores uncoalesced.
constexpr int kGroups3 = 3;
constexpr int kNT3 = kGroups3 * kGT;  // 768 threads

struct Tc3Smem {
  uint32_t bop, ytile, stage, colinv1, colinv2, colmax, tmu, mbar, total;
};

// The B operand and the Y tile are never live together (the second build reads the whole Y tile
// into registers before its column-maximum barrier, and writes B after it), so they share one
// region; the room this frees holds the staged next tile.
__host__ __device__ inline Tc3Smem tc3_layout(int n) {
  const int h = n / 2;
  Tc3Smem L{};
  const uint32_t bbytes = 2u * 2u * kTN * h * 2u, ybytes = (uint32_t)n * kYS * 4u;
  uint32_t o = 0;
  L.bop = o;
  L.ytile = o;
  o += bbytes > ybytes ? bbytes : ybytes;
  o = (o + 15u) & ~15u;
  L.stage = o;  // the next tile, [t][32] floats, loaded with cp.async
  o += (uint32_t)n * kTN * 4u;
  L.colinv1 = o;
  o += kTN * 4u;
  L.colinv2 = o;
  o += kTN * 4u;
  L.colmax = o;
  o += 8u * kTN * 4u;
  L.tmu = o;
  o += kTN * 4u;
  L.mbar = o;
  o += 8;
  L.total = (o + 1023u) & ~1023u;
  return L;
}

__host__ __device__ inline uint32_t tc3_block_bytes(int n) { return kGroups3 * tc3_layout(n).total + 16u; }

// S pieces into tensor memory: 24 warps, warp w writes piece (w / 4) % 4 for quadrant w % 4 (the
// first 16 warps cover the four pieces once; the others skip)
__device__ __forceinline__ void load_a_tmem(const __half *sop_g, int h, uint32_t a_base, int warp,
                                            int lane) {
  if (warp >= 16) return;
  const int q = warp & 3, piece = warp >> 2;
  const int r = q * 32 + lane;
  const unsigned char *img = reinterpret_cast<const unsigned char *>(sop_g) +
                             (size_t)piece * kM * h * 2u;
  const uint32_t lanes = (uint32_t)(q * 32) << 16;
  for (int ks = 0; ks < h / 16; ++ks) {
    uint32_t w[8];
    const uint4 c0 = *reinterpret_cast<const uint4 *>(img + canon_off(r, ks * 16, h));
    const uint4 c1 = *reinterpret_cast<const uint4 *>(img + canon_off(r, ks * 16 + 8, h));
    w[0] = c0.x; w[1] = c0.y; w[2] = c0.z; w[3] = c0.w;
    w[4] = c1.x; w[5] = c1.y; w[6] = c1.z; w[7] = c1.w;
    tmem_st8(a_base + lanes + (uint32_t)piece * 64u + (uint32_t)ks * 8u, w);
  }
  asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
}

__global__ void __launch_bounds__(kNT3, 1)
    k_time_tc3(float *data, int n, long long m, int mx, Spec<float> sp, const __half *sop_g,
               State *S, int tmode, double *__restrict__ partials, int gk) {
  __shared__ double red[32];
  if (gate_closed(S, gk)) return;
  extern __shared__ __align__(1024) unsigned char smem[];
  const int h = n >> 1;
  const Tc3Smem L = tc3_layout(n);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int grp = warp >> 3, gt = tid & (kGT - 1), w8 = warp & 7;
  const int bar = 1 + grp;
  unsigned char *gs = smem + (uint32_t)grp * L.total;
  uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(smem + kGroups3 * L.total);
  float *colinv1 = reinterpret_cast<float *>(gs + L.colinv1);
  float *colinv2 = reinterpret_cast<float *>(gs + L.colinv2);
  float *part = reinterpret_cast<float *>(gs + L.colmax);
  float *ytile = reinterpret_cast<float *>(gs + L.ytile);
  float *tmus = reinterpret_cast<float *>(gs + L.tmu);
  const uint32_t mbar = smem_u32(gs + L.mbar);
  const long long ntiles = (m + kTN - 1) / kTN;
  if (gt == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(mbar) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 512;" ::"r"(
                     smem_u32(tmem_slot))
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tmem = *tmem_slot;
  const uint32_t a_base = tmem;
  const uint32_t dcol = tmem + 256u + (uint32_t)grp * 64u;
  load_a_tmem(sop_g, h, a_base, warp, lane);
  fence_before();
  __syncthreads();
  fence_after();
  uint32_t phase = 0;
  bool ok = true, outstanding = false;
  float esum = 0.f, ecomp = 0.f;
  float *stage = reinterpret_cast<float *>(gs + L.stage);
  // copy the tile's n rows x 32 columns into the stage (zeros beyond the last column)
  auto prefetch = [&](long long tile) {
    const long long tj0 = tile * kTN;
    const int tje = (int)min((long long)kTN, m - tj0);
    const int c = gt & (kTN - 1), t0 = gt >> 5;
    const float *gp = data + (long long)t0 * m + tj0 + c;
    const long long gstep = (long long)(kGT / kTN) * m;
    uint32_t sa = smem_u32(stage) + 4u * (uint32_t)gt;
    for (int t = t0; t < n; t += kGT / kTN, gp += gstep, sa += 4u * kGT) {
      if (c < tje)
        cp_async4(sa, gp);
      else
        stage[t * kTN + c] = 0.f;
    }
    cp_async_commit();
  };
  const int q = warp & 3, P = w8 >> 2;
  const int r = (q << 5) + lane;
  const uint32_t tl = dcol + ((uint32_t)(q * 32) << 16) + (uint32_t)(P * kTN);
  const SymRow sr = sym_row(sp, r < h ? (P == 0 ? 2 * r + 1 : 2 * r + 2) : 1);
  float *yrow = ytile + (P * h + r) * kYS;
  auto ycell = [&](int t, int c) -> float & { return ytile[((t & 1) * h + (t >> 1)) * kYS + c]; };
  // one transform: MMAs from the operand just built, then the bounded wait (uniform in the group)
  auto run_mmas = [&]() -> bool {
    fence_async_smem();
    group_sync(bar, kGT);
    fence_after();
    if (gt == 0) issue_mmas_ta(a_base, smem_u32(gs + L.bop), h, dcol, mbar);
    outstanding = true;
    const bool w = group_sync_and(mbar_wait(mbar, phase), bar, kGT);
    if (!w) return false;
    outstanding = false;
    phase ^= 1u;
    fence_after();
    return true;
  };
  const long long tstride = (long long)kGroups3 * gridDim.x;
  const long long tfirst = (long long)blockIdx.x * kGroups3 + grp;
  if (tfirst < ntiles) prefetch(tfirst);
  for (long long tile = tfirst; tile < ntiles; tile += tstride) {
    const long long j0 = tile * kTN;
    const int je = (int)min((long long)kTN, m - j0);
    if (gt < kTN) {
      float t = 0.f;
      if (gt < je) {
        const long long j = j0 + gt;
        const long long jy = j / mx, jx = j - jy * mx;
        t = sp.mux[jx] + sp.muy[jy];
      }
      tmus[gt] = t;
    }
    cp_async_wait_all();
    group_sync(bar, kGT);  // this tile is staged
    {
      float a[2][8], b[2][8];
      load_b_g_src(n, gt, [&](int t, int c) -> float { return stage[t * kTN + c]; }, a, b);
      build_b_g(gs + L.bop, colinv1, part, n, a, b, gt, bar);
    }
    // every thread has read the stage (the column-maximum barrier inside the build): load the
    // next tile while this one is transformed
    if (tile + tstride < ntiles) prefetch(tile + tstride);
    if (!(ok = run_mmas())) break;
    // first epilogue: unscale, spectral scaling, energy; scaled Y into the parity-split tile
    {
      float v[16];
#pragma unroll
      for (int half = 0; half < 2; ++half) {
        tmem_ld16(tl + 16u * half, v);
        if (r < h) {
          float rs = 0.f;
#pragma unroll
          for (int c = 0; c < 16; ++c) {
            const int cc = 16 * half + c;
            const float y = v[c] * colinv1[cc];
            const float yi = y * inv_sym(sp, sr, tmus[cc]);
            if (cc < je) rs = fmaf(y, yi, rs);
            yrow[cc] = yi;
          }
          const float term = rs - ecomp;
          const float t = esum + term;
          ecomp = (t - esum) - term;
          esum = t;
        }
      }
    }
    fence_before();
    group_sync(bar, kGT);
    fence_after();
    {
      float a[2][8], b[2][8];
      load_b_g_src(n, gt, [&](int t, int c) -> float { return ycell(t, c); }, a, b);
      build_b_g(gs + L.bop, colinv2, part, n, a, b, gt, bar);
    }
    if (!(ok = run_mmas())) break;
    {
      float v[16];
#pragma unroll
      for (int half = 0; half < 2; ++half) {
        tmem_ld16(tl + 16u * half, v);
        if (r < h) {
#pragma unroll
          for (int c = 0; c < 16; ++c) yrow[16 * half + c] = v[c] * colinv2[16 * half + c];
        }
      }
    }
    fence_before();
    group_sync(bar, kGT);
    fence_after();
    for (int idx = gt; idx < n * kTN; idx += kGT) {
      const int t = idx >> 5, c = idx & (kTN - 1);
      if (c < je) data[(long long)t * m + j0 + c] = ycell(t, c);
    }
    group_sync(bar, kGT);
  }
  cp_async_wait_all();
  tc_release_cols<512>(ok, outstanding, mbar, phase, false, 0u, 0u, tmem, S);
  if (tmode != TM_NONE) {
    const double e = (double)esum - (double)ecomp;
    double tot;
    if (last_block_reduce<kNT3>(e, partials, &S->counter[CNT_TIME], gridDim.x, blockIdx.x, red,
                                &tot) &&
        tid == 0) {
      if (tmode == TM_INIT || tmode == TM_RESTART)
        minres_init_scalars_dev(S, tot);
      else
        minres_givens_dev(S, tot);
    }
  }
}

// ------------------------------------------------------------------ long time axes (n > 256)
// For 256 < n <= 512 the S_n operand (both parities, two 128-row M tiles each, K padded to 256,
// hi and lo: 512 KB) does not fit in shared memory.  It is laid out in global memory as 16
// chunks of 32 KB, chunk q = (P*2 + mt)*4 + kc holding rows mt*128.. of parity P and K range
// kc*64.., each piece canonical K-major with K = 64, and one thread streams the chunks through a
// two-slot ring with cp.async.bulk (mbarrier transaction counts), one chunk ahead of the MMAs.
// The B operand holds both parities for K = 256 (zero beyond h); the four accumulators
// (parity x M tile, 32 columns each) take 128 tensor-memory columns.
constexpr int kKP2 = 256;                 // padded K of the long kernel
constexpr uint32_t kChunk2 = 32768u;      // bytes per streamed A chunk (2 pieces x 128 x 64 fp16)
constexpr uint32_t kPiece2 = kChunk2 / 2; // one piece of a chunk

struct Tc2Smem {
  uint32_t ring, bop, ytile, colscale, colinv1, colinv2, colmax, tmu, mbar, tmem, total;
};

__host__ __device__ inline Tc2Smem tc2_layout(int n) {
  const int h = n / 2;
  Tc2Smem L{};
  uint32_t o = 0;
  L.ring = o;
  o += 2u * kChunk2;
  L.bop = o;
  o += 2u * 2u * kTN * kKP2 * 2u;  // [parity][piece][32][256] fp16
  L.ytile = o;
  o += 2u * h * kYS * 4u;
  L.colscale = o;
  o += kTN * 4u;
  L.colinv1 = o;
  o += kTN * 4u;
  L.colinv2 = o;
  o += kTN * 4u;
  L.colmax = o;
  o += kTN * 4u;
  L.tmu = o;
  o += kTN * 4u;
  L.mbar = o;  // full[2], empty[2], done
  o += 5 * 8;
  L.tmem = o;
  o += 8;
  L.total = o;
  return L;
}

__device__ __forceinline__ void mbar_expect_tx(uint32_t mbar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(mbar), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void *src, uint32_t bytes,
                                         uint32_t mbar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::
          "r"(dst),
      "l"(src), "r"(bytes), "r"(mbar)
      : "memory");
}

// Fold, scale and split for K = 256 (h <= 256 folded rows): thread (column c, group g) handles
// the t-blocks g and g + 16 of 8 rows each.  Same arithmetic as build_b.
template <class Src>
__device__ __forceinline__ void build_b_long(unsigned char *smem, const Tc2Smem &L,
                                             uint32_t colinv_off, int n, Src src, int tid) {
  const int h = n >> 1, hb = h >> 3;
  unsigned int *colmax = reinterpret_cast<unsigned int *>(smem + L.colmax);
  float *colscale = reinterpret_cast<float *>(smem + L.colscale);
  float *colinv = reinterpret_cast<float *>(smem + colinv_off);
  const int c = tid & (kTN - 1), g = tid >> 5;
  if (tid < kTN) colmax[tid] = 0u;
  float u[2][8], d[2][8];
  float mx = 0.f;
#pragma unroll
  for (int it = 0; it < 2; ++it) {
    const int tb = g + 16 * it;
    if (tb < hb) {
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        const int t = tb * 8 + q;
        const float a = src(t, c), b = src(n - 1 - t, c);
        u[it][q] = a + b;
        d[it][q] = a - b;
        mx = fmaxf(mx, fmaxf(fabsf(u[it][q]), fabsf(d[it][q])));
      }
    }
  }
  __syncthreads();
  atomicMax(&colmax[c], __float_as_uint(mx));
  __syncthreads();
  if (tid < kTN) {
    const float m = __uint_as_float(colmax[tid]);
    float s = 1.0f;
    if (m > 0.f && isfinite(m)) {
      int e;
      frexpf(m, &e);
      s = ldexpf(1.0f, 14 - e);
    }
    colscale[tid] = s;
    colinv[tid] = 1.0f / (s * kSScale);
  }
  __syncthreads();
  const float s = colscale[c];
  unsigned char *bop = smem + L.bop;
  const uint32_t piece = (uint32_t)kTN * kKP2 * 2u;
#pragma unroll
  for (int it = 0; it < 2; ++it) {
    const int tb = g + 16 * it;
    if (tb < hb) {
      uint32_t uh[4], ul[4], dh[4], dl[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        split_h2(u[it][2 * q] * s, u[it][2 * q + 1] * s, uh[q], ul[q]);
        split_h2(d[it][2 * q] * s, d[it][2 * q + 1] * s, dh[q], dl[q]);
      }
      const uint32_t off = canon_off(c, tb * 8, kKP2);
      *reinterpret_cast<uint4 *>(bop + 0 * piece + off) = make_uint4(uh[0], uh[1], uh[2], uh[3]);
      *reinterpret_cast<uint4 *>(bop + 1 * piece + off) = make_uint4(ul[0], ul[1], ul[2], ul[3]);
      *reinterpret_cast<uint4 *>(bop + 2 * piece + off) = make_uint4(dh[0], dh[1], dh[2], dh[3]);
      *reinterpret_cast<uint4 *>(bop + 3 * piece + off) = make_uint4(dl[0], dl[1], dl[2], dl[3]);
    }
  }
}

// Issued by one thread: one transform (16 streamed A chunks x 4 K steps x 3 products into the
// four accumulators), then a commit to `done`, which tracks every MMA issued before it.  The ring
// phases persist across calls.  Returns false if a wait ran out (the caller records the
// timeout); *fills_drained is false if, after such a timeout, a bulk copy into the ring could
// still be in flight.
__device__ __forceinline__ bool stream_mmas(unsigned char *smem, const Tc2Smem &L,
                                            const unsigned char *A_g, uint32_t tmem,
                                            uint32_t *fph, uint32_t *eph, bool *fills_drained) {
  const uint32_t full0 = smem_u32(smem + L.mbar), empty0 = full0 + 16, done = full0 + 32;
  const uint32_t ring = smem_u32(smem + L.ring), bbase = smem_u32(smem + L.bop);
  const uint32_t bpiece = (uint32_t)kTN * kKP2 * 2u;
  auto fill = [&](int q, int slot) {
    mbar_expect_tx(full0 + 8u * slot, kChunk2);
    bulk_g2s(ring + (uint32_t)slot * kChunk2, A_g + (size_t)q * kChunk2, kChunk2,
             full0 + 8u * slot);
  };
  bool ok = true;
  int pending[2] = {0, 0};  // fills not yet waited for, per slot
  fill(0, 0);
  fill(1, 1);
  pending[0] = pending[1] = 1;
  for (int q = 0; q < 16; ++q) {
    const int slot = q & 1;
    if (!mbar_wait(full0 + 8u * slot, fph[slot])) {
      ok = false;
      break;
    }
    fph[slot] ^= 1u;
    --pending[slot];
    const int P = q >> 3, mt = (q >> 2) & 1, kc = q & 3;
    const uint32_t d = tmem + (uint32_t)((P * 2 + mt) * kTN);
    const uint32_t a_hi = ring + (uint32_t)slot * kChunk2, a_lo = a_hi + kPiece2;
    const uint32_t b_hi = bbase + (2 * P) * bpiece, b_lo = b_hi + bpiece;
#pragma unroll
    for (int ks = 0; ks < 4; ++ks) {
      const uint32_t aoff = (uint32_t)ks * 256u, boff = (uint32_t)(kc * 4 + ks) * 256u;
      mma_f16(d, make_desc(a_hi + aoff, 64), make_desc(b_hi + boff, kKP2),
              (kc > 0 || ks > 0) ? 1u : 0u);
      mma_f16(d, make_desc(a_hi + aoff, 64), make_desc(b_lo + boff, kKP2), 1u);
      mma_f16(d, make_desc(a_lo + aoff, 64), make_desc(b_hi + boff, kKP2), 1u);
    }
    mma_commit(empty0 + 8u * slot);
    // chunk q-1 (other slot) is read by MMAs issued before; once they are done, load chunk q+1
    if (q >= 1 && q + 1 < 16) {
      const int other = slot ^ 1;
      if (!mbar_wait(empty0 + 8u * other, eph[other])) {
        ok = false;
        break;
      }
      eph[other] ^= 1u;
      fill(q + 1, other);
      ++pending[other];
    }
  }
  if (ok) {
    // the commits of the last two chunks (slots 0 and 1) complete one more phase of each empty
    // barrier: consume them so that the phases stay in step for the next transform
    for (int sl = 0; sl < 2 && ok; ++sl) {
      if (!mbar_wait(empty0 + 8u * sl, eph[sl])) ok = false;
      eph[sl] ^= 1u;
    }
  } else {
    // after a timeout: wait (bounded) for copies still in flight before the block moves on
    for (int sl = 0; sl < 2; ++sl)
      if (pending[sl] > 0 && !mbar_wait(full0 + 8u * sl, fph[sl])) *fills_drained = false;
  }
  mma_commit(done);
  return ok;
}

__global__ void __launch_bounds__(kNT, 1)
    k_time_tc_long(float *data, int n, long long m, int mx, Spec<float> sp,
                   const unsigned char *A_g, State *S, int tmode, double *__restrict__ partials,
                   int gk) {
  __shared__ double red[32];
  if (gate_closed(S, gk)) return;
  extern __shared__ __align__(1024) unsigned char smem[];
  const int h = n >> 1;
  const Tc2Smem L = tc2_layout(n);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(smem + L.tmem);
  const float *colinv1 = reinterpret_cast<const float *>(smem + L.colinv1);
  const float *colinv2 = reinterpret_cast<const float *>(smem + L.colinv2);
  float *ytile = reinterpret_cast<float *>(smem + L.ytile);
  float *tmus = reinterpret_cast<float *>(smem + L.tmu);
  const uint32_t full0 = smem_u32(smem + L.mbar), done = full0 + 32;
  const long long ntiles = (m + kTN - 1) / kTN;
  {  // B rows t >= h stay zero for the whole launch
    uint4 *b = reinterpret_cast<uint4 *>(smem + L.bop);
    const int cnt = (int)((2u * 2u * kTN * kKP2 * 2u) / 16u);
    for (int i = tid; i < cnt; i += kNT) b[i] = make_uint4(0u, 0u, 0u, 0u);
  }
  if (tid == 0) {
    for (int i = 0; i < 5; ++i)
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(full0 + 8u * i) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 128;" ::"r"(
                     smem_u32(tmem_slot))
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tmem = *tmem_slot;
  uint32_t fph[2] = {0u, 0u}, eph[2] = {0u, 0u}, dph = 0u;  // phases (used by thread 0)
  bool ok = true;
  bool out_done = false;      // a commit to `done` whose completion has not been seen
  bool fills_drained = true;  // thread 0: no bulk copy into the ring left in flight
  float esum = 0.f, ecomp = 0.f;
  // accumulator view: TMEM lanes 32q.. (rows r = mt*128 + 32q + lane), parity P, columns 16ch..
  const int qq = warp & 3, P = (warp >> 2) & 1, ch = warp >> 3;
  const int c0 = ch * 16;
  const uint32_t lanes = (uint32_t)(qq * 32) << 16;
  SymRow sr[2];
#pragma unroll
  for (int mt = 0; mt < 2; ++mt) {
    const int r = mt * 128 + (qq << 5) + lane;
    sr[mt] = sym_row(sp, r < h ? (P == 0 ? 2 * r + 1 : 2 * r + 2) : 1);
  }
  auto ycell = [&](int t, int c) -> float { return ytile[((t & 1) * h + (t >> 1)) * kYS + c]; };
  auto run_mmas = [&]() {
    fence_async_smem();
    __syncthreads();
    fence_after();
    bool w = true;
    if (tid == 0) w = stream_mmas(smem, L, A_g, tmem, fph, eph, &fills_drained);
    const bool d = __syncthreads_and(mbar_wait(done, dph) ? 1 : 0) != 0;
    if (d) {
      dph ^= 1u;
    } else {
      out_done = true;
    }
    ok = (__syncthreads_and((w && d) ? 1 : 0) != 0) && ok;
    fence_after();
  };
  for (long long tile = blockIdx.x; tile < ntiles && ok; tile += gridDim.x) {
    const long long j0 = tile * kTN;
    const int je = (int)min((long long)kTN, m - j0);
    if (tid < kTN) {
      float t = 0.f;
      if (tid < je) {
        const long long j = j0 + tid;
        const long long jy = j / mx, jx = j - jy * mx;
        t = sp.mux[jx] + sp.muy[jy];
      }
      tmus[tid] = t;
    }
    build_b_long(smem, L, L.colinv1, n,
                 [&](int t, int c) -> float {
                   return (c < je) ? data[(long long)t * m + j0 + c] : 0.f;
                 },
                 tid);
    run_mmas();
    if (!ok) break;  // uniform
    // unscale, spectral scaling, energy; Y into the parity-split tile
#pragma unroll
    for (int mt = 0; mt < 2; ++mt) {
      float v[16];
      tmem_ld16(tmem + lanes + (uint32_t)((P * 2 + mt) * kTN + c0), v);
      const int r = mt * 128 + (qq << 5) + lane;
      if (r < h) {
        float *yrow = ytile + (P * h + r) * kYS;
        float rs = 0.f;
#pragma unroll
        for (int c = 0; c < 16; ++c) {
          const float y = v[c] * colinv1[c0 + c];
          const float yi = y * inv_sym(sp, sr[mt], tmus[c0 + c]);
          if (c0 + c < je) rs = fmaf(y, yi, rs);
          yrow[c0 + c] = yi;
        }
        const float term = rs - ecomp;
        const float t = esum + term;
        ecomp = (t - esum) - term;
        esum = t;
      }
    }
    fence_before();
    __syncthreads();
    fence_after();
    build_b_long(smem, L, L.colinv2, n, [&](int t, int c) -> float { return ycell(t, c); }, tid);
    run_mmas();
    if (!ok) break;  // uniform
#pragma unroll
    for (int mt = 0; mt < 2; ++mt) {
      float v[16];
      tmem_ld16(tmem + lanes + (uint32_t)((P * 2 + mt) * kTN + c0), v);
      const int r = mt * 128 + (qq << 5) + lane;
      if (r < h) {
        float *yrow = ytile + (P * h + r) * kYS;
#pragma unroll
        for (int c = 0; c < 16; ++c) yrow[c0 + c] = v[c] * colinv2[c0 + c];
      }
    }
    fence_before();
    __syncthreads();
    fence_after();
    for (int idx = tid; idx < n * kTN; idx += kNT) {
      const int t = idx >> 5, c = idx & (kTN - 1);
      if (c < je) data[(long long)t * m + j0 + c] = ycell(t, c);
    }
    __syncthreads();
  }
  // a bulk copy that may still land in the ring keeps the block from handing its resources back
  // as well: it counts as an outstanding completion
  const bool fills_ok = __syncthreads_and(fills_drained ? 1 : 0) != 0;
  tc_release_cols<128>(ok, out_done, done, dph, false, 0u, 0u, tmem, S, fills_ok);
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

// n a multiple of 32 up to 256, and the whole tile layout (plus 1 KB of static shared memory)
// within the 227 KB a block may opt into
bool time_tc_supported(int n) {
  return n >= 32 && n <= 256 && (n % 32) == 0 && tc3_block_bytes(n) + 1024u <= 227u * 1024u;
}

size_t time_tc_sop_halves(int n) { return (size_t)2 * 2 * kM * ((n + 1) / 2); }

// Host: canonical fp16 image of 8 S_len restricted to each parity of k (rows k = 2r+1 and 2r+2,
// k <= len; columns t = 1..h, h = (len+1)/2), hi and lo pieces.  Serves the time kernel
// (len = n, even) and the spatial kernel (len = my, odd).
void time_tc_build_sop(int len, unsigned short *out) {
  const int h = (len + 1) / 2;
  const double PI = 3.14159265358979323846;
  const double sn = std::sqrt(2.0 / (len + 1));
  const size_t piece = (size_t)kM * h;  // halves per piece
  for (size_t i = 0; i < 4 * piece; ++i) out[i] = 0;
  for (int P = 0; P < 2; ++P)
    for (int r = 0; r < h; ++r) {
      const int k = (P == 0) ? 2 * r + 1 : 2 * r + 2;
      if (k > len) continue;
      for (int t = 0; t < h; ++t) {
        const double v = kSScale * sn * std::sin(PI * (double)k * (t + 1) / (len + 1));
        const __half hi = __float2half_rn((float)v);
        const __half lo = __float2half_rn((float)(v - (double)__half2float(hi)));
        const uint32_t off = canon_off(r, t, h) / 2;  // in halves
        __half_raw rh = hi, rl = lo;
        out[(2 * P) * piece + off] = rh.x;
        out[(2 * P + 1) * piece + off] = rl.x;
      }
    }
}

// len + 1 in {32, 64, 128, 256} (h = 16..128 folded rows, a multiple of the MMA K step) and the
// layout within 227 KB with 1 KB of static shared memory
bool dst_tc_supported(int len) {
  const int L1 = len + 1;
  return (L1 == 32 || L1 == 64 || L1 == 128 || L1 == 256) &&
         tcyw_layout(len).total + 1024u <= 227u * 1024u;
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

// three tile pipelines per block, S_n in tensor memory
cudaError_t launch_time_tc(float *data, const Geom &g, const Spec<float> &sp,
                           const unsigned short *sop, State *S, int tmode, double *partials,
                           int gk, cudaStream_t st) {
  const uint32_t smem_bytes = tc3_block_bytes(g.n);
  cudaError_t e = cudaFuncSetAttribute(k_time_tc3, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem_bytes);
  if (e != cudaSuccess) return e;
  const long long ntiles = (g.m + kTN - 1) / kTN;
  const long long need = (ntiles + kGroups3 - 1) / kGroups3;
  int grid = time_tc_grid();
  if (need < grid) grid = (int)need;
  prof_begin(KC_TIME, st);
  k_time_tc3<<<grid, kNT3, smem_bytes, st>>>(data, g.n, g.m, g.mx, sp,
                                             reinterpret_cast<const __half *>(sop), S, tmode,
                                             partials, gk);
  prof_end(st);
  return cudaGetLastError();
}

// A multiple of 32 up to 256 (time axes: h = len/2 folded rows, a multiple of the K step) is
// also accepted by the single-transform kernel, with the same layout limit
bool dst_tc_len_supported(int len) {
  if (dst_tc_supported(len)) return true;
  return len >= 32 && len <= 256 && (len % 32) == 0 &&
         tcyw_layout(len).total + 1024u <= 227u * 1024u;
}

// One DST-I of length len along lines `stride` apart, nplanes planes `plane` apart, 32 adjacent
// lines per tile (k_dst_tc_yw, S_len in tensor memory), from `in` to `out` (the same array, or
// one that does not overlap).
cudaError_t launch_dst_tc_lines(const float *in, float *out, int len, int stride, long long plane,
                                long long nplanes, const unsigned short *sop, State *S, int gk,
                                int kc, cudaStream_t st) {
  const uint32_t smem_bytes = tcyw_layout(len).total;
  cudaError_t e = cudaFuncSetAttribute(k_dst_tc_yw<false>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_bytes);
  if (e != cudaSuccess) return e;
  const long long ntiles = nplanes * ((stride + kTN - 1) / kTN);
  int grid = time_tc_grid();
  if (ntiles < grid) grid = (int)ntiles;
  prof_begin(kc, st);
  k_dst_tc_yw<false><<<grid, kNTW, smem_bytes, st>>>(in, out, len, stride, plane, nplanes,
                                                     reinterpret_cast<const __half *>(sop), S, gk);
  prof_end(st);
  return cudaGetLastError();
}

// x lines (contiguous, n*my*mz of them), in place
cudaError_t launch_dst_tc_x(float *data, const Geom &g, const unsigned short *sop, State *S,
                            int gk, cudaStream_t st) {
  const uint32_t smem_bytes = tcyw_layout(g.mx).total;
  cudaError_t e = cudaFuncSetAttribute(k_dst_tc_yw<true>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_bytes);
  if (e != cudaSuccess) return e;
  const long long nlines = (long long)g.n * g.my * g.mz;
  const long long ntiles = (nlines + kTN - 1) / kTN;
  int grid = time_tc_grid();
  if (ntiles < grid) grid = (int)ntiles;
  prof_begin(KC_DSTX, st);
  k_dst_tc_yw<true><<<grid, kNTW, smem_bytes, st>>>(data, data, g.mx, 0, 0, nlines,
                                                    reinterpret_cast<const __half *>(sop), S, gk);
  prof_end(st);
  return cudaGetLastError();
}

// y lines: mx apart, in planes of mx*my (one per time level and z), in place
cudaError_t launch_dst_tc_y(float *data, const Geom &g, const unsigned short *sop, State *S,
                            int gk, cudaStream_t st) {
  return launch_dst_tc_lines(data, data, g.my, g.mx, (long long)g.mx * g.my,
                             (long long)g.n * g.mz, sop, S, gk, KC_DSTY, st);
}

// z lines (3D): mx*my apart, in planes of m (one per time level), in place
cudaError_t launch_dst_tc_z(float *data, const Geom &g, const unsigned short *sop, State *S,
                            int gk, cudaStream_t st) {
  return launch_dst_tc_lines(data, data, g.mz, g.mx * g.my, g.m, (long long)g.n, sop, S, gk,
                             KC_DSTY, st);
}

// The time DST alone (no scaling): lines of n values m apart, one plane of all m columns.
cudaError_t launch_time_tc_single(const float *in, float *out, const Geom &g,
                                  const unsigned short *sop, State *S, int gk, cudaStream_t st) {
  return launch_dst_tc_lines(in, out, g.n, (int)g.m, g.N, 1, sop, S, gk, KC_TIME, st);
}

// ------------------------------------------------------------------ long time axes: host side
bool time_tc_long_supported(int n) {
  return n > 256 && n <= 512 && (n % 32) == 0 && tc2_layout(n).total + 1024u <= 227u * 1024u;
}

size_t time_tc_long_bytes(int) { return (size_t)16 * kChunk2; }

// Host: the 16 streamed chunks of 8 S_n (rows of parity P, M tile mt, K range kc*64..), hi and
// lo pieces, each canonical K-major with K = 64.  Rows beyond h or with k > n, and columns
// t >= h, are zero.
void time_tc_long_build(int n, unsigned short *out) {
  const int h = n / 2;
  const double PI = 3.14159265358979323846;
  const double sn = std::sqrt(2.0 / (n + 1));
  const size_t halves = kChunk2 / 2, piece = kPiece2 / 2;
  for (size_t i = 0; i < 16 * halves; ++i) out[i] = 0;
  for (int P = 0; P < 2; ++P)
    for (int mt = 0; mt < 2; ++mt)
      for (int kc = 0; kc < 4; ++kc) {
        unsigned short *chunk = out + (size_t)((P * 2 + mt) * 4 + kc) * halves;
        for (int rr = 0; rr < kM; ++rr) {
          const int r = mt * kM + rr;
          const int k = (P == 0) ? 2 * r + 1 : 2 * r + 2;
          if (r >= h || k > n) continue;
          for (int kk = 0; kk < 64; ++kk) {
            const int t = kc * 64 + kk;
            if (t >= h) continue;
            const double v = kSScale * sn * std::sin(PI * (double)k * (t + 1) / (n + 1));
            const __half hi = __float2half_rn((float)v);
            const __half lo = __float2half_rn((float)(v - (double)__half2float(hi)));
            const uint32_t off = canon_off(rr, kk, 64) / 2;
            __half_raw rh = hi, rl = lo;
            chunk[off] = rh.x;
            chunk[piece + off] = rl.x;
          }
        }
      }
}

cudaError_t launch_time_tc_long(float *data, const Geom &g, const Spec<float> &sp,
                                const unsigned short *A, State *S, int tmode, double *partials,
                                int gk, cudaStream_t st) {
  const uint32_t smem_bytes = tc2_layout(g.n).total;
  cudaError_t e = cudaFuncSetAttribute(k_time_tc_long,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem_bytes);
  if (e != cudaSuccess) return e;
  const long long ntiles = (g.m + kTN - 1) / kTN;
  int grid = time_tc_grid();
  if (ntiles < grid) grid = (int)ntiles;
  prof_begin(KC_TIME, st);
  k_time_tc_long<<<grid, kNT, smem_bytes, st>>>(data, g.n, g.m, g.mx, sp,
                                                reinterpret_cast<const unsigned char *>(A), S,
                                                tmode, partials, gk);
  prof_end(st);
  return cudaGetLastError();
}

// ------------------------------------------------------------------ float64-accurate time DST
// The time stage of the float64 preconditioner (Sec. 3.1.1, steps 1-3 along time) on the tensor
// cores, for double-float data.  An fp16 MMA with float32 accumulation is exact on integers as
// long as every partial sum stays below 2^24, so both operands are cut into integer digits:
//   S^ = S 2^eS = sum_i S_i 2^-7i,   X^ = X 2^ec = sum_j B_j 2^-7j,   i, j = 0..6,
// with |S_i|, |B_j| <= 2^7 (one scale for S, one per column c of X and parity).  S's digits are
// rounded ones taken in float64 on the host; X's are the 7-bit fields of the folded double-float
// value as a 64-bit fixed-point integer (2^42 X^, rounded), the top one signed.  One product
// S_i B_j over K = h <= 128 folded rows is at most 2^21 in magnitude, and the at most seven
// products of a digit group g = i + j sum below 2^24, so each group accumulates exactly in
// float32.  The groups g <= 6 are kept (28 products per parity); the dropped ones and the
// digits' remainders are below 2^-41 of the column's largest entry.  The groups are summed in
// double-float (sum_g acc_g 2^-7g, TwoSum) and unscaled by 2^-(eS + ec).
//
// With S's digits read from shared memory each MMA (M = 128, N = 32) costs about ten times one
// that reads A from tensor memory, so the seven digits of one parity (448 tensor-memory columns)
// stay resident for a whole phase: a block takes its tiles of 32 spatial columns once for each
// parity.  Within a phase three roles work on different tiles at once, handing off through
// mbarriers (every wait bounded):
//   - eight build warps fold a tile's rows for the parity (x_t + x_{n+1-t}, or the difference),
//     choose each column's scale from its largest folded entry and write the seven digits as fp16
//     B operands (canonical K-major, [digit][32][h]) into one of two buffers;
//   - one thread issues the digit groups g = 0..6 of a tile in order, alternating between two
//     32-column accumulators, and frees the B buffer after the tile's last group;
//   - eight drain warps take each group out of tensor memory (tcgen05.ld; one row, 16 columns
//     per thread), add it into double-float sums, release the accumulator, and after group 6
//     unscale the tile's rows (and in the first launch multiply by 1/p and accumulate
//     <v, P^-1 v>), stage them in shared memory and write them out row by row.
// A row of output depends on every input row, so the transform cannot run in place: the first
// launch reads the data and writes the scaled transform into a scratch vector, the second
// transforms the scratch vector back into the data.
namespace {

constexpr int kDg = 7;                                   // digits per operand
constexpr int kDgW = 7;                                  // bits per digit
constexpr int kDrainW = 8;                               // warps 0..7: drain and epilogue
constexpr int kBuildW = 8;                               // warps 8..15: digits of the next tile
constexpr int kNTG = (kDrainW + kBuildW + 1) * 32;       // and warp 16: the MMA thread
constexpr int kBarD = 1, kBarB = 2;                      // named barriers of the two groups

struct TcdSmem {
  uint32_t bdig, ytile, part, cdown, tmu, mbar, tmem, total;
};

__host__ __device__ inline TcdSmem tcd_layout(int n) {
  const int h = n / 2;
  TcdSmem L{};
  uint32_t o = 0;
  L.bdig = o;  // two buffers of [digit][32][h] fp16
  o += 2u * kDg * kTN * (uint32_t)h * 2u;
  L.ytile = o;  // the drain warps' staged rows: hi floats then lo floats, [h][kYS]
  o += 2u * (uint32_t)h * kYS * 4u;
  L.part = o;  // 8 build warps x 32 per-column partial maxima
  o += (uint32_t)kBuildW * kTN * 4u;
  L.cdown = o;  // per buffer and column: 2^-(eS + e_c), the factor that undoes both scales
  o += 2u * kTN * 4u;
  L.tmu = o;  // per column: tau mu_j and the symbol's column factor w_j, double-float
  o += 2u * kTN * 8u;
  L.mbar = o;  // bfull[2], bempty[2], afull[2], aempty[2], done
  o += 9u * 8u;
  L.tmem = o;
  o += 8u;
  L.total = o;
  return L;
}

__device__ __forceinline__ dd ld_dd(const dd *p) {
  const float2 v = *reinterpret_cast<const float2 *>(p);
  return dd(v.x, v.y);
}
__device__ __forceinline__ void st_dd(dd *p, dd v) {
  *reinterpret_cast<float2 *>(p) = make_float2(v.hi, v.lo);
}

// 2^e as a float (exact; e outside the normal range through ldexpf)
__device__ __forceinline__ float pow2f(int e) {
  return (e >= -126 && e <= 127) ? __int_as_float((e + 127) << 23) : ldexpf(1.0f, e);
}

// 1/p in double-float with the per-row parts hoisted (the double-float form of inv_symbol):
// theta and BDF2 take 1/sqrt((a + tmu b)^2 + (w c)^2) with a, b, c per time frequency and
// w per column (w = -1 + (1 - theta) tmu for theta, 1 for BDF2); P_theta takes 1/(a + b tmu).
struct SymRowDD {
  dd a, b, c;
};
__device__ __forceinline__ SymRowDD sym_row_dd(const Spec<dd> &sp, int k) {
  SymRowDD r;
  const dd hk = sp.hk[k - 1], ck = sp.ck[k - 1], sk = sp.sk[k - 1];
  if (sp.prec == ST_PREC_PTHETA) {
    r.a = sp.lh[k - 1];
    r.b = sp.lht[k - 1];
    r.c = dd(0.f, 0.f);
  } else if (sp.scheme == ST_THETA) {
    r.a = hk;
    r.b = sp.theta + (dd(1) - sp.theta) * ck;
    r.c = sk;
  } else {
    r.a = hk * hk;
    r.b = dd(1);
    r.c = -(sk * (dd(1) + hk));
  }
  return r;
}
__device__ __forceinline__ dd sym_col_w(const Spec<dd> &sp, dd tmu) {
  if (sp.prec != ST_PREC_PTHETA && sp.scheme == ST_THETA)
    return dd(-1) + (dd(1) - sp.theta) * tmu;
  return dd(1);
}
__device__ __forceinline__ dd inv_sym_dd(const Spec<dd> &sp, const SymRowDD &r, dd tmu, dd w) {
  if (sp.prec == ST_PREC_PTHETA) return dd(1) / (r.a + r.b * tmu);
  const dd re = dd_fma(tmu, r.b, r.a), im = w * r.c;
  return rsqrt_dd(dd_fma(re, re, im * im));
}

// The seven 7-bit digits of x 2^e (|x 2^e| < 2^7, double-float): X = 2^42 x 2^e rounded to an
// integer, held as H 2^21 + Lo with 0 <= Lo < 2^21 (32-bit parts: no float64 conversion), is
// d_0 2^42 + sum_k d_k 2^(42-7k) with d_0 = H >> 21 (signed) and d_k the 7-bit fields below.
__device__ __forceinline__ void digits7(dd x, float up21, int (&d)[kDg]) {
  const float xh = x.hi * up21, xl = x.lo * up21;  // exact: powers of two
  int H = __float2int_rn(xh);                      // |H| <= 2^28; exact when |xh| >= 2^24
  const float r = xh - (float)H;                   // exact, |r| <= 1/2
  int Lo = __float2int_rn((r + xl) * 2097152.0f);  // (r + xl) 2^21; the rounding is below 1
  const int carry = Lo >> 21;                      // floor(Lo / 2^21)
  Lo -= carry * 2097152;
  H += carry;
  d[0] = H >> 21;
  d[1] = (H >> 14) & 127;
  d[2] = (H >> 7) & 127;
  d[3] = H & 127;
  d[4] = (Lo >> 14) & 127;
  d[5] = (Lo >> 7) & 127;
  d[6] = Lo & 127;
}

// scaled: out = (S_n x)/p per column with <in, P^-1 in> into the MINRES state (tmode);
// otherwise out = S_n x.  in and out do not overlap.
__global__ void __launch_bounds__(kNTG, 1)
    k_time_tcd(const dd *__restrict__ in, dd *__restrict__ out, int n, long long m, int mx,
               Spec<dd> sp, const unsigned char *A_g, int eS, int scaled, State *S, int tmode,
               double *__restrict__ partials, int gk) {
  __shared__ double red[32];
  if (gate_closed(S, gk)) return;
  extern __shared__ __align__(1024) unsigned char smem[];
  const int h = n >> 1, hb = h >> 3;
  const TcdSmem L = tcd_layout(n);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const uint32_t bop = (uint32_t)kTN * h * 2u;   // one digit's B operand
  const uint32_t bbytes = (uint32_t)kDg * bop;   // one B buffer
  uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(smem + L.tmem);
  float *yhi = reinterpret_cast<float *>(smem + L.ytile);
  float *ylo = yhi + (size_t)h * kYS;
  float *part = reinterpret_cast<float *>(smem + L.part);
  float *cdown = reinterpret_cast<float *>(smem + L.cdown);
  dd *tmus = reinterpret_cast<dd *>(smem + L.tmu);
  const uint32_t mb = smem_u32(smem + L.mbar);
  const uint32_t bfull = mb, bempty = mb + 16u, afull = mb + 32u, aempty = mb + 48u,
                 done = mb + 64u;
  const long long ntiles = (m + kTN - 1) / kTN;
  if (tid == 0) {
    for (int i = 0; i < 9; ++i) {
      const uint32_t cnt = (i == 6 || i == 7) ? (uint32_t)kDrainW : 1u;  // aempty: every drain warp
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(mb + 8u * i), "r"(cnt)
                   : "memory");
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 512;" ::"r"(
                     smem_u32(tmem_slot))
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  fence_before();
  __syncthreads();
  fence_after();
  if (tid == 0) {  // both B buffers and both accumulators start free
    mbar_arrive(bempty);
    mbar_arrive(bempty + 8u);
    for (int k = 0; k < kDrainW; ++k) {
      mbar_arrive(aempty);
      mbar_arrive(aempty + 8u);
    }
  }
  const uint32_t tmem = *tmem_slot;
  const uint32_t acol = (uint32_t)(h / 2);            // tensor-memory columns of one S digit
  const uint32_t dcol = tmem + (uint32_t)kDg * acol;  // the two accumulators follow S
  bool ok = true;
  // phases of bfull, bempty, afull and aempty as this thread's role waits on them
  // mbarrier phases, one bit per buffer (registers; an indexed array would live in local memory)
  uint32_t pbf = 0u, pbe = 0u, paf = 0u, pae = 0u;
  uint32_t G = 0;  // digit groups this thread's role has handled (accumulator G & 1)
  MacAcc<dd> en;   // drain threads: their part of <v, P^-1 v>
  en.zero();
  __syncthreads();

  for (int P = 0; P < 2 && ok; ++P) {
    // this parity's seven S digits into tensor memory: warp w writes lanes 32 (w % 4).., pieces
    // split among the warps of that quadrant
    {
      const int q = warp & 3, nq = (kNTG / 32 - q + 3) / 4, r = (q << 5) + lane;
      const uint32_t tl = (uint32_t)(q * 32) << 16;
      for (int pc = warp >> 2; pc < kDg; pc += nq) {
        const unsigned char *img = A_g + (size_t)(P * kDg + pc) * kM * h * 2u;
        for (int ks = 0; ks < h / 16; ++ks) {
          uint32_t w[8];
          const uint4 a0 = *reinterpret_cast<const uint4 *>(img + canon_off(r, ks * 16, h));
          const uint4 a1 = *reinterpret_cast<const uint4 *>(img + canon_off(r, ks * 16 + 8, h));
          w[0] = a0.x; w[1] = a0.y; w[2] = a0.z; w[3] = a0.w;
          w[4] = a1.x; w[5] = a1.y; w[6] = a1.z; w[7] = a1.w;
          tmem_st8(tmem + tl + (uint32_t)pc * acol + (uint32_t)ks * 8u, w);
        }
      }
      asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
    }
    fence_before();
    __syncthreads();
    fence_after();
    if (warp == kDrainW + kBuildW) {
      // ---------------------------------------------------------------- MMA thread
      if (lane == 0) {
        int u = 0;
        for (long long tile = blockIdx.x; tile < ntiles && ok; tile += gridDim.x, ++u) {
          const int b = u & 1;
          if (!mbar_wait(bfull + 8u * b, ((pbf >> b) & 1u))) {
            ok = false;
            break;
          }
          pbf ^= 1u << b;
          // descriptors differ only in their start-address field (address / 16), so each MMA
          // takes one add on a descriptor built once per tile
          const uint64_t bdesc = make_desc(smem_u32(smem + L.bdig) + (uint32_t)b * bbytes, h);
          const int ksteps = h / 16;
          for (int g = 0; g < kDg; ++g) {
            const int a = (int)(G & 1u);
            if (!mbar_wait(aempty + 8u * a, ((pae >> a) & 1u))) {
              ok = false;
              break;
            }
            pae ^= 1u << a;
            fence_after();
            const uint32_t d = dcol + (uint32_t)(kTN * a);
            uint32_t acc = 0u;
            for (int i = 0; i <= g; ++i) {
              const uint32_t at = tmem + (uint32_t)i * acol;
              const uint64_t bd = bdesc + (uint64_t)(((uint32_t)(g - i) * bop) >> 4);
#pragma unroll 8
              for (int ks = 0; ks < ksteps; ++ks) {
                mma_f16_ta(d, at + (uint32_t)ks * 8u, bd + (uint64_t)(16 * ks), acc);
                acc = 1u;
              }
            }
            mma_commit(afull + 8u * a);
            ++G;
          }
          if (!ok) break;
          mma_commit(bempty + 8u * b);  // the buffer is free once this tile's MMAs are done
        }
      }
      __syncwarp();
    } else if (warp >= kDrainW) {
      // ---------------------------------------------------------------- build warps
      const int bw = warp - kDrainW, bc = lane;
      int u = 0;
      for (long long tile = blockIdx.x; tile < ntiles; tile += gridDim.x, ++u) {
        const int b = u & 1;
        const long long j0 = tile * kTN;
        const int je = (int)min((long long)kTN, m - j0);
        ok = group_sync_and(mbar_wait(bempty + 8u * b, ((pbe >> b) & 1u)), kBarB, kBuildW * 32);
        if (!ok) break;
        pbe ^= 1u << b;
        dd f[2][8];
        float mxv = 0.f;
#pragma unroll
        for (int it = 0; it < 2; ++it) {
          const int tb = bw + kBuildW * it;
#pragma unroll
          for (int q = 0; q < 8; ++q) {
            f[it][q] = dd(0.f, 0.f);
            if (tb < hb && bc < je) {
              const int t = tb * 8 + q;
              const dd x1 = ld_dd(in + (long long)t * m + j0 + bc);
              const dd x2 = ld_dd(in + (long long)(n - 1 - t) * m + j0 + bc);
              f[it][q] = P == 0 ? x1 + x2 : x1 - x2;
              mxv = fmaxf(mxv, fabsf(f[it][q].hi));
            }
          }
        }
        part[bw * kTN + bc] = mxv;
        group_sync(kBarB, kBuildW * 32);
        float cm = 0.f;
#pragma unroll
        for (int k = 0; k < kBuildW; ++k) cm = fmaxf(cm, part[k * kTN + bc]);
        int e = 0;
        if (cm > 0.f && isfinite(cm)) {
          int E;
          frexpf(cm, &E);
          e = 7 - E;  // cm 2^e in [2^6, 2^7)
        }
        if (bw == 0) cdown[b * kTN + bc] = pow2f(-(eS + e));
        const float up21 = pow2f(e + 21);
        unsigned char *bb = smem + L.bdig + (uint32_t)b * bbytes;
#pragma unroll
        for (int it = 0; it < 2; ++it) {
          const int tb = bw + kBuildW * it;
          if (tb >= hb) continue;
          int dq[8][kDg];
#pragma unroll
          for (int q = 0; q < 8; ++q) digits7(f[it][q], up21, dq[q]);
          const uint32_t off = canon_off(bc, tb * 8, h);
#pragma unroll
          for (int dg = 0; dg < kDg; ++dg) {
            uint32_t pk[4];
#pragma unroll
            for (int q2 = 0; q2 < 4; ++q2) {
              const __half2 hv = __floats2half2_rn((float)dq[2 * q2][dg], (float)dq[2 * q2 + 1][dg]);
              pk[q2] = *reinterpret_cast<const uint32_t *>(&hv);
            }
            *reinterpret_cast<uint4 *>(bb + (uint32_t)dg * bop + off) =
                make_uint4(pk[0], pk[1], pk[2], pk[3]);
          }
        }
        fence_async_smem();
        group_sync(kBarB, kBuildW * 32);  // the buffer is written (and `part` read)
        if (bw == 0 && lane == 0) mbar_arrive(bfull + 8u * b);
      }
    } else {
      // ---------------------------------------------------------------- drain warps
      const int q4 = warp & 3, c0 = (warp >> 2) * 16;
      const int r = (q4 << 5) + lane;
      const int krow = (P == 0) ? 2 * r + 1 : 2 * r + 2;  // time frequency of row r (1-based)
      const bool row_ok = r < h && krow <= n;
      const SymRowDD srow = sym_row_dd(sp, row_ok ? krow : 1);
      const uint32_t lanes = (uint32_t)(q4 * 32) << 16;
      int u = 0;
      for (long long tile = blockIdx.x; tile < ntiles; tile += gridDim.x, ++u) {
        const int b = u & 1;
        const long long j0 = tile * kTN;
        const int je = (int)min((long long)kTN, m - j0);
        // each warp waits on its own (warp-uniform result); the drain group combines the results
        // once per tile, before its first named barrier, so that no warp leaves a barrier early
        if (ok) {
          ok = __all_sync(0xffffffffu, mbar_wait(bfull + 8u * b, ((pbf >> b) & 1u)) ? 1 : 0) != 0;
          if (ok) pbf ^= 1u << b;
        }
        float cd[16];
#pragma unroll
        for (int c = 0; c < 16; ++c) cd[c] = cdown[b * kTN + c0 + c];
        if (scaled && warp == 0) {
          dd tv(0.f, 0.f);
          if (lane < je) {
            const long long jj = j0 + lane;
            const long long jy = jj / mx, jx = jj - jy * mx;
            tv = sp.mux[jx] + sp.muy[jy];
          }
          tmus[lane] = tv;
          tmus[kTN + lane] = sym_col_w(sp, tv);
        }
        float s[16], t[16];
        for (int g = 0; g < kDg; ++g) {
          const int a = (int)(G & 1u);
          ++G;
          if (!ok) continue;
          ok = __all_sync(0xffffffffu, mbar_wait(afull + 8u * a, ((paf >> a) & 1u)) ? 1 : 0) != 0;
          if (!ok) continue;
          paf ^= 1u << a;
          fence_after();
          float v[16];
          tmem_ld16(dcol + lanes + (uint32_t)(kTN * a + c0), v);
          // the values are in registers: the accumulator is free for group g + 2
          fence_before();
          __syncwarp();
          if (lane == 0) mbar_arrive(aempty + 8u * a);
          const float sc = pow2f(-kDgW * g);
#pragma unroll
          for (int c = 0; c < 16; ++c) {
            const float x = v[c] * sc;
            if (g == 0) {
              s[c] = x;
              t[c] = 0.f;
            } else {
              float ss, er;
              two_sum(s[c], x, ss, er);
              s[c] = ss;
              t[c] += er;
            }
          }
        }
        ok = group_sync_and(ok, kBarD, kDrainW * 32);
        if (!ok) break;
        if (row_ok) {
#pragma unroll
          for (int c = 0; c < 16; ++c) {
            const int col = c0 + c;
            const dd v = dd_norm(s[c], t[c]);
            dd y(v.hi * cd[c], v.lo * cd[c]);
            if (scaled) {
              const dd yi = y * inv_sym_dd(sp, srow, tmus[col], tmus[kTN + col]);
              if (col < je) en.add(y, yi);
              y = yi;
            }
            yhi[r * kYS + col] = y.hi;
            ylo[r * kYS + col] = y.lo;
          }
        }
        group_sync(kBarD, kDrainW * 32);
        for (int idx = tid; idx < h * kTN; idx += kDrainW * 32) {
          const int rr = idx >> 5, c = idx & (kTN - 1);
          const int k = (P == 0) ? 2 * rr + 1 : 2 * rr + 2;
          if (c < je && k <= n)
            st_dd(out + (long long)(k - 1) * m + j0 + c, dd(yhi[rr * kYS + c], ylo[rr * kYS + c]));
        }
        group_sync(kBarD, kDrainW * 32);  // the staged rows and tmus are free again
      }
    }
    fence_before();
    ok = __syncthreads_and(ok ? 1 : 0) != 0;  // every role done: all MMAs of the phase drained
    fence_after();
  }
  if (warp == kDrainW + kBuildW && lane == 0) mma_commit(done);
  // after a timeout `done` tracks every MMA issued: tc_release_cols waits for it (bounded)
  tc_release_cols<512>(ok, true, done, 0u, false, 0u, 0u, tmem, S, true);
  if (scaled && tmode != TM_NONE) {
    const double e = (double)en.get();
    double tot;
    if (last_block_reduce<kNTG>(e, partials, &S->counter[CNT_TIME], gridDim.x, blockIdx.x, red,
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

// n a multiple of 32 up to 256 (h = n/2 folded rows, a multiple of the MMA K step; seven S
// digits of h/2 columns plus two 32-column accumulators within the 512 tensor-memory columns),
// and the layout within the 227 KB a block may opt into (with 1 KB of static shared memory)
bool time_tcd_supported(int n) {
  if (n < 32 || n > 256 || (n % 32) != 0) return false;
  if (kDg * (n / 4) + 2 * kTN > 512) return false;
  return tcd_layout(n).total + 1024u <= 227u * 1024u;
}

size_t time_tcd_bytes(int n) { return (size_t)2 * kDg * kM * (size_t)(n / 2) * 2; }

// Host: the digit image of S_n for k_time_tcd: piece (parity P, digit i) at index P * 7 + i, the
// rows r of parity P (k = 2r+1 or 2r+2) by K = h folded columns, canonical K-major fp16; the
// digits of S 2^eS (integers, |.| <= 2^7) are taken in float64, where they are exact.
// Returns eS.
int time_tcd_build(int n, unsigned char *out) {
  const int h = n / 2;
  const double PI = 3.14159265358979323846;
  const double sn = std::sqrt(2.0 / (n + 1));
  double smax = 0.0;
  for (int k = 1; k <= n; ++k)
    for (int t = 1; t <= h; ++t)
      smax = std::fmax(smax, std::fabs(sn * std::sin(PI * (double)k * t / (n + 1))));
  int E = 0;
  std::frexp(smax, &E);
  const int eS = 7 - E;  // smax 2^eS in [2^6, 2^7)
  unsigned short *o = reinterpret_cast<unsigned short *>(out);
  const size_t piece = (size_t)kM * h;  // halves
  for (size_t i = 0; i < time_tcd_bytes(n) / 2; ++i) o[i] = 0;
  for (int P = 0; P < 2; ++P)
    for (int r = 0; r < h; ++r) {
      const int k = (P == 0) ? 2 * r + 1 : 2 * r + 2;
      if (k > n) continue;
      for (int t = 0; t < h; ++t) {
        double v = std::ldexp(sn * std::sin(PI * (double)k * (t + 1) / (n + 1)), eS);
        for (int dg = 0; dg < kDg; ++dg) {
          const double q = std::nearbyint(v);
          v = (v - q) * 128.0;
          const __half hq = __float2half_rn((float)q);
          __half_raw raw = hq;
          o[(size_t)(P * kDg + dg) * piece + canon_off(r, t, h) / 2] = raw.x;
        }
      }
    }
  return eS;
}

// scaled: scratch = (S_n data)/p with <v, P^-1 v> and the MINRES step; then data = S_n scratch
cudaError_t launch_time_tcd(dd *data, dd *scratch, const Geom &g, const Spec<dd> &sp,
                            const unsigned char *img, int eS, State *S, int tmode,
                            double *partials, int gk, cudaStream_t st) {
  // at least 116 KB of shared memory, so that one block runs per SM: each allocates all 512
  // tensor-memory columns
  uint32_t smem_bytes = tcd_layout(g.n).total;
  if (smem_bytes < 116u * 1024u) smem_bytes = 116u * 1024u;
  cudaError_t e = cudaFuncSetAttribute(k_time_tcd, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem_bytes);
  if (e != cudaSuccess) return e;
  const long long ntiles = (g.m + kTN - 1) / kTN;
  int grid = time_tc_grid();
  if (ntiles < grid) grid = (int)ntiles;
  prof_begin(KC_TIME, st);
  k_time_tcd<<<grid, kNTG, smem_bytes, st>>>(data, scratch, g.n, g.m, g.mx, sp, img, eS, 1, S,
                                             tmode, partials, gk);
  k_time_tcd<<<grid, kNTG, smem_bytes, st>>>(scratch, data, g.n, g.m, g.mx, sp, img, eS, 0, S,
                                             TM_NONE, partials, gk);
  prof_end(st);
  return cudaGetLastError();
}

}  // namespace st
