// st_residual_noalloc: the residual-mode space-time stencil (r = Y f_H - Y T u and its squared
// norm) for callers that must not allocate device memory.
//
// Some callers cannot call cudaMalloc/cudaFree at the point where they need a residual check:
// code recording a CUDA graph (allocation calls are not captured and would break the capture),
// latency-critical loops where cudaFree's implicit device synchronisation is unacceptable, and
// hosts that hand all device memory to their own arena up front.  The regular path keeps its
// per-block partial sums in workspace that st_setup allocates; this variant keeps them in a
// fixed file-scope __device__ array instead, and takes the diffusion coefficient as a device
// array, so nothing is allocated by the call (no handle either).
#include <mutex>

#include "st_internal.cuh"

namespace {

constexpr int kNT = 256;
constexpr int kMaxBlocks = 4096;  // capacity of the static scratch (partial sums per block)

// [0, kMaxBlocks): partial ||r||^2, [kMaxBlocks, 2 kMaxBlocks): partial ||f_H||^2,
// then one completion counter.  Every GPU that loads the library holds these 64 KB until exit.
static __device__ __align__(256) double g_scratch[2 * kMaxBlocks + 32];

constexpr int kMaxDevices = 64;
void *g_scratch_addr[kMaxDevices];  // resolved device address per device (null: not yet)
std::mutex g_scratch_mu;

// The array's name is a host-side stand-in in host code; the device address comes from the
// runtime, per device, with that device current.  Only a successful lookup is kept: a lookup
// that failed (for instance one made while a stream was being captured) is tried again by the
// next call.
cudaError_t scratch_for_current_device(double **out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lk(g_scratch_mu);
  if (!g_scratch_addr[dev]) {
    void *p = nullptr;
    e = cudaGetSymbolAddress(&p, g_scratch);
    if (e != cudaSuccess) {
      cudaGetLastError();  // the failed lookup must not surface in a later, unrelated check
      return e;
    }
    g_scratch_addr[dev] = p;
  }
  *out = static_cast<double *>(g_scratch_addr[dev]);
  return cudaSuccess;
}

// [a, a + n) and [b, b + n) share an element
bool overlaps(const double *a, const double *b, long long n) {
  const char *pa = reinterpret_cast<const char *>(a), *pb = reinterpret_cast<const char *>(b);
  const long long bytes = n * (long long)sizeof(double);
  return pa < pb + bytes && pb < pa + bytes;
}

__device__ __forceinline__ double anode(const double *a, int dim, int mx, int J, int I) {
  if (!a) return 1.0;
  return (dim == 1) ? a[I] : a[(long long)J * (mx + 2) + I];
}

// One thread per spatial node and chunk of time levels; face coefficients come straight from
// the nodal a (mean of the two nodes of a face), times tau/h^2.
__global__ void __launch_bounds__(kNT)
    k_residual_static(st::Geom g, const double *__restrict__ a, const double *__restrict__ fH,
                      const double *__restrict__ u, double *__restrict__ r, double *scratch,
                      double *__restrict__ sums, int kc) {
  __shared__ double red[32];
  __shared__ bool is_last;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y * blockDim.y + threadIdx.y;
  const int mx = g.mx, my = g.my, n = g.n, dim = g.dim;
  const long long m = g.m;
  const int k0 = blockIdx.z * kc, k1 = min(n, k0 + kc);
  double rr = 0.0, ff = 0.0;
  if (i < mx && j < my) {
    const double hx = 1.0 / (mx + 1), hy = (dim == 2) ? 1.0 / (my + 1) : 1.0;
    const double sx = g.tau / (hx * hx), sy = g.tau / (hy * hy);
    const int J = j + 1, I = i + 1;
    const double ac = anode(a, dim, mx, J, I);
    const double cw = sx * 0.5 * (anode(a, dim, mx, J, I - 1) + ac);
    const double ce = sx * 0.5 * (ac + anode(a, dim, mx, J, I + 1));
    double cs = 0.0, cn = 0.0;
    if (dim == 2) {
      cs = sy * 0.5 * (anode(a, dim, mx, J - 1, I) + ac);
      cn = sy * 0.5 * (ac + anode(a, dim, mx, J + 1, I));
    }
    const long long p = (long long)j * mx + i;
    auto tK = [&](int k) -> double {
      const double *b = u + (long long)k * m;
      const double c = b[p];
      double t = (cw + ce + cs + cn) * c;
      if (i > 0) t -= cw * b[p - 1];
      if (i < mx - 1) t -= ce * b[p + 1];
      if (dim == 2) {
        if (j > 0) t -= cs * b[p - mx];
        if (j < my - 1) t -= cn * b[p + mx];
      }
      return t;
    };
    for (int k = k0; k < k1; ++k) {
      const double c = u[(long long)k * m + p];
      double y;
      if (g.scheme == ST_THETA) {
        const double c1 = (k > 0) ? u[(long long)(k - 1) * m + p] : 0.0;
        const double K1 = (k > 0) ? tK(k - 1) : 0.0;
        y = (c - c1) + g.theta * tK(k) + (1.0 - g.theta) * K1;
      } else {
        const double c1 = (k > 0) ? u[(long long)(k - 1) * m + p] : 0.0;
        const double c2 = (k > 1) ? u[(long long)(k - 2) * m + p] : 0.0;
        y = 1.5 * c - 2.0 * c1 + 0.5 * c2 + tK(k);
      }
      const double fk = fH[(long long)k * m + p];
      const double res = fk - y;  // block n-1-k of Y f_H - Y T u
      if (r) r[(long long)(n - 1 - k) * m + p] = res;
      rr += res * res;
      ff += fk * fk;
    }
  }
  // deterministic two-level reduction through the static scratch
  const int tid = threadIdx.x + threadIdx.y * blockDim.x;
  const int nb = gridDim.x * gridDim.y * gridDim.z;
  const int bid = blockIdx.x + gridDim.x * (blockIdx.y + gridDim.y * blockIdx.z);
  double s1 = st::block_sum<kNT>(rr, red);
  double s2 = st::block_sum<kNT>(ff, red);
  unsigned int *counter = reinterpret_cast<unsigned int *>(scratch + 2 * kMaxBlocks);
  if (tid == 0) {
    scratch[bid] = s1;
    scratch[kMaxBlocks + bid] = s2;
    __threadfence();
    is_last = (atomicAdd(counter, 1u) == (unsigned int)(nb - 1));
  }
  __syncthreads();
  if (!is_last) return;
  __threadfence();
  double a1 = 0.0, a2 = 0.0;
  for (int b = tid; b < nb; b += kNT) {
    a1 += ((volatile double *)scratch)[b];
    a2 += ((volatile double *)scratch)[kMaxBlocks + b];
  }
  a1 = st::block_sum<kNT>(a1, red);
  a2 = st::block_sum<kNT>(a2, red);
  if (tid == 0) {
    sums[0] = a1;
    sums[1] = a2;
    *counter = 0u;
  }
}

bool pow2(int v) { return v > 0 && (v & (v - 1)) == 0; }

}  // namespace

extern "C" int st_residual_noalloc(const st_problem *prob, const double *a_nodal_dev,
                                   const double *fH_dev, const double *u_dev, double *r_dev,
                                   double *sums_dev) {
  if (!prob || !fH_dev || !u_dev || !sums_dev) return ST_ERR_ARG;
  if (prob->a_nodal != nullptr) return ST_ERR_ARG;  // the coefficient comes in a_nodal_dev
  if (prob->dim != 1 && prob->dim != 2) return ST_ERR_ARG;
  if (prob->mx < 3 || prob->mx > 1023 || !pow2(prob->mx + 1)) return ST_ERR_ARG;
  if (prob->dim == 1 && prob->my != 1) return ST_ERR_ARG;
  if (prob->dim == 2 && (prob->my < 3 || prob->my > 1023 || !pow2(prob->my + 1))) return ST_ERR_ARG;
  if (prob->n < 1 || prob->n > 1024 || !(prob->T > 0.0)) return ST_ERR_ARG;
  if (prob->scheme != ST_THETA && prob->scheme != ST_BDF2) return ST_ERR_ARG;
  if (prob->scheme == ST_THETA && !(prob->theta >= 0.0 && prob->theta <= 1.0)) return ST_ERR_ARG;
  st::Geom g{};
  g.dim = prob->dim;
  g.mx = prob->mx;
  g.my = (prob->dim == 1) ? 1 : prob->my;
  g.n = prob->n;
  g.m = (long long)g.mx * g.my;
  g.N = g.m * g.n;
  g.scheme = prob->scheme;
  g.tau = prob->T / prob->n;
  g.theta = (prob->scheme == ST_THETA) ? prob->theta : 1.0;
  // every block reads f_H and u across time levels while other blocks write r: an r that shares
  // memory with either input would be read after it has been overwritten
  if (r_dev && (overlaps(r_dev, fH_dev, g.N) || overlaps(r_dev, u_dev, g.N))) return ST_ERR_ARG;
  dim3 block = (g.dim == 1) ? dim3(256, 1) : dim3(32, 8);
  const int gx = (g.mx + (int)block.x - 1) / (int)block.x;
  const int gy = (g.my + (int)block.y - 1) / (int)block.y;
  const long long tiles = (long long)gx * gy;
  if (tiles > kMaxBlocks) return ST_ERR_ARG;  // beyond the static scratch's capacity
  long long nchunk = kMaxBlocks / tiles;
  if (nchunk > 1216 / tiles + 1) nchunk = 1216 / tiles + 1;
  if (nchunk > g.n) nchunk = g.n;
  if (nchunk < 1) nchunk = 1;
  const int kc = (int)((g.n + nchunk - 1) / nchunk);
  const int nz = (g.n + kc - 1) / kc;
  if (tiles * nz > kMaxBlocks) return ST_ERR_ARG;
  double *scratch = nullptr;
  cudaError_t e = scratch_for_current_device(&scratch);
  if (e != cudaSuccess) return ST_ERR_CUDA;
  cudaStream_t st = (cudaStream_t)prob->stream;
  // the completion counter must start at zero (a faulted earlier call could have left it set)
  e = cudaMemsetAsync(scratch + 2 * kMaxBlocks, 0, sizeof(double), st);
  if (e != cudaSuccess) return ST_ERR_CUDA;
  k_residual_static<<<dim3(gx, gy, nz), block, 0, st>>>(g, a_nodal_dev, fH_dev, u_dev, r_dev,
                                                        scratch, sums_dev, kc);
  e = cudaGetLastError();
  return e == cudaSuccess ? ST_OK : ST_ERR_CUDA;
}
