// Batched mixed-precision solves: many independent instances of uneven size (mx, my, n, theta,
// a(x)) run concurrently in one CUDA graph, launched once per solve.
//
// The graph holds one conditional WHILE node per instance; the nodes have no dependencies, so the
// instances run side by side.  The body of instance i is four MINRES iterations (z in a ring of
// four vectors, with a grouped direction/solution update after the second and the fourth)
// followed by a refinement block: convert the double-float x to float64, recompute the float64
// residual, and let the residual kernel's last block decide (done, or restart the inner run with
// the residual as right-hand side).  A restart zeroes the direction buffers and re-initialises
// the inner run through a preconditioner pass gated on the state's `restart` flag, so the next
// trip starts again at the ring's first slot.  The body ends with a one-thread
// kernel that sets the loop's condition from the device state: the loop of an instance ends as
// soon as it is done, so a finished instance launches nothing more, and no host decision sits
// anywhere inside the solve.  Each loop also stops after a fixed number of trips (maxit + 64),
// whatever the state says, and the instance then reports ST_ERR_NOT_CONVERGED.
#include <algorithm>
#include <cstring>
#include <new>
#include <vector>

#include "st_internal.cuh"

using namespace st;

namespace {

constexpr int kNT = 256;
constexpr int kStreamBlocks = 152 * 8;

__global__ void k_zero3_gated(long long N, df *a, df *b, df *c, const State *S) {
  if (!S->restart) return;
  const df z{0.f, 0.f};
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < N;
       e += (long long)gridDim.x * blockDim.x) {
    a[e] = z;
    b[e] = z;
    c[e] = z;
  }
}

__global__ void k_df_to_double_gated(long long N, const df *__restrict__ src,
                                     double *__restrict__ dst, const State *S) {
  if (!(S->finish && !S->done)) return;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < N;
       e += (long long)gridDim.x * blockDim.x)
    dst[e] = df_to_double(src[e]);
}

// End of one trip of an instance's loop: continue while the instance is not done and the trip
// budget lasts; a loop stopped by the budget marks the instance done and not converged.
__global__ void k_loop_control(cudaGraphConditionalHandle cond, State *S, int *trips,
                               int max_trips) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  const int t = ++(*trips);
  bool go = !S->done;
  if (go && t >= max_trips) {
    go = false;
    S->done = 1;
    S->active = 0;
    if (S->status == 0) S->status = ST_ERR_NOT_CONVERGED;
  }
  cudaGraphSetConditional(cond, go ? 1u : 0u);
}

struct BatchInfo {
  double rho, est;
  int done, status, total, outer, tmem_held;
};

__global__ void k_gather(State *const *states, int count, BatchInfo *out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= count) return;
  const State *S = states[i];
  BatchInfo b;
  b.rho = S->rho;
  b.est = S->est;
  b.done = S->done;
  b.status = S->status;
  b.total = S->total;
  b.outer = S->outer;
  b.tmem_held = S->tmem_held;
  out[i] = b;
}

// MINRES iteration b (0..3) of a trip: iterations 4t + 1 .. 4t + 4 of an inner run, z_k in ring
// slot (k - 1) % 4 (st_setup_batch gives the instance handles four z vectors), the Lanczos
// vectors alternating with the parity of k; the direction/solution update runs after b = 1 and
// b = 3 and applies the iterations pending since the previous one (k_update_group_df)
cudaError_t iteration(st_handle *h, int b, cudaStream_t st) {
  const int c = b & 1, o = c ^ 1;
  const Geom &g = h->g;
  const float *zc = zslot(h, b);
  float *zn = zslot(h, (b + 1) & 3);
  df *V0 = (df *)h->V[c], *V1 = (df *)h->V[o];
  df *q = (df *)h->q;
  cudaError_t e;
  if ((e = launch_stencil_df(g, zc, q, h->S, h->partials, st)) != cudaSuccess) return e;
  // Lanczos step fused into the first transform of the preconditioner pass
  if ((e = launch_prec_lanczos<float, df, float>(g, h->pp, q, V0, V1, zn, h->S, h->partials,
                                                 st)) != cudaSuccess)
    return e;
  return (b & 1) ? launch_update_group(h, st) : cudaSuccess;
}

// refinement block: x (float64) <- x (df); r <- Y f_H - Y T x with decision; restart if asked
cudaError_t refine(st_handle *h, const double *fH, double *u, cudaStream_t st) {
  const Geom &g = h->g;
  cudaError_t e;
  k_df_to_double_gated<<<kStreamBlocks, kNT, 0, st>>>(g.N, h->Xdf, u, h->S);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  if ((e = launch_resid_outer(g, u, (df *)h->V[0], fH, h->S, h->partials, st)) != cudaSuccess)
    return e;
  k_zero3_gated<<<kStreamBlocks, kNT, 0, st>>>(g.N, (df *)h->D[0], (df *)h->D[1], (df *)h->V[1],
                                              h->S);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  return launch_prec<float, df, float>(g, h->pp, (const df *)h->V[0], (float *)h->Z[0], h->S,
                                       TM_RESTART, h->partials, st);
}

int map_err(cudaError_t e) {
  if (e == cudaSuccess) return ST_OK;
  return e == cudaErrorMemoryAllocation ? ST_ERR_OOM : ST_ERR_CUDA;
}

}  // namespace

struct st_batch {
  int count;
  int device;
  cudaStream_t stream;                // caller's stream (may be the legacy default stream)
  cudaStream_t cstream;               // the batch's own stream: capture and graph launches
  std::vector<st_handle *> h;
  std::vector<cudaStream_t> streams;  // one per instance
  std::vector<cudaEvent_t> events;    // one per instance: joins of the start-up work
  std::vector<cudaEvent_t> cevents;   // one per instance: joins inside the captured graph
  cudaEvent_t fork, cfork, done_ev;
  State **d_states;
  BatchInfo *d_info, *h_info;
  int *d_trips;                       // per instance: trips of its loop in the current solve
  cudaGraphExec_t exec;
  std::vector<const double *> cap_fH;  // pointers the graph was captured with
  std::vector<double *> cap_u;
  int cap_maxit;                       // trip budget the graph was built with
};

namespace {

void free_batch(st_batch *b) {
  if (!b) return;
  if (b->exec) cudaGraphExecDestroy(b->exec);
  for (auto h : b->h) st_destroy(h);
  for (auto s : b->streams) cudaStreamDestroy(s);
  for (auto e : b->events) cudaEventDestroy(e);
  for (auto e : b->cevents) cudaEventDestroy(e);
  if (b->fork) cudaEventDestroy(b->fork);
  if (b->cfork) cudaEventDestroy(b->cfork);
  if (b->done_ev) cudaEventDestroy(b->done_ev);
  if (b->cstream) cudaStreamDestroy(b->cstream);
  cudaFree(b->d_states);
  cudaFree(b->d_info);
  cudaFree(b->d_trips);
  if (b->h_info) cudaFreeHost(b->h_info);
  delete b;
}

#define BT_TRY(expr)                          \
  do {                                        \
    cudaError_t _e = (expr);                  \
    if (_e != cudaSuccess) return map_err(_e); \
  } while (0)

// Build the graph: one WHILE node per instance, its body captured from the instance's own stream.
int capture(st_batch *b, const double *const *fH, double *const *u, int maxit) {
  if (b->exec) {
    cudaGraphExecDestroy(b->exec);
    b->exec = nullptr;
  }
  cudaGraph_t graph = nullptr;
  BT_TRY(cudaGraphCreate(&graph, 0));
  cudaError_t e = cudaSuccess;
  const int max_trips = maxit + 64;
  for (int i = 0; i < b->count && e == cudaSuccess; ++i) {
    cudaGraphConditionalHandle cond;
    e = cudaGraphConditionalHandleCreate(&cond, graph, 1, cudaGraphCondAssignDefault);
    if (e != cudaSuccess) break;
    cudaGraphNodeParams np = {};
    np.type = cudaGraphNodeTypeConditional;
    np.conditional.handle = cond;
    np.conditional.type = cudaGraphCondTypeWhile;
    np.conditional.size = 1;
    cudaGraphNode_t node;
    e = cudaGraphAddNode(&node, graph, nullptr, nullptr, 0, &np);
    if (e != cudaSuccess) break;
    cudaGraph_t body = np.conditional.phGraph_out[0];
    cudaStream_t s = b->streams[i];
    e = cudaStreamBeginCaptureToGraph(s, body, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed);
    if (e != cudaSuccess) break;
    for (int it = 0; it < 4 && e == cudaSuccess; ++it) e = iteration(b->h[i], it, s);
    if (e == cudaSuccess) e = refine(b->h[i], fH[i], u[i], s);
    if (e == cudaSuccess) {
      k_loop_control<<<1, 32, 0, s>>>(cond, b->h[i]->S, b->d_trips + i, max_trips);
      e = cudaGetLastError();
    }
    cudaGraph_t captured = nullptr;
    const cudaError_t e2 = cudaStreamEndCapture(s, &captured);
    if (e == cudaSuccess) e = e2;
  }
  if (e == cudaSuccess) e = cudaGraphInstantiate(&b->exec, graph, 0);
  cudaGraphDestroy(graph);
  if (e != cudaSuccess) {
    cudaGetLastError();
    if (b->exec) cudaGraphExecDestroy(b->exec);
    b->exec = nullptr;
    return map_err(e);
  }
  b->cap_fH.assign(fH, fH + b->count);
  b->cap_u.assign(u, u + b->count);
  b->cap_maxit = maxit;
  return ST_OK;
}

}  // namespace

extern "C" {

int st_setup_batch(const st_problem *probs, int count, void *stream, st_batch **out) {
  if (!out || !probs || count < 1 || count > 4096) return ST_ERR_ARG;
  *out = nullptr;
  for (int i = 0; i < count; ++i) {
    if (probs[i].precision != ST_MIXED) return ST_ERR_ARG;
    size_t bytes = 0;
    int r = st_workspace_bytes(&probs[i], &bytes);
    if (r) return r;
  }
  st_batch *b = new (std::nothrow) st_batch();
  if (!b) return ST_ERR_OOM;
  b->count = count;
  b->stream = (cudaStream_t)stream;
  if (cudaGetDevice(&b->device) != cudaSuccess) {
    delete b;
    return ST_ERR_CUDA;
  }
  auto fail = [&](int code) {
    free_batch(b);
    return code;
  };
  if (cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&b->cfork, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&b->done_ev, cudaEventDisableTiming) != cudaSuccess ||
      cudaStreamCreateWithFlags(&b->cstream, cudaStreamNonBlocking) != cudaSuccess)
    return fail(ST_ERR_CUDA);
  b->h.assign(count, nullptr);
  b->streams.assign(count, nullptr);
  b->events.assign(count, nullptr);
  b->cevents.assign(count, nullptr);
  for (int i = 0; i < count; ++i) {
    if (cudaStreamCreateWithFlags(&b->streams[i], cudaStreamNonBlocking) != cudaSuccess)
      return fail(ST_ERR_CUDA);
    if (cudaEventCreateWithFlags(&b->events[i], cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&b->cevents[i], cudaEventDisableTiming) != cudaSuccess)
      return fail(ST_ERR_CUDA);
    // instance handles serve the caller's own calls (st_assemble_rhs, st_apply_op, ...) on the
    // caller's stream; the batch solve passes its internal streams explicitly
    st_problem p = probs[i];
    p.stream = stream;
    // group of 3 (four z vectors): the captured trip uses the ring of four with an update pass
    // after every second iteration
    int r = setup_handle(&p, &b->h[i], 3);
    if (r) return fail(r);
    // launch shapes per (size, precision), cached across instances of the same shape
    r = st_autotune(b->h[i], 5);
    if (r) return fail(r);
  }
  std::vector<State *> sp(count);
  for (int i = 0; i < count; ++i) sp[i] = b->h[i]->S;
  if (cudaMalloc(&b->d_states, count * sizeof(State *)) != cudaSuccess) return fail(ST_ERR_OOM);
  if (cudaMemcpy(b->d_states, sp.data(), count * sizeof(State *), cudaMemcpyHostToDevice) !=
      cudaSuccess)
    return fail(ST_ERR_CUDA);
  if (cudaMalloc(&b->d_info, count * sizeof(BatchInfo)) != cudaSuccess) return fail(ST_ERR_OOM);
  if (cudaMalloc(&b->d_trips, count * sizeof(int)) != cudaSuccess) return fail(ST_ERR_OOM);
  if (cudaMallocHost(&b->h_info, count * sizeof(BatchInfo)) != cudaSuccess)
    return fail(ST_ERR_OOM);
  *out = b;
  return ST_OK;
}

void st_destroy_batch(st_batch *b) {
  if (!b) return;
  cudaSetDevice(b->device);
  cudaStreamSynchronize(b->stream);
  if (b->cstream) cudaStreamSynchronize(b->cstream);
  for (auto s : b->streams) cudaStreamSynchronize(s);
  free_batch(b);
}

int st_solve_batch(st_batch *b, const double *const *fH_devs, double *const *u_devs, double tol,
                   int maxit, st_stats *stats) {
  if (!b || !fH_devs || !u_devs || !(tol > 0.0) || maxit < 1) return ST_ERR_ARG;
  for (int i = 0; i < b->count; ++i)
    if (!fH_devs[i] || !u_devs[i] || fH_devs[i] == u_devs[i]) return ST_ERR_ARG;
  BT_TRY(cudaSetDevice(b->device));
  if (device_closed(b->device)) return ST_ERR_TIMEOUT;
  // start of every instance (regular launches on the instance streams, after the caller's work)
  BT_TRY(cudaEventRecord(b->fork, b->stream));
  for (int i = 0; i < b->count; ++i) {
    st_handle *h = b->h[i];
    cudaStream_t s = b->streams[i];
    const Geom &g = h->g;
    BT_TRY(cudaStreamWaitEvent(s, b->fork, 0));
    State &S = *h->hS;
    std::memset(&S, 0, sizeof(State));
    S.active = 1;
    S.tol_outer = tol;
    S.maxit_total = maxit;
    S.maxit = maxit;
    S.inner_floor = inner_floor();
    S.target = std::max(0.5 * tol, S.inner_floor);
    BT_TRY(cudaMemcpyAsync(h->S, h->hS, kStatePushBytes, cudaMemcpyHostToDevice, s));
    BT_TRY(cudaMemsetAsync(h->Xdf, 0, g.N * sizeof(df), s));
    BT_TRY(cudaMemsetAsync(u_devs[i], 0, g.N * sizeof(double), s));
    BT_TRY(cudaMemsetAsync(h->D[0], 0, g.N * sizeof(df), s));
    BT_TRY(cudaMemsetAsync(h->D[1], 0, g.N * sizeof(df), s));
    BT_TRY(cudaMemsetAsync(h->V[1], 0, g.N * sizeof(df), s));
    BT_TRY(launch_flip_to_df(g, fH_devs[i], (df *)h->V[0], s));
    BT_TRY(launch_norm2(g.N, fH_devs[i], h->S, h->partials, s));
    BT_TRY((launch_prec<float, df, float>(g, h->pp, (const df *)h->V[0], (float *)h->Z[0], h->S,
                                          TM_INIT, h->partials, s)));
    BT_TRY(cudaEventRecord(b->events[i], s));
    BT_TRY(cudaStreamWaitEvent(b->cstream, b->events[i], 0));
  }
  bool same = b->exec && b->cap_fH.size() == (size_t)b->count && b->cap_maxit == maxit;
  for (int i = 0; same && i < b->count; ++i)
    same = (b->cap_fH[i] == fH_devs[i] && b->cap_u[i] == u_devs[i]);
  if (!same) {
    int r = capture(b, fH_devs, u_devs, maxit);
    if (r) return r;
  }
  // one launch runs every instance's loop to its end
  BT_TRY(cudaMemsetAsync(b->d_trips, 0, b->count * sizeof(int), b->cstream));
  BT_TRY(cudaGraphLaunch(b->exec, b->cstream));
  k_gather<<<(b->count + 127) / 128, 128, 0, b->cstream>>>(b->d_states, b->count, b->d_info);
  BT_TRY(cudaGetLastError());
  BT_TRY(cudaMemcpyAsync(b->h_info, b->d_info, b->count * sizeof(BatchInfo),
                         cudaMemcpyDeviceToHost, b->cstream));
  BT_TRY(cudaStreamSynchronize(b->cstream));
  for (int i = 0; i < b->count; ++i) {
    if (b->h_info[i].tmem_held) {
      close_device(b->device);
      return ST_ERR_TIMEOUT;
    }
  }
  // later work on the caller's stream sees the solutions
  BT_TRY(cudaEventRecord(b->done_ev, b->cstream));
  BT_TRY(cudaStreamWaitEvent(b->stream, b->done_ev, 0));
  int worst = ST_OK;
  for (int i = 0; i < b->count; ++i) {
    const BatchInfo &bi = b->h_info[i];
    int st = bi.done ? bi.status : ST_ERR_NOT_CONVERGED;
    if (st == 0 && bi.rho > tol) st = ST_ERR_NOT_CONVERGED;
    if (stats) {
      stats[i] = st_stats{};
      stats[i].iterations = bi.total;
      stats[i].outer_steps = bi.outer;
      stats[i].true_checks = bi.outer;
      stats[i].status = st;
      stats[i].est_rel_res = bi.est;
      stats[i].true_rel_res = bi.rho;
    }
    if (st != ST_OK && worst == ST_OK) worst = st;
  }
  return worst;
}

int st_batch_instance(st_batch *b, int i, st_handle **out) {
  if (!b || !out || i < 0 || i >= b->count) return ST_ERR_ARG;
  *out = b->h[i];
  return ST_OK;
}

}  // extern "C"
