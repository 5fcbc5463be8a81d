// Restarted right-preconditioned GMRES / flexible GMRES (Sec. 3.2 and 4;
// Saad 1993 for the flexible form) on device vectors, entirely on the device.
//
// Arnoldi step j (all FP64):
//   z_j = M^{-1} v_j   (kept in Z for the flexible form)
//   w   = F z_j
//   h   = V_j^T w ;  w -= V_j h          classical Gram-Schmidt ...
//   h2  = V_j^T w ;  w -= V_j h2         ... applied twice (CGS2)
//   column j of H = h + h2, H[j+1][j] = ||w||
//   Givens rotations, residual estimate |g_{j+1}| / ||b||, stop test  (gm_givens)
//   v_{j+1} = w / ||w||
// The rotations, the estimate, the stop decision and the back substitution
// run in single-thread kernels on the device state (GmresState), and every
// kernel of a step is gated by the state's `active` flag: once the cycle has
// stopped, the remaining steps' kernels return at once.  A restart cycle is
// therefore a fixed sequence of launches, which the outer solver captures
// into a CUDA graph once and replays, with one host round trip per cycle to
// read the state (true residual, flag).  Dot products are reduced in a fixed
// order (block partials, then one block per vector), so results are
// deterministic.

#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "internal.cuh"

namespace {

constexpr int kDotBlocks = 304;   // 2 x 152 SMs (1216 measured slower: the coarse-level dots are short)
constexpr int kDotThreads = 256;

// partial[k * kDotBlocks + b] = sum over block b's part of V_k . w.  Block
// (k, b) runs with k fastest, so the m blocks that read the same part of w
// run together and w comes from L2 after its first read; V_k is read once,
// with evict-first loads that leave L2 to w.
__global__ void __launch_bounds__(kDotThreads) multidot_partial(const double* __restrict__ V, long long ldv,
                                                                const double* __restrict__ w, long long n,
                                                                double* __restrict__ part, const int* gate) {
  if (gated_off(gate)) return;
  __shared__ double red[kDotThreads / 32];
  const int k = blockIdx.x, b = blockIdx.y, nb = gridDim.y;
  const double* v = V + (long long)k * ldv;
  double acc = 0.0;
  for (long long i = b * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)nb * blockDim.x)
    acc = fma(__ldcs(v + i), w[i], acc);
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int q = 0; q < kDotThreads / 32; ++q) s += red[q];
    part[k * nb + b] = s;
  }
}

// out[k] = sum_b partial[k * nb + b], fixed order; one block per k
__global__ void multidot_final(const double* __restrict__ part, int nb, double* __restrict__ out, const int* gate) {
  if (gated_off(gate)) return;
  __shared__ double red[32];
  const int k = blockIdx.x;
  double acc = 0.0;
  for (int b = threadIdx.x; b < nb; b += blockDim.x) acc += part[k * nb + b];
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int q = 0; q < (int)(blockDim.x + 31) / 32; ++q) s += red[q];
    out[k] = s;
  }
}

// w -= sum_{k < m} V_k h[k]
__global__ void multi_axpy(double* __restrict__ w, const double* __restrict__ V, long long ldv,
                           const double* __restrict__ h, int m, long long n, const int* gate) {
  if (gated_off(gate)) return;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    double acc = w[i];
    for (int k = 0; k < m; ++k) acc = fma(-V[(long long)k * ldv + i], h[k], acc);
    w[i] = acc;
  }
}

// x += sum_{i < *k} Z_i y[i]  (the column count is read from the device state)
__global__ void multi_update(double* __restrict__ x, const double* __restrict__ Z, long long ldz,
                             const double* __restrict__ y, const int* __restrict__ k, long long n, const int* gate) {
  if (gated_off(gate)) return;
  const int m = *k;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    double acc = x[i];
    for (int q = 0; q < m; ++q) acc = fma(Z[(long long)q * ldz + i], y[q], acc);
    x[i] = acc;
  }
}

// y = *a x  (the factor is read from the device state)
__global__ void scale_dev(double* __restrict__ y, const double* __restrict__ x, const double* __restrict__ a,
                          long long n, const int* gate) {
  if (gated_off(gate)) return;
  const double f = *a;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    y[i] = f * x[i];
}

__global__ void axpby_kernel(double* __restrict__ y, double a, const double* __restrict__ x, double b, long long n,
                             const int* gate) {
  if (gated_off(gate)) return;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    y[i] = a * x[i] + b * y[i];
}

__global__ void copy_kernel(double* __restrict__ y, const double* __restrict__ x, long long n, const int* gate) {
  if (gated_off(gate)) return;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    y[i] = x[i];
}

// ---------------------------------------------------------------------------
// the single-thread kernels on the solver state
// ---------------------------------------------------------------------------

// First call of a solve: ||b|| from its squared norm; the iteration budget.
__global__ void gm_init(GmresState* st, double rtol, int maxit, const int* parent) {
  if (threadIdx.x != 0) return;
  st->bnorm = sqrt(st->b2);
  st->rtol = rtol;
  st->maxit = maxit;
  st->iters = 0;
  st->steps = 0;
  st->k = 0;
  st->ran = 0;
  st->active = 0;
  st->est = 1.0;
  st->flag = (parent != nullptr && *parent == 0) || isfinite(st->bnorm) ? kGmRunning : kGmNonFinite;
}

// Start of a restart cycle: beta = ||r|| from its squared norm, g = beta e_1;
// the cycle runs while the residual is above the tolerance, iterations are
// left and the parent step (if any) is live.
__global__ void gm_begin(GmresState* st, double* g, int m, const int* parent) {
  if (threadIdx.x != 0) return;
  st->k = 0;
  st->ran = 0;
  st->steps = 0;
  if ((parent != nullptr && *parent == 0) || st->flag == kGmNonFinite || st->flag == kGmBreakdown) {
    st->active = 0;
    return;
  }
  const double beta = sqrt(st->r2);
  st->beta = beta;
  for (int i = 0; i <= m; ++i) g[i] = 0.0;
  g[0] = beta;
  st->est = st->bnorm > 0.0 ? beta / st->bnorm : 0.0;
  if (!isfinite(beta)) {
    st->flag = kGmNonFinite;
    st->active = 0;
    return;
  }
  st->flag = kGmRunning;
  st->active = beta > st->rtol * st->bnorm && st->iters < st->maxit ? 1 : 0;
  st->inv = st->active ? 1.0 / beta : 0.0;
}

// Column j of the Hessenberg matrix, the previous rotations applied to it,
// the new rotation, the residual estimate and the stop test.  H is stored by
// columns (column j at H + j (m+1)).
__global__ void gm_givens(GmresState* st, int j, int m, const double* __restrict__ h, const double* __restrict__ h2,
                          double* __restrict__ H, double* __restrict__ cs, double* __restrict__ sn,
                          double* __restrict__ g) {
  if (threadIdx.x != 0 || !st->active) return;
  st->steps += 1;
  st->iters += 1;
  double* col = H + (size_t)j * (m + 1);
  for (int i = 0; i <= j; ++i) col[i] = h[i] + h2[i];
  const double hn = sqrt(h[j + 1]);
  col[j + 1] = hn;
  bool bad = !isfinite(hn);
  for (int i = 0; i <= j; ++i) bad = bad || !isfinite(col[i]);
  if (bad) {
    st->flag = kGmNonFinite;
    st->active = 0;
    st->k = j;
    return;
  }
  for (int i = 0; i < j; ++i) {
    const double t = cs[i] * col[i] + sn[i] * col[i + 1];
    col[i + 1] = -sn[i] * col[i] + cs[i] * col[i + 1];
    col[i] = t;
  }
  const double den = hypot(col[j], col[j + 1]);
  if (den == 0.0) {
    // F M^{-1} v_j lies in span(v_0 .. v_{j-1}) with a zero rotated diagonal:
    // column j adds nothing to the least-squares problem; the cycle ends on
    // columns 0 .. j-1 with a breakdown
    st->flag = kGmBreakdown;
    st->active = 0;
    st->k = j;
    return;
  }
  cs[j] = col[j] / den;
  sn[j] = col[j + 1] / den;
  col[j] = den;
  col[j + 1] = 0.0;
  g[j + 1] = -sn[j] * g[j];
  g[j] = cs[j] * g[j];
  st->k = j + 1;
  st->est = fabs(g[j + 1]) / st->bnorm;
  if (hn == 0.0 || st->est <= st->rtol || st->iters >= st->maxit) {
    st->active = 0;
    st->flag = st->est <= st->rtol ? kGmConverged : (hn == 0.0 ? kGmBreakdown : kGmLimit);
  } else {
    st->inv = 1.0 / hn;
  }
}

// End of a cycle: back substitution R y = g on the k columns; `ran` gates the
// solution update.
__global__ void gm_solve_y(GmresState* st, int m, const double* __restrict__ H, const double* __restrict__ g,
                           double* __restrict__ y) {
  if (threadIdx.x != 0) return;
  st->active = 0;
  const int k = st->k;
  for (int i = k - 1; i >= 0; --i) {
    double acc = g[i];
    for (int q = i + 1; q < k; ++q) acc -= H[(size_t)q * (m + 1) + i] * y[q];
    y[i] = acc / H[(size_t)i * (m + 1) + i];
  }
  st->ran = k > 0 ? 1 : 0;
}

constexpr unsigned kVecBlocks = 1216;   // 8 x 152 SMs

// out[0..m) = V_k . w  for k < m
kkt_status multidot(const double* V, long long ldv, int m, const double* w, long long n, double* part, double* out,
                    cudaStream_t s, const int* gate) {
  dim3 g(m, kDotBlocks);
  multidot_partial<<<g, kDotThreads, 0, s>>>(V, ldv, w, n, part, gate);
  multidot_final<<<m, 256, 0, s>>>(part, kDotBlocks, out, gate);
  KKT_COUNT(2);
  KKT_TRY_CUDA(cudaGetLastError());
  return KKT_OK;
}

kkt_status launched(int n = 1) {
  KKT_COUNT(n);
  KKT_TRY_CUDA(cudaGetLastError());
  return KKT_OK;
}

// One restart cycle: V_0 = r / ||r||, up to m Arnoldi steps, the back
// substitution and the update of x; with check_true also the true residual
// r = b - A x and its squared norm.  Every launch is stream-ordered on s and
// nothing reads the device state on the host, so the cycle can be captured.
kkt_status enqueue_cycle(Operator& A, Operator* M, const double* b, double* x, GmresWork& ws, int m,
                         bool check_true, const int* parent, cudaStream_t s) {
  const long long n = ws.n;
  GmresState* st = ws.st;
  const int* active = &st->active;
  const int* ran = &st->ran;
  gm_begin<<<1, 32, 0, s>>>(st, ws.g(), m, parent);
  KKT_TRY(launched());
  scale_dev<<<kVecBlocks, 256, 0, s>>>(ws.V, ws.r, &st->inv, n, active);
  KKT_TRY(launched());
  // the outer cycle tags its captured timing pairs with the step (the inner coarse cycle
  // runs inside an outer step and leaves the tag alone)
  const bool tag = g_capture != nullptr && check_true;
  for (int j = 0; j < m; ++j) {
    if (tag) g_capture->step = j;
    double* vj = ws.V + (size_t)j * n;
    double* zj = ws.flexible ? ws.Z + (size_t)j * n : ws.r;
    if (M) KKT_TRY(M->apply(vj, zj, s, active));
    else KKT_TRY(vec_copy(zj, vj, n, s, active));
    KKT_TRY(A.apply(zj, ws.w, s, active));
    KKT_TRY(multidot(ws.V, n, j + 1, ws.w, n, ws.part, ws.h(), s, active));
    multi_axpy<<<kVecBlocks, 256, 0, s>>>(ws.w, ws.V, n, ws.h(), j + 1, n, active);
    KKT_TRY(launched());
    KKT_TRY(multidot(ws.V, n, j + 1, ws.w, n, ws.part, ws.h2(), s, active));
    multi_axpy<<<kVecBlocks, 256, 0, s>>>(ws.w, ws.V, n, ws.h2(), j + 1, n, active);
    KKT_TRY(launched());
    KKT_TRY(multidot(ws.w, 0, 1, ws.w, n, ws.part, ws.h() + j + 1, s, active));
    gm_givens<<<1, 32, 0, s>>>(st, j, m, ws.h(), ws.h2(), ws.H(), ws.cs(), ws.sn(), ws.g());
    KKT_TRY(launched());
    if (j + 1 < m) {
      scale_dev<<<kVecBlocks, 256, 0, s>>>(ws.V + (size_t)(j + 1) * n, ws.w, &st->inv, n, active);
      KKT_TRY(launched());
    }
  }
  if (tag) g_capture->step = -1;
  gm_solve_y<<<1, 32, 0, s>>>(st, m, ws.H(), ws.g(), ws.y());
  KKT_TRY(launched());
  if (ws.flexible) {
    multi_update<<<kVecBlocks, 256, 0, s>>>(x, ws.Z, n, ws.y(), &st->k, n, ran);
    KKT_TRY(launched());
  } else {
    // x += M^{-1} (V y): V y in w, preconditioned into r
    KKT_TRY(vec_zero(ws.w, n, s));
    multi_update<<<kVecBlocks, 256, 0, s>>>(ws.w, ws.V, n, ws.y(), &st->k, n, ran);
    KKT_TRY(launched());
    if (M) KKT_TRY(M->apply(ws.w, ws.r, s, ran));
    else KKT_TRY(vec_copy(ws.r, ws.w, n, s, ran));
    KKT_TRY(vec_axpby(x, 1.0, ws.r, 1.0, n, s, ran));
  }
  if (check_true) {
    // true residual r = b - A x and its squared norm, for the next cycle or the exit
    KKT_TRY(A.apply(x, ws.w, s, nullptr));
    KKT_TRY(vec_copy(ws.r, b, n, s));
    KKT_TRY(vec_axpby(ws.r, -1.0, ws.w, 1.0, n, s));
    KKT_TRY(multidot(ws.r, 0, 1, ws.r, n, ws.part, &st->r2, s, nullptr));
  }
  return KKT_OK;
}

kkt_status read_state(GmresWork& ws, cudaStream_t s) {
  KKT_TRY_CUDA(cudaMemcpyAsync(ws.st_host, ws.st, sizeof(GmresState), cudaMemcpyDeviceToHost, s));
  KKT_TRY_CUDA(cudaStreamSynchronize(s));
  return KKT_OK;
}

// Replay bookkeeping of a captured cycle: the launch count and the timing
// pairs of the steps that ran.
kkt_status after_replay(CycleGraph& gr, int steps) {
  g_kernel_launches.fetch_add(gr.launches, std::memory_order_relaxed);
  for (auto& e : gr.timing.entries) {
    if (e.step >= steps) continue;
    float ms = 0.f;
    const cudaError_t err = cudaEventElapsedTime(&ms, e.e0, e.e1);
    if (err != cudaSuccess) {
      cudaGetLastError();
      set_error(std::string("gmres: timing of a captured launch: ") + cudaGetErrorString(err));
      return KKT_ERR_CUDA;
    }
    e.log->total_ms += ms;
    e.log->count += 1;
  }
  return KKT_OK;
}

// Capture one restart cycle, enqueued by `enqueue` on the given stream, into
// gr (on the work's own stream, which forks from and joins into nothing: the
// graph is launched on the caller's stream).
template <typename Enqueue>
kkt_status capture_cycle(GmresWork& ws, int m, const unsigned long long* key, int timed_per_step,
                         Enqueue&& enqueue) {
  CycleGraph& gr = ws.graph;
  gr.release();
  if (!ws.cap) KKT_TRY_CUDA(cudaStreamCreateWithFlags(&ws.cap, cudaStreamNonBlocking));
  CaptureTiming& ct = gr.timing;
  ct.clear();
  if (g_timing_on.load()) {
    // launches timed per step: outer matvecs, fine and coarse subdomain solves
    const size_t npairs = (size_t)timed_per_step * m + 16;
    for (size_t i = 0; i < npairs; ++i) {
      cudaEvent_t e0, e1;
      KKT_TRY_CUDA(cudaEventCreate(&e0));
      KKT_TRY_CUDA(cudaEventCreate(&e1));
      ct.pool.emplace_back(e0, e1);
    }
  }
  const long long before = g_kernel_launches.load();
  KKT_TRY_CUDA(cudaStreamBeginCapture(ws.cap, cudaStreamCaptureModeThreadLocal));
  g_capture = &ct;
  const kkt_status st = enqueue(ws.cap);
  g_capture = nullptr;
  cudaGraph_t graph = nullptr;
  const cudaError_t ce = cudaStreamEndCapture(ws.cap, &graph);
  gr.launches = g_kernel_launches.load() - before;
  g_kernel_launches.fetch_sub(gr.launches, std::memory_order_relaxed);   // counted per replay instead
  if (st != KKT_OK) {
    if (graph) cudaGraphDestroy(graph);
    return st;
  }
  if (ce != cudaSuccess) {
    set_error(std::string("gmres: cycle capture failed: ") + cudaGetErrorString(ce));
    return KKT_ERR_CUDA;
  }
  const cudaError_t ie = cudaGraphInstantiate(&gr.exec, graph, 0);
  cudaGraphDestroy(graph);
  if (ie != cudaSuccess) {
    gr.exec = nullptr;
    set_error(std::string("gmres: graph instantiation failed: ") + cudaGetErrorString(ie));
    return KKT_ERR_CUDA;
  }
  std::memcpy(gr.key, key, sizeof(gr.key));
  return KKT_OK;
}

}  // namespace

thread_local CaptureTiming* g_capture = nullptr;

void CaptureTiming::clear() {
  for (auto& e : pool) {
    cudaEventDestroy(e.first);
    cudaEventDestroy(e.second);
  }
  pool.clear();
  entries.clear();
  used = 0;
  step = -1;
}

void CycleGraph::release() {
  if (exec) cudaGraphExecDestroy(exec);
  exec = nullptr;
  std::memset(key, 0, sizeof(key));
  launches = 0;
  timing.clear();
}

kkt_status vec_copy(double* y, const double* x, long long n, cudaStream_t s, const int* gate) {
  copy_kernel<<<kVecBlocks, 256, 0, s>>>(y, x, n, gate);
  return launched();
}

kkt_status vec_zero(double* y, long long n, cudaStream_t s) {
  KKT_TRY_CUDA(cudaMemsetAsync(y, 0, n * sizeof(double), s));
  return KKT_OK;
}

kkt_status vec_axpby(double* y, double a, const double* x, double b, long long n, cudaStream_t s, const int* gate) {
  axpby_kernel<<<kVecBlocks, 256, 0, s>>>(y, a, x, b, n, gate);
  return launched();
}

kkt_status GmresWork::alloc(long long n_, int m_, bool flex) {
  if (n_ == n && m_ <= m && (!flex || flexible)) return KKT_OK;
  release();
  n = n_;
  m = m_;
  flexible = flex;
  nparts = kDotBlocks;
  if (cudaMalloc(&V, (size_t)(m + 1) * n * sizeof(double)) != cudaSuccess ||
      (flex && cudaMalloc(&Z, (size_t)m * n * sizeof(double)) != cudaSuccess) ||
      cudaMalloc(&w, n * sizeof(double)) != cudaSuccess || cudaMalloc(&r, n * sizeof(double)) != cudaSuccess ||
      cudaMalloc(&hbuf, doubles(m) * sizeof(double)) != cudaSuccess ||
      cudaMalloc(&st, sizeof(GmresState)) != cudaSuccess ||
      cudaMalloc(&part, (size_t)(m + 2) * kDotBlocks * sizeof(double)) != cudaSuccess ||
      cudaMallocHost(&st_host, sizeof(GmresState)) != cudaSuccess ||
      cudaMemset(hbuf, 0, doubles(m) * sizeof(double)) != cudaSuccess ||
      cudaMemset(st, 0, sizeof(GmresState)) != cudaSuccess) {
    cudaGetLastError();
    release();
    set_error("gmres: workspace allocation failed");
    return KKT_ERR_NOMEM;
  }
  return KKT_OK;
}

void GmresWork::release() {
  graph.release();
  if (cap) cudaStreamDestroy(cap);
  cap = nullptr;
  cudaFree(V);
  cudaFree(Z);
  cudaFree(w);
  cudaFree(r);
  cudaFree(hbuf);
  cudaFree(st);
  cudaFree(part);
  if (st_host) cudaFreeHost(st_host);
  V = Z = w = r = hbuf = part = nullptr;
  st = nullptr;
  st_host = nullptr;
  n = 0;
  m = 0;
}

kkt_status gmres_run(Operator& A, Operator* M, const double* b, double* x, GmresWork& ws, int restart, double rtol,
                     int maxit, bool check_true, bool zero_guess, GmresResult* res, cudaStream_t s,
                     const int* parent, bool graph) {
  const long long n = ws.n;
  const int m = restart;
  res->iters = 0;
  res->relres = 0.0;
  res->status = KKT_OK;
  if (m > ws.m) {
    set_error("gmres: restart longer than the workspace");
    return KKT_ERR_ARG;
  }
  GmresState* st = ws.st;

  if (!check_true) {
    // inner solve (the coarse level): one cycle from a zero guess, enqueued only
    KKT_TRY(vec_zero(x, n, s));
    KKT_TRY(vec_copy(ws.r, b, n, s, parent));
    KKT_TRY(multidot(b, 0, 1, b, n, ws.part, &st->b2, s, parent));
    KKT_TRY(multidot(b, 0, 1, b, n, ws.part, &st->r2, s, parent));
    gm_init<<<1, 32, 0, s>>>(st, rtol, maxit, parent);
    KKT_TRY(launched());
    return enqueue_cycle(A, M, b, x, ws, m, false, parent, s);
  }

  // outer solve: ||b|| and the initial residual, then one host round trip per cycle
  KKT_TRY(multidot(b, 0, 1, b, n, ws.part, &st->b2, s, nullptr));
  gm_init<<<1, 32, 0, s>>>(st, rtol, maxit, nullptr);
  KKT_TRY(launched());
  KKT_TRY(read_state(ws, s));
  const double bnorm = ws.st_host->bnorm;
  if (!std::isfinite(bnorm)) {
    set_error("gmres: right-hand side is not finite");
    res->status = KKT_ERR_NONFINITE;
    return KKT_ERR_NONFINITE;
  }
  if (bnorm == 0.0) {
    KKT_TRY(vec_zero(x, n, s));
    return KKT_OK;
  }
  if (zero_guess) {
    KKT_TRY(vec_zero(x, n, s));
    KKT_TRY(vec_copy(ws.r, b, n, s));
  } else {
    KKT_TRY(A.apply(x, ws.w, s, nullptr));
    KKT_TRY(vec_copy(ws.r, b, n, s));
    KKT_TRY(vec_axpby(ws.r, -1.0, ws.w, 1.0, n, s));
  }
  KKT_TRY(multidot(ws.r, 0, 1, ws.r, n, ws.part, &st->r2, s, nullptr));

  // what a captured cycle depends on besides the device state
  const unsigned long long key[10] = {A.uid(),
                                      M ? M->uid() : 0ull,
                                      (unsigned long long)(uintptr_t)b,
                                      (unsigned long long)(uintptr_t)x,
                                      (unsigned long long)m,
                                      (unsigned long long)ws.flexible,
                                      (unsigned long long)g_timing_on.load(),
                                      (unsigned long long)(uintptr_t)ws.V,
                                      1ull,
                                      0ull};
  bool converged = false;
  double beta = 0.0;
  kkt_status status = KKT_NOT_CONVERGED;
  for (;;) {
    if (graph) {
      if (!ws.graph.exec || std::memcmp(ws.graph.key, key, sizeof(key)) != 0)
        KKT_TRY(capture_cycle(ws, m, key, 8, [&](cudaStream_t cs) {
          return enqueue_cycle(A, M, b, x, ws, m, true, nullptr, cs);
        }));
      KKT_TRY_CUDA(cudaGraphLaunch(ws.graph.exec, s));
    } else {
      KKT_TRY(enqueue_cycle(A, M, b, x, ws, m, true, nullptr, s));
    }
    KKT_TRY(read_state(ws, s));
    const GmresState& h = *ws.st_host;
    if (graph) KKT_TRY(after_replay(ws.graph, h.steps));
    beta = std::sqrt(h.r2);
    res->iters = h.iters;
    if (h.flag == kGmNonFinite || !std::isfinite(beta)) {
      set_error("gmres: non-finite value in the Arnoldi process");
      res->status = KKT_ERR_NONFINITE;
      return KKT_ERR_NONFINITE;
    }
    converged = beta <= rtol * bnorm;
    if (converged) {
      status = KKT_OK;
      break;
    }
    if (h.flag == kGmBreakdown) {
      status = KKT_BREAKDOWN;
      break;
    }
    if (h.iters >= maxit || h.steps == 0) {
      status = KKT_NOT_CONVERGED;
      break;
    }
  }
  res->relres = beta / bnorm;
  res->status = status;
  return KKT_OK;
}

// ---------------------------------------------------------------------------
// Several independent problems in lockstep (gmres_solve_batch).  Their
// unknowns are concatenated (problem k from off[k]); V, Z, w, r hold all of
// them, every problem has its own state, Hessenberg column and rotations.
// Step j applies the preconditioner to all problems at once (the subdomain
// solve over all boxes, each box gated by its problem's state), then each
// problem's matvec, CGS2 and rotation on its own part, gated by its state.
// ---------------------------------------------------------------------------
kkt_status BatchWork::alloc(const std::vector<long long>& off_, int m_) {
  if (off_ == off && m_ <= ws.m) return KKT_OK;
  release();
  off = off_;
  const int np = (int)off.size() - 1;
  KKT_TRY(ws.alloc(off.back(), m_, true));
  if (cudaMalloc(&st, np * sizeof(GmresState)) != cudaSuccess ||
      cudaMalloc(&small, (size_t)np * GmresWork::doubles(ws.m) * sizeof(double)) != cudaSuccess ||
      cudaMallocHost(&st_host, np * sizeof(GmresState)) != cudaSuccess ||
      cudaMemset(st, 0, np * sizeof(GmresState)) != cudaSuccess ||
      cudaMemset(small, 0, (size_t)np * GmresWork::doubles(ws.m) * sizeof(double)) != cudaSuccess) {
    cudaGetLastError();
    release();
    set_error("gmres_solve_batch: workspace allocation failed");
    return KKT_ERR_NOMEM;
  }
  return KKT_OK;
}

void BatchWork::release() {
  ws.release();
  cudaFree(st);
  cudaFree(small);
  if (st_host) cudaFreeHost(st_host);
  st = nullptr;
  small = nullptr;
  st_host = nullptr;
  off.clear();
}

namespace {

// the small arrays of problem k, laid out as in GmresWork
struct Small {
  double *h, *h2, *y, *cs, *sn, *g, *H;
};
Small small_of(const BatchWork& bw, int k) {
  const int m = bw.ws.m;
  double* b = bw.small + (size_t)k * GmresWork::doubles(m);
  Small o;
  o.h = b;
  o.h2 = b + (m + 2);
  o.y = b + 2 * (m + 2);
  o.cs = o.y + m;
  o.sn = o.cs + m;
  o.g = o.sn + m;
  o.H = o.g + (m + 1);
  return o;
}

kkt_status enqueue_cycle_batch(std::vector<Operator*>& A, Operator& M, const double* b, double* x, BatchWork& bw,
                               int m, cudaStream_t s) {
  GmresWork& ws = bw.ws;
  const long long N = ws.n;   // all problems
  const int np = (int)bw.off.size() - 1;
  for (int k = 0; k < np; ++k) {
    gm_begin<<<1, 32, 0, s>>>(bw.st + k, small_of(bw, k).g, m, nullptr);
    KKT_TRY(launched());
    const long long o = bw.off[k];
    scale_dev<<<kVecBlocks, 256, 0, s>>>(ws.V + o, ws.r + o, &bw.st[k].inv, bw.off[k + 1] - o, &bw.st[k].active);
    KKT_TRY(launched());
  }
  constexpr int kStride = (int)(sizeof(GmresState) / sizeof(int));
  for (int j = 0; j < m; ++j) {
    if (g_capture) g_capture->step = j;
    double* Vj = ws.V + (size_t)j * N;
    double* Zj = ws.Z + (size_t)j * N;
    // the preconditioner of every problem in one launch, boxes gated by their problem
    KKT_TRY(M.apply(Vj, Zj, s, &bw.st[0].active));
    static_assert(sizeof(GmresState) % sizeof(int) == 0, "state stride");
    (void)kStride;
    for (int k = 0; k < np; ++k) {
      const long long o = bw.off[k], nk = bw.off[k + 1] - o;
      const int* act = &bw.st[k].active;
      const Small sm = small_of(bw, k);
      KKT_TRY(A[k]->apply(Zj + o, ws.w + o, s, act));
      KKT_TRY(multidot(ws.V + o, N, j + 1, ws.w + o, nk, ws.part, sm.h, s, act));
      multi_axpy<<<kVecBlocks, 256, 0, s>>>(ws.w + o, ws.V + o, N, sm.h, j + 1, nk, act);
      KKT_TRY(launched());
      KKT_TRY(multidot(ws.V + o, N, j + 1, ws.w + o, nk, ws.part, sm.h2, s, act));
      multi_axpy<<<kVecBlocks, 256, 0, s>>>(ws.w + o, ws.V + o, N, sm.h2, j + 1, nk, act);
      KKT_TRY(launched());
      KKT_TRY(multidot(ws.w + o, 0, 1, ws.w + o, nk, ws.part, sm.h + j + 1, s, act));
      gm_givens<<<1, 32, 0, s>>>(bw.st + k, j, m, sm.h, sm.h2, sm.H, sm.cs, sm.sn, sm.g);
      KKT_TRY(launched());
      if (j + 1 < m) {
        scale_dev<<<kVecBlocks, 256, 0, s>>>(ws.V + (size_t)(j + 1) * N + o, ws.w + o, &bw.st[k].inv, nk, act);
        KKT_TRY(launched());
      }
    }
  }
  if (g_capture) g_capture->step = -1;
  for (int k = 0; k < np; ++k) {
    const long long o = bw.off[k], nk = bw.off[k + 1] - o;
    const Small sm = small_of(bw, k);
    gm_solve_y<<<1, 32, 0, s>>>(bw.st + k, m, sm.H, sm.g, sm.y);
    KKT_TRY(launched());
    multi_update<<<kVecBlocks, 256, 0, s>>>(x + o, ws.Z + o, N, sm.y, &bw.st[k].k, nk, &bw.st[k].ran);
    KKT_TRY(launched());
    // true residual of problem k and its squared norm
    KKT_TRY(A[k]->apply(x + o, ws.w + o, s, nullptr));
    KKT_TRY(vec_copy(ws.r + o, b + o, nk, s));
    KKT_TRY(vec_axpby(ws.r + o, -1.0, ws.w + o, 1.0, nk, s));
    KKT_TRY(multidot(ws.r + o, 0, 1, ws.r + o, nk, ws.part, &bw.st[k].r2, s, nullptr));
  }
  return KKT_OK;
}

}  // namespace

kkt_status gmres_run_batch(std::vector<Operator*>& A, Operator& M, const double* b, double* x, BatchWork& bw,
                           int restart, double rtol, int maxit, std::vector<GmresResult>& res, cudaStream_t s,
                           bool graph) {
  GmresWork& ws = bw.ws;
  const int np = (int)bw.off.size() - 1;
  const int m = restart;
  if (m > ws.m || (int)A.size() != np) {
    set_error("gmres_solve_batch: restart longer than the workspace or operator count mismatch");
    return KKT_ERR_ARG;
  }
  res.assign(np, GmresResult{});
  // ||b_k||, zero guess: r = b
  KKT_TRY(vec_zero(x, ws.n, s));
  KKT_TRY(vec_copy(ws.r, b, ws.n, s));
  for (int k = 0; k < np; ++k) {
    const long long o = bw.off[k], nk = bw.off[k + 1] - o;
    KKT_TRY(multidot(b + o, 0, 1, b + o, nk, ws.part, &bw.st[k].b2, s, nullptr));
    KKT_TRY(multidot(b + o, 0, 1, b + o, nk, ws.part, &bw.st[k].r2, s, nullptr));
    gm_init<<<1, 32, 0, s>>>(bw.st + k, rtol, maxit, nullptr);
    KKT_TRY(launched());
  }
  KKT_TRY_CUDA(cudaMemcpyAsync(bw.st_host, bw.st, np * sizeof(GmresState), cudaMemcpyDeviceToHost, s));
  KKT_TRY_CUDA(cudaStreamSynchronize(s));
  std::vector<char> done(np, 0);
  for (int k = 0; k < np; ++k) {
    const double bn = bw.st_host[k].bnorm;
    if (!std::isfinite(bn)) {
      res[k].status = KKT_ERR_NONFINITE;
      done[k] = 1;
    } else if (bn == 0.0) {
      res[k].status = KKT_OK;
      done[k] = 1;
    }
  }
  unsigned long long key[10] = {M.uid(), (unsigned long long)(uintptr_t)b, (unsigned long long)(uintptr_t)x,
                                (unsigned long long)m, (unsigned long long)g_timing_on.load(),
                                (unsigned long long)(uintptr_t)ws.V, (unsigned long long)np, 2ull, 0ull, 0ull};
  for (int k = 0; k < np; ++k) key[8] = key[8] * 1000003ull + A[k]->uid();
  for (;;) {
    bool any = false;
    for (int k = 0; k < np; ++k) any = any || !done[k];
    if (!any) break;
    if (graph) {
      if (!ws.graph.exec || std::memcmp(ws.graph.key, key, sizeof(key)) != 0)
        KKT_TRY(capture_cycle(ws, m, key, 2 * np + 2, [&](cudaStream_t cs) {
          return enqueue_cycle_batch(A, M, b, x, bw, m, cs);
        }));
      KKT_TRY_CUDA(cudaGraphLaunch(ws.graph.exec, s));
    } else {
      KKT_TRY(enqueue_cycle_batch(A, M, b, x, bw, m, s));
    }
    KKT_TRY_CUDA(cudaMemcpyAsync(bw.st_host, bw.st, np * sizeof(GmresState), cudaMemcpyDeviceToHost, s));
    KKT_TRY_CUDA(cudaStreamSynchronize(s));
    int steps = 0;
    for (int k = 0; k < np; ++k) steps = std::max(steps, bw.st_host[k].steps);
    if (graph) KKT_TRY(after_replay(ws.graph, steps));
    for (int k = 0; k < np; ++k) {
      if (done[k]) continue;
      const GmresState& h = bw.st_host[k];
      const double beta = std::sqrt(h.r2);
      res[k].iters = h.iters;
      res[k].relres = beta / h.bnorm;
      if (h.flag == kGmNonFinite || !std::isfinite(beta)) {
        res[k].status = KKT_ERR_NONFINITE;
        done[k] = 1;
      } else if (beta <= rtol * h.bnorm) {
        res[k].status = KKT_OK;
        done[k] = 1;
      } else if (h.flag == kGmBreakdown) {
        res[k].status = KKT_BREAKDOWN;
        done[k] = 1;
      } else if (h.iters >= maxit || h.steps == 0) {
        res[k].status = KKT_NOT_CONVERGED;
        done[k] = 1;
      }
    }
  }
  return KKT_OK;
}
