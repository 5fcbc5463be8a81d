// Internal declarations shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>

#include <atomic>
#include <cstdint>
#include <string>
#include <utility>
#include <vector>

#include "stkkt.h"

// NVTX ranges around the library's host entry points (tracing under a
// profiler; no-ops without one attached): the header-only NVTX 3 C API of
// the CUDA toolkit, left out where the toolkit has no such header.
#if defined(__has_include)
#if __has_include(<nvtx3/nvToolsExt.h>)
#include <nvtx3/nvToolsExt.h>
#define KKT_HAVE_NVTX 1
#endif
#endif
struct NvtxRange {
  explicit NvtxRange(const char* name) {
#ifdef KKT_HAVE_NVTX
    nvtxRangePushA(name);
#else
    (void)name;
#endif
  }
  ~NvtxRange() {
#ifdef KKT_HAVE_NVTX
    nvtxRangePop();
#endif
  }
  NvtxRange(const NvtxRange&) = delete;
  NvtxRange& operator=(const NvtxRange&) = delete;
};

void set_error(const std::string& msg);

#define KKT_TRY_CUDA(call)                                                        \
  do {                                                                            \
    cudaError_t err_ = (call);                                                    \
    if (err_ != cudaSuccess) {                                                    \
      set_error(std::string(#call) + ": " + cudaGetErrorString(err_));            \
      return KKT_ERR_CUDA;                                                        \
    }                                                                             \
  } while (0)

#define KKT_TRY(call)                 \
  do {                                \
    kkt_status st_ = (call);          \
    if (st_ < 0) return st_;          \
  } while (0)

// True when the spans [a, a + n) and [b, b + n) of doubles share an element.
inline bool spans_overlap(const double* a, const double* b, long long n) {
  const uintptr_t pa = (uintptr_t)a, pb = (uintptr_t)b, len = (uintptr_t)n * sizeof(double);
  return pa < pb + len && pb < pa + len;
}

// Count of kernel launches made by the library (kkt_launch_count).
extern std::atomic<long long> g_kernel_launches;
#define KKT_COUNT(n) g_kernel_launches.fetch_add((n), std::memory_order_relaxed)

// CUDA-event timing of selected launches (kkt_timing_enable / *_timing_read).
extern std::atomic<int> g_timing_on;
struct TimingLog {
  std::vector<std::pair<cudaEvent_t, cudaEvent_t>> pending;
  double total_ms = 0.0;
  long long count = 0;
  void drain();            // synchronise on pending events and accumulate
  void reset();
  ~TimingLog();
};

// Timing of launches captured into a CUDA graph (an FGMRES cycle): the event
// pairs are created before the capture, recorded as graph nodes, and read
// after every replay; each pair is tagged with the outer Arnoldi step whose
// launches it brackets, so pairs of steps the cycle skipped (after it
// converged, their kernels return at once) are not counted.
struct CaptureTiming {
  struct Entry {
    TimingLog* log;
    int step;                // outer step, -1 outside the steps (counted always)
    cudaEvent_t e0, e1;
  };
  std::vector<std::pair<cudaEvent_t, cudaEvent_t>> pool;   // created before the capture
  size_t used = 0;
  std::vector<Entry> entries;
  int step = -1;             // step being captured
  void clear();
  ~CaptureTiming() { clear(); }
};
extern thread_local CaptureTiming* g_capture;   // set while this thread captures a cycle

// Records an event pair around the launches issued in its scope when timing is on.
struct TimedScope {
  TimingLog* log;
  cudaStream_t s;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  bool captured = false;
  TimedScope(TimingLog* l, cudaStream_t st);
  ~TimedScope();
};

// 27-point stencil offsets: d = (dx+1) + 3 (dy+1) + 9 (dz+1), centre d = 13.
constexpr int kStencil = 27;
constexpr int kCentre = 13;

// Everything a kernel needs to evaluate F_h on one problem (passed by value).
struct DevProblem {
  int nx, ny, nz, N, M, L;
  long long P;                              // points N * (M+1)
  double tau, theta, beta1, beta2;
  int reg;                                  // beta2 term: 0 stiffness K (H1-H1), 1 mass B (H1-L2)
  int elem;                                 // KKT_ELEM_Q1 or KKT_ELEM_P1 (kkt_set_element)
  double hx, hy, hz;                        // mesh widths (Q1: B and K are tensor products of 1D factors)
  const double *S, *ST, *B, *K;             // [27][N] row coefficients (FP64)
  const float *S32, *ST32, *B32, *K32;      // FP32 copies
  const unsigned char* dir;                 // [N] 1 on Dirichlet nodes
  const double* sens;                       // [N] sensor counts, 0 on Dirichlet nodes
  const int* gate;                          // device flag: the kernels return at once when it reads 0
                                            // (an Arnoldi step after convergence); nullptr = always run
};

// True when a gated kernel should return without work.
__device__ __forceinline__ bool gated_off(const int* gate) { return gate != nullptr && *gate == 0; }

// Device state of one (F)GMRES instance: the Givens rotations, residual
// estimate and stop test run on the device, so a restart cycle needs no host
// round trip (and can be captured into a CUDA graph).
enum GmresFlag : int { kGmRunning = 0, kGmConverged = 1, kGmBreakdown = 2, kGmNonFinite = 3, kGmLimit = 4 };
struct GmresState {
  double bnorm;            // ||b||
  double beta;             // residual norm at the start of the cycle
  double rtol;
  double est;              // Arnoldi residual estimate / ||b||
  double inv;              // 1 / the norm the next Arnoldi vector is scaled by
  double b2, r2;           // squared norms of b and of the residual (dot results)
  int k;                   // columns of the least-squares problem of the cycle
  int active;              // gate of the cycle's kernels
  int ran;                 // gate of the update after the cycle (k > 0)
  int steps;               // Arnoldi steps executed in this cycle
  int iters;               // steps of all cycles
  int maxit;
  int flag;                // GmresFlag
  int pad_;
};

// A captured restart cycle of the outer solver and what it was captured for.
struct CycleGraph {
  cudaGraphExec_t exec = nullptr;
  unsigned long long key[10] = {};
  long long launches = 0;    // kernel launches per replay
  CaptureTiming timing;
  void release();
};

struct GmresWork {
  long long n = 0;
  int m = 0;
  bool flexible = false;
  double* V = nullptr;      // (m+1) * n
  double* Z = nullptr;      // m * n (flexible)
  double* w = nullptr;      // n
  double* r = nullptr;      // n
  double* hbuf = nullptr;   // device: h, h2 (m+2 each), y (m), cs, sn (m), g (m+1), H ((m+1) m)
  GmresState* st = nullptr; // device state
  GmresState* st_host = nullptr;   // pinned host mirror
  double* part = nullptr;   // partial sums
  int nparts = 0;
  cudaStream_t cap = nullptr;      // stream the outer cycle is captured on
  CycleGraph graph;
  kkt_status alloc(long long n_, int m_, bool flex);
  void release();
  double* h() const { return hbuf; }
  double* h2() const { return hbuf + (m + 2); }
  double* y() const { return hbuf + 2 * (m + 2); }
  double* cs() const { return y() + m; }
  double* sn() const { return cs() + m; }
  double* g() const { return sn() + m; }
  double* H() const { return g() + (m + 1); }
  static size_t doubles(int m_) { return 2 * (size_t)(m_ + 2) + 3 * (size_t)m_ + (m_ + 1) + (size_t)(m_ + 1) * m_; }
};

// Identity of a handle for the cache of captured graphs (never reused).
unsigned long long next_handle_uid();

struct kkt_problem {
  unsigned long long uid = next_handle_uid();
  kkt_grid grid;
  int nx, ny, nz, N, M, L;
  long long P, n;                           // points, unknowns
  double hx, hy, hz, tau, T, theta, beta1, beta2;
  int reg = 0;                              // kkt_set_regularization
  int elem = 0;                             // kkt_set_element
  // host copies used by the coarse level and by kkt_set_element
  std::vector<double> a_cell, v_cell;
  std::vector<int> sensor_node;
  // device memory
  double* coef64 = nullptr;                 // S, ST, B, K   (4 * 27 * N)
  float* coef32 = nullptr;                  // FP32 copies
  unsigned char* dir = nullptr;
  double* sens = nullptr;
  int* sens_ptr = nullptr;                  // CSR: sensors of each node (N+1)
  int* sens_idx = nullptr;                  // sensor ids ordered by node
  int nsens = 0;
  GmresWork* ws = nullptr;                  // outer Krylov workspace (lazily allocated)
  TimingLog mv_timing;                      // outer FP64 matvec launches
  DevProblem dev() const;
};

// matvec.cu (kernels return at once while *p.gate reads 0)
kkt_status matvec_prepare();   // raises the kernels' shared-memory limit on the current device
kkt_status launch_matvec64(const DevProblem& p, const double* x, double* y, cudaStream_t s);
kkt_status launch_matvec32(const DevProblem& p, const float* x, float* y, cudaStream_t s);
kkt_status launch_residual(const DevProblem& p, const double* b, const double* x, double* r, cudaStream_t s);
kkt_status launch_residual32(const DevProblem& p, const double* b, const double* x, double* r,
                             float* x32, float* y32, cudaStream_t s);
kkt_status launch_matvec32_d(const DevProblem& p, const double* x, double* y, float* x32, float* y32,
                             cudaStream_t s);

// problem.cu
kkt_status create_problem(const kkt_grid* g, int nt, double dt, const double* a_cell, const double* v_cell,
                          const int* sensor_node, int nsens, double beta1, double beta2, double theta,
                          kkt_problem** out);

// krylov.cu -- device vector helpers used by the solvers
// An operator y = A x enqueued on stream s; its kernels return at once while
// *gate reads 0 (gate nullptr: always run).
struct Operator {
  virtual ~Operator() = default;
  virtual kkt_status apply(const double* x, double* y, cudaStream_t s, const int* gate) = 0;
  virtual unsigned long long uid() const = 0;   // identity for the graph cache
};

struct GmresResult {
  int iters = 0;
  double relres = 0.0;
  kkt_status status = KKT_OK;
};

// Restarted right-preconditioned (F)GMRES with CGS2 on device vectors, the
// Givens rotations and stop test on the device.  The outer form
// (check_true: stop on the true residual) runs one host round trip per
// restart cycle, replaying the cycle as a captured CUDA graph when `graph`;
// the inner form (!check_true, zero guess, one cycle: the coarse solve)
// only enqueues its kernels, gated by `parent` (the outer step's gate).
kkt_status gmres_run(Operator& A, Operator* M, const double* b, double* x, GmresWork& ws, int restart,
                     double rtol, int maxit, bool check_true, bool zero_guess, GmresResult* res,
                     cudaStream_t s, const int* parent = nullptr, bool graph = false);

// Workspace of gmres_run_batch: one FGMRES workspace over the concatenated
// unknowns of all problems, one state and set of small arrays per problem.
struct BatchWork {
  GmresWork ws;
  std::vector<long long> off;   // nprob + 1 offsets of the problems' unknowns
  GmresState* st = nullptr;     // device, one per problem
  GmresState* st_host = nullptr;
  double* small = nullptr;      // device, GmresWork::doubles(m) per problem
  kkt_status alloc(const std::vector<long long>& off_, int m_);
  void release();
  ~BatchWork() { release(); }
};

// Flexible GMRES on several independent problems in lockstep (one captured
// cycle for all when `graph`); A[k] is problem k's operator on its part of the
// concatenated vectors, M the preconditioner of all problems, whose kernels
// read the gate of problem k at stride sizeof(GmresState) ints; res[k] gets
// problem k's iterations, true relative residual and status.
kkt_status gmres_run_batch(std::vector<Operator*>& A, Operator& M, const double* b, double* x, BatchWork& bw,
                           int restart, double rtol, int maxit, std::vector<GmresResult>& res, cudaStream_t s,
                           bool graph);

kkt_status vec_copy(double* y, const double* x, long long n, cudaStream_t s, const int* gate = nullptr);
kkt_status vec_zero(double* y, long long n, cudaStream_t s);
kkt_status vec_axpby(double* y, double a, const double* x, double b, long long n, cudaStream_t s,
                     const int* gate = nullptr);
