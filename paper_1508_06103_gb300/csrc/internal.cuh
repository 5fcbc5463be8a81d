// Internal declarations shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>

#include <atomic>
#include <cstdint>
#include <string>
#include <utility>
#include <vector>

#include "stkkt.h"

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
// Records an event pair around the launches issued in its scope when timing is on.
struct TimedScope {
  TimingLog* log;
  cudaStream_t s;
  cudaEvent_t e0 = nullptr;
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
  double hx, hy, hz;                        // mesh widths (B and K are tensor products of 1D factors)
  const double *S, *ST, *B, *K;             // [27][N] row coefficients (FP64)
  const float *S32, *ST32, *B32, *K32;      // FP32 copies
  const unsigned char* dir;                 // [N] 1 on Dirichlet nodes
  const double* sens;                       // [N] sensor counts, 0 on Dirichlet nodes
};

struct GmresWork {
  long long n = 0;
  int m = 0;
  bool flexible = false;
  double* V = nullptr;      // (m+1) * n
  double* Z = nullptr;      // m * n (flexible)
  double* w = nullptr;      // n
  double* r = nullptr;      // n
  double* hbuf = nullptr;   // device scalars: 2 * (m+2)
  double* part = nullptr;   // partial sums
  double* hhost = nullptr;  // pinned host mirror
  int nparts = 0;
  kkt_status alloc(long long n_, int m_, bool flex);
  void release();
};

struct kkt_problem {
  kkt_grid grid;
  int nx, ny, nz, N, M, L;
  long long P, n;                           // points, unknowns
  double hx, hy, hz, tau, T, theta, beta1, beta2;
  int reg = 0;                              // kkt_set_regularization
  // host copies used by the coarse level
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

// matvec.cu
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
struct Operator {
  virtual ~Operator() = default;
  virtual kkt_status apply(const double* x, double* y, cudaStream_t s) = 0;
};

struct GmresResult {
  int iters = 0;
  double relres = 0.0;
  kkt_status status = KKT_OK;
};

// Restarted right-preconditioned (F)GMRES with CGS2 on device vectors.
// `check_true` = form the true residual to confirm convergence.
kkt_status gmres_run(Operator& A, Operator* M, const double* b, double* x, GmresWork& ws, int restart,
                     double rtol, int maxit, bool check_true, bool zero_guess, GmresResult* res,
                     cudaStream_t s);

kkt_status vec_copy(double* y, const double* x, long long n, cudaStream_t s);
kkt_status vec_zero(double* y, long long n, cudaStream_t s);
kkt_status vec_axpby(double* y, double a, const double* x, double b, long long n, cudaStream_t s);
