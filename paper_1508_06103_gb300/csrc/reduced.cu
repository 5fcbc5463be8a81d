// The reduced-space ("traditional") method of Sec. 1 on the GPU: the source f
// is the only unknown; for a given f the state comes from a forward march of
// the time steps of Eq. 8, the adjoint from a backward march driven by the
// data misfit, and the first-order condition of the f rows (Eq. 9, Appendix)
//
//     H f = W f - D G_lin(C_lin(f)) = g,   g = D G0,
//     W = beta1 Lt (x) B + beta2 Mt (x) K  (H1-L2: Mt (x) B),  D = Mt (x) B,
//
// is solved by right-preconditioned GMRES.  Each application of H is two
// sequential sweeps of M spatial solves, the cost the all-at-once method of
// the paper avoids.  (C, G, f) is then the KKT solution of F_h U = b.
//
// Spatial step solves: (B + theta tau S) x = r (state) and (B + theta tau S^T)
// x = r (adjoint), identity rows on the Dirichlet nodes; GMRES with Jacobi
// preconditioning on the device, one restart cycle per captured graph replay,
// from the neighbouring level as the initial guess.
//
// Preconditioner of the outer GMRES: P = W + sigma Mt (x) B applied by fast
// diagonalisation.  Under trilinear elements on the uniform grid B and K are
// Kronecker products of the 1D linear-element mass and stiffness matrices, so
// P = (V (x) U)^{-T} diag(beta1 lt + beta2 (lx + ly + lz) + sigma) (V (x) U)^{-1}
// with the generalised eigenvectors of the 1D pairs (Lt, Mt) in time and
// (Kx, Mx) per axis; P^{-1} is four dense 1D transforms each way around a
// diagonal scaling.  Under P1 elements on the Kuhn split the same P (built
// from the trilinear 1D factors) is only an approximation of the regulariser:
// it changes the iteration count, not the solution.

#include <algorithm>
#include <cmath>
#include <vector>

#include "internal.cuh"

namespace {

// ---------------------------------------------------------------------------
// Level kernels (one thread per node j = ix + nx (iy + ny iz)).
// ---------------------------------------------------------------------------

struct LevelGrid {
  int nx, ny, nz, N;
};

__device__ __forceinline__ bool nbr(const LevelGrid& g, int j, int d, int& k) {
  const int ix = j % g.nx, iy = (j / g.nx) % g.ny, iz = j / (g.nx * g.ny);
  const int x = ix + d % 3 - 1, y = iy + (d / 3) % 3 - 1, z = iz + d / 9 - 1;
  if (x < 0 || x >= g.nx || y < 0 || y >= g.ny || z < 0 || z >= g.nz) return false;
  k = x + g.nx * (y + g.ny * z);
  return true;
}

// y = (B + w A) x with A = S (state) or S^T (adjoint) from its row stencils;
// identity rows on the Dirichlet nodes.
__global__ void step_apply(LevelGrid g, const double* __restrict__ B, const double* __restrict__ A, double w,
                           const unsigned char* __restrict__ dir, const double* __restrict__ x,
                           double* __restrict__ y, const int* gate) {
  if (gated_off(gate)) return;
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= g.N) return;
  if (dir[j]) {
    y[j] = x[j];
    return;
  }
  double acc = 0.0;
  for (int d = 0; d < kStencil; ++d) {
    int k;
    if (nbr(g, j, d, k)) acc += (B[(size_t)d * g.N + j] + w * A[(size_t)d * g.N + j]) * x[k];
  }
  y[j] = acc;
}

// inv[j] = 1 / diagonal of (B + w A) (1 on the Dirichlet nodes)
__global__ void step_diag_inv(LevelGrid g, const double* __restrict__ B, const double* __restrict__ A, double w,
                              const unsigned char* __restrict__ dir, double* __restrict__ inv) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= g.N) return;
  constexpr int c = 13;   // the centre offset (0, 0, 0)
  inv[j] = dir[j] ? 1.0 : 1.0 / (B[(size_t)c * g.N + j] + w * A[(size_t)c * g.N + j]);
}

__global__ void scale_by(const double* __restrict__ inv, const double* __restrict__ x, double* __restrict__ y,
                         int N, const int* gate) {
  if (gated_off(gate)) return;
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j < N) y[j] = inv[j] * x[j];
}

// Right-hand side of state step n (Eq. 8, theta scheme):
//   r = (B - (1-theta) tau S) C^{n-1} + tau B ((1-theta) f^{n-1} + theta f^n),  r = 0 on Dirichlet nodes.
__global__ void rhs_state(LevelGrid g, const double* __restrict__ B, const double* __restrict__ S, double tau,
                          double theta, const unsigned char* __restrict__ dir, const double* __restrict__ Cm,
                          const double* __restrict__ fm, const double* __restrict__ f0, double* __restrict__ r) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= g.N) return;
  if (dir[j]) {
    r[j] = 0.0;
    return;
  }
  const double th1 = 1.0 - theta;
  double acc = 0.0;
  for (int d = 0; d < kStencil; ++d) {
    int k;
    if (!nbr(g, j, d, k)) continue;
    const double b = B[(size_t)d * g.N + j], s = S[(size_t)d * g.N + j];
    acc += (b - th1 * tau * s) * Cm[k] + tau * b * (th1 * fm[k] + theta * f0[k]);
  }
  r[j] = acc;
}

// Right-hand side of adjoint step n (the G rows of the Appendix, n < M):
//   r = (B - (1-theta) tau S^T) G^{n+1} - tau ((1-theta) m^n + theta m^{n+1}),
//   m^l_j = s_j C^l_j - sum of the observations c_obs[l, k] of the sensors k at node j
// (no observation term when c_obs is null), r = 0 on Dirichlet nodes.
__global__ void rhs_adjoint(LevelGrid g, const double* __restrict__ B, const double* __restrict__ ST, double tau,
                            double theta, const unsigned char* __restrict__ dir, const double* __restrict__ sens,
                            const int* __restrict__ sptr, const int* __restrict__ sidx,
                            const double* __restrict__ Gp, const double* __restrict__ C0,
                            const double* __restrict__ Cp, const double* __restrict__ obs0,
                            const double* __restrict__ obsp, double* __restrict__ r) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= g.N) return;
  if (dir[j]) {
    r[j] = 0.0;
    return;
  }
  const double th1 = 1.0 - theta;
  double acc = 0.0;
  for (int d = 0; d < kStencil; ++d) {
    int k;
    if (nbr(g, j, d, k)) acc += (B[(size_t)d * g.N + j] - th1 * tau * ST[(size_t)d * g.N + j]) * Gp[k];
  }
  double m0 = sens[j] * C0[j], mp = sens[j] * Cp[j];
  if (obs0 != nullptr)
    for (int q = sptr[j]; q < sptr[j + 1]; ++q) {
      m0 -= obs0[sidx[q]];
      mp -= obsp[sidx[q]];
    }
  r[j] = acc - tau * (th1 * m0 + theta * mp);
}

// U (point-block order) = (C, G, f) from three level-major fields; a null
// field gives zeros.
__global__ void interleave(const double* __restrict__ C, const double* __restrict__ G,
                           const double* __restrict__ f, double* __restrict__ U, long long P) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i >= P) return;
  U[3 * i] = C ? C[i] : 0.0;
  U[3 * i + 1] = G ? G[i] : 0.0;
  U[3 * i + 2] = f ? f[i] : 0.0;
}

__global__ void take_f(const double* __restrict__ U, double* __restrict__ f, long long P, double sign) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i < P) f[i] = sign * U[3 * i + 2];
}

// out = (A or A^T along one axis of the 4D array [t][z][y][x]) in, A n x n
// row-major; one thread per output value.
__global__ void mode_product(const double* __restrict__ A, int n, bool transpose, long long inner,
                             long long total, const double* __restrict__ in, double* __restrict__ out,
                             const int* gate) {
  if (gated_off(gate)) return;
  const long long o = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (o >= total) return;
  const long long lo = o % inner, rest = o / inner;
  const int i = (int)(rest % n);
  const long long base = (rest / n) * n * inner + lo;
  double acc = 0.0;
  for (int k = 0; k < n; ++k) acc += (transpose ? A[(size_t)k * n + i] : A[(size_t)i * n + k]) * in[base + k * inner];
  out[o] = acc;
}

__global__ void scale_div(const double* __restrict__ dg, double* __restrict__ x, long long n, const int* gate) {
  if (gated_off(gate)) return;
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i < n) x[i] /= dg[i];
}

unsigned blocks_for(long long n, int t) { return (unsigned)((n + t - 1) / t); }

}  // namespace

namespace {

// ---------------------------------------------------------------------------
// Host: generalised symmetric eigenproblems K u = lambda M u of the 1D
// linear-element pairs, by a Cholesky factor of M and cyclic Jacobi rotations
// on L^{-1} K L^{-T} (n <= a few hundred).
// ---------------------------------------------------------------------------

// 1D linear-element mass and stiffness on n_cells uniform cells of width h (dense, row-major)
void mass_stiff_1d(int n_cells, double h, std::vector<double>& Mx, std::vector<double>& Kx) {
  const int n = n_cells + 1;
  Mx.assign((size_t)n * n, 0.0);
  Kx.assign((size_t)n * n, 0.0);
  for (int e = 0; e < n_cells; ++e)
    for (int a = 0; a < 2; ++a)
      for (int b = 0; b < 2; ++b) {
        const size_t ij = (size_t)(e + a) * n + (e + b);
        Mx[ij] += h / 6.0 * (a == b ? 2.0 : 1.0);
        Kx[ij] += (a == b ? 1.0 : -1.0) / h;
      }
}

// U (n x n, row-major, columns the eigenvectors, U^T M U = I) and lambda.
bool gen_eig(int n, const std::vector<double>& Kx, const std::vector<double>& Mx, std::vector<double>& U,
             std::vector<double>& lam) {
  // Cholesky M = L L^T
  std::vector<double> L((size_t)n * n, 0.0);
  for (int i = 0; i < n; ++i)
    for (int j = 0; j <= i; ++j) {
      double s = Mx[(size_t)i * n + j];
      for (int k = 0; k < j; ++k) s -= L[(size_t)i * n + k] * L[(size_t)j * n + k];
      if (i == j) {
        if (!(s > 0)) return false;
        L[(size_t)i * n + i] = std::sqrt(s);
      } else {
        L[(size_t)i * n + j] = s / L[(size_t)j * n + j];
      }
    }
  // C = L^{-1} K L^{-T}: first X = L^{-1} K (forward substitution per column), then C = L^{-1} X^T
  auto lsolve = [&](std::vector<double>& Y) {   // Y <- L^{-1} Y, Y n x n row-major, column by column
    for (int c = 0; c < n; ++c)
      for (int i = 0; i < n; ++i) {
        double s = Y[(size_t)i * n + c];
        for (int k = 0; k < i; ++k) s -= L[(size_t)i * n + k] * Y[(size_t)k * n + c];
        Y[(size_t)i * n + c] = s / L[(size_t)i * n + i];
      }
  };
  std::vector<double> X = Kx;
  lsolve(X);
  std::vector<double> C((size_t)n * n);
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) C[(size_t)i * n + j] = X[(size_t)j * n + i];
  lsolve(C);
  for (int i = 0; i < n; ++i)   // symmetrise the rounding
    for (int j = 0; j < i; ++j) {
      const double v = 0.5 * (C[(size_t)i * n + j] + C[(size_t)j * n + i]);
      C[(size_t)i * n + j] = C[(size_t)j * n + i] = v;
    }
  // cyclic Jacobi: C <- J^T C J until the off-diagonal part vanishes; Q accumulates J
  std::vector<double> Q((size_t)n * n, 0.0);
  for (int i = 0; i < n; ++i) Q[(size_t)i * n + i] = 1.0;
  for (int sweep = 0; sweep < 100; ++sweep) {
    double off = 0.0, tot = 0.0;
    for (int i = 0; i < n; ++i)
      for (int j = 0; j < n; ++j) {
        const double v = C[(size_t)i * n + j] * C[(size_t)i * n + j];
        tot += v;
        if (i != j) off += v;
      }
    if (off <= 1e-30 * tot) break;
    for (int p = 0; p < n - 1; ++p)
      for (int q = p + 1; q < n; ++q) {
        const double apq = C[(size_t)p * n + q];
        if (apq == 0.0) continue;
        const double app = C[(size_t)p * n + p], aqq = C[(size_t)q * n + q];
        const double tau = (aqq - app) / (2.0 * apq);
        const double t = (tau >= 0 ? 1.0 : -1.0) / (std::fabs(tau) + std::sqrt(1.0 + tau * tau));
        const double c = 1.0 / std::sqrt(1.0 + t * t), s = t * c;
        for (int k = 0; k < n; ++k) {   // columns p, q
          const double ckp = C[(size_t)k * n + p], ckq = C[(size_t)k * n + q];
          C[(size_t)k * n + p] = c * ckp - s * ckq;
          C[(size_t)k * n + q] = s * ckp + c * ckq;
        }
        for (int k = 0; k < n; ++k) {   // rows p, q
          const double cpk = C[(size_t)p * n + k], cqk = C[(size_t)q * n + k];
          C[(size_t)p * n + k] = c * cpk - s * cqk;
          C[(size_t)q * n + k] = s * cpk + c * cqk;
        }
        for (int k = 0; k < n; ++k) {
          const double qkp = Q[(size_t)k * n + p], qkq = Q[(size_t)k * n + q];
          Q[(size_t)k * n + p] = c * qkp - s * qkq;
          Q[(size_t)k * n + q] = s * qkp + c * qkq;
        }
      }
  }
  lam.resize(n);
  for (int i = 0; i < n; ++i) lam[i] = C[(size_t)i * n + i];
  // U = L^{-T} Q: back substitution with L^T per column
  U = Q;
  for (int c = 0; c < n; ++c)
    for (int i = n - 1; i >= 0; --i) {
      double s = U[(size_t)i * n + c];
      for (int k = i + 1; k < n; ++k) s -= L[(size_t)k * n + i] * U[(size_t)k * n + c];
      U[(size_t)i * n + c] = s / L[(size_t)i * n + i];
    }
  return true;
}

}  // namespace

namespace {

// ---------------------------------------------------------------------------
// Operators and the two marches
// ---------------------------------------------------------------------------

struct StepOp : Operator {   // B + theta tau S (state) or B + theta tau S^T (adjoint)
  const kkt_problem* p;
  bool adjoint;
  unsigned long long id = next_handle_uid();
  StepOp(const kkt_problem* p_, bool adj) : p(p_), adjoint(adj) {}
  kkt_status apply(const double* x, double* y, cudaStream_t s, const int* gate) override {
    const DevProblem d = p->dev();
    const LevelGrid g{p->nx, p->ny, p->nz, p->N};
    step_apply<<<blocks_for(p->N, 256), 256, 0, s>>>(g, d.B, adjoint ? d.ST : d.S, p->theta * p->tau, d.dir, x, y,
                                                      gate);
    KKT_COUNT(1);
    KKT_TRY_CUDA(cudaGetLastError());
    return KKT_OK;
  }
  unsigned long long uid() const override { return id; }
};

struct JacobiOp : Operator {
  const double* inv;
  int N;
  unsigned long long id = next_handle_uid();
  JacobiOp(const double* i, int n) : inv(i), N(n) {}
  kkt_status apply(const double* x, double* y, cudaStream_t s, const int* gate) override {
    scale_by<<<blocks_for(N, 256), 256, 0, s>>>(inv, x, y, N, gate);
    KKT_COUNT(1);
    KKT_TRY_CUDA(cudaGetLastError());
    return KKT_OK;
  }
  unsigned long long uid() const override { return id; }
};

// P^{-1} of the regulariser by fast diagonalisation (see the file header).
struct FastDiagOp : Operator {
  int dims[4];          // L, nz, ny, nx
  double* mats[4] = {}; // device n x n eigenvector matrices: time, z, y, x
  double* dg = nullptr; // device diagonal over the 4D array
  double* tmp = nullptr;
  long long total = 0;
  unsigned long long id = next_handle_uid();
  kkt_status init(const kkt_problem* p) {
    dims[0] = p->L;
    dims[1] = p->nz;
    dims[2] = p->ny;
    dims[3] = p->nx;
    total = p->P;
    std::vector<double> lam[4];
    const int cells[4] = {p->M, p->grid.cz, p->grid.cy, p->grid.cx};
    const double h[4] = {p->tau, p->hz, p->hy, p->hx};
    for (int a = 0; a < 4; ++a) {
      std::vector<double> Mx, Kx, U;
      mass_stiff_1d(cells[a], h[a], Mx, Kx);
      if (!gen_eig(cells[a] + 1, Kx, Mx, U, lam[a])) {
        set_error("reduced_solve: 1D mass matrix not positive definite");
        return KKT_ERR_ARG;
      }
      KKT_TRY_CUDA(cudaMalloc(&mats[a], U.size() * sizeof(double)));
      KKT_TRY_CUDA(cudaMemcpy(mats[a], U.data(), U.size() * sizeof(double), cudaMemcpyHostToDevice));
    }
    std::vector<double> base((size_t)total);
    double bmax = 0.0;
    size_t o = 0;
    for (int t = 0; t < dims[0]; ++t)
      for (int z = 0; z < dims[1]; ++z)
        for (int y = 0; y < dims[2]; ++y)
          for (int x = 0; x < dims[3]; ++x, ++o) {
            const double space = p->reg == 0 ? lam[1][z] + lam[2][y] + lam[3][x] : 1.0;
            base[o] = p->beta1 * lam[0][t] + p->beta2 * space;
            bmax = std::max(bmax, base[o]);
          }
    // sigma: 1e-3 of the smallest non-zero eigenvalue (the constant source is in W's null space)
    double bmin = bmax;
    for (double v : base)
      if (v > 1e-12 * bmax) bmin = std::min(bmin, v);
    const double sigma = 1e-3 * (bmax > 0 ? bmin : 1.0);
    for (double& v : base) v += sigma;
    KKT_TRY_CUDA(cudaMalloc(&dg, total * sizeof(double)));
    KKT_TRY_CUDA(cudaMalloc(&tmp, total * sizeof(double)));
    KKT_TRY_CUDA(cudaMemcpy(dg, base.data(), total * sizeof(double), cudaMemcpyHostToDevice));
    return KKT_OK;
  }
  ~FastDiagOp() override {
    for (double* m : mats) cudaFree(m);
    cudaFree(dg);
    cudaFree(tmp);
  }
  // y <- (A_t (x) A_z (x) A_y (x) A_x) x with A = U^T (forward) or U; ping-pong between y and tmp
  kkt_status transform(const double* x, double* y, bool forward, cudaStream_t s, const int* gate) {
    const double* in = x;
    long long inner = total;
    double* outs[4] = {tmp, y, tmp, y};
    for (int a = 0; a < 4; ++a) {
      inner /= dims[a];
      mode_product<<<blocks_for(total, 256), 256, 0, s>>>(mats[a], dims[a], forward, inner, total, in, outs[a],
                                                          gate);
      KKT_COUNT(1);
      in = outs[a];
    }
    KKT_TRY_CUDA(cudaGetLastError());
    return KKT_OK;
  }
  kkt_status apply(const double* x, double* y, cudaStream_t s, const int* gate) override {
    KKT_TRY(transform(x, y, true, s, gate));
    scale_div<<<blocks_for(total, 256), 256, 0, s>>>(dg, y, total, gate);
    KKT_COUNT(1);
    return transform(y, y, false, s, gate);
  }
  unsigned long long uid() const override { return id; }
};

// Everything one reduced-space solve needs (device buffers freed on exit).
struct Reduced {
  kkt_problem* p;
  cudaStream_t s;
  double step_rtol;
  int step_restart, step_maxit;
  StepOp state, adj;
  double *inv_state = nullptr, *inv_adj = nullptr;
  JacobiOp *jac_state = nullptr, *jac_adj = nullptr;
  GmresWork ws_state, ws_adj;       // step solves (each keeps its captured cycle)
  double *rb = nullptr, *xb = nullptr;   // fixed step right-hand side and iterate (the graphs' pointers)
  double *C = nullptr, *G = nullptr;     // level-major L x N
  double *U = nullptr, *Y = nullptr;     // point-block 3P scratch for the f rows
  const double* c_obs = nullptr;         // device (M+1) x nsens, or null
  const double* c0 = nullptr;
  long long step_iters = 0, step_solves = 0;
  int step_iters_max = 0;
  long long hess_applies = 0;

  Reduced(kkt_problem* p_, cudaStream_t s_) : p(p_), s(s_), state(p_, false), adj(p_, true) {}
  ~Reduced() {
    delete jac_state;
    delete jac_adj;
    ws_state.release();
    ws_adj.release();
    for (double* b : {inv_state, inv_adj, rb, xb, C, G, U, Y}) cudaFree(b);
  }
  kkt_status init() {
    const long long N = p->N, P = p->P;
    KKT_TRY_CUDA(cudaMalloc(&inv_state, N * sizeof(double)));
    KKT_TRY_CUDA(cudaMalloc(&inv_adj, N * sizeof(double)));
    KKT_TRY_CUDA(cudaMalloc(&rb, N * sizeof(double)));
    KKT_TRY_CUDA(cudaMalloc(&xb, N * sizeof(double)));
    KKT_TRY_CUDA(cudaMalloc(&C, P * sizeof(double)));
    KKT_TRY_CUDA(cudaMalloc(&G, P * sizeof(double)));
    KKT_TRY_CUDA(cudaMalloc(&U, 3 * P * sizeof(double)));
    KKT_TRY_CUDA(cudaMalloc(&Y, 3 * P * sizeof(double)));
    const DevProblem d = p->dev();
    const LevelGrid g{p->nx, p->ny, p->nz, p->N};
    const double w = p->theta * p->tau;
    step_diag_inv<<<blocks_for(N, 256), 256, 0, s>>>(g, d.B, d.S, w, d.dir, inv_state);
    step_diag_inv<<<blocks_for(N, 256), 256, 0, s>>>(g, d.B, d.ST, w, d.dir, inv_adj);
    KKT_COUNT(2);
    KKT_TRY_CUDA(cudaGetLastError());
    jac_state = new JacobiOp(inv_state, p->N);
    jac_adj = new JacobiOp(inv_adj, p->N);
    KKT_TRY(ws_state.alloc(N, step_restart, false));
    KKT_TRY(ws_adj.alloc(N, step_restart, false));
    return KKT_OK;
  }

  // x_out = step matrix^{-1} rb from the initial guess x_in (fixed buffers rb, xb)
  kkt_status step_solve(bool adjoint, const double* x_in, double* x_out) {
    KKT_TRY(vec_copy(xb, x_in, p->N, s));
    GmresResult res;
    const kkt_status st = gmres_run(adjoint ? (Operator&)adj : (Operator&)state, adjoint ? jac_adj : jac_state, rb, xb,
                                    adjoint ? ws_adj : ws_state, step_restart, step_rtol, step_maxit, true, false,
                                    &res, s, nullptr, true);
    if (st != KKT_OK) return st;
    if (res.status != KKT_OK) {   // iteration limit or breakdown before step_rtol
      set_error("reduced_solve: a time-step solve did not reach its tolerance within its iteration limit");
      return res.status == KKT_BREAKDOWN ? KKT_BREAKDOWN : KKT_NOT_CONVERGED;
    }
    step_iters += res.iters;
    step_solves += 1;
    step_iters_max = std::max(step_iters_max, res.iters);
    return vec_copy(x_out, xb, p->N, s);
  }

  // C = states for sources f (L x N, null = 0) and initial state c0 (null = 0)
  kkt_status march_state(const double* f, const double* c0_, double* Cout) {
    const long long N = p->N;
    const DevProblem d = p->dev();
    const LevelGrid g{p->nx, p->ny, p->nz, p->N};
    if (c0_) {
      KKT_TRY(vec_copy(Cout, c0_, N, s));
      interleave_dir_zero(Cout);
    } else {
      KKT_TRY(vec_zero(Cout, N, s));
    }
    for (int n = 1; n <= p->M; ++n) {
      const double* fm = f ? f + (n - 1) * N : xb;
      const double* f0 = f ? f + n * N : xb;
      if (!f) KKT_TRY(vec_zero(xb, N, s));   // no source: a zero level in xb (overwritten by the solve)
      rhs_state<<<blocks_for(N, 256), 256, 0, s>>>(g, d.B, d.S, p->tau, p->theta, d.dir, Cout + (n - 1) * N, fm, f0,
                                                   rb);
      KKT_COUNT(1);
      KKT_TRY_CUDA(cudaGetLastError());
      KKT_TRY(step_solve(false, Cout + (n - 1) * N, Cout + n * N));
    }
    return KKT_OK;
  }

  // G = adjoint states for states Cin and observations obs ((M+1) x nsens, null = none)
  kkt_status march_adjoint(const double* Cin, const double* obs, double* Gout) {
    const long long N = p->N;
    const DevProblem d = p->dev();
    const LevelGrid g{p->nx, p->ny, p->nz, p->N};
    KKT_TRY(vec_zero(Gout + (long long)p->M * N, N, s));
    for (int n = p->M - 1; n >= 0; --n) {
      const double* o0 = obs ? obs + (long long)n * p->nsens : nullptr;
      const double* op = obs ? obs + (long long)(n + 1) * p->nsens : nullptr;
      rhs_adjoint<<<blocks_for(N, 256), 256, 0, s>>>(g, d.B, d.ST, p->tau, p->theta, d.dir, d.sens, p->sens_ptr,
                                                     p->sens_idx, Gout + (n + 1) * N, Cin + n * N, Cin + (n + 1) * N,
                                                     o0, op, rb);
      KKT_COUNT(1);
      KKT_TRY_CUDA(cudaGetLastError());
      KKT_TRY(step_solve(true, Gout + (n + 1) * N, Gout + n * N));
    }
    return KKT_OK;
  }

  // out = sign * (f rows of F_h at (., Gin, f)): -Mt (x) B G + W f, through the KKT matvec
  kkt_status f_rows(const double* Gin, const double* f, double* out, double sign) {
    interleave<<<blocks_for(p->P, 256), 256, 0, s>>>(nullptr, Gin, f, U, p->P);
    KKT_COUNT(1);
    KKT_TRY(launch_matvec64(p->dev(), U, Y, s));
    take_f<<<blocks_for(p->P, 256), 256, 0, s>>>(Y, out, p->P, sign);
    KKT_COUNT(1);
    KKT_TRY_CUDA(cudaGetLastError());
    return KKT_OK;
  }

  void interleave_dir_zero(double* level);
};

__global__ void zero_dirichlet(const unsigned char* __restrict__ dir, double* __restrict__ x, int N) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j < N && dir[j]) x[j] = 0.0;
}

void Reduced::interleave_dir_zero(double* level) {
  zero_dirichlet<<<blocks_for(p->N, 256), 256, 0, s>>>(p->dev().dir, level, p->N);
  KKT_COUNT(1);
}

struct HessOp : Operator {   // H f = W f - D G_lin(C_lin(f)): one forward and one backward march
  Reduced* r;
  unsigned long long id = next_handle_uid();
  explicit HessOp(Reduced* r_) : r(r_) {}
  kkt_status apply(const double* x, double* y, cudaStream_t s, const int* gate) override {
    if (gate != nullptr) {   // an Arnoldi step after convergence: skip the marches
      int on = 1;
      KKT_TRY_CUDA(cudaMemcpyAsync(&on, gate, sizeof(int), cudaMemcpyDeviceToHost, s));
      KKT_TRY_CUDA(cudaStreamSynchronize(s));
      if (on == 0) return KKT_OK;
    }
    KKT_TRY(r->march_state(x, nullptr, r->C));
    KKT_TRY(r->march_adjoint(r->C, nullptr, r->G));
    r->hess_applies += 1;
    return r->f_rows(r->G, x, y, 1.0);
  }
  unsigned long long uid() const override { return id; }
};

}  // namespace

extern "C" kkt_status reduced_solve(kkt_problem* p, const double* c_obs, const double* c0, double* U, int restart,
                                    double rtol, int maxit, double step_rtol, int* iters, double* relres,
                                    long long stats[4], void* stream) {
  NvtxRange nvtx_("reduced_solve");
  if (!p || !U || (p->nsens > 0 && !c_obs) || restart < 1 || maxit < 1 || !(rtol > 0) || !(step_rtol > 0)) {
    set_error("reduced_solve: null argument, or restart, maxit, rtol or step_rtol not positive");
    return KKT_ERR_ARG;
  }
  cudaStream_t s = (cudaStream_t)stream;
  Reduced r(p, s);
  r.step_rtol = step_rtol;
  r.step_restart = 40;
  r.step_maxit = 2000;
  KKT_TRY(r.init());
  // steps 1-2 of the method: the affine part (f = 0, the data) and g = D G0
  KKT_TRY(r.march_state(nullptr, c0, r.C));
  KKT_TRY(r.march_adjoint(r.C, c_obs, r.G));
  double *g = nullptr, *f = nullptr;
  KKT_TRY_CUDA(cudaMalloc(&g, p->P * sizeof(double)));
  if (cudaMalloc(&f, p->P * sizeof(double)) != cudaSuccess) {
    cudaGetLastError();
    cudaFree(g);
    set_error("reduced_solve: device allocation failed");
    return KKT_ERR_NOMEM;
  }
  struct Bufs {
    double *a, *b;
    ~Bufs() {
      cudaFree(a);
      cudaFree(b);
    }
  } bufs{g, f};
  KKT_TRY(r.f_rows(r.G, nullptr, g, -1.0));
  // step 3: GMRES on H f = g, right-preconditioned by the regulariser
  FastDiagOp P;
  KKT_TRY(P.init(p));
  HessOp H(&r);
  GmresWork wo;
  struct WsGuard {
    GmresWork& w;
    ~WsGuard() { w.release(); }
  } guard{wo};
  KKT_TRY(wo.alloc(p->P, restart, false));
  GmresResult res;
  KKT_TRY(gmres_run(H, &P, g, f, wo, restart, rtol, maxit, true, true, &res, s, nullptr, false));
  if (iters) *iters = res.iters;
  if (relres) *relres = res.relres;
  const kkt_status st = res.status;   // OK, NOT_CONVERGED or BREAKDOWN: U is written in every case
  // step 4: the state and adjoint of the solution, U = (C, G, f)
  KKT_TRY(r.march_state(f, c0, r.C));
  KKT_TRY(r.march_adjoint(r.C, c_obs, r.G));
  interleave<<<blocks_for(p->P, 256), 256, 0, s>>>(r.C, r.G, f, U, p->P);
  KKT_COUNT(1);
  KKT_TRY_CUDA(cudaGetLastError());
  KKT_TRY_CUDA(cudaStreamSynchronize(s));
  if (stats) {
    stats[0] = r.hess_applies;
    stats[1] = r.step_solves;
    stats[2] = r.step_iters;
    stats[3] = r.step_iters_max;
  }
  return st;
}
