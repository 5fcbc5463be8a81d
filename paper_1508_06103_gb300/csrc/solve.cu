// Two-level space-time Schwarz preconditioner and the outer solver (Sec. 3.2, 4).
//
// Coarse level.  The coarse space-time mesh is nested in the fine one (every
// coarse node and level is a fine node and level).  The coarse operator F_c is
// rediscretised on it: a and v of a coarse cell are the means over its fine
// cells and each fine sensor node goes to the nearest coarse node (ties toward
// the lower index).  Interpolation I^h_c is multilinear in (x, y, z, t) and
// acts on C, G and f alike; restriction is its transpose I^c_h = (I^h_c)^T.
//
// Two-level multiplicative hybrid:
//   y = I^h_c F_c^{-1} I^c_h x,   z = y + M_one^{-1} (x - F_h y),
// where F_c^{-1} is GMRES right-preconditioned by the coarse one-level RAS,
// stopped at relative residual c_rtol or after c_maxit iterations; since it
// changes with x the outer solver is flexible GMRES.

#include <algorithm>
#include <cmath>
#include <vector>

#include "internal.cuh"
#include "ras.cuh"

struct coarse_level {
  unsigned long long uid = next_handle_uid();
  kkt_problem* fine = nullptr;
  kkt_problem* cp = nullptr;         // coarse problem (owned)
  ras_precond* cras = nullptr;       // coarse one-level RAS (owned)
  int rx = 1, ry = 1, rz = 1, rt = 1;
  double c_rtol = 0.1;
  int c_maxit = 4;
  double *rc = nullptr, *yc = nullptr, *y = nullptr, *t = nullptr;
  int prec = 64;                     // precision of everything inside the preconditioner
  float *cx32 = nullptr, *cy32 = nullptr;   // coarse FP32 scratch
  float *fx32 = nullptr, *fy32 = nullptr;   // fine FP32 scratch
  GmresWork ws;
  cudaStream_t aux = nullptr;        // two_level_refactor: stream of the coarse factorisation
  cudaEvent_t fork = nullptr, join = nullptr;
};

namespace {

struct Grid4 {
  int nx, ny, nz, L, N;
};

// fine y = I^h_c yc (multilinear in x, y, z, t); one thread per fine point.
// Per axis the fine index i = I r + rem takes (1 - rem/r) of coarse I and
// rem/r of coarse I + 1 (the second weight is 0 on coarse points).  A is the
// arithmetic type: FP64, or FP32 inside the mixed-precision preconditioner
// (vectors stay FP64 in memory).
template <typename A>
__global__ void interp_kernel(Grid4 f, Grid4 c, int rx, int ry, int rz, int rt, const double* __restrict__ yc,
                              double* __restrict__ y, const int* gate) {
  if (gated_off(gate)) return;
  const long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (idx >= (long long)f.N * f.L) return;
  const int n = (int)(idx / f.N);
  const int j = (int)(idx - (long long)n * f.N);
  const int ix = j % f.nx, iy = (j / f.nx) % f.ny, iz = j / (f.nx * f.ny);
  const int X0 = ix / rx, Y0 = iy / ry, Z0 = iz / rz, T0 = n / rt;
  const A wx = (A)(ix - X0 * rx) / (A)rx, wy = (A)(iy - Y0 * ry) / (A)ry;
  const A wz = (A)(iz - Z0 * rz) / (A)rz, wt = (A)(n - T0 * rt) / (A)rt;
  const int X1 = wx > 0 ? X0 + 1 : X0, Y1 = wy > 0 ? Y0 + 1 : Y0, Z1 = wz > 0 ? Z0 + 1 : Z0, T1 = wt > 0 ? T0 + 1 : T0;
  const int xs[2] = {X0, X1}, ys[2] = {Y0, Y1}, zs[2] = {Z0, Z1}, ts[2] = {T0, T1};
  const A wxs[2] = {(A)1 - wx, wx}, wys[2] = {(A)1 - wy, wy}, wzs[2] = {(A)1 - wz, wz}, wts[2] = {(A)1 - wt, wt};
  A a0 = 0, a1 = 0, a2 = 0;
#pragma unroll
  for (int at = 0; at < 2; ++at)
#pragma unroll
    for (int az = 0; az < 2; ++az)
#pragma unroll
      for (int ay = 0; ay < 2; ++ay) {
        const A w3 = wts[at] * wzs[az] * wys[ay];
        const double* src = yc + 3 * ((long long)ts[at] * c.N + c.nx * (ys[ay] + c.ny * zs[az]));
#pragma unroll
        for (int ax = 0; ax < 2; ++ax) {
          const A w = w3 * wxs[ax];
          const double* q = src + 3 * xs[ax];
          a0 += w * (A)q[0];
          a1 += w * (A)q[1];
          a2 += w * (A)q[2];
        }
      }
  y[3 * idx] = a0;
  y[3 * idx + 1] = a1;
  y[3 * idx + 2] = a2;
}

// coarse rc = (I^h_c)^T x; one thread per coarse point gathers its fine
// support: fine index I r + a, |a| < r, weight 1 - |a|/r per axis.  A as in
// interp_kernel.
template <typename A>
__global__ void restrict_kernel(Grid4 f, Grid4 c, int rx, int ry, int rz, int rt, const double* __restrict__ x,
                                double* __restrict__ rc, const int* gate) {
  if (gated_off(gate)) return;
  const long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (idx >= (long long)c.N * c.L) return;
  const int n = (int)(idx / c.N);
  const int j = (int)(idx - (long long)n * c.N);
  const int I = j % c.nx, J = (j / c.nx) % c.ny, K = j / (c.nx * c.ny);
  const int x0 = max(I * rx - rx + 1, 0), x1 = min(I * rx + rx - 1, f.nx - 1);
  const int y0 = max(J * ry - ry + 1, 0), y1 = min(J * ry + ry - 1, f.ny - 1);
  const int z0 = max(K * rz - rz + 1, 0), z1 = min(K * rz + rz - 1, f.nz - 1);
  const int t0 = max(n * rt - rt + 1, 0), t1 = min(n * rt + rt - 1, f.L - 1);
  const A irx = (A)1 / (A)rx, iry = (A)1 / (A)ry, irz = (A)1 / (A)rz, irt = (A)1 / (A)rt;
  A a0 = 0, a1 = 0, a2 = 0;
  for (int ft = t0; ft <= t1; ++ft) {
    const A wt = (A)1 - (A)abs(ft - n * rt) * irt;
    for (int fz = z0; fz <= z1; ++fz) {
      const A wz = wt * ((A)1 - (A)abs(fz - K * rz) * irz);
      for (int fy = y0; fy <= y1; ++fy) {
        const A wy = wz * ((A)1 - (A)abs(fy - J * ry) * iry);
        const double* row = x + 3 * ((long long)ft * f.N + f.nx * (fy + f.ny * fz));
        for (int fx = x0; fx <= x1; ++fx) {
          const A w = wy * ((A)1 - (A)abs(fx - I * rx) * irx);
          const double* q = row + 3 * fx;
          a0 += w * (A)q[0];
          a1 += w * (A)q[1];
          a2 += w * (A)q[2];
        }
      }
    }
  }
  rc[3 * idx] = a0;
  rc[3 * idx + 1] = a1;
  rc[3 * idx + 2] = a2;
}

Grid4 grid_of(const kkt_problem* p) { return Grid4{p->nx, p->ny, p->nz, p->L, p->N}; }

// The outer operator: FP64 KKT matvec (timed for the roofline report).
struct KktOp : Operator {
  kkt_problem* p;
  explicit KktOp(kkt_problem* p_) : p(p_) {}
  kkt_status apply(const double* x, double* y, cudaStream_t s, const int* gate) override {
    TimedScope t(&p->mv_timing, s);
    DevProblem d = p->dev();
    d.gate = gate;
    return launch_matvec64(d, x, y, s);
  }
  unsigned long long uid() const override { return p->uid * 4 + (unsigned long long)(p->reg + 2 * p->elem); }
};

// The coarse operator inside the preconditioner: FP64, or FP32 arithmetic on
// FP64 vectors in the mixed form.
struct CoarseOp : Operator {
  kkt_problem* p;
  int prec;
  float *x32, *y32;
  CoarseOp(kkt_problem* p_, int prec_, float* a, float* b) : p(p_), prec(prec_), x32(a), y32(b) {}
  kkt_status apply(const double* x, double* y, cudaStream_t s, const int* gate) override {
    DevProblem d = p->dev();
    d.gate = gate;
    if (prec == 64) return launch_matvec64(d, x, y, s);
    return launch_matvec32_d(d, x, y, x32, y32, s);
  }
  unsigned long long uid() const override { return p->uid * 4 + (unsigned long long)(p->reg + 2 * p->elem); }
};

struct RasOp : Operator {
  ras_precond* m;
  explicit RasOp(ras_precond* m_) : m(m_) {}
  kkt_status apply(const double* x, double* y, cudaStream_t s, const int* gate) override {
    return ras_launch(m, x, y, s, gate);
  }
  unsigned long long uid() const override { return m->uid; }
};

// The multiplicative two-level hybrid; every kernel returns at once while
// *gate reads 0 (the coarse GMRES is gated by its own state, which starts
// only when *gate is live).
kkt_status two_level(coarse_level* c, ras_precond* fine, const double* x, double* z, cudaStream_t s,
                     const int* gate) {
  kkt_problem* pf = c->fine;
  kkt_problem* pc = c->cp;
  const Grid4 gf = grid_of(pf), gc = grid_of(pc);
  const unsigned rblocks = (unsigned)((pc->P + 255) / 256), iblocks = (unsigned)((pf->P + 255) / 256);
  if (c->prec == 64)
    restrict_kernel<double><<<rblocks, 256, 0, s>>>(gf, gc, c->rx, c->ry, c->rz, c->rt, x, c->rc, gate);
  else
    restrict_kernel<float><<<rblocks, 256, 0, s>>>(gf, gc, c->rx, c->ry, c->rz, c->rt, x, c->rc, gate);
  KKT_COUNT(1);
  KKT_TRY_CUDA(cudaGetLastError());
  CoarseOp Ac(pc, c->prec, c->cx32, c->cy32);
  RasOp Mc(c->cras);
  GmresResult r;
  KKT_TRY(gmres_run(Ac, &Mc, c->rc, c->yc, c->ws, c->c_maxit, c->c_rtol, c->c_maxit, false, true, &r, s, gate));
  if (c->prec == 64)
    interp_kernel<double><<<iblocks, 256, 0, s>>>(gf, gc, c->rx, c->ry, c->rz, c->rt, c->yc, c->y, gate);
  else
    interp_kernel<float><<<iblocks, 256, 0, s>>>(gf, gc, c->rx, c->ry, c->rz, c->rt, c->yc, c->y, gate);
  KKT_COUNT(1);
  KKT_TRY_CUDA(cudaGetLastError());
  DevProblem df = pf->dev();
  df.gate = gate;
  if (c->prec == 64) KKT_TRY(launch_residual(df, x, c->y, c->t, s));   // t = x - F_h y
  else KKT_TRY(launch_residual32(df, x, c->y, c->t, c->fx32, c->fy32, s));
  KKT_TRY(ras_launch(fine, c->t, z, s, gate));
  KKT_TRY(vec_axpby(z, 1.0, c->y, 1.0, pf->n, s, gate));   // z = M^{-1} t + y
  return KKT_OK;
}

// The one-level RAS of several problems: one subdomain solve over all their
// boxes, box b gated by its problem's FGMRES state.
struct BatchRasOp : Operator {
  ras_precond* m;
  explicit BatchRasOp(ras_precond* m_) : m(m_) {}
  kkt_status apply(const double* x, double* y, cudaStream_t s, const int* gate) override {
    return ras_launch(m, x, y, s, gate, gate ? (int)(sizeof(GmresState) / sizeof(int)) : 0);
  }
  unsigned long long uid() const override { return m->uid; }
};

struct TwoLevelOp : Operator {
  coarse_level* c;
  ras_precond* fine;
  TwoLevelOp(coarse_level* c_, ras_precond* f_) : c(c_), fine(f_) {}
  kkt_status apply(const double* x, double* y, cudaStream_t s, const int* gate) override {
    return two_level(c, fine, x, y, s, gate);
  }
  unsigned long long uid() const override { return (c->uid << 32) ^ fine->uid; }
};

}  // namespace

extern "C" kkt_status coarse_setup(kkt_problem* fine, int ccx, int ccy, int ccz, int cnt, const int nsub_c[4],
                                   int c_overlap, double c_rtol, int c_maxit, int factor_prec, coarse_level** out) {
  NvtxRange nvtx_("coarse_setup");
  if (!fine || !nsub_c || !out) {
    set_error("coarse_setup: null argument");
    return KKT_ERR_ARG;
  }
  *out = nullptr;
  const kkt_grid& g = fine->grid;
  if (ccx < 1 || ccy < 1 || ccz < 1 || cnt < 1 || g.cx % ccx || g.cy % ccy || g.cz % ccz || fine->M % cnt ||
      c_maxit < 1 || !(c_rtol > 0)) {
    set_error("coarse_setup: the coarse mesh must be nested (divisors of the fine cells and steps)");
    return KKT_ERR_ARG;
  }
  coarse_level* c = new (std::nothrow) coarse_level();
  if (!c) return KKT_ERR_NOMEM;
  c->fine = fine;
  c->rx = g.cx / ccx;
  c->ry = g.cy / ccy;
  c->rz = g.cz / ccz;
  c->rt = fine->M / cnt;
  c->c_rtol = c_rtol;
  c->c_maxit = c_maxit;
  c->prec = factor_prec == 64 ? 64 : 32;   // FP32 arithmetic with FP32 or BF16-stored factors
  // coarse coefficients: cell means of the fine cells
  const int ncc = ccx * ccy * ccz;
  std::vector<double> ac(ncc, 0.0), vc(3 * (size_t)ncc, 0.0);
  const double inv = 1.0 / ((double)c->rx * c->ry * c->rz);
  for (int ez = 0; ez < g.cz; ++ez)
    for (int ey = 0; ey < g.cy; ++ey)
      for (int ex = 0; ex < g.cx; ++ex) {
        const int e = ex + g.cx * (ey + g.cy * ez);
        const int E = ex / c->rx + ccx * (ey / c->ry + ccy * (ez / c->rz));
        ac[E] += inv * fine->a_cell[e];
        for (int d = 0; d < 3; ++d) vc[3 * (size_t)E + d] += inv * fine->v_cell[3 * (size_t)e + d];
      }
  // sensors: nearest coarse node of each fine sensor node, ties toward the lower index
  std::vector<int> sc(fine->sensor_node.size());
  auto snap = [](int i, int r) { return (i + (r - 1) / 2) / r; };
  for (size_t q = 0; q < sc.size(); ++q) {
    const int j = fine->sensor_node[q];
    const int ix = j % fine->nx, iy = (j / fine->nx) % fine->ny, iz = j / (fine->nx * fine->ny);
    sc[q] = snap(ix, c->rx) + (ccx + 1) * (snap(iy, c->ry) + (ccy + 1) * snap(iz, c->rz));
  }
  kkt_grid cg = g;
  cg.cx = ccx;
  cg.cy = ccy;
  cg.cz = ccz;
  kkt_status st = create_problem(&cg, cnt, fine->tau * c->rt, ac.data(), vc.data(), sc.empty() ? nullptr : sc.data(),
                                 (int)sc.size(), fine->beta1, fine->beta2, fine->theta, &c->cp);
  if (st == KKT_OK) c->cp->reg = fine->reg;   // the coarse operator is the same discretisation
  if (st == KKT_OK && fine->elem != KKT_ELEM_Q1) st = kkt_set_element(c->cp, fine->elem);
  if (st == KKT_OK) st = ras_create(&c->cp, 1, nsub_c, c_overlap, 0, factor_prec, nullptr, &c->cras);
  // The coarse GMRES keeps z_j = M_c^{-1} v_j (the flexible form's store, c_maxit
  // coarse vectors) and forms y_c = Z y: for its fixed preconditioner this is
  // the right-preconditioned iterate M_c^{-1} V y with one application less.
  if (st == KKT_OK) st = c->ws.alloc(c->cp->n, c_maxit, true);
  if (st == KKT_OK &&
      (cudaMalloc(&c->rc, c->cp->n * sizeof(double)) != cudaSuccess ||
       cudaMalloc(&c->yc, c->cp->n * sizeof(double)) != cudaSuccess ||
       cudaMalloc(&c->y, fine->n * sizeof(double)) != cudaSuccess ||
       cudaMalloc(&c->t, fine->n * sizeof(double)) != cudaSuccess ||
       (c->prec == 32 && (cudaMalloc(&c->cx32, c->cp->n * sizeof(float)) != cudaSuccess ||
                          cudaMalloc(&c->cy32, c->cp->n * sizeof(float)) != cudaSuccess ||
                          cudaMalloc(&c->fx32, fine->n * sizeof(float)) != cudaSuccess ||
                          cudaMalloc(&c->fy32, fine->n * sizeof(float)) != cudaSuccess)))) {
    cudaGetLastError();
    set_error("coarse_setup: device allocation failed");
    st = KKT_ERR_NOMEM;
  }
  if (st != KKT_OK) {
    coarse_destroy(c);
    return st;
  }
  *out = c;
  return KKT_OK;
}

extern "C" kkt_status two_level_apply(coarse_level* c, ras_precond* fine, const double* x, double* z, void* stream) {
  NvtxRange nvtx_("two_level_apply");
  if (!c || !fine || !x || !z || x == z) {
    set_error("two_level_apply: bad argument");
    return KKT_ERR_ARG;
  }
  if (fine->prob != c->fine) {
    set_error("two_level_apply: the fine preconditioner belongs to another problem");
    return KKT_ERR_ARG;
  }
  return two_level(c, fine, x, z, (cudaStream_t)stream, nullptr);
}

extern "C" kkt_status coarse_refactor(coarse_level* c, void* stream) {
  NvtxRange nvtx_("coarse_refactor");
  if (!c) {
    set_error("coarse_refactor: null argument");
    return KKT_ERR_ARG;
  }
  return ras_factor(c->cras, (cudaStream_t)stream);
}

extern "C" kkt_status two_level_refactor(coarse_level* c, ras_precond* fine, void* stream) {
  if (!c || !fine || fine->prob != c->fine) {
    set_error("two_level_refactor: bad argument");
    return KKT_ERR_ARG;
  }
  const cudaStream_t s = (cudaStream_t)stream;
  if (!c->aux) {
    KKT_TRY_CUDA(cudaStreamCreateWithFlags(&c->aux, cudaStreamNonBlocking));
    KKT_TRY_CUDA(cudaEventCreateWithFlags(&c->fork, cudaEventDisableTiming));
    KKT_TRY_CUDA(cudaEventCreateWithFlags(&c->join, cudaEventDisableTiming));
  }
  // the coarse factorisation fills the SMs the fine one leaves idle
  KKT_TRY_CUDA(cudaEventRecord(c->fork, s));
  KKT_TRY_CUDA(cudaStreamWaitEvent(c->aux, c->fork, 0));
  KKT_TRY(ras_factor_enqueue(fine, s));
  KKT_TRY(ras_factor_enqueue(c->cras, c->aux));
  KKT_TRY_CUDA(cudaEventRecord(c->join, c->aux));
  KKT_TRY_CUDA(cudaStreamWaitEvent(s, c->join, 0));
  KKT_TRY_CUDA(cudaStreamSynchronize(s));
  KKT_TRY(ras_factor_status(fine));
  return ras_factor_status(c->cras);
}

extern "C" void coarse_destroy(coarse_level* c) {
  if (!c) return;
  if (c->aux) cudaStreamDestroy(c->aux);
  if (c->fork) cudaEventDestroy(c->fork);
  if (c->join) cudaEventDestroy(c->join);
  ras_destroy(c->cras);
  kkt_destroy(c->cp);
  cudaFree(c->rc);
  cudaFree(c->yc);
  cudaFree(c->y);
  cudaFree(c->t);
  cudaFree(c->cx32);
  cudaFree(c->cy32);
  cudaFree(c->fx32);
  cudaFree(c->fy32);
  c->ws.release();
  delete c;
}

extern "C" kkt_status gmres_solve(kkt_problem* p, ras_precond* m, coarse_level* c, const double* b, double* x,
                                  int restart, double rtol, int maxit, int flexible, int* iters, double* true_relres,
                                  void* stream) {
  NvtxRange nvtx_("gmres_solve");
  if (!p || !b || !x || b == x || restart < 1 || maxit < 0 || !(rtol > 0)) {
    set_error("gmres_solve: bad argument");
    return KKT_ERR_ARG;
  }
  if (c && (!m || !flexible)) {
    set_error("gmres_solve: the two-level method needs a fine RAS and flexible GMRES");
    return KKT_ERR_ARG;
  }
  if ((m && m->prob != p) || (c && c->fine != p)) {
    set_error("gmres_solve: preconditioner built for another problem");
    return KKT_ERR_ARG;
  }
  cudaStream_t s = (cudaStream_t)stream;
  if (!p->ws) {
    p->ws = new (std::nothrow) GmresWork();
    if (!p->ws) return KKT_ERR_NOMEM;
  }
  GmresWork& ws = *p->ws;
  KKT_TRY(ws.alloc(p->n, restart, flexible != 0));
  KktOp A(p);
  RasOp R(m);
  TwoLevelOp T(c, m);
  Operator* M = c ? (Operator*)&T : (m ? (Operator*)&R : nullptr);
  GmresResult res;
  KKT_TRY(gmres_run(A, M, b, x, ws, restart, rtol, maxit, true, false, &res, s, nullptr, true));
  if (m) KKT_TRY(ras_check(m));
  if (c) KKT_TRY(ras_check(c->cras));
  if (iters) *iters = res.iters;
  if (true_relres) *true_relres = res.relres;
  return res.status;
}

extern "C" kkt_status gmres_solve_batch(kkt_problem* const* probs, int nprob, ras_precond* m, const double* b,
                                        double* x, int restart, double rtol, int maxit, int* iters,
                                        double* true_relres, int* status, void* stream) {
  NvtxRange nvtx_("gmres_solve_batch");
  if (!probs || nprob < 1 || !m || !b || !x || restart < 1 || maxit < 0 || !(rtol > 0)) {
    set_error("gmres_solve_batch: bad argument");
    return KKT_ERR_ARG;
  }
  if ((int)m->probs.size() != nprob || !std::equal(m->probs.begin(), m->probs.end(), probs)) {
    set_error("gmres_solve_batch: the preconditioner was set up for another list of problems");
    return KKT_ERR_ARG;
  }
  if (spans_overlap(b, x, m->n_total)) {
    set_error("gmres_solve_batch: b and x must not overlap");
    return KKT_ERR_ARG;
  }
  if (!m->bw) {
    m->bw = new (std::nothrow) BatchWork();
    if (!m->bw) return KKT_ERR_NOMEM;
  }
  KKT_TRY(m->bw->alloc(m->vec_off, restart));
  std::vector<KktOp> ops;
  ops.reserve(nprob);
  std::vector<Operator*> A;
  for (int k = 0; k < nprob; ++k) {
    ops.emplace_back(probs[k]);
    A.push_back(&ops.back());
  }
  BatchRasOp M(m);
  std::vector<GmresResult> res;
  KKT_TRY(gmres_run_batch(A, M, b, x, *m->bw, restart, rtol, maxit, res, (cudaStream_t)stream, true));
  KKT_TRY(ras_check(m));
  kkt_status worst = KKT_OK;
  for (int k = 0; k < nprob; ++k) {
    if (iters) iters[k] = res[k].iters;
    if (true_relres) true_relres[k] = res[k].relres;
    if (status) status[k] = res[k].status;
    if (res[k].status < 0 && (worst >= 0 || res[k].status < worst)) worst = res[k].status;
    else if (worst >= 0 && res[k].status > worst) worst = res[k].status;
  }
  if (worst < 0) set_error("gmres_solve_batch: a problem met a non-finite value");
  return worst;
}
