// Problem set-up: stencil coefficients of the KKT blocks, right-hand side and
// source extraction (Sec. 3.1-3.2, Appendix).
//
// On the uniform box every trilinear element matrix is a tensor product of
// the 1D linear-element matrices on [0, h]:
//   mass      m(h)[a][b] = h/6 * (a == b ? 2 : 1)
//   stiffness k(h)[a][b] = (a == b ? 1 : -1) / h
//   derivative g[a][b]   = int psi_a psi_b' = (b == 1 ? +1/2 : -1/2)
// so a cell with constant a_e, v_e contributes, for test node a and trial b,
//   A: a_e (kx my mz + mx ky mz + mx my kz)
//   B: mx my mz,   K: the Laplacian part of A with a = 1
//   E_s (state convection, Eq. 8: row = test): sum_d v_e,d  G_d[a][b]
// where G_x[a][b] = g[ax][bx] my mz, etc.  The adjoint uses E_s^T, i.e.
// G_d[b][a].  Each node stores the 27 row coefficients of S = A + E_s,
// ST = A + E_s^T, B and K; the matvec and the subdomain factorisation read
// only these.

#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>

#include "internal.cuh"

static thread_local std::string g_last_error;
std::atomic<long long> g_kernel_launches{0};
std::atomic<int> g_timing_on{0};

void TimingLog::drain() {
  for (auto& ev : pending) {
    float ms = 0.f;
    if (cudaEventSynchronize(ev.second) == cudaSuccess && cudaEventElapsedTime(&ms, ev.first, ev.second) == cudaSuccess) {
      total_ms += ms;
      ++count;
    }
    cudaEventDestroy(ev.first);
    cudaEventDestroy(ev.second);
  }
  pending.clear();
}

void TimingLog::reset() {
  drain();
  total_ms = 0.0;
  count = 0;
}

TimingLog::~TimingLog() {
  for (auto& ev : pending) {
    cudaEventDestroy(ev.first);
    cudaEventDestroy(ev.second);
  }
}

TimedScope::TimedScope(TimingLog* l, cudaStream_t st) : log(l), s(st) {
  if (!g_timing_on.load()) return;
  if (g_capture) {
    // inside a graph capture: a pair made before the capture, read after each replay
    if (g_capture->used < g_capture->pool.size()) {
      const auto& pr = g_capture->pool[g_capture->used++];
      e0 = pr.first;
      e1 = pr.second;
      captured = true;
      // an external record becomes an event-record node of the graph (a plain
      // record in a capturing stream only orders the capture)
      cudaEventRecordWithFlags(e0, s, cudaEventRecordExternal);
    }
    return;
  }
  if (cudaEventCreate(&e0) == cudaSuccess) cudaEventRecord(e0, s);
  else e0 = nullptr;
}

TimedScope::~TimedScope() {
  if (!e0) return;
  if (captured) {
    cudaEventRecordWithFlags(e1, s, cudaEventRecordExternal);
    if (g_capture) g_capture->entries.push_back({log, g_capture->step, e0, e1});
    return;
  }
  if (cudaEventCreate(&e1) == cudaSuccess) {
    cudaEventRecord(e1, s);
    log->pending.emplace_back(e0, e1);
  } else {
    cudaEventDestroy(e0);
  }
}

unsigned long long next_handle_uid() {
  static std::atomic<unsigned long long> next{1};
  return next.fetch_add(1);
}

extern "C" long long kkt_launch_count(void) { return g_kernel_launches.load(); }
extern "C" int kkt_timing_enable(int on) { return g_timing_on.exchange(on ? 1 : 0); }

extern "C" kkt_status kkt_timing_read(kkt_problem* p, double* total_ms, long long* launches) {
  if (!p) {
    set_error("kkt_timing_read: null problem");
    return KKT_ERR_ARG;
  }
  p->mv_timing.drain();
  if (total_ms) *total_ms = p->mv_timing.total_ms;
  if (launches) *launches = p->mv_timing.count;
  return KKT_OK;
}

void set_error(const std::string& msg) { g_last_error = msg; }

extern "C" const char* kkt_last_error(void) { return g_last_error.c_str(); }
extern "C" const char* kkt_version(void) { return "stkkt 0.1 (sm_103a)"; }

DevProblem kkt_problem::dev() const {
  DevProblem d;
  d.nx = nx; d.ny = ny; d.nz = nz; d.N = N; d.M = M; d.L = L; d.P = P;
  d.tau = tau; d.theta = theta; d.beta1 = beta1; d.beta2 = beta2; d.reg = reg; d.elem = elem;
  d.hx = hx; d.hy = hy; d.hz = hz;
  const size_t c = (size_t)kStencil * N;
  d.S = coef64; d.ST = coef64 + c; d.B = coef64 + 2 * c; d.K = coef64 + 3 * c;
  d.S32 = coef32; d.ST32 = coef32 + c; d.B32 = coef32 + 2 * c; d.K32 = coef32 + 3 * c;
  d.dir = dir;
  d.sens = sens;
  d.gate = nullptr;
  return d;
}

namespace {

struct CellGeom {
  int cx, cy, cz, nx, ny, nz;
  double hx, hy, hz;
};

__device__ __forceinline__ double m1(double h, int a, int b) { return h / 6.0 * (a == b ? 2.0 : 1.0); }
__device__ __forceinline__ double k1(double h, int a, int b) { return (a == b ? 1.0 : -1.0) / h; }
__device__ __forceinline__ double g1(int /*a*/, int b) { return b == 1 ? 0.5 : -0.5; }

// One thread per node: sum the contributions of the (up to 8) cells around it.
__global__ void assemble_stencils(CellGeom g, const double* __restrict__ a_cell,
                                  const double* __restrict__ v_cell, double* __restrict__ S,
                                  double* __restrict__ ST, double* __restrict__ B, double* __restrict__ K) {
  const int N = g.nx * g.ny * g.nz;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  const int ix = i % g.nx, iy = (i / g.nx) % g.ny, iz = i / (g.nx * g.ny);
  double s[kStencil], st[kStencil], b[kStencil], k[kStencil];
  for (int d = 0; d < kStencil; ++d) s[d] = st[d] = b[d] = k[d] = 0.0;
  for (int ez = iz - 1; ez <= iz; ++ez) {
    if (ez < 0 || ez >= g.cz) continue;
    for (int ey = iy - 1; ey <= iy; ++ey) {
      if (ey < 0 || ey >= g.cy) continue;
      for (int ex = ix - 1; ex <= ix; ++ex) {
        if (ex < 0 || ex >= g.cx) continue;
        const int e = ex + g.cx * (ey + g.cy * ez);
        const double ae = a_cell[e];
        const double vx = v_cell[3 * e], vy = v_cell[3 * e + 1], vz = v_cell[3 * e + 2];
        const int ax = ix - ex, ay = iy - ey, az = iz - ez;   // local coords of the test node
        for (int bz = 0; bz < 2; ++bz)
          for (int by = 0; by < 2; ++by)
            for (int bx = 0; bx < 2; ++bx) {
              const int d = (ex + bx - ix + 1) + 3 * (ey + by - iy + 1) + 9 * (ez + bz - iz + 1);
              const double mx = m1(g.hx, ax, bx), my = m1(g.hy, ay, by), mz = m1(g.hz, az, bz);
              const double kx = k1(g.hx, ax, bx), ky = k1(g.hy, ay, by), kz = k1(g.hz, az, bz);
              const double lap = kx * my * mz + mx * ky * mz + mx * my * kz;
              const double conv = vx * g1(ax, bx) * my * mz + vy * mx * g1(ay, by) * mz + vz * mx * my * g1(az, bz);
              const double convT = vx * g1(bx, ax) * my * mz + vy * mx * g1(by, ay) * mz + vz * mx * my * g1(bz, az);
              s[d] += ae * lap + conv;
              st[d] += ae * lap + convT;
              b[d] += mx * my * mz;
              k[d] += lap;
            }
      }
    }
  }
  for (int d = 0; d < kStencil; ++d) {
    S[(size_t)d * N + i] = s[d];
    ST[(size_t)d * N + i] = st[d];
    B[(size_t)d * N + i] = b[d];
    K[(size_t)d * N + i] = k[d];
  }
}

// 8x8 matrices of one cell, local node l = lx + 2 ly + 4 lz:
//   Me[a][b] = int phi_a phi_b,  Ke[a][b] = int grad phi_a . grad phi_b,
//   G[d][a][b] = int (d phi_b / d x_d) phi_a.
struct CellMats {
  double Me[64], Ke[64], G[3][64];
};

// P1 elements on the Kuhn split of the cell (Sec. 3.1: piecewise-linear
// elements on a regular triangulation).  For each ordering (i, j, k) of the
// axes the tetrahedron {1 >= x_i/h_i >= x_j/h_j >= x_k/h_k >= 0} has the
// vertices 0, e_i, e_i + e_j, (1,1,1) and the barycentric coordinates
//   1 - s_i,  s_i - s_j,  s_j - s_k,  s_k      (s = x / h),
// whose gradients are constant.  With |T| = hx hy hz / 6 the closed forms are
//   mass |T| (1 + delta_ab) / 20,  stiffness |T| grad l_a . grad l_b,
//   convection |T| / 4 * d l_b / d x_d  (the mean of l_a is 1/4).
CellMats p1_cell_matrices(double hx, double hy, double hz) {
  CellMats m{};
  const double h[3] = {hx, hy, hz};
  const double T = hx * hy * hz / 6.0;
  const int perm[6][3] = {{0, 1, 2}, {0, 2, 1}, {1, 0, 2}, {1, 2, 0}, {2, 0, 1}, {2, 1, 0}};
  for (const auto& pm : perm) {
    const int i = pm[0], j = pm[1], k = pm[2];
    const int node[4] = {0, 1 << i, (1 << i) | (1 << j), 7};
    double g[4][3] = {};
    g[0][i] = -1.0 / h[i];
    g[1][i] = 1.0 / h[i];
    g[1][j] = -1.0 / h[j];
    g[2][j] = 1.0 / h[j];
    g[2][k] = -1.0 / h[k];
    g[3][k] = 1.0 / h[k];
    for (int a = 0; a < 4; ++a)
      for (int b = 0; b < 4; ++b) {
        const int ab = node[a] * 8 + node[b];
        m.Me[ab] += T * (a == b ? 2.0 : 1.0) / 20.0;
        m.Ke[ab] += T * (g[a][0] * g[b][0] + g[a][1] * g[b][1] + g[a][2] * g[b][2]);
        for (int d = 0; d < 3; ++d) m.G[d][ab] += 0.25 * T * g[b][d];
      }
  }
  return m;
}

// One thread per node: the stencils from the cell matrices of the (up to 8)
// cells around the node, with a and v constant per cell.
__global__ void assemble_from_cells(CellGeom g, CellMats cm, const double* __restrict__ a_cell,
                                    const double* __restrict__ v_cell, double* __restrict__ S,
                                    double* __restrict__ ST, double* __restrict__ B, double* __restrict__ K) {
  const int N = g.nx * g.ny * g.nz;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  const int ix = i % g.nx, iy = (i / g.nx) % g.ny, iz = i / (g.nx * g.ny);
  double s[kStencil], st[kStencil], b[kStencil], k[kStencil];
  for (int d = 0; d < kStencil; ++d) s[d] = st[d] = b[d] = k[d] = 0.0;
  for (int ez = iz - 1; ez <= iz; ++ez) {
    if (ez < 0 || ez >= g.cz) continue;
    for (int ey = iy - 1; ey <= iy; ++ey) {
      if (ey < 0 || ey >= g.cy) continue;
      for (int ex = ix - 1; ex <= ix; ++ex) {
        if (ex < 0 || ex >= g.cx) continue;
        const int e = ex + g.cx * (ey + g.cy * ez);
        const double ae = a_cell[e];
        const double vx = v_cell[3 * e], vy = v_cell[3 * e + 1], vz = v_cell[3 * e + 2];
        const int la = (ix - ex) + 2 * (iy - ey) + 4 * (iz - ez);   // local id of the test node
        for (int lb = 0; lb < 8; ++lb) {
          const int bx = lb & 1, by = (lb >> 1) & 1, bz = lb >> 2;
          const int d = (ex + bx - ix + 1) + 3 * (ey + by - iy + 1) + 9 * (ez + bz - iz + 1);
          const int ab = la * 8 + lb, ba = lb * 8 + la;
          const double kab = cm.Ke[ab];
          s[d] += ae * kab + vx * cm.G[0][ab] + vy * cm.G[1][ab] + vz * cm.G[2][ab];
          st[d] += ae * kab + vx * cm.G[0][ba] + vy * cm.G[1][ba] + vz * cm.G[2][ba];
          b[d] += cm.Me[ab];
          k[d] += kab;
        }
      }
    }
  }
  for (int d = 0; d < kStencil; ++d) {
    S[(size_t)d * N + i] = s[d];
    ST[(size_t)d * N + i] = st[d];
    B[(size_t)d * N + i] = b[d];
    K[(size_t)d * N + i] = k[d];
  }
}

__global__ void to_float(const double* __restrict__ x, float* __restrict__ y, size_t n) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    y[i] = (float)x[i];
}

__global__ void rhs_kernel(DevProblem p, const double* __restrict__ c_obs, int nsens, const double* __restrict__ c0,
                           const int* __restrict__ sptr, const int* __restrict__ sidx, double* __restrict__ b) {
  const long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (idx >= p.P) return;
  const int n = (int)(idx / p.N);
  const int j = (int)(idx - (long long)n * p.N);
  const bool dirj = p.dir[j] != 0;
  double bc = 0.0, bg = 0.0;
  if (n == 0 && c0 != nullptr && !dirj) bc = c0[j];
  if (n < p.M && !dirj) {
    double acc = 0.0;
    for (int q = sptr[j]; q < sptr[j + 1]; ++q) {
      const int k = sidx[q];
      acc += (1.0 - p.theta) * c_obs[(size_t)n * nsens + k] + p.theta * c_obs[(size_t)(n + 1) * nsens + k];
    }
    bg = p.tau * acc;
  }
  b[3 * idx] = bc;
  b[3 * idx + 1] = bg;
  b[3 * idx + 2] = 0.0;
}

__global__ void source_kernel(const double* __restrict__ U, double* __restrict__ f, long long P) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i < P) f[i] = U[3 * i + 2];
}

}  // namespace

// S, ST, B, K of the problem's element from its host a and v (FP64), and the
// FP32 copies; synchronous.
kkt_status assemble_coefficients(kkt_problem* p, const char* who) {
  const kkt_grid* g = &p->grid;
  const size_t ncell = (size_t)g->cx * g->cy * g->cz;
  const long long N = p->N;
  const size_t ncoef = 4 * (size_t)kStencil * N;
  double *d_a = nullptr, *d_v = nullptr;
  if (cudaMalloc(&d_a, ncell * sizeof(double)) != cudaSuccess ||
      cudaMalloc(&d_v, 3 * ncell * sizeof(double)) != cudaSuccess) {
    cudaGetLastError();
    cudaFree(d_a);
    set_error(std::string(who) + ": device allocation failed");
    return KKT_ERR_NOMEM;
  }
  cudaError_t e = cudaMemcpy(d_a, p->a_cell.data(), ncell * sizeof(double), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(d_v, p->v_cell.data(), 3 * ncell * sizeof(double), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) {
    CellGeom geo{g->cx, g->cy, g->cz, p->nx, p->ny, p->nz, p->hx, p->hy, p->hz};
    const size_t c = (size_t)kStencil * N;
    const unsigned blocks = (unsigned)((N + 127) / 128);
    if (p->elem == KKT_ELEM_P1)
      assemble_from_cells<<<blocks, 128>>>(geo, p1_cell_matrices(p->hx, p->hy, p->hz), d_a, d_v, p->coef64,
                                           p->coef64 + c, p->coef64 + 2 * c, p->coef64 + 3 * c);
    else
      assemble_stencils<<<blocks, 128>>>(geo, d_a, d_v, p->coef64, p->coef64 + c, p->coef64 + 2 * c,
                                         p->coef64 + 3 * c);
    to_float<<<1024, 256>>>(p->coef64, p->coef32, ncoef);
    KKT_COUNT(2);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  cudaFree(d_a);
  cudaFree(d_v);
  if (e != cudaSuccess) {
    set_error(std::string(who) + ": " + cudaGetErrorString(e));
    return KKT_ERR_CUDA;
  }
  return KKT_OK;
}

kkt_status create_problem(const kkt_grid* g, int nt, double dt, const double* a_cell, const double* v_cell,
                          const int* sensor_node, int nsens, double beta1, double beta2, double theta,
                          kkt_problem** out) {
  if (!g || !out || !a_cell || !v_cell || (nsens > 0 && !sensor_node)) {
    set_error("kkt_create: null argument");
    return KKT_ERR_ARG;
  }
  *out = nullptr;
  if (g->cx < 1 || g->cy < 1 || g->cz < 1 || nt < 1 || !(dt > 0) || !(g->lx > 0) || !(g->ly > 0) ||
      !(g->lz > 0) || nsens < 0 || !(theta >= 0.5 && theta <= 1.0) || !(beta1 >= 0) || !(beta2 >= 0) ||
      g->dirichlet_faces > 63u) {
    set_error("kkt_create: invalid grid, step, theta, beta or face mask");
    return KKT_ERR_ARG;
  }
  const long long nx = g->cx + 1, ny = g->cy + 1, nz = g->cz + 1;
  const long long N = nx * ny * nz;
  if (N > (1LL << 30) || N * (nt + 1LL) * 3LL > (1LL << 40)) {
    set_error("kkt_create: problem too large");
    return KKT_ERR_ARG;
  }
  const int ncell = g->cx * g->cy * g->cz;
  for (int q = 0; q < nsens; ++q)
    if (sensor_node[q] < 0 || sensor_node[q] >= N) {
      set_error("kkt_create: sensor node out of range");
      return KKT_ERR_ARG;
    }
  for (int e = 0; e < ncell; ++e)
    if (!std::isfinite(a_cell[e]) || !std::isfinite(v_cell[3 * e]) || !std::isfinite(v_cell[3 * e + 1]) ||
        !std::isfinite(v_cell[3 * e + 2])) {
      set_error("kkt_create: non-finite coefficient");
      return KKT_ERR_ARG;
    }

  kkt_problem* p = new (std::nothrow) kkt_problem();
  if (!p) return KKT_ERR_NOMEM;
  p->grid = *g;
  p->nx = (int)nx; p->ny = (int)ny; p->nz = (int)nz; p->N = (int)N;
  p->M = nt; p->L = nt + 1; p->P = N * (nt + 1LL); p->n = 3 * p->P;
  p->hx = g->lx / g->cx; p->hy = g->ly / g->cy; p->hz = g->lz / g->cz;
  p->tau = dt; p->T = dt * nt; p->theta = theta; p->beta1 = beta1; p->beta2 = beta2;
  p->a_cell.assign(a_cell, a_cell + ncell);
  p->v_cell.assign(v_cell, v_cell + 3 * (size_t)ncell);
  p->sensor_node.assign(sensor_node, sensor_node + nsens);
  p->nsens = nsens;

  // host-side masks: Dirichlet nodes, sensor counts and the per-node sensor lists
  std::vector<unsigned char> dir(N, 0);
  for (long long iz = 0; iz < nz; ++iz)
    for (long long iy = 0; iy < ny; ++iy)
      for (long long ix = 0; ix < nx; ++ix) {
        const unsigned f = g->dirichlet_faces;
        bool d = ((f & KKT_FACE_X0) && ix == 0) || ((f & KKT_FACE_X1) && ix == nx - 1) ||
                 ((f & KKT_FACE_Y0) && iy == 0) || ((f & KKT_FACE_Y1) && iy == ny - 1) ||
                 ((f & KKT_FACE_Z0) && iz == 0) || ((f & KKT_FACE_Z1) && iz == nz - 1);
        dir[ix + nx * (iy + ny * iz)] = d ? 1 : 0;
      }
  std::vector<double> sens(N, 0.0);
  std::vector<int> sptr(N + 1, 0), sidx(nsens);
  for (int q = 0; q < nsens; ++q) sptr[sensor_node[q] + 1]++;
  for (long long j = 0; j < N; ++j) sptr[j + 1] += sptr[j];
  {
    std::vector<int> fill(sptr.begin(), sptr.end() - 1);
    for (int q = 0; q < nsens; ++q) sidx[fill[sensor_node[q]]++] = q;
  }
  for (long long j = 0; j < N; ++j) sens[j] = dir[j] ? 0.0 : (double)(sptr[j + 1] - sptr[j]);

  auto fail = [&](kkt_status st) {
    kkt_destroy(p);
    return st;
  };
  const size_t ncoef = 4 * (size_t)kStencil * N;
  if (cudaMalloc(&p->coef64, ncoef * sizeof(double)) != cudaSuccess ||
      cudaMalloc(&p->coef32, ncoef * sizeof(float)) != cudaSuccess ||
      cudaMalloc(&p->dir, N) != cudaSuccess || cudaMalloc(&p->sens, N * sizeof(double)) != cudaSuccess ||
      cudaMalloc(&p->sens_ptr, (N + 1) * sizeof(int)) != cudaSuccess ||
      cudaMalloc(&p->sens_idx, std::max(nsens, 1) * sizeof(int)) != cudaSuccess) {
    cudaGetLastError();
    set_error("kkt_create: device allocation failed");
    return fail(KKT_ERR_NOMEM);
  }
  cudaError_t e = cudaSuccess;
  if (e == cudaSuccess) e = cudaMemcpy(p->dir, dir.data(), N, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(p->sens, sens.data(), N * sizeof(double), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(p->sens_ptr, sptr.data(), (N + 1) * sizeof(int), cudaMemcpyHostToDevice);
  if (e == cudaSuccess && nsens > 0) e = cudaMemcpy(p->sens_idx, sidx.data(), nsens * sizeof(int), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) {
    set_error(std::string("kkt_create: ") + cudaGetErrorString(e));
    return fail(KKT_ERR_CUDA);
  }
  {
    const kkt_status as = assemble_coefficients(p, "kkt_create");
    if (as != KKT_OK) return fail(as);
  }
  {
    const kkt_status ms = matvec_prepare();
    if (ms != KKT_OK) return fail(ms);
  }
  *out = p;
  return KKT_OK;
}

extern "C" kkt_status kkt_create(const kkt_grid* g, int nt, double dt, const double* a_cell, const double* v_cell,
                                 const int* sensor_node, int nsens, double beta1, double beta2, double theta,
                                 kkt_problem** out) {
  NvtxRange nvtx_("kkt_create");
  return create_problem(g, nt, dt, a_cell, v_cell, sensor_node, nsens, beta1, beta2, theta, out);
}

extern "C" kkt_status kkt_set_regularization(kkt_problem* p, int reg) {
  if (!p || (reg != 0 && reg != 1)) {
    set_error("kkt_set_regularization: null problem, or reg not 0 (H1-H1) or 1 (H1-L2)");
    return KKT_ERR_ARG;
  }
  p->reg = reg;
  return KKT_OK;
}

extern "C" kkt_status kkt_set_element(kkt_problem* p, int elem) {
  if (!p || (elem != KKT_ELEM_Q1 && elem != KKT_ELEM_P1)) {
    set_error("kkt_set_element: null problem, or elem not KKT_ELEM_Q1 or KKT_ELEM_P1");
    return KKT_ERR_ARG;
  }
  if (elem == p->elem) return KKT_OK;
  const int old = p->elem;
  p->elem = elem;
  const kkt_status st = assemble_coefficients(p, "kkt_set_element");
  if (st != KKT_OK) p->elem = old;   // the coefficients may be partly written: reassemble the old ones
  if (st != KKT_OK) assemble_coefficients(p, "kkt_set_element");
  return st;
}

extern "C" kkt_status kkt_sizes(const kkt_problem* p, int* nx, int* ny, int* nz, int* levels, long long* unknowns) {
  if (!p) {
    set_error("kkt_sizes: null problem");
    return KKT_ERR_ARG;
  }
  if (nx) *nx = p->nx;
  if (ny) *ny = p->ny;
  if (nz) *nz = p->nz;
  if (levels) *levels = p->L;
  if (unknowns) *unknowns = p->n;
  return KKT_OK;
}

extern "C" kkt_status kkt_rhs(kkt_problem* p, const double* c_obs, const double* c0, double* b, void* stream) {
  if (!p || !b || (p->nsens > 0 && !c_obs)) {
    set_error("kkt_rhs: null argument");
    return KKT_ERR_ARG;
  }
  const unsigned blocks = (unsigned)((p->P + 255) / 256);
  rhs_kernel<<<blocks, 256, 0, (cudaStream_t)stream>>>(p->dev(), c_obs, p->nsens, c0, p->sens_ptr, p->sens_idx, b);
  KKT_COUNT(1);
  KKT_TRY_CUDA(cudaGetLastError());
  return KKT_OK;
}

extern "C" kkt_status recover_source(kkt_problem* p, const double* U, double* f, void* stream) {
  if (!p || !U || !f) {
    set_error("recover_source: null argument");
    return KKT_ERR_ARG;
  }
  source_kernel<<<(unsigned)((p->P + 255) / 256), 256, 0, (cudaStream_t)stream>>>(U, f, p->P);
  KKT_COUNT(1);
  KKT_TRY_CUDA(cudaGetLastError());
  return KKT_OK;
}

extern "C" void kkt_destroy(kkt_problem* p) {
  if (!p) return;
  cudaFree(p->coef64);
  cudaFree(p->coef32);
  cudaFree(p->dir);
  cudaFree(p->sens);
  cudaFree(p->sens_ptr);
  cudaFree(p->sens_idx);
  if (p->ws) {
    p->ws->release();
    delete p->ws;
  }
  delete p;
}
