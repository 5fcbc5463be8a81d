// One-level space-time restricted additive Schwarz preconditioner (Sec. 3.2)
// with ILU(0) subdomain solves, all subdomains in one launch.
//
// Subdomains.  The node range of each axis and the level range 0..M are cut
// into nsub parts (part k of n holds floor(n/p) + (k < n mod p)); a box is the
// product of one part per axis (owned set), extended by `overlap` on every
// side and trimmed to the domain (extended set, Fig. 1).  The subdomain
// matrix M_ij is the principal submatrix of F_h on the extended set, i.e. the
// discretisation with homogeneous Dirichlet data on every cut face in space
// and time (Eq. 10-12).
//
// Storage.  A row of F_h is described by its row type (C, G or f) and a fixed
// list of slots (level offset dt, spatial offset, column component) -- the
// structural stencil of that block row, ordered as the columns are ordered
// (time slowest, then z, y, x, then component).  Every point of a box stores
// 108 + 56 + 162 = 326 slot values, no column indices; slots whose column is
// outside the box hold 0, which is the same as leaving them out of the
// pattern.  Values are laid out [slot][point in wavefront order] per box so
// that the threads working on one wavefront read consecutive addresses.
//
// Ordering and parallelism.  Points are processed in the natural
// (lexicographic) order of the box; with this stencil every lower-triangular
// dependency of point (x, y, z, t) lies on a wavefront w' < w where
// w = x + 2y + 4z + 8t, so all points of one wavefront are independent.  Within
// a point the rows go C, G, f.  One CTA owns one box and steps through its
// wavefronts with a barrier between them.
//
// ILU(0) (IKJ form, on the structural pattern):
//   for each row i in order, for each k < i in pattern(i) ascending:
//     a_ik /= u_kk;  a_ij -= a_ik u_kj  for j > k in pattern(i) and pattern(k).
// The (row slot, column slot) pairs of the inner update are precomputed per
// row type as tables of slot indices.
//
// Solve.  The local vector of each box has a ghost layer of zeros one point
// wide in every direction, so the triangular sweeps need no bounds tests:
// a slot whose column leaves the box reads 0 and has factor value 0.

#include <algorithm>
#include <array>
#include <cmath>
#include <cstring>
#include <vector>

#include "internal.cuh"
#include "ras.cuh"

namespace {

// ---------------------------------------------------------------------------
// slot tables (host-built, copied to constant memory)
// ---------------------------------------------------------------------------
struct SlotTables {
  // per slot (0..325): packed offsets
  int8_t dt[kSlots], dz[kSlots], dy[kSlots], dx[kSlots], comp[kSlots];
  int base[3], count[3], diag[3];       // diag = absolute slot index of the diagonal
  // update lists of the factorisation, for every absolute L-slot s of each type:
  // entries [uptr[s], uptr[s+1]) of (t, s2): a[s2] -= l * u_k[t]
  std::vector<int> uptr;
  std::vector<short2> upd;
};

SlotTables build_tables() {
  SlotTables T;
  int s = 0;
  for (int c = 0; c < 3; ++c) {
    T.base[c] = s;
    const int dt_lo = (c == 1) ? 0 : -1;
    const int dt_hi = (c == 0) ? 0 : 1;
    for (int dt = dt_lo; dt <= dt_hi; ++dt)
      for (int dz = -1; dz <= 1; ++dz)
        for (int dy = -1; dy <= 1; ++dy)
          for (int dx = -1; dx <= 1; ++dx)
            for (int cc = 0; cc < 3; ++cc) {
              bool use;
              if (c == 0) use = (cc == 0 || cc == 2);
              else if (c == 1) use = (cc == 1) || (cc == 0 && dx == 0 && dy == 0 && dz == 0);
              else use = (cc == 1 || cc == 2);
              if (!use) continue;
              T.dt[s] = (int8_t)dt; T.dz[s] = (int8_t)dz; T.dy[s] = (int8_t)dy; T.dx[s] = (int8_t)dx;
              T.comp[s] = (int8_t)cc;
              if (dt == 0 && dz == 0 && dy == 0 && dx == 0 && cc == c) T.diag[c] = s;
              ++s;
            }
    T.count[c] = s - T.base[c];
  }
  // lookup (type c, offset, comp) -> slot
  auto find = [&](int c, int dt, int dz, int dy, int dx, int cc) {
    for (int q = T.base[c]; q < T.base[c] + T.count[c]; ++q)
      if (T.dt[q] == dt && T.dz[q] == dz && T.dy[q] == dy && T.dx[q] == dx && T.comp[q] == cc) return q;
    return -1;
  };
  T.uptr.assign(kSlots + 1, 0);
  std::vector<std::vector<short2>> lists(kSlots);
  for (int c = 0; c < 3; ++c)
    for (int q = T.base[c]; q < T.diag[c]; ++q) {    // L-slots of row type c
      const int ck = T.comp[q];                        // row type of the pivot row k
      for (int t = T.diag[ck] + 1; t < T.base[ck] + T.count[ck]; ++t) {   // U-slots of row k
        const int s2 = find(c, T.dt[q] + T.dt[t], T.dz[q] + T.dz[t], T.dy[q] + T.dy[t], T.dx[q] + T.dx[t], T.comp[t]);
        if (s2 >= 0) lists[q].push_back(make_short2((short)t, (short)s2));
      }
    }
  for (int q = 0; q < kSlots; ++q) T.uptr[q + 1] = T.uptr[q] + (int)lists[q].size();
  for (int q = 0; q < kSlots; ++q) T.upd.insert(T.upd.end(), lists[q].begin(), lists[q].end());
  return T;
}

const SlotTables& tables() {
  static const SlotTables T = build_tables();
  return T;
}

__constant__ int8_t c_dt[kSlots], c_dz[kSlots], c_dy[kSlots], c_dx[kSlots], c_comp[kSlots];
__constant__ int c_base[3], c_count[3], c_diag[3];

// ---------------------------------------------------------------------------
// kernels
// ---------------------------------------------------------------------------

// Matrix entry of F_h in row (point, type c) at slot s (global coordinates).
__device__ double kkt_entry(const DevProblem& p, int c, int s, int j, int n, int jn, int d) {
  const double tau = p.tau, th = p.theta, th1 = 1.0 - p.theta;
  const int dt = c_dt[s], cc = c_comp[s];
  const size_t ci = (size_t)d * p.N + j;
  const bool dirj = p.dir[j] != 0;
  if (c == 0) {
    if (n == 0 || dirj) return (s == c_diag[0]) ? 1.0 : 0.0;
    if (cc == 0) return dt == 0 ? p.B[ci] + th * tau * p.S[ci] : -p.B[ci] + th1 * tau * p.S[ci];
    return dt == 0 ? -th * tau * p.B[ci] : -th1 * tau * p.B[ci];
  }
  if (c == 1) {
    if (n == p.M || dirj) return (s == c_diag[1]) ? 1.0 : 0.0;
    if (cc == 1) return dt == 0 ? p.B[ci] + th * tau * p.ST[ci] : -p.B[ci] + th1 * tau * p.ST[ci];
    return (dt == 0 ? th1 : th) * tau * p.sens[j];
  }
  // f row: time mass / stiffness weights of the linear hats
  const int m = n + dt;
  double mt, lt;
  if (dt == 0) {
    mt = (n > 0 ? tau / 3 : 0.0) + (n < p.M ? tau / 3 : 0.0);
    lt = (n > 0 ? 1.0 / tau : 0.0) + (n < p.M ? 1.0 / tau : 0.0);
  } else {
    mt = tau / 6;
    lt = -1.0 / tau;
  }
  (void)m;
  (void)jn;
  if (cc == 1) return -mt * p.B[ci];
  return p.beta1 * lt * p.B[ci] + p.beta2 * mt * p.K[ci];
}

// Fill the slot values of every point of every box from the stencil coefficients.
template <typename T>
__global__ void gather_matrix(DevProblem p, const BoxDesc* __restrict__ boxes, const int* __restrict__ perm,
                              T* __restrict__ F) {
  const BoxDesc bx = boxes[blockIdx.y];
  const long long P = bx.P;
  T* Fb = F + bx.foff;
  for (long long r = blockIdx.x * (long long)blockDim.x + threadIdx.x; r < P * kSlots;
       r += (long long)gridDim.x * blockDim.x) {
    const int s = (int)(r / P);
    const long long q = r - (long long)s * P;      // wavefront-order position
    const int lex = perm[bx.poff + q];
    const int kx = lex % bx.lx, ky = (lex / bx.lx) % bx.ly, kz = (lex / (bx.lx * bx.ly)) % bx.lz;
    const int kt = lex / (bx.lx * bx.ly * bx.lz);
    const int c = s < c_base[1] ? 0 : (s < c_base[2] ? 1 : 2);
    const int nx_ = kx + c_dx[s], ny_ = ky + c_dy[s], nz_ = kz + c_dz[s], nt_ = kt + c_dt[s];
    double v = 0.0;
    if (nx_ >= 0 && nx_ < bx.lx && ny_ >= 0 && ny_ < bx.ly && nz_ >= 0 && nz_ < bx.lz && nt_ >= 0 && nt_ < bx.lt) {
      const int gx = bx.x0 + kx, gy = bx.y0 + ky, gz = bx.z0 + kz, gt = bx.t0 + kt;
      const int j = gx + p.nx * (gy + p.ny * gz);
      const int d = (c_dx[s] + 1) + 3 * (c_dy[s] + 1) + 9 * (c_dz[s] + 1);
      v = kkt_entry(p, c, s, j, gt, 0, d);
    }
    Fb[(size_t)s * P + q] = (T)v;
  }
}

// ILU(0) of every box: one CTA per box, wavefront by wavefront.
template <typename T>
__global__ void __launch_bounds__(256) ilu0_factor(const BoxDesc* __restrict__ boxes, const int* __restrict__ perm,
                                                   const int* __restrict__ iperm, const int* __restrict__ lptr,
                                                   const int* __restrict__ uptr, const short2* __restrict__ upd,
                                                   T* __restrict__ F, int* __restrict__ status) {
  const BoxDesc bx = boxes[blockIdx.x];
  const long long P = bx.P;
  T* Fb = F + bx.foff;
  const int* lp = lptr + bx.loff;
  for (int w = 0; w < bx.nlev; ++w) {
    for (int q = lp[w] + threadIdx.x; q < lp[w + 1]; q += blockDim.x) {
      const int lex = perm[bx.poff + q];
      const int kx = lex % bx.lx, ky = (lex / bx.lx) % bx.ly, kz = (lex / (bx.lx * bx.ly)) % bx.lz;
      const int kt = lex / (bx.lx * bx.ly * bx.lz);
      for (int c = 0; c < 3; ++c) {
        for (int s = c_base[c]; s < c_diag[c]; ++s) {
          const int ax = kx + c_dx[s], ay = ky + c_dy[s], az = kz + c_dz[s], at = kt + c_dt[s];
          if (ax < 0 || ax >= bx.lx || ay < 0 || ay >= bx.ly || az < 0 || az >= bx.lz || at < 0 || at >= bx.lt)
            continue;
          const int klex = ax + bx.lx * (ay + bx.ly * (az + bx.lz * at));
          const long long kq = iperm[bx.poff + klex];
          const T aik = Fb[(size_t)s * P + q];
          if (aik == (T)0) continue;
          const T ukk = Fb[(size_t)c_diag[c_comp[s]] * P + kq];
          const T l = aik / ukk;
          Fb[(size_t)s * P + q] = l;
          for (int e = uptr[s]; e < uptr[s + 1]; ++e) {
            const short2 u = upd[e];
            Fb[(size_t)u.y * P + q] -= l * Fb[(size_t)u.x * P + kq];
          }
        }
        const T dg = Fb[(size_t)c_diag[c] * P + q];
        if (!(fabs((double)dg) > 1e-300) || !isfinite((double)dg)) atomicExch(status, 1);
      }
    }
    __syncthreads();
  }
}

// z = sum_boxes (R^0)^T M^{-1} R^delta r; one CTA per box.
template <typename T>
__global__ void __launch_bounds__(256) ras_solve(const BoxDesc* __restrict__ boxes, const int* __restrict__ perm,
                                                 const int* __restrict__ lptr, const T* __restrict__ F,
                                                 T* __restrict__ V, const double* __restrict__ r,
                                                 double* __restrict__ z, int nx, int ny, int N) {
  __shared__ int off[kSlots];
  const BoxDesc bx = boxes[blockIdx.x];
  const long long P = bx.P;
  const T* Fb = F + bx.foff;
  T* v = V + bx.voff;
  const int* lp = lptr + bx.loff;
  const int px = bx.lx + 2, py = bx.ly + 2, pz = bx.lz + 2;
  const long long sy = px, sz = (long long)px * py, st = (long long)px * py * pz;
  for (int s = threadIdx.x; s < kSlots; s += blockDim.x)
    off[s] = (int)(3 * (c_dx[s] + sy * c_dy[s] + sz * c_dz[s] + st * c_dt[s]) + c_comp[s]);
  // gather R^delta r into the padded local vector
  for (long long q = threadIdx.x; q < P; q += blockDim.x) {
    const int kx = (int)(q % bx.lx), ky = (int)((q / bx.lx) % bx.ly), kz = (int)((q / (bx.lx * bx.ly)) % bx.lz);
    const int kt = (int)(q / ((long long)bx.lx * bx.ly * bx.lz));
    const long long g = ((long long)(bx.t0 + kt) * N + (bx.x0 + kx) + (long long)nx * ((bx.y0 + ky) + (long long)ny * (bx.z0 + kz))) * 3;
    const long long pq = 3 * ((kx + 1) + sy * (ky + 1) + sz * (kz + 1) + st * (kt + 1));
    v[pq] = (T)r[g];
    v[pq + 1] = (T)r[g + 1];
    v[pq + 2] = (T)r[g + 2];
  }
  __syncthreads();
  // forward sweep with the unit lower factor
  for (int w = 0; w < bx.nlev; ++w) {
    for (int q = lp[w] + threadIdx.x; q < lp[w + 1]; q += blockDim.x) {
      const int lex = perm[bx.poff + q];
      const int kx = lex % bx.lx, ky = (lex / bx.lx) % bx.ly, kz = (lex / (bx.lx * bx.ly)) % bx.lz;
      const int kt = lex / (bx.lx * bx.ly * bx.lz);
      T* vp = v + 3 * ((kx + 1) + sy * (ky + 1) + sz * (kz + 1) + st * (kt + 1));
      for (int c = 0; c < 3; ++c) {
        T acc = vp[c];
        for (int s = c_base[c]; s < c_diag[c]; ++s) acc -= Fb[(size_t)s * P + q] * vp[off[s]];
        vp[c] = acc;
      }
    }
    __syncthreads();
  }
  // backward sweep with the upper factor
  for (int w = bx.nlev - 1; w >= 0; --w) {
    for (int q = lp[w] + threadIdx.x; q < lp[w + 1]; q += blockDim.x) {
      const int lex = perm[bx.poff + q];
      const int kx = lex % bx.lx, ky = (lex / bx.lx) % bx.ly, kz = (lex / (bx.lx * bx.ly)) % bx.lz;
      const int kt = lex / (bx.lx * bx.ly * bx.lz);
      T* vp = v + 3 * ((kx + 1) + sy * (ky + 1) + sz * (kz + 1) + st * (kt + 1));
      for (int c = 2; c >= 0; --c) {
        T acc = vp[c];
        const int end = c_base[c] + c_count[c];
        for (int s = c_diag[c] + 1; s < end; ++s) acc -= Fb[(size_t)s * P + q] * vp[off[s]];
        vp[c] = acc / Fb[(size_t)c_diag[c] * P + q];
      }
    }
    __syncthreads();
  }
  // scatter the owned part: (R^0)^T
  const int ox = bx.ox1 - bx.ox0, oy = bx.oy1 - bx.oy0, oz = bx.oz1 - bx.oz0, ot = bx.ot1 - bx.ot0;
  const long long nown = (long long)ox * oy * oz * ot;
  for (long long q = threadIdx.x; q < nown; q += blockDim.x) {
    const int gx = bx.ox0 + (int)(q % ox), gy = bx.oy0 + (int)((q / ox) % oy);
    const int gz = bx.oz0 + (int)((q / ((long long)ox * oy)) % oz), gt = bx.ot0 + (int)(q / ((long long)ox * oy * oz));
    const int kx = gx - bx.x0, ky = gy - bx.y0, kz = gz - bx.z0, kt = gt - bx.t0;
    const long long pq = 3 * ((kx + 1) + sy * (ky + 1) + sz * (kz + 1) + st * (kt + 1));
    const long long g = ((long long)gt * N + gx + (long long)nx * (gy + (long long)ny * gz)) * 3;
    z[g] = (double)v[pq];
    z[g + 1] = (double)v[pq + 1];
    z[g + 2] = (double)v[pq + 2];
  }
}

std::vector<std::pair<int, int>> parts(int n, int p) {
  std::vector<std::pair<int, int>> out;
  const int base = n / p, extra = n % p;
  int s = 0;
  for (int k = 0; k < p; ++k) {
    const int e = s + base + (k < extra ? 1 : 0);
    out.emplace_back(s, e);
    s = e;
  }
  return out;
}

}  // namespace

kkt_status ras_create(kkt_problem* p, const int nsub[4], int overlap, int local, int factor_prec,
                      ras_precond** out) {
  if (!p || !nsub || !out) {
    set_error("ras_setup: null argument");
    return KKT_ERR_ARG;
  }
  *out = nullptr;
  const int dims[4] = {p->nx, p->ny, p->nz, p->L};
  for (int a = 0; a < 4; ++a)
    if (nsub[a] < 1 || nsub[a] > dims[a]) {
      set_error("ras_setup: each nsub must lie in [1, points along that axis]");
      return KKT_ERR_ARG;
    }
  if (overlap < 0 || local != 0 || (factor_prec != 64 && factor_prec != 32)) {
    set_error("ras_setup: overlap must be >= 0, local 0 (ILU(0)), factor_prec 64 or 32");
    return KKT_ERR_ARG;
  }
  const SlotTables& T = tables();
  static bool consts_done = false;   // constant memory is per module; upload once per process
  if (!consts_done) {
    KKT_TRY_CUDA(cudaMemcpyToSymbol(c_dt, T.dt, kSlots));
    KKT_TRY_CUDA(cudaMemcpyToSymbol(c_dz, T.dz, kSlots));
    KKT_TRY_CUDA(cudaMemcpyToSymbol(c_dy, T.dy, kSlots));
    KKT_TRY_CUDA(cudaMemcpyToSymbol(c_dx, T.dx, kSlots));
    KKT_TRY_CUDA(cudaMemcpyToSymbol(c_comp, T.comp, kSlots));
    KKT_TRY_CUDA(cudaMemcpyToSymbol(c_base, T.base, sizeof(T.base)));
    KKT_TRY_CUDA(cudaMemcpyToSymbol(c_count, T.count, sizeof(T.count)));
    KKT_TRY_CUDA(cudaMemcpyToSymbol(c_diag, T.diag, sizeof(T.diag)));
    consts_done = true;
  }

  ras_precond* m = new (std::nothrow) ras_precond();
  if (!m) return KKT_ERR_NOMEM;
  m->prob = p;
  m->prec = factor_prec;
  std::vector<std::pair<int, int>> pr[4];
  for (int a = 0; a < 4; ++a) pr[a] = parts(dims[a], nsub[a]);
  std::vector<BoxDesc> boxes;
  std::vector<int> perm, iperm, lptr;
  long long foff = 0, voff = 0;
  for (int it = 0; it < nsub[3]; ++it)
    for (int iz = 0; iz < nsub[2]; ++iz)
      for (int iy = 0; iy < nsub[1]; ++iy)
        for (int ix = 0; ix < nsub[0]; ++ix) {
          BoxDesc b{};
          const std::pair<int, int>* own[4] = {&pr[0][ix], &pr[1][iy], &pr[2][iz], &pr[3][it]};
          int lo[4], hi[4];
          for (int a = 0; a < 4; ++a) {
            lo[a] = std::max(0, own[a]->first - overlap);
            hi[a] = std::min(dims[a], own[a]->second + overlap);
          }
          b.x0 = lo[0]; b.y0 = lo[1]; b.z0 = lo[2]; b.t0 = lo[3];
          b.lx = hi[0] - lo[0]; b.ly = hi[1] - lo[1]; b.lz = hi[2] - lo[2]; b.lt = hi[3] - lo[3];
          b.ox0 = own[0]->first; b.ox1 = own[0]->second; b.oy0 = own[1]->first; b.oy1 = own[1]->second;
          b.oz0 = own[2]->first; b.oz1 = own[2]->second; b.ot0 = own[3]->first; b.ot1 = own[3]->second;
          b.P = (long long)b.lx * b.ly * b.lz * b.lt;
          b.nlev = (b.lx - 1) + 2 * (b.ly - 1) + 4 * (b.lz - 1) + 8 * (b.lt - 1) + 1;
          b.foff = foff;
          b.voff = voff;
          b.poff = (long long)perm.size();
          b.loff = (long long)lptr.size();
          foff += b.P * kSlots;
          voff += 3LL * (b.lx + 2) * (b.ly + 2) * (b.lz + 2) * (b.lt + 2);
          // counting sort of the points by wavefront
          std::vector<int> cnt(b.nlev + 1, 0);
          for (int kt = 0; kt < b.lt; ++kt)
            for (int kz = 0; kz < b.lz; ++kz)
              for (int ky = 0; ky < b.ly; ++ky)
                for (int kx = 0; kx < b.lx; ++kx) cnt[kx + 2 * ky + 4 * kz + 8 * kt + 1]++;
          for (int w = 0; w < b.nlev; ++w) cnt[w + 1] += cnt[w];
          for (int w = 0; w <= b.nlev; ++w) lptr.push_back(cnt[w]);
          std::vector<int> bp(b.P), bi(b.P);
          std::vector<int> fill(cnt.begin(), cnt.end() - 1);
          int lex = 0;
          for (int kt = 0; kt < b.lt; ++kt)
            for (int kz = 0; kz < b.lz; ++kz)
              for (int ky = 0; ky < b.ly; ++ky)
                for (int kx = 0; kx < b.lx; ++kx, ++lex) {
                  const int q = fill[kx + 2 * ky + 4 * kz + 8 * kt]++;
                  bp[q] = lex;
                  bi[lex] = q;
                }
          perm.insert(perm.end(), bp.begin(), bp.end());
          iperm.insert(iperm.end(), bi.begin(), bi.end());
          boxes.push_back(b);
        }
  m->nbox = (int)boxes.size();
  m->boxes_h = boxes;
  m->fcount = foff;
  const size_t esz = factor_prec == 64 ? sizeof(double) : sizeof(float);
  auto fail = [&](kkt_status st, const char* what) {
    cudaGetLastError();
    set_error(std::string("ras_setup: ") + what);
    ras_destroy(m);
    return st;
  };
  if (cudaMalloc(&m->boxes, boxes.size() * sizeof(BoxDesc)) != cudaSuccess ||
      cudaMalloc(&m->perm, perm.size() * sizeof(int)) != cudaSuccess ||
      cudaMalloc(&m->iperm, iperm.size() * sizeof(int)) != cudaSuccess ||
      cudaMalloc(&m->lptr, lptr.size() * sizeof(int)) != cudaSuccess ||
      cudaMalloc(&m->uptr, T.uptr.size() * sizeof(int)) != cudaSuccess ||
      cudaMalloc(&m->upd, T.upd.size() * sizeof(short2)) != cudaSuccess ||
      cudaMalloc(&m->F, foff * esz) != cudaSuccess || cudaMalloc(&m->V, voff * esz) != cudaSuccess ||
      cudaMalloc(&m->status, sizeof(int)) != cudaSuccess)
    return fail(KKT_ERR_NOMEM, "device allocation failed");
  cudaError_t e = cudaSuccess;
  if (e == cudaSuccess) e = cudaMemcpy(m->boxes, boxes.data(), boxes.size() * sizeof(BoxDesc), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(m->perm, perm.data(), perm.size() * sizeof(int), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(m->iperm, iperm.data(), iperm.size() * sizeof(int), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(m->lptr, lptr.data(), lptr.size() * sizeof(int), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(m->uptr, T.uptr.data(), T.uptr.size() * sizeof(int), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(m->upd, T.upd.data(), T.upd.size() * sizeof(short2), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemset(m->V, 0, voff * esz);
  if (e == cudaSuccess) e = cudaMemset(m->status, 0, sizeof(int));
  if (e != cudaSuccess) return fail(KKT_ERR_CUDA, cudaGetErrorString(e));
  kkt_status st = ras_factor(m);
  if (st != KKT_OK) {
    ras_destroy(m);
    return st;
  }
  *out = m;
  return KKT_OK;
}

kkt_status ras_factor(ras_precond* m) {
  const DevProblem dp = m->prob->dev();
  dim3 g(152, m->nbox);
  if (m->prec == 64) {
    gather_matrix<double><<<g, 256>>>(dp, m->boxes, m->perm, (double*)m->F);
    ilu0_factor<double><<<m->nbox, 256>>>(m->boxes, m->perm, m->iperm, m->lptr, m->uptr, m->upd, (double*)m->F,
                                          m->status);
  } else {
    gather_matrix<float><<<g, 256>>>(dp, m->boxes, m->perm, (float*)m->F);
    ilu0_factor<float><<<m->nbox, 256>>>(m->boxes, m->perm, m->iperm, m->lptr, m->uptr, m->upd, (float*)m->F,
                                         m->status);
  }
  KKT_TRY_CUDA(cudaGetLastError());
  KKT_TRY_CUDA(cudaDeviceSynchronize());
  int st = 0;
  KKT_TRY_CUDA(cudaMemcpy(&st, m->status, sizeof(int), cudaMemcpyDeviceToHost));
  if (st != 0) {
    set_error("ras_setup: zero or non-finite pivot in a subdomain ILU(0)");
    return KKT_ERR_ZERO_PIVOT;
  }
  return KKT_OK;
}

kkt_status ras_launch(ras_precond* m, const double* r, double* z, cudaStream_t s) {
  const kkt_problem* p = m->prob;
  if (m->prec == 64)
    ras_solve<double><<<m->nbox, 256, 0, s>>>(m->boxes, m->perm, m->lptr, (const double*)m->F, (double*)m->V, r, z,
                                              p->nx, p->ny, p->N);
  else
    ras_solve<float><<<m->nbox, 256, 0, s>>>(m->boxes, m->perm, m->lptr, (const float*)m->F, (float*)m->V, r, z,
                                             p->nx, p->ny, p->N);
  KKT_TRY_CUDA(cudaGetLastError());
  return KKT_OK;
}

extern "C" kkt_status ras_setup(kkt_problem* p, const int nsub[4], int overlap, int local, int factor_prec,
                                ras_precond** out) {
  return ras_create(p, nsub, overlap, local, factor_prec, out);
}

extern "C" kkt_status ras_apply(ras_precond* m, const double* r, double* z, void* stream) {
  if (!m || !r || !z) {
    set_error("ras_apply: null argument");
    return KKT_ERR_ARG;
  }
  if (r == z) {
    set_error("ras_apply: r and z must not overlap");
    return KKT_ERR_ARG;
  }
  return ras_launch(m, r, z, (cudaStream_t)stream);
}

extern "C" void ras_destroy(ras_precond* m) {
  if (!m) return;
  cudaFree(m->boxes);
  cudaFree(m->perm);
  cudaFree(m->iperm);
  cudaFree(m->lptr);
  cudaFree(m->uptr);
  cudaFree(m->upd);
  cudaFree(m->F);
  cudaFree(m->V);
  cudaFree(m->status);
  delete m;
}
