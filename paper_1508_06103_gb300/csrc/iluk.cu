// Subdomain solvers beyond ILU(0) (Sec. 4, Table 1; Sec. 3.2): ILU(1), the
// incomplete factorisation on the pattern grown by one level of fill, and the
// 3x3 point-block ILU(0), the incomplete factorisation on the pattern of whole
// point blocks (the point-block ordering of Sec. 3.2: C, G, f of a space-time
// point together).  Both run one pattern-driven elimination:
//
// Pattern.  Every row type c (C, G, f) has a list of slots (point offset
// (dt, dz, dy, dx), column component) in column order: the pattern of an
// interior point.  ILU(1): the level-1 pattern, found on the host by the
// symbolic elimination (levels of fill) on a box of 5^4 points around one
// point; block ILU(0): all components of the 81 points at offsets in
// {-1, 0, 1}^4.  A point near a box face or the domain boundary uses a subset:
// the per-point levels decide which slots it keeps.
//
// Values and levels.  Point-major per box, by the point's lexicographic index
// in the box (so a column's address is arithmetic on the point's, with no
// index lookup): slot s of point lex at F[foff + lex * S + s] (a warp takes
// one point, its lanes consecutive slots), its level of fill at LV[...] (0 for
// an entry of F_h's structural pattern, 255 for a slot the point does not
// have).  The local vectors of the solve are indexed the same way.
//
// Elimination (IKJ, rows in the natural point-block order, as the oracle's
// ILU0 on the same pattern).  For row (p, c): a symbolic pass over the L slots
// s in column order lowers the levels of the row's later slots through each
// pivot row's kept U entries (lev(s) + lev_piv(t) + 1); a numeric pass then
// divides by the pivot and updates every kept target.  The pairs (t, u) of a
// pivot slot t that lands on the row's slot u are tabulated on the host per
// (row type, L slot).  Schedule: wavefronts w = x + b y + b^2 z + b^3 t with
// b = R + 1 for the largest offset R of an L slot, so every L-slot column of
// a point lies on an earlier wavefront.
//
// Solve.  One CTA per box: gather R^delta r, forward and backward sweeps by
// wavefront over the same slot lists (a warp per point), scatter the owned
// points.

#include <algorithm>
#include <array>
#include <cstring>
#include <map>
#include <mutex>
#include <vector>

#include "ras.cuh"
#include "slotval.cuh"

namespace {

constexpr int kGpMaxRow = 800;       // slots of one row type at most (ILU(1): 780 in the C row)

struct GpSlot {
  int dt, dz, dy, dx, cc;
};

bool slot_less(const GpSlot& a, const GpSlot& b) {
  if (a.dt != b.dt) return a.dt < b.dt;
  if (a.dz != b.dz) return a.dz < b.dz;
  if (a.dy != b.dy) return a.dy < b.dy;
  if (a.dx != b.dx) return a.dx < b.dx;
  return a.cc < b.cc;
}

// Structural columns of row c of an interior point (all sensor couplings
// present): C rows couple C and f at levels n-1, n; G rows G at n, n+1 and C
// at the node itself at n, n+1; f rows G and f at n-1, n, n+1 (Appendix).
std::vector<GpSlot> structural_row(int c) {
  std::vector<GpSlot> out;
  for (int dt = -1; dt <= 1; ++dt)
    for (int dz = -1; dz <= 1; ++dz)
      for (int dy = -1; dy <= 1; ++dy)
        for (int dx = -1; dx <= 1; ++dx) {
          if (c == 0 && dt <= 0) {
            out.push_back({dt, dz, dy, dx, 0});
            out.push_back({dt, dz, dy, dx, 2});
          } else if (c == 1 && dt >= 0) {
            out.push_back({dt, dz, dy, dx, 1});
            if (dz == 0 && dy == 0 && dx == 0) out.push_back({dt, 0, 0, 0, 0});
          } else if (c == 2) {
            out.push_back({dt, dz, dy, dx, 1});
            out.push_back({dt, dz, dy, dx, 2});
          }
        }
  std::sort(out.begin(), out.end(), slot_less);
  return out;
}

// Interior level-1 pattern per row type: the symbolic IKJ elimination with
// levels of fill on a box of 5^4 points (every level-1 path of the centre
// point's rows runs through points within distance 2), read at the centre.
std::array<std::vector<GpSlot>, 3> ilu1_interior_rows() {
  constexpr int E = 5, NP = E * E * E * E, NR = 3 * NP;
  auto col_of = [&](int x, int y, int z, int t, int c) { return 3 * (x + E * (y + E * (z + E * t))) + c; };
  std::vector<std::vector<std::pair<int, int>>> ulev(NR);   // kept upper entries (column, level)
  std::array<std::vector<GpSlot>, 3> rows;
  std::vector<int> lev(NR);
  const int centre = 2 + E * (2 + E * (2 + E * 2));
  for (int i = 0; i < NR; ++i) {
    const int pt = i / 3, c = i % 3;
    const int x = pt % E, y = (pt / E) % E, z = (pt / (E * E)) % E, t = pt / (E * E * E);
    std::fill(lev.begin(), lev.end(), 1 << 20);
    for (const GpSlot& s : structural_row(c)) {
      const int X = x + s.dx, Y = y + s.dy, Z = z + s.dz, T = t + s.dt;
      if (X < 0 || X >= E || Y < 0 || Y >= E || Z < 0 || Z >= E || T < 0 || T >= E) continue;
      lev[col_of(X, Y, Z, T, s.cc)] = 0;
    }
    for (int m = 0; m < i; ++m) {   // L entries in column order (fill joins before it is reached)
      if (lev[m] > 1) continue;
      for (const auto& e : ulev[m]) {
        const int nl = lev[m] + e.second + 1;
        if (nl <= 1 && nl < lev[e.first]) lev[e.first] = nl;
      }
    }
    for (int j = i + 1; j < NR; ++j)
      if (lev[j] <= 1) ulev[i].push_back({j, lev[j]});
    if (pt == centre)
      for (int j = 0; j < NR; ++j)
        if (lev[j] <= 1) {
          const int q = j / 3;
          rows[c].push_back({q / (E * E * E) - 2, (q / (E * E)) % E - 2, (q / E) % E - 2, q % E - 2, j % 3});
        }
  }
  for (auto& r : rows) std::sort(r.begin(), r.end(), slot_less);
  return rows;
}

std::array<std::vector<GpSlot>, 3> block_rows() {
  std::array<std::vector<GpSlot>, 3> rows;
  for (int c = 0; c < 3; ++c) {
    for (int dt = -1; dt <= 1; ++dt)
      for (int dz = -1; dz <= 1; ++dz)
        for (int dy = -1; dy <= 1; ++dy)
          for (int dx = -1; dx <= 1; ++dx)
            for (int cc = 0; cc < 3; ++cc) rows[c].push_back({dt, dz, dy, dx, cc});
    std::sort(rows[c].begin(), rows[c].end(), slot_less);
  }
  return rows;
}

std::array<std::vector<GpSlot>, 3> gp_rows(int local) {
  static std::array<std::vector<GpSlot>, 3> ilu1, blk;   // built once per process
  static bool have1 = false, haveb = false;
  static std::mutex mu;
  std::lock_guard<std::mutex> lock(mu);
  if (local == 2) {
    if (!have1) {
      ilu1 = ilu1_interior_rows();
      have1 = true;
    }
    return ilu1;
  }
  if (!haveb) {
    blk = block_rows();
    haveb = true;
  }
  return blk;
}

}  // namespace

// Slots per row type of an interior point under the local solver `local`
// (0 ILU(0), 2 ILU(1), 3 point-block ILU(0)); host only.
extern "C" kkt_status ras_local_pattern(int local, int counts[3]) {
  if (!counts || (local != 0 && local != 2 && local != 3)) {
    set_error("ras_local_pattern: counts is null, or local is not 0, 2 or 3");
    return KKT_ERR_ARG;
  }
  if (local == 0) {
    for (int c = 0; c < 3; ++c) counts[c] = (int)structural_row(c).size();
    return KKT_OK;
  }
  const auto rows = gp_rows(local);
  for (int c = 0; c < 3; ++c) counts[c] = (int)rows[c].size();
  return KKT_OK;
}

// ---------------------------------------------------------------------------
// Device side
// ---------------------------------------------------------------------------

// Per-box storage of the pattern-driven factors.
struct GpBox {
  long long foff;   // values / levels: slot s of point lex (box-lexicographic) at foff + lex * S + s
  long long voff;   // local vector: 3 values per point
  long long poff;   // schedule array (perm: schedule position -> lexicographic index)
  long long loff;   // wavefront pointers
  int nlev;
  int P;
};

struct GpTables {
  const signed char* slot;   // [S][5]: dt, dz, dy, dx, column component
  const short* smap;         // [S]: the slot's index among the ILU(0) slots (its value), or -1
  const int* tptr;           // [S + 1]: update pairs of each L slot (global slot numbering)
  const int* tt;             // pivot-row slot (global index) of each pair
  const short* tu;           // target slot (row-local index) of each pair
  int base[3], cnt[3], diag[3];   // row types: first global slot, slots, row-local diagonal
  int S;                     // slots per point
  int K;                     // kept level of fill (ILU(1): 1, point-block ILU(0): 0)
};

struct GpFactor {
  int local = 2;
  int prec = 64;
  GpTables tab{};
  std::vector<GpBox> boxes_h;
  GpBox* boxes = nullptr;
  int* perm = nullptr;
  int* lptr = nullptr;
  signed char* slot = nullptr;
  short* smap = nullptr;
  int* tptr = nullptr;
  int* tt = nullptr;
  short* tu = nullptr;
  void* F = nullptr;
  unsigned char* LV = nullptr;
  void* V = nullptr;
  long long fcount = 0, vcount = 0;
  ~GpFactor() {
    cudaFree(boxes);
    cudaFree(perm);
    cudaFree(lptr);
    cudaFree(slot);
    cudaFree(smap);
    cudaFree(tptr);
    cudaFree(tt);
    cudaFree(tu);
    cudaFree(F);
    cudaFree(LV);
    cudaFree(V);
  }
};

namespace {

constexpr int kGpThreads = 192;        // factor CTA (row buffers: 6 warps x 800 slots fit 48 KB in FP64)
constexpr int kGpSolveThreads = 256;

__device__ __forceinline__ int gp_row_of(const GpTables& tb, int s) {
  return s < tb.base[1] ? 0 : (s < tb.base[2] ? 1 : 2);
}

// Lexicographic box index of the column point of slot s, or -1 outside the box.
__device__ __forceinline__ int gp_col_lex(const BoxDesc& bx, const signed char* sl, int kx, int ky, int kz, int kt) {
  const int ax = kx + sl[3], ay = ky + sl[2], az = kz + sl[1], at = kt + sl[0];
  if (ax < 0 || ax >= bx.lx || ay < 0 || ay >= bx.ly || az < 0 || az >= bx.lz || at < 0 || at >= bx.lt) return -1;
  return ax + bx.lx * (ay + bx.ly * (az + bx.lz * at));
}

// Initial values (the principal submatrix of F_h on the box, Eq. 10-12) and
// levels (0: F_h's structural pattern; 255: not kept unless fill reaches it).
// One warp per point, its lanes over the slots (point-major storage).
template <typename T>
__global__ void gp_gather(const DevProblem* __restrict__ probs, const BoxDesc* __restrict__ boxes,
                          const GpBox* __restrict__ gb, const int* __restrict__ perm, GpTables tb, T* __restrict__ F,
                          unsigned char* __restrict__ LV) {
  const BoxDesc bx = boxes[blockIdx.y];
  const GpBox g = gb[blockIdx.y];
  const int q = blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32;
  const int lane = threadIdx.x & 31;
  if (q >= g.P) return;
  const DevProblem p = probs[bx.prob];
  const Coefs<T> cf = coefs<T>(p);
  const int lex = perm[g.poff + q];
  const PointRow<T> pr = point_row<T>(p, bx, lex);
  const bool idC = pr.n == 0 || pr.dirj, idG = pr.n == p.M || pr.dirj;
  const long long o = g.foff + (long long)lex * tb.S;
  for (int s = lane; s < tb.S; s += 32) {
    const signed char* sl = tb.slot + 5 * s;
    const int c = gp_row_of(tb, s);
    const bool inb = gp_col_lex(bx, sl, pr.kx, pr.ky, pr.kz, pr.kt) >= 0;
    const int ss = tb.smap[s];
    T v = (T)0;
    bool structural = false;
    if (inb && ss >= 0) {
      bool ib;
      v = slot_value<T>(p, bx, cf, pr, ss, &ib);
      const bool diag = s - tb.base[c] == tb.diag[c];
      structural = !((c == 0 && idC && !diag) || (c == 1 && idG && !diag) ||
                     (c == 1 && sl[4] == 0 && pr.sj == (T)0));
    }
    const bool keep0 = tb.K == 0 ? inb : structural;   // point-block: every in-box slot
    F[o + s] = v;
    LV[o + s] = keep0 ? 0 : 255;
  }
}

__device__ __forceinline__ void gp_check_pivot(double d, int* status) {
  if (!(fabs(d) > 1e-300) || !isfinite(d)) atomicExch(status, 1);
}

constexpr int kGpWarps = kGpThreads / 32;

// One CTA per box; wavefronts in order with a barrier between them; one warp
// per point, its C, G and f rows in turn (IKJ, see the file header).  The row
// (values and levels) sits in the warp's shared memory during its
// elimination; the L slots go in order, the update pairs of one L slot
// (distinct targets) are split over the lanes.
template <typename T>
__global__ void __launch_bounds__(kGpThreads) gp_factor(const BoxDesc* __restrict__ boxes,
                                                        const GpBox* __restrict__ gb, const int* __restrict__ perm,
                                                        const int* __restrict__ lptr,
                                                        GpTables tb, T* __restrict__ F, unsigned char* __restrict__ LV,
                                                        int* __restrict__ status) {
  __shared__ T rowv[kGpWarps][kGpMaxRow];
  __shared__ unsigned char rowl[kGpWarps][kGpMaxRow];
  const BoxDesc bx = boxes[blockIdx.x];
  const GpBox g = gb[blockIdx.x];
  const int lane = threadIdx.x & 31, wp = threadIdx.x / 32;
  T* rv = rowv[wp];
  unsigned char* rl = rowl[wp];
  const int K = tb.K;
  for (int w = 0; w < g.nlev; ++w) {
    const int l0 = lptr[g.loff + w], l1 = lptr[g.loff + w + 1];
    for (int q = l0 + wp; q < l1; q += kGpWarps) {
      const int lex = perm[g.poff + q];
      const int kx = lex % bx.lx, ky = (lex / bx.lx) % bx.ly, kz = (lex / (bx.lx * bx.ly)) % bx.lz;
      const int kt = lex / (bx.lx * bx.ly * bx.lz);
      T* own = F + g.foff + (long long)lex * tb.S;
      unsigned char* ownl = LV + g.foff + (long long)lex * tb.S;
      for (int c = 0; c < 3; ++c) {
        const int b = tb.base[c], nrow = tb.cnt[c], dg = tb.diag[c];
        for (int u = lane; u < nrow; u += 32) {
          rv[u] = own[b + u];
          rl[u] = ownl[b + u];
        }
        __syncwarp();
        if (K > 0) {   // symbolic pass: final levels of the row
          for (int s = 0; s < dg; ++s) {
            const int ls = rl[s];
            if (ls > K) continue;
            const int qp = gp_col_lex(bx, tb.slot + 5 * (b + s), kx, ky, kz, kt);
            const unsigned char* pl = LV + g.foff + (long long)qp * tb.S;
            for (int e = tb.tptr[b + s] + lane; e < tb.tptr[b + s + 1]; e += 32) {
              const int lp = pl[tb.tt[e]];
              const int nl = ls + lp + 1;
              const int u = tb.tu[e];
              if (lp <= K && nl <= K && nl < rl[u]) rl[u] = (unsigned char)nl;
            }
            __syncwarp();
          }
        }
        // numeric pass (a pivot's dropped entries hold 0, so every pair may update)
        for (int s = 0; s < dg; ++s) {
          if (rl[s] > K) continue;
          const int sc = tb.slot[5 * (b + s) + 4];
          const int qp = gp_col_lex(bx, tb.slot + 5 * (b + s), kx, ky, kz, kt);
          const T* pv = F + g.foff + (long long)qp * tb.S;
          const T l = rv[s] * pv[tb.base[sc] + tb.diag[sc]];
          for (int e = tb.tptr[b + s] + lane; e < tb.tptr[b + s + 1]; e += 32) {
            const int u = tb.tu[e];
            if (rl[u] <= K) rv[u] -= l * pv[tb.tt[e]];
          }
          __syncwarp();
          if (lane == 0) rv[s] = l;
        }
        __syncwarp();
        if (lane == 0) {
          const T d = rv[dg];
          gp_check_pivot((double)d, status);
          rv[dg] = (T)1 / d;
        }
        __syncwarp();
        for (int u = lane; u < nrow; u += 32) {
          own[b + u] = rv[u];
          ownl[b + u] = rl[u] <= K ? rl[u] : 255;
        }
        __syncwarp();
      }
    }
    __syncthreads();
  }
}

// z = sum over boxes (R^0)^T M^{-1} R^delta r with the pattern-driven factors:
// one CTA per box gathers its residual, sweeps forward and backward by
// wavefront, one warp per point and row, its lanes summing over the slots
// (slots whose column leaves the box are skipped; dropped entries hold 0),
// and writes its owned points.
template <typename T>
__global__ void __launch_bounds__(kGpSolveThreads) gp_solve(const DevProblem* __restrict__ probs,
                                                       const BoxDesc* __restrict__ boxes, const GpBox* __restrict__ gb,
                                                       const int* __restrict__ perm,
                                                       const int* __restrict__ lptr, GpTables tb,
                                                       const T* __restrict__ F, T* __restrict__ V,
                                                       const double* __restrict__ r, double* __restrict__ z,
                                                       const int* gate) {
  if (gated_off(gate)) return;
  const BoxDesc bx = boxes[blockIdx.x];
  const GpBox g = gb[blockIdx.x];
  const DevProblem p = probs[bx.prob];
  T* Vb = V + g.voff;
  const int lane = threadIdx.x & 31, wp = threadIdx.x / 32;
  auto global_point = [&](int lex) {
    const int kx = lex % bx.lx, ky = (lex / bx.lx) % bx.ly, kz = (lex / (bx.lx * bx.ly)) % bx.lz;
    const int kt = lex / (bx.lx * bx.ly * bx.lz);
    return (long long)(bx.t0 + kt) * p.N + (bx.x0 + kx) + (long long)p.nx * ((bx.y0 + ky) + (long long)p.ny * (bx.z0 + kz));
  };
  for (int lex = threadIdx.x; lex < g.P; lex += blockDim.x) {   // R^delta r
    const long long gi = 3 * global_point(lex);
    for (int c = 0; c < 3; ++c) Vb[3 * lex + c] = (T)r[gi + c];
  }
  __syncthreads();
  for (int pass = 0; pass < 2; ++pass) {
    for (int wi = 0; wi < g.nlev; ++wi) {
      const int w = pass == 0 ? wi : g.nlev - 1 - wi;
      const int l0 = lptr[g.loff + w], l1 = lptr[g.loff + w + 1];
      for (int q = l0 + wp; q < l1; q += kGpSolveThreads / 32) {
        const int lex = perm[g.poff + q];
        const int kx = lex % bx.lx, ky = (lex / bx.lx) % bx.ly, kz = (lex / (bx.lx * bx.ly)) % bx.lz;
        const int kt = lex / (bx.lx * bx.ly * bx.lz);
        const T* Fp = F + g.foff + (long long)lex * tb.S;
        for (int ci = 0; ci < 3; ++ci) {
          const int c = pass == 0 ? ci : 2 - ci;
          const int b = tb.base[c], dg = tb.diag[c];
          const int s0 = pass == 0 ? 0 : dg + 1, s1 = pass == 0 ? dg : tb.cnt[c];
          T part = (T)0;
#pragma unroll 4
          for (int s = s0 + lane; s < s1; s += 32) {
            // the column from the slot table alone, so the value and vector loads are independent
            const signed char* sl = tb.slot + 5 * (b + s);
            const int cl = gp_col_lex(bx, sl, kx, ky, kz, kt);
            const T v = Fp[b + s];
            if (cl >= 0) part += v * Vb[3 * cl + sl[4]];
          }
          for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
          if (lane == 0) {
            T acc = Vb[3 * lex + c] - part;
            if (pass == 1) acc *= Fp[b + dg];   // the stored 1 / u_ii
            Vb[3 * lex + c] = acc;
          }
          __syncwarp();
        }
      }
      __syncthreads();
    }
  }
  for (int lex = threadIdx.x; lex < g.P; lex += blockDim.x) {   // (R^0)^T: owned points only
    const int kx = lex % bx.lx, ky = (lex / bx.lx) % bx.ly, kz = (lex / (bx.lx * bx.ly)) % bx.lz;
    const int kt = lex / (bx.lx * bx.ly * bx.lz);
    const int x = bx.x0 + kx, y = bx.y0 + ky, zz = bx.z0 + kz, t = bx.t0 + kt;
    if (x < bx.ox0 || x >= bx.ox1 || y < bx.oy0 || y >= bx.oy1 || zz < bx.oz0 || zz >= bx.oz1 || t < bx.ot0 ||
        t >= bx.ot1)
      continue;
    const long long gi = 3 * global_point(lex);
    for (int c = 0; c < 3; ++c) z[gi + c] = (double)Vb[3 * lex + c];
  }
}

template <typename T>
kkt_status gp_factor_t(ras_precond* m, cudaStream_t s) {
  GpFactor* f = m->gp;
  int pmax = 0;
  for (const GpBox& b : f->boxes_h) pmax = std::max(pmax, b.P);
  gp_gather<T><<<dim3((pmax + 7) / 8, m->nbox), 256, 0, s>>>(m->dprobs, m->boxes, f->boxes, f->perm, f->tab,
                                                             (T*)f->F, f->LV);
  KKT_COUNT(1);
  KKT_TRY_CUDA(cudaGetLastError());
  {
    TimedScope timed(&m->factor_timing, s);
    gp_factor<T><<<m->nbox, kGpThreads, 0, s>>>(m->boxes, f->boxes, f->perm, f->lptr, f->tab, (T*)f->F,
                                                f->LV, m->status);
  }
  KKT_COUNT(1);
  KKT_TRY_CUDA(cudaGetLastError());
  return KKT_OK;
}

}  // namespace

kkt_status gp_factor(ras_precond* m, cudaStream_t s) {
  return m->gp->prec == 64 ? gp_factor_t<double>(m, s) : gp_factor_t<float>(m, s);
}

kkt_status gp_solve(ras_precond* m, const double* r, double* z, cudaStream_t s, const int* gate) {
  GpFactor* f = m->gp;
  if (f->prec == 64)
    gp_solve<double><<<m->nbox, kGpSolveThreads, 0, s>>>(m->dprobs, m->boxes, f->boxes, f->perm, f->lptr, f->tab,
                                                    (const double*)f->F, (double*)f->V, r, z, gate);
  else
    gp_solve<float><<<m->nbox, kGpSolveThreads, 0, s>>>(m->dprobs, m->boxes, f->boxes, f->perm, f->lptr, f->tab,
                                                   (const float*)f->F, (float*)f->V, r, z, gate);
  KKT_COUNT(1);
  KKT_TRY_CUDA(cudaGetLastError());
  return KKT_OK;
}

void gp_destroy(ras_precond* m) {
  delete m->gp;
  m->gp = nullptr;
}

// Tables, schedule and storage of the pattern-driven factors of m's boxes.
kkt_status gp_create(ras_precond* m, int local, int prec) {
  GpFactor* f = new (std::nothrow) GpFactor();
  if (!f) return KKT_ERR_NOMEM;
  m->gp = f;
  f->local = local;
  f->prec = prec;
  const auto rows = gp_rows(local);
  GpTables& tb = f->tab;
  tb.K = local == 2 ? 1 : 0;
  std::vector<GpSlot> all;
  for (int c = 0; c < 3; ++c) {
    if ((int)rows[c].size() > kGpMaxRow) {
      set_error("ras_setup: internal error: a pattern row exceeds the kernel's level buffer");
      return KKT_ERR_ARG;
    }
    tb.base[c] = (int)all.size();
    tb.cnt[c] = (int)rows[c].size();
    tb.diag[c] = -1;
    for (int u = 0; u < tb.cnt[c]; ++u) {
      const GpSlot& sl = rows[c][u];
      if (sl.dt == 0 && sl.dz == 0 && sl.dy == 0 && sl.dx == 0 && sl.cc == c) tb.diag[c] = u;
      all.push_back(sl);
    }
    if (tb.diag[c] < 0) {
      set_error("ras_setup: internal error: a pattern row has no diagonal");
      return KKT_ERR_ARG;
    }
  }
  tb.S = (int)all.size();
  // the ILU(0) slot of each slot (its value comes from slot_value)
  signed char gen[kSlots][5];
  KKT_TRY_CUDA(cudaMemcpyFromSymbol(gen, c_gen_slot, sizeof(gen)));
  auto key = [](int c, int dt, int dz, int dy, int dx, int cc) {
    return ((((c * 3 + dt + 1) * 3 + dz + 1) * 3 + dy + 1) * 3 + dx + 1) * 3 + cc;
  };
  std::map<int, int> gen_of;
  for (int s = 0; s < kSlots; ++s) {
    const int c = s < kGenRowSlots0 ? 0 : (s < kGenRowSlots0 + kGenRowSlots1 ? 1 : 2);
    gen_of[key(c, gen[s][0], gen[s][1], gen[s][2], gen[s][3], gen[s][4])] = s;
  }
  std::vector<signed char> slot(5 * (size_t)tb.S);
  std::vector<short> smap(tb.S, -1);
  int R = 0;
  for (int c = 0; c < 3; ++c)
    for (int u = 0; u < tb.cnt[c]; ++u) {
      const GpSlot& sl = all[tb.base[c] + u];
      const int s = tb.base[c] + u;
      slot[5 * s] = (signed char)sl.dt;
      slot[5 * s + 1] = (signed char)sl.dz;
      slot[5 * s + 2] = (signed char)sl.dy;
      slot[5 * s + 3] = (signed char)sl.dx;
      slot[5 * s + 4] = (signed char)sl.cc;
      if (std::abs(sl.dt) <= 1 && std::abs(sl.dz) <= 1 && std::abs(sl.dy) <= 1 && std::abs(sl.dx) <= 1) {
        const auto it = gen_of.find(key(c, sl.dt, sl.dz, sl.dy, sl.dx, sl.cc));
        if (it != gen_of.end()) smap[s] = (short)it->second;
      }
      if (u < tb.diag[c])
        R = std::max({R, std::abs(sl.dt), std::abs(sl.dz), std::abs(sl.dy), std::abs(sl.dx)});
    }
  // update pairs: L slot s of row c (pivot row type cc_s at offset o_s) and U
  // slot t of the pivot row land on the row's slot u at o_s + o_t
  std::map<std::array<int, 6>, int> local_of;
  for (int c = 0; c < 3; ++c)
    for (int u = 0; u < tb.cnt[c]; ++u) {
      const GpSlot& sl = rows[c][u];
      local_of[{c, sl.dt, sl.dz, sl.dy, sl.dx, sl.cc}] = u;
    }
  std::vector<int> tptr(tb.S + 1, 0), tt;
  std::vector<short> tu;
  for (int c = 0; c < 3; ++c)
    for (int s = 0; s < tb.cnt[c]; ++s) {
      tptr[tb.base[c] + s] = (int)tt.size();
      if (s >= tb.diag[c]) continue;
      const GpSlot& a = rows[c][s];
      const int cs = a.cc;
      for (int t = tb.diag[cs] + 1; t < tb.cnt[cs]; ++t) {
        const GpSlot& b = rows[cs][t];
        const auto it = local_of.find({c, a.dt + b.dt, a.dz + b.dz, a.dy + b.dy, a.dx + b.dx, b.cc});
        if (it == local_of.end()) continue;
        if (it->second <= s) {
          set_error("ras_setup: internal error: an update lands left of its pivot slot");
          return KKT_ERR_ARG;
        }
        tt.push_back(tb.base[cs] + t);
        tu.push_back((short)it->second);
      }
    }
  tptr[tb.S] = (int)tt.size();
  // schedule: wavefronts x + b y + b^2 z + b^3 t, b = R + 1 (every L-slot column earlier)
  const int bw = R + 1;
  for (int c = 0; c < 3; ++c)
    for (int s = 0; s < tb.diag[c]; ++s) {
      const GpSlot& a = rows[c][s];
      if (a.dx + bw * (a.dy + bw * (a.dz + bw * a.dt)) >= 0 && !(a.dt == 0 && a.dz == 0 && a.dy == 0 && a.dx == 0)) {
        set_error("ras_setup: internal error: a pivot column is not on an earlier wavefront");
        return KKT_ERR_ARG;
      }
    }
  std::vector<int> perm, lptr;
  long long foff = 0, voff = 0;
  for (const BoxDesc& bx : m->boxes_h) {
    GpBox g{};
    g.P = (int)bx.P;
    g.foff = foff;
    g.voff = voff;
    g.poff = (long long)perm.size();
    g.loff = (long long)lptr.size();
    g.nlev = (bx.lx - 1) + bw * ((bx.ly - 1) + bw * ((bx.lz - 1) + bw * (bx.lt - 1))) + 1;
    std::vector<int> cnt(g.nlev + 1, 0);
    auto wof = [&](int lex) {
      const int kx = lex % bx.lx, ky = (lex / bx.lx) % bx.ly, kz = (lex / (bx.lx * bx.ly)) % bx.lz;
      const int kt = lex / (bx.lx * bx.ly * bx.lz);
      return kx + bw * (ky + bw * (kz + bw * kt));
    };
    for (int lex = 0; lex < g.P; ++lex) cnt[wof(lex) + 1]++;
    for (int w = 0; w < g.nlev; ++w) cnt[w + 1] += cnt[w];
    for (int w = 0; w <= g.nlev; ++w) lptr.push_back(cnt[w]);
    std::vector<int> pb(g.P);
    std::vector<int> fill(cnt.begin(), cnt.end() - 1);
    for (int lex = 0; lex < g.P; ++lex) {
      const int q = fill[wof(lex)]++;
      pb[q] = lex;
    }
    perm.insert(perm.end(), pb.begin(), pb.end());
    f->boxes_h.push_back(g);
    foff += (long long)tb.S * g.P;
    voff += 3LL * g.P;
  }
  f->fcount = foff;
  f->vcount = voff;
  const size_t esz = prec == 64 ? sizeof(double) : sizeof(float);
  auto up = [&](auto** dst, const auto& v) -> kkt_status {
    using E = typename std::remove_reference<decltype(v[0])>::type;
    if (cudaMalloc((void**)dst, std::max<size_t>(1, v.size()) * sizeof(E)) != cudaSuccess) {
      cudaGetLastError();
      set_error("ras_setup: device allocation failed (pattern tables)");
      return KKT_ERR_NOMEM;
    }
    if (!v.empty()) KKT_TRY_CUDA(cudaMemcpy(*dst, v.data(), v.size() * sizeof(E), cudaMemcpyHostToDevice));
    return KKT_OK;
  };
  KKT_TRY(up(&f->boxes, f->boxes_h));
  KKT_TRY(up(&f->perm, perm));
  KKT_TRY(up(&f->lptr, lptr));
  KKT_TRY(up(&f->slot, slot));
  KKT_TRY(up(&f->smap, smap));
  KKT_TRY(up(&f->tptr, tptr));
  KKT_TRY(up(&f->tt, tt));
  KKT_TRY(up(&f->tu, tu));
  if (cudaMalloc(&f->F, std::max<long long>(1, f->fcount) * esz) != cudaSuccess ||
      cudaMalloc(&f->LV, std::max<long long>(1, f->fcount)) != cudaSuccess ||
      cudaMalloc(&f->V, std::max<long long>(1, f->vcount) * esz) != cudaSuccess) {
    cudaGetLastError();
    set_error("ras_setup: device allocation failed (" + std::to_string(f->fcount) + " factor values)");
    return KKT_ERR_NOMEM;
  }
  tb.slot = f->slot;
  tb.smap = f->smap;
  tb.tptr = f->tptr;
  tb.tt = f->tt;
  tb.tu = f->tu;
  return KKT_OK;
}

long long gp_factor_count(const ras_precond* m) { return m->gp ? m->gp->fcount : 0; }
