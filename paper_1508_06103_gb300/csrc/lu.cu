// Exact local solves of the one-level RAS: LU with partial pivoting of every
// subdomain matrix M_ij = R^delta F_h (R^delta)^T (Sec. 3.2, Eq. 10-12), FP64.
//
// Storage.  The unknowns of a box are numbered in its natural point-block
// order, u = 3 lex + c with lex = kx + lx (ky + ly (kz + lz kt)).  Every
// coupling of the KKT stencil then lies within kl = 3 (1 + lx + lx ly +
// lx ly lz) + 2 of the diagonal on either side, so the matrix is stored as a
// band, column-major with leading dimension ld = 3 kl + 1 (kl rows below the
// diagonal, kl above, and kl more for the fill that row interchanges bring
// into U): A(i, k) sits at A[(2 kl + i - k) + ld k].
//
// Factorisation (the column-by-column LU with partial pivoting of a band
// matrix): at step j the pivot is the first entry of largest magnitude in
// column j on or below the diagonal; rows j and p are interchanged in the
// columns j..ju (ju: the last column that fill can have reached), and the
// rank-1 update A(i, k) -= l_i u_k is applied below row j.  One launch per
// step covers all boxes; several CTAs share a box, each finds the pivot
// itself from column j and updates its own columns, and column j's own
// interchange and scaling by 1/pivot are written at the next step, when no
// CTA reads it any more.
//
// Solve.  One CTA per box: gather R^delta r, forward sweep with the row
// interchanges and the unit lower factor, backward sweep with U, scatter the
// owned part (R^0)^T; the box vector lives in shared memory.

#include <algorithm>
#include <cmath>

#include "slotval.cuh"

namespace {

constexpr int kLuThreads = 1024;
constexpr int kLuGather = 256;

__device__ __forceinline__ double* band_col(double* AB, const BoxDesc& bx, int k) {
  const int kl = bx.kl, ld = 3 * kl + 1;
  return AB + bx.aoff + (long long)ld * k + 2 * kl - k;   // [i] = A(i, k)
}

// the entries of every box matrix into its band (the band is zeroed before)
__global__ void __launch_bounds__(kLuGather) gather_band(DevProblem p, const BoxDesc* __restrict__ boxes,
                                                         double* __restrict__ AB) {
  const BoxDesc bx = boxes[blockIdx.y];
  const long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (q >= bx.P) return;
  const int lex = (int)q;
  const Coefs<double> cf = coefs<double>(p);
  const PointRow<double> pr = point_row<double>(p, bx, lex);
  for (int s = 0; s < kSlots; ++s) {
    bool inb;
    const double v = slot_value<double>(p, bx, cf, pr, s, &inb);
    if (!inb) continue;
    const int c = s < kGenRowSlots0 ? 0 : (s < kGenRowSlots0 + kGenRowSlots1 ? 1 : 2);
    const int dt = c_gen_slot[s][0], dz = c_gen_slot[s][1], dy = c_gen_slot[s][2], dx = c_gen_slot[s][3];
    const int cc = c_gen_slot[s][4];
    const int lex2 = lex + dx + bx.lx * (dy + bx.ly * (dz + bx.lz * dt));
    const int i = 3 * lex + c, k = 3 * lex2 + cc;
    band_col(AB, bx, k)[i] = v;
  }
}

// One elimination step j for every box (grid: CTAs per box x boxes).  At
// j = n it only finishes column n - 1.
__global__ void __launch_bounds__(kLuThreads) lu_step(const BoxDesc* __restrict__ boxes, double* __restrict__ AB,
                                                      int* __restrict__ ipiv, int* __restrict__ ju2,
                                                      int* __restrict__ status, int j) {
  __shared__ double col[kMaxLuBand + 1];
  __shared__ double red_v[kLuThreads / 32];
  __shared__ int red_i[kLuThreads / 32];
  const BoxDesc bx = boxes[blockIdx.y];
  const int n = 3 * (int)bx.P, kl = bx.kl;
  int* ip = ipiv + 3 * bx.poff;
  // finish column j - 1: its interchange and its multipliers
  if (blockIdx.x == 0 && j >= 1 && j - 1 < n) {
    double* Ac = band_col(AB, bx, j - 1);
    const int jj = j - 1, p = ip[jj], km = min(kl, n - 1 - jj);
    const double a = Ac[jj], b = Ac[p];
    const double piv = b;
    const double rp = piv != 0.0 ? 1.0 / piv : 0.0;
    for (int t = 1 + threadIdx.x; t <= km; t += blockDim.x) {
      const double v = (jj + t == p) ? a : Ac[jj + t];
      Ac[jj + t] = v * rp;
    }
    __syncthreads();
    if (threadIdx.x == 0) Ac[jj] = piv;
  }
  if (j >= n) return;
  const double* Aj = band_col(AB, bx, j);
  const int km = min(kl, n - 1 - j);
  // pivot: first entry of largest magnitude on or below the diagonal
  double best = -1.0;
  int bi = 0;
  for (int t = threadIdx.x; t <= km; t += blockDim.x) {
    const double v = Aj[j + t];
    col[t] = v;
    if (fabs(v) > best) {
      best = fabs(v);
      bi = t;
    }
  }
  for (int o = 16; o > 0; o >>= 1) {
    const double ov = __shfl_xor_sync(0xffffffffu, best, o);
    const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
    if (ov > best || (ov == best && oi < bi)) {
      best = ov;
      bi = oi;
    }
  }
  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32, nw = blockDim.x / 32;
  if (lane == 0) {
    red_v[warp] = best;
    red_i[warp] = bi;
  }
  __syncthreads();
  best = red_v[0];
  bi = red_i[0];
  for (int w = 1; w < nw; ++w)
    if (red_v[w] > best || (red_v[w] == best && red_i[w] < bi)) {
      best = red_v[w];
      bi = red_i[w];
    }
  const int jp = bi;
  const double piv = col[jp];
  const int ju_in = ju2[2 * blockIdx.y + (j & 1)];
  const int ju = max(ju_in, min(j + kl + jp, n - 1));
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    ju2[2 * blockIdx.y + ((j + 1) & 1)] = ju;
    ip[j] = j + jp;
    if (!(piv != 0.0) || !isfinite(piv)) atomicExch(status, 1);
  }
  const double rp = piv != 0.0 ? 1.0 / piv : 0.0;
  // columns j+1..ju, one warp per column
  for (int k = j + 1 + blockIdx.x * nw + warp; k <= ju; k += gridDim.x * nw) {
    double* Ak = band_col(AB, bx, k);
    double u = Ak[j];
    if (jp != 0) {
      const double w = Ak[j + jp];
      if (lane == 0) {
        Ak[j + jp] = u;
        Ak[j] = w;
      }
      u = w;
    }
    __syncwarp();
    if (u != 0.0)
      for (int t = 1 + lane; t <= km; t += 32) {
        const double l = (t == jp ? col[0] : col[t]) * rp;
        Ak[j + t] -= l * u;
      }
  }
}

// z = sum over boxes (R^0)^T M_ij^{-1} R^delta r with the band LU factors
__global__ void __launch_bounds__(kLuThreads) lu_solve(const BoxDesc* __restrict__ boxes,
                                                       const double* __restrict__ AB, const int* __restrict__ ipiv,
                                                       const double* __restrict__ r, double* __restrict__ z, int nx,
                                                       int ny, int N, const int* gate) {
  if (gated_off(gate)) return;
  extern __shared__ __align__(16) double bvec[];
  const BoxDesc bx = boxes[blockIdx.x];
  const int n = 3 * (int)bx.P, kl = bx.kl;
  const int* ip = ipiv + 3 * bx.poff;
  for (int u = threadIdx.x; u < n; u += blockDim.x) {
    const int lex = u / 3, c = u - 3 * lex;
    const int kx = lex % bx.lx, ky = (lex / bx.lx) % bx.ly, kz = (lex / (bx.lx * bx.ly)) % bx.lz;
    const int kt = lex / (bx.lx * bx.ly * bx.lz);
    const long long g =
        ((long long)(bx.t0 + kt) * N + (bx.x0 + kx) + (long long)nx * ((bx.y0 + ky) + (long long)ny * (bx.z0 + kz))) * 3;
    bvec[u] = r[g + c];
  }
  __syncthreads();
  // forward: interchanges and the unit lower factor
  for (int j = 0; j < n - 1; ++j) {
    const int p = ip[j];
    const double bj = bvec[p];
    __syncthreads();
    if (threadIdx.x == 0 && p != j) {
      bvec[p] = bvec[j];
      bvec[j] = bj;
    }
    const double* Aj = band_col(const_cast<double*>(AB), bx, j);
    const int km = min(kl, n - 1 - j);
    for (int t = 1 + threadIdx.x; t <= km; t += blockDim.x)
      if (j + t != p) bvec[j + t] -= Aj[j + t] * bj;
    if (threadIdx.x == 0 && p != j) bvec[p] -= Aj[p] * bj;
    __syncthreads();
  }
  // backward: U has 2 kl superdiagonals
  for (int j = n - 1; j >= 0; --j) {
    const double* Aj = band_col(const_cast<double*>(AB), bx, j);
    const double xj = bvec[j] / Aj[j];
    __syncthreads();
    if (threadIdx.x == 0) bvec[j] = xj;
    const int lo = max(0, j - 2 * kl);
    for (int i = lo + threadIdx.x; i < j; i += blockDim.x) bvec[i] -= Aj[i] * xj;
    __syncthreads();
  }
  // scatter the owned part
  const int ox = bx.ox1 - bx.ox0, oy = bx.oy1 - bx.oy0, oz = bx.oz1 - bx.oz0, ot = bx.ot1 - bx.ot0;
  const long long nown = (long long)ox * oy * oz * ot;
  for (long long q = threadIdx.x; q < nown; q += blockDim.x) {
    const int gx = bx.ox0 + (int)(q % ox), gy = bx.oy0 + (int)((q / ox) % oy);
    const int gz = bx.oz0 + (int)((q / ((long long)ox * oy)) % oz), gt = bx.ot0 + (int)(q / ((long long)ox * oy * oz));
    const int lex = (gx - bx.x0) + bx.lx * ((gy - bx.y0) + bx.ly * ((gz - bx.z0) + bx.lz * (gt - bx.t0)));
    const long long g = ((long long)gt * N + gx + (long long)nx * (gy + (long long)ny * gz)) * 3;
    z[g] = bvec[3 * lex];
    z[g + 1] = bvec[3 * lex + 1];
    z[g + 2] = bvec[3 * lex + 2];
  }
}

}  // namespace

kkt_status ras_lu_factor(ras_precond* m, cudaStream_t s) {
  const DevProblem dp = m->prob->dev();
  long long pmax = 0;
  int nmax = 0;
  for (const BoxDesc& b : m->boxes_h) {
    pmax = std::max(pmax, b.P);
    nmax = std::max(nmax, 3 * (int)b.P);
  }
  // the solve keeps a box's vector in shared memory (at most kMaxLuUnknowns values); the
  // limit is raised here, at set-up, so the solve's launch needs no attribute call
  KKT_TRY_CUDA(cudaFuncSetAttribute(lu_solve, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)(kMaxLuUnknowns * sizeof(double))));
  KKT_TRY_CUDA(cudaMemsetAsync(m->AB, 0, m->ab_count * sizeof(double), s));
  KKT_TRY_CUDA(cudaMemsetAsync(m->lu_ju, 0, 2 * m->nbox * sizeof(int), s));
  const dim3 g((unsigned)((pmax + kLuGather - 1) / kLuGather), m->nbox);
  gather_band<<<g, kLuGather, 0, s>>>(dp, m->boxes, m->AB);
  KKT_COUNT(1);
  KKT_TRY_CUDA(cudaGetLastError());
  const dim3 sg(m->lu_ctas, m->nbox);
  for (int j = 0; j <= nmax; ++j) {
    lu_step<<<sg, kLuThreads, 0, s>>>(m->boxes, m->AB, m->ipiv, m->lu_ju, m->status, j);
    KKT_COUNT(1);
  }
  KKT_TRY_CUDA(cudaGetLastError());
  return KKT_OK;
}

kkt_status ras_lu_solve(ras_precond* m, const double* r, double* z, cudaStream_t s, const int* gate) {
  const kkt_problem* p = m->prob;
  int nmax = 0;
  for (const BoxDesc& b : m->boxes_h) nmax = std::max(nmax, 3 * (int)b.P);
  const size_t smem = (size_t)nmax * sizeof(double);
  lu_solve<<<m->nbox, kLuThreads, smem, s>>>(m->boxes, m->AB, m->ipiv, r, z, p->nx, p->ny, p->N, gate);
  KKT_COUNT(1);
  KKT_TRY_CUDA(cudaGetLastError());
  return KKT_OK;
}
