// ILU(0) factorisation of all subdomain matrices (Sec. 3.2), in place on the
// chunk layout that the subdomain solve streams.  Included by factor32.cu and
// factor64.cu, one translation unit per precision (the generated elimination
// code is large, and the two compile in parallel).
//
// Values.  gather_chunks forms every slot value of every box point from the
// stencil coefficients (the principal submatrix of F_h on the extended box,
// Eq. 10-12; a slot whose column leaves the box holds 0) and writes it to the
// point's column of its chunk block, row c_gen_rank[slot] (c_gen_rank_of by
// the slot's offsets).
//
// Elimination.  One CTA per box steps through the wavefronts
// w = x + 2y + 4z + 8t with a barrier between them; one thread takes one point
// of the wavefront and eliminates its C, G and f rows in turn with the
// straight-line code of ilu_rows.inc.  The thread first lists where the
// columns of its 41 possible pivot points are (offset and row stride of their
// chunk blocks); a pivot point outside the box is sent to the box's unit row
// (stride 1, 1 at the three diagonal ranks, 0 elsewhere).  The diagonal slot
// of a finished row holds 1/u_kk.
#pragma once

#include "slotval.cuh"

namespace {

#include "ilu_rows.inc"

constexpr int kGatherThreads = 256;
// Threads per factor CTA, two CTAs per SM (all 256 boxes of the 4x4x4x4
// partition resident at once).  FP32 rows fit 192 threads without large
// spills; FP64 rows need the registers of 128.
template <typename T>
constexpr int factor_threads = sizeof(T) == 4 ? 192 : 128;

// One thread per point (wavefront order, so the threads of a chunk write
// consecutive addresses); all threads of a warp on the same slot.  Entries are
// formed in the factor precision, with the arithmetic of slot_value, but one
// spatial offset at a time: the point's B, S, S^T and K coefficients of that
// offset are loaded once and give all 12 slots that share it (C row: C and f
// columns at levels n-1, n; G row: G column at n, n+1; f row: G and f columns
// at n-1, n, n+1), plus the G row's two sensor slots at the centre.  Also
// writes each box's unit row.
template <typename T>
__global__ void __launch_bounds__(kGatherThreads) gather_chunks(const DevProblem* __restrict__ probs,
                                                                const BoxDesc* __restrict__ boxes,
                                                                const int* __restrict__ perm,
                                                                const int2* __restrict__ ptab, T* __restrict__ F) {
  const BoxDesc bx = boxes[blockIdx.y];
  const DevProblem p = probs[bx.prob];
  T* Fb = F + bx.foff;
  if (blockIdx.x == 0)
    for (int s = threadIdx.x; s < kSlots; s += blockDim.x)
      Fb[bx.unit + c_gen_rank[s]] = (s == kDiagC || s == kDiagG || s == kDiagF) ? (T)1 : (T)0;
  const long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (q >= bx.P) return;
  const Coefs<T> cf = coefs<T>(p);
  const PointRow<T> pr = point_row<T>(p, bx, perm[bx.poff + q]);
  const int2 pt = ptab[bx.poff + q];
  T* dst = Fb + pt.x;
  const long long st = pt.y;
  const T tau = (T)p.tau, th = (T)p.theta, th1 = (T)(1.0 - p.theta), b1 = (T)p.beta1, b2 = (T)p.beta2;
  const T mt1 = tau / (T)6, lt1 = -(T)1 / tau;
  const bool idC = pr.n == 0 || pr.dirj, idG = pr.n == p.M || pr.dirj;   // identity rows
  const bool tm = pr.kt > 0, tp = pr.kt + 1 < bx.lt;                      // levels n-1, n+1 in the box
  const T z = (T)0;
  // slot (row type c, level offset dt, spatial offset d, column component cc)
#define PUT(c, dt, d, cc, v) dst[(long long)c_gen_rank_of[c][(dt) + 1][d][cc] * st] = (v)
#pragma unroll
  for (int d = 0; d < kStencil; ++d) {
    const int dx = d % 3 - 1, dy = (d / 3) % 3 - 1, dz = d / 9 - 1;
    const int ax = pr.kx + dx, ay = pr.ky + dy, az = pr.kz + dz;
    const bool sp = ax >= 0 && ax < bx.lx && ay >= 0 && ay < bx.ly && az >= 0 && az < bx.lz;
    T Bv = z, Sv = z, STv = z, Kv = z;
    if (sp) {
      const size_t ci = (size_t)d * p.N + pr.j;
      Bv = cf.B[ci];
      Sv = cf.S[ci];
      STv = cf.ST[ci];
      Kv = p.reg ? Bv : cf.K[ci];   // beta2 term: K (H1-H1) or B (H1-L2)
    }
    constexpr int kCentre = 13;
    // C row
    PUT(0, 0, d, 0, !sp ? z : idC ? (d == kCentre ? (T)1 : z) : Bv + th * tau * Sv);
    PUT(0, 0, d, 2, !sp || idC ? z : -th * tau * Bv);
    PUT(0, -1, d, 0, !sp || !tm || idC ? z : -Bv + th1 * tau * Sv);
    PUT(0, -1, d, 2, !sp || !tm || idC ? z : -th1 * tau * Bv);
    // G row
    PUT(1, 0, d, 1, !sp ? z : idG ? (d == kCentre ? (T)1 : z) : Bv + th * tau * STv);
    PUT(1, 1, d, 1, !sp || !tp || idG ? z : -Bv + th1 * tau * STv);
    if (d == kCentre) {
      PUT(1, 0, d, 0, idG ? z : th1 * tau * pr.sj);
      PUT(1, 1, d, 0, !tp || idG ? z : th * tau * pr.sj);
    }
    // f row
    PUT(2, -1, d, 1, !sp || !tm ? z : -mt1 * Bv);
    PUT(2, -1, d, 2, !sp || !tm ? z : b1 * lt1 * Bv + b2 * mt1 * Kv);
    PUT(2, 0, d, 1, !sp ? z : -pr.mt0 * Bv);
    PUT(2, 0, d, 2, !sp ? z : b1 * pr.lt0 * Bv + b2 * pr.mt0 * Kv);
    PUT(2, 1, d, 1, !sp || !tp ? z : -mt1 * Bv);
    PUT(2, 1, d, 2, !sp || !tp ? z : b1 * lt1 * Bv + b2 * mt1 * Kv);
  }
#undef PUT
}

__device__ __forceinline__ void check_pivot(double d, int* status) {
  if (!(fabs(d) > 1e-300) || !isfinite(d)) atomicExch(status, 1);
}

template <typename T>
__global__ void __launch_bounds__(factor_threads<T>, 2) ilu0_factor(const BoxDesc* __restrict__ boxes,
                                                                    const int* __restrict__ iperm,
                                                                    const int* __restrict__ perm,
                                                                    const int* __restrict__ lptr,
                                                                    const int2* __restrict__ ptab,
                                                                    T* __restrict__ F, int* __restrict__ status) {
  // per thread and pivot point: {offset of its column in Fb, row stride of its block}
  constexpr int NS = factor_threads<T>;
  __shared__ int2 nbs[kGenNbrs * NS];
  const BoxDesc bx = boxes[blockIdx.x];
  T* Fb = F + bx.foff;
  const int* lp = lptr + bx.loff;
  const int* ip = iperm + bx.poff;
  const int2* pb = ptab + bx.poff;
  int2* nb = nbs + threadIdx.x;
  const int unit = (int)bx.unit;
  for (int w = 0; w < bx.nlev; ++w) {
    const int npts = lp[w + 1] - lp[w];
    for (int j = threadIdx.x; j < npts; j += blockDim.x) {
      const int q = lp[w] + j;
      const int lex = perm[bx.poff + q];
      const int kx = lex % bx.lx, ky = (lex / bx.lx) % bx.ly, kz = (lex / (bx.lx * bx.ly)) % bx.lz;
      const int kt = lex / (bx.lx * bx.ly * bx.lz);
#pragma unroll 1
      for (int i = 0; i < kGenNbrs; ++i) {
        const int dt = c_gen_nbr[i][0], dz = c_gen_nbr[i][1], dy = c_gen_nbr[i][2], dx = c_gen_nbr[i][3];
        const int ax = kx + dx, ay = ky + dy, az = kz + dz, at = kt + dt;
        int2 e = make_int2(unit, 1);
        if (ax >= 0 && ax < bx.lx && ay >= 0 && ay < bx.ly && az >= 0 && az < bx.lz && at >= 0 && at < bx.lt)
          e = pb[ip[ax + bx.lx * (ay + bx.ly * (az + bx.lz * at))]];
        nb[i * NS] = e;
      }
      const int2 pt = pb[q];
      T* own = Fb + pt.x;
      // the G and f rows read the U parts of this point's C and G rows
      if constexpr (sizeof(T) == 4) {
        check_pivot((double)ilu_row0_32<T, NS>(own, pt.y, Fb, nb), status);
        asm volatile("" ::: "memory");
        check_pivot((double)ilu_row1_32<T, NS>(own, pt.y, Fb, nb), status);
        asm volatile("" ::: "memory");
        check_pivot((double)ilu_row2_32<T, NS>(own, pt.y, Fb, nb), status);
      } else {
        check_pivot((double)ilu_row0_64<T, NS>(own, pt.y, Fb, nb), status);
        asm volatile("" ::: "memory");
        check_pivot((double)ilu_row1_64<T, NS>(own, pt.y, Fb, nb), status);
        asm volatile("" ::: "memory");
        check_pivot((double)ilu_row2_64<T, NS>(own, pt.y, Fb, nb), status);
      }
    }
    __syncthreads();
  }
}

// gather, then factor, in place on F (chunk layout); both on stream s
template <typename T>
kkt_status factor_launch(ras_precond* m, T* F, cudaStream_t s) {
  long long pmax = 0;
  for (const BoxDesc& b : m->boxes_h) pmax = std::max(pmax, b.P);
  const dim3 g((unsigned)((pmax + kGatherThreads - 1) / kGatherThreads), m->nbox);
  gather_chunks<T><<<g, kGatherThreads, 0, s>>>(m->dprobs, m->boxes, m->perm, m->ptab, F);
  KKT_COUNT(1);
  KKT_TRY_CUDA(cudaGetLastError());
  {
    TimedScope timed(&m->factor_timing, s);
    ilu0_factor<T><<<m->nbox, factor_threads<T>, 0, s>>>(m->boxes, m->iperm, m->perm, m->lptr, m->ptab, F,
                                                      m->status);
  }
  KKT_COUNT(1);
  KKT_TRY_CUDA(cudaGetLastError());
  return KKT_OK;
}

}  // namespace
