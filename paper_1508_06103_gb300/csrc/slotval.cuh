// Values of the subdomain matrices M_ij = R^delta F_h (R^delta)^T (Eq. 10-12),
// slot by slot: the principal submatrix of F_h on an extended box, so a slot
// whose column leaves the box is 0.  The exact banded LU (lu.cu) gathers
// with slot_value; the ILU(0) gather (factor.cuh) uses the per-point
// constants and forms the same values one spatial offset at a time.
// Entries are formed in the precision T of the factorisation from the
// stencil coefficients of problem.cu (the Appendix block rows with the theta
// scheme).
#pragma once

#include "internal.cuh"
#include "ras.cuh"

namespace {

#include "ilu_slots.inc"

static_assert(kGenSlots == kSlots, "slot count");

template <typename T>
struct Coefs {
  const T *S, *ST, *B, *K;
};
template <typename T>
__device__ __forceinline__ Coefs<T> coefs(const DevProblem& p);
template <>
__device__ __forceinline__ Coefs<double> coefs<double>(const DevProblem& p) {
  return {p.S, p.ST, p.B, p.K};
}
template <>
__device__ __forceinline__ Coefs<float> coefs<float>(const DevProblem& p) {
  return {p.S32, p.ST32, p.B32, p.K32};
}

// diagonal slots of the C, G and f rows
constexpr int kDiagC = 80, kDiagG = 122, kDiagF = 245;

// Per-point constants of the slot values.
template <typename T>
struct PointRow {
  int kx, ky, kz, kt;       // box-local position
  int j, n;                 // global node and level
  bool dirj;                // Dirichlet node
  T sj;                     // sensor count
  T mt0, lt0;               // time weights of the f row at this level
};

template <typename T>
__device__ __forceinline__ PointRow<T> point_row(const DevProblem& p, const BoxDesc& bx, int lex) {
  PointRow<T> pr;
  pr.kx = lex % bx.lx;
  pr.ky = (lex / bx.lx) % bx.ly;
  pr.kz = (lex / (bx.lx * bx.ly)) % bx.lz;
  pr.kt = lex / (bx.lx * bx.ly * bx.lz);
  const int gx = bx.x0 + pr.kx, gy = bx.y0 + pr.ky, gz = bx.z0 + pr.kz;
  pr.n = bx.t0 + pr.kt;
  pr.j = gx + p.nx * (gy + p.ny * gz);
  pr.dirj = p.dir[pr.j] != 0;
  pr.sj = (T)p.sens[pr.j];
  const T tau = (T)p.tau;
  pr.mt0 = (pr.n > 0 ? tau / (T)3 : (T)0) + (pr.n < p.M ? tau / (T)3 : (T)0);
  pr.lt0 = (pr.n > 0 ? (T)1 / tau : (T)0) + (pr.n < p.M ? (T)1 / tau : (T)0);
  return pr;
}

// Value of slot s of the point (0 when the slot's column leaves the box);
// *in_box tells whether the column is inside.
template <typename T>
__device__ __forceinline__ T slot_value(const DevProblem& p, const BoxDesc& bx, const Coefs<T>& cf,
                                        const PointRow<T>& pr, int s, bool* in_box) {
  const int dt = c_gen_slot[s][0], dz = c_gen_slot[s][1], dy = c_gen_slot[s][2], dx = c_gen_slot[s][3];
  const int cc = c_gen_slot[s][4];
  const int ax = pr.kx + dx, ay = pr.ky + dy, az = pr.kz + dz, at = pr.kt + dt;
  const bool inb = ax >= 0 && ax < bx.lx && ay >= 0 && ay < bx.ly && az >= 0 && az < bx.lz && at >= 0 && at < bx.lt;
  *in_box = inb;
  if (!inb) return (T)0;
  const T tau = (T)p.tau, th = (T)p.theta, th1 = (T)(1.0 - p.theta), b1 = (T)p.beta1, b2 = (T)p.beta2;
  const int d = (dx + 1) + 3 * (dy + 1) + 9 * (dz + 1);
  const size_t ci = (size_t)d * p.N + pr.j;
  const int n = pr.n;
  if (s < kGenRowSlots0) {
    if (n == 0 || pr.dirj) return (s == kDiagC) ? (T)1 : (T)0;
    if (cc == 0) return dt == 0 ? cf.B[ci] + th * tau * cf.S[ci] : -cf.B[ci] + th1 * tau * cf.S[ci];
    return dt == 0 ? -th * tau * cf.B[ci] : -th1 * tau * cf.B[ci];
  }
  if (s < kGenRowSlots0 + kGenRowSlots1) {
    if (n == p.M || pr.dirj) return (s == kDiagG) ? (T)1 : (T)0;
    if (cc == 1) return dt == 0 ? cf.B[ci] + th * tau * cf.ST[ci] : -cf.B[ci] + th1 * tau * cf.ST[ci];
    return (dt == 0 ? th1 : th) * tau * pr.sj;
  }
  const T mt1 = tau / (T)6, lt1 = -(T)1 / tau;
  const T mt = dt == 0 ? pr.mt0 : mt1, lt = dt == 0 ? pr.lt0 : lt1;
  return cc == 1 ? -mt * cf.B[ci] : b1 * lt * cf.B[ci] + b2 * mt * (p.reg ? cf.B[ci] : cf.K[ci]);
}

}  // namespace
