// KKT matvec y = F_h x: one fused pass of the 4D (x, y, z, t) stencil over
// the three fields (Appendix block rows; Eq. 8-9).  With S = A + E_s and the
// theta weights (theta = 1/2: Crank-Nicolson):
//   C row, n >= 1 : B (C^n - C^{n-1}) + tau S (theta C^n + (1-theta) C^{n-1})
//                   - tau B (theta f^n + (1-theta) f^{n-1})
//   G row, n < M  : B (G^n - G^{n+1}) + tau S^T (theta G^n + (1-theta) G^{n+1})
//                   + tau s_j (theta C_j^{n+1} + (1-theta) C_j^n)
//   f row         : B (-sum_m Mt[n,m] G^m + beta1 sum_m Lt[n,m] f^m)
//                   + beta2 K (sum_m Mt[n,m] f^m)
//   identity rows : C^0, G^M and C, G on Dirichlet nodes.
// Mt, Lt are the 1D linear-element time mass and stiffness (tau/6 [1 4 1],
// [-1 2 -1]/tau, halved diagonals at the end levels).
//
// matvec_tiled below computes all three output slots of a space-time point
// in one pass: four spatial operators applied to six time combinations, B and
// K by sum factorisation, S and S^T as 27-point stencils.  Under P1 elements
// on the Kuhn split (kkt_set_element) B and K are no tensor products: all four
// operators are applied as stencils over the 15 offsets the split couples.

#include "internal.cuh"

namespace {

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

// ---------------------------------------------------------------------------
// Tiled matvec: one CTA owns a TX x TY x TZ tile of nodes and a run of NT time
// levels (NT = levels_per_cta<T>(): 4 in FP64, 8 in FP32); one thread per
// output node.  Per level the six time combinations
//   u1 = (C^n - C^{n-1}) - tau (theta f^n + (1-theta) f^{n-1})   (C row, via B)
//   u2 = tau (theta C^n + (1-theta) C^{n-1})                        (C row, via S)
//   u3 = G^n - G^{n+1}                                              (G row, via B)
//   u4 = tau (theta G^n + (1-theta) G^{n+1})                        (G row, via S^T)
//   u5 = -(Mt G)_n + beta1 (Lt f)_n                                 (f row, via B)
//   u6 = beta2 (Mt f)_n                                             (f row, via K;
//        via B, added to u5, under the H1-L2 regularisation)
// are formed once per halo node.  B = Mx (x) My (x) Mz and K = Kx My Mz +
// Mx Ky Mz + Mx My Kz are tensor products of the 1D linear-element mass and
// stiffness matrices on the uniform grid, so B u1, B u3, B u5 and K u6 are
// applied by sum factorisation: a pass along x over the tile and its y, z
// halo, one along y, one along z, with 1D factors computed from the mesh
// widths (no coefficient loads).  S and S^T, whose coefficients vary from
// node to node, are applied as 27-point stencils; in FP32 each thread keeps
// its node's 54 coefficients in registers for all NT levels.  Levels of x
// stream into a ring of four shared-memory slots with cp.async two levels
// ahead of their use; halo nodes outside the domain are zero-filled, so the
// passes need no bounds tests.
// ---------------------------------------------------------------------------
// Tile shapes (nodes per CTA along x, y, z): 8 x 8 x 4, or 11 x 11 x 2, which
// covers grids of 11 k nodes per axis without ragged tiles (33^3 and 65^3
// nodes: 40 x 40 x 36 / 33^3 = 1.6x the nodes with 8 x 8 x 4 tiles); the host
// picks the shape with the least estimated work (launch_tiled).
// Levels per CTA: shorter runs give more CTAs for the same work (two halo
// levels more per run).  Measured at 32^3 x 64 with the inputs out of L2
// (runs of 16 / 8 / 4 levels): FP64 1.127 / 1.047 / 1.018 ms, FP32 0.158 /
// 0.153 / 0.159 ms.
template <typename T>
__host__ __device__ constexpr int levels_per_cta() {
  return sizeof(T) == 8 ? 4 : 8;
}
template <int TX_, int TY_, int TZ_>
struct Tile {
  static constexpr int TX = TX_, TY = TY_, TZ = TZ_;
  static constexpr int HX = TX + 2, HY = TY + 2, HZ = TZ + 2, NH = HX * HY * HZ;
  static constexpr int NXP = TX * HY * HZ;   // x-pass outputs: tile in x, halo in y and z
  static constexpr int NYP = TX * TY * HZ;   // y-pass outputs: tile in x and y, halo in z
  static constexpr int kThreads = TX * TY * TZ;
};
using TileA = Tile<8, 8, 4>;
using TileB = Tile<11, 11, 2>;

template <typename T, typename Tl, bool kP1 = false>
constexpr size_t mv_smem() {
  return kP1 ? sizeof(T) * (4 * 3 * Tl::NH + 6 * Tl::NH)
             : sizeof(T) * (4 * 3 * Tl::NH + 6 * Tl::NH + 5 * Tl::NXP + 5 * Tl::NYP);
}

// Stencil offset d = (dx+1) + 3 (dy+1) + 9 (dz+1) is an edge of the Kuhn split
// (or the node itself) when its nonzero components all have one sign.
__host__ __device__ constexpr bool kuhn_offset(int d) {
  const int dx = d % 3 - 1, dy = (d / 3) % 3 - 1, dz = d / 9 - 1;
  return !((dx > 0 || dy > 0 || dz > 0) && (dx < 0 || dy < 0 || dz < 0));
}

// 1D linear-element mass and stiffness rows on one axis of n nodes with
// width h: row i has (i > 0) + (i < n - 1) elements; the entries are chosen
// from values formed once on the host (no arithmetic per node).
template <typename T>
struct Axis1D {
  int n;
  T m1, m2, mo, k1, k2, ko;   // mass diagonal (one / two elements), off-diagonal; the same for stiffness
  T hh;                       // the width
  __host__ __device__ void init(int n_, double h) {
    n = n_;
    m1 = (T)(h / 3.0);
    m2 = (T)(2.0 * h / 3.0);
    mo = (T)(h / 6.0);
    k1 = (T)(1.0 / h);
    k2 = (T)(2.0 / h);
    ko = (T)(-1.0 / h);
    hh = (T)h;
  }
  // entries (i, i-1), (i, i), (i, i+1) of the mass (m) and stiffness (k) rows
  __device__ __forceinline__ void row(int i, T& m_, T& m0, T& mp, T& k_, T& k0, T& kp) const {
    const bool lo = i > 0, hi = i < n - 1;
    if constexpr (sizeof(T) == 8) {   // FP64: select only (the FP64 pipe is the limit)
      m_ = lo ? mo : (T)0;
      mp = hi ? mo : (T)0;
      m0 = lo && hi ? m2 : (lo || hi ? m1 : (T)0);
      k_ = lo ? ko : (T)0;
      kp = hi ? ko : (T)0;
      k0 = lo && hi ? k2 : (lo || hi ? k1 : (T)0);
    } else {                          // FP32: from the width per node (measured 4 % faster)
      m0 = (T)((i > 0) + (i < n - 1)) * hh / (T)3;
      m_ = lo ? hh / (T)6 : (T)0;
      mp = hi ? hh / (T)6 : (T)0;
      k0 = (T)((i > 0) + (i < n - 1)) / hh;
      k_ = lo ? -(T)1 / hh : (T)0;
      kp = hi ? -(T)1 / hh : (T)0;
    }
  }
};

// Weights of the six time combinations: the theta weights and the rows of
// the 1D linear-element time mass Mt (tau/6 [1 4 1]) and stiffness Lt
// ([-1 2 -1]/tau) scaled by beta1 and beta2.  A level has one time element
// on each side it has a neighbour; the diagonal entries for one and two
// elements are formed on the host, in T, so a level only selects.
template <typename T>
struct LevelW {
  T wt0, wt1;          // tau theta, tau (1 - theta)
  T mto, mtd1, mtd2;   // Mt: off-diagonal; diagonal with one, two elements
  T lo, ld1, ld2;      // beta1 Lt
  T ko, kd1, kd2;      // beta2 Mt
  void init(double tau_, double theta, double beta1, double beta2) {
    const T tau = (T)tau_, th = (T)theta, th1 = (T)(1.0 - theta), b1 = (T)beta1, b2 = (T)beta2;
    const T m6 = tau / (T)6, m3 = tau / (T)3, l1 = (T)1 / tau;
    wt0 = tau * th;
    wt1 = tau * th1;
    mto = m6;
    mtd1 = m3;
    mtd2 = m3 + m3;
    lo = b1 * -l1;
    ld1 = b1 * l1;
    ld2 = b1 * (l1 + l1);
    ko = b2 * m6;
    kd1 = b2 * m3;
    kd2 = b2 * (m3 + m3);
  }
};

// asynchronous global -> shared copy of one value; zero-filled when !valid
template <typename T>
__device__ __forceinline__ void cp_async_value(T* dst, const T* src, bool valid) {
  const unsigned d = static_cast<unsigned>(__cvta_generic_to_shared(dst));
  if constexpr (sizeof(T) == 8)
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;" ::"r"(d), "l"(src), "r"(valid ? 8 : 0) : "memory");
  else
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;" ::"r"(d), "l"(src), "r"(valid ? 4 : 0) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

// kL2: the H1-L2 regularisation (its beta2 term goes through B), a template
// argument so the H1-H1 kernel carries no test for it.  kP1: P1 elements, B and
// K as stored 15-point stencils (no x and y passes, two barriers per level).
template <typename T, bool kL2, typename Tl, bool kP1 = false>
__global__ void __launch_bounds__(Tl::kThreads) matvec_tiled(DevProblem p, const T* __restrict__ x,
                                                             T* __restrict__ y, const double* __restrict__ b,
                                                             int tiles_x, int tiles_y, Axis1D<T> ax, Axis1D<T> ay,
                                                             Axis1D<T> az, LevelW<T> W) {
  constexpr int TX = Tl::TX, TY = Tl::TY, TZ = Tl::TZ;
  constexpr int HX = Tl::HX, HY = Tl::HY, NH = Tl::NH, NXP = Tl::NXP, NYP = Tl::NYP;
  if (gated_off(p.gate)) return;
  extern __shared__ __align__(16) unsigned char mv_sm[];
  T* Xs = reinterpret_cast<T*>(mv_sm);   // [4 slots][3 components][NH]
  T* U = Xs + 4 * 3 * NH;                // [6][NH]
  T* PX = U + 6 * NH;                    // [5][NXP]
  T* PY = PX + 5 * NXP;                  // [5][NYP]
  const int N = p.N, M = p.M;
  const int tile = blockIdx.x;
  const int bx0 = (tile % tiles_x) * TX, by0 = ((tile / tiles_x) % tiles_y) * TY, bz0 = (tile / (tiles_x * tiles_y)) * TZ;
  constexpr int NT = levels_per_cta<T>();
  const int n0 = blockIdx.y * NT, n1 = min(n0 + NT, M + 1);
  const Coefs<T> c = coefs<T>(p);
  const T tau = (T)p.tau, th = (T)p.theta, th1 = (T)(1.0 - p.theta);
  const int t = threadIdx.x;
  const int tx = t % TX, ty = (t / TX) % TY, tz = t / (TX * TY);
  const int ix = bx0 + tx, iy = by0 + ty, iz = bz0 + tz;
  const bool own = ix < p.nx && iy < p.ny && iz < p.nz;
  const int j = own ? ix + p.nx * (iy + p.ny * iz) : 0;
  const int hc = (tx + 1) + HX * ((ty + 1) + HY * (tz + 1));

  auto prefetch = [&](int m) {   // level m of x on the halo into ring slot m mod 4
    T* dst = Xs + (size_t)(((m % 4) + 4) % 4) * 3 * NH;
    for (int h = t; h < NH; h += blockDim.x) {
      const int hx_ = h % HX, hy_ = (h / HX) % HY, hz_ = h / (HX * HY);
      const int gx = bx0 - 1 + hx_, gy = by0 - 1 + hy_, gz = bz0 - 1 + hz_;
      const bool valid = m >= 0 && m <= M && gx >= 0 && gx < p.nx && gy >= 0 && gy < p.ny && gz >= 0 && gz < p.nz;
      const T* src = valid ? x + 3 * ((long long)m * N + gx + (long long)p.nx * (gy + (long long)p.ny * gz)) : x;
      cp_async_value(dst + h, src, valid);
      cp_async_value(dst + NH + h, src + (valid ? 1 : 0), valid);
      cp_async_value(dst + 2 * NH + h, src + (valid ? 2 : 0), valid);
    }
  };
  // S and S^T (and under P1, B and K) of the thread's node: registers in
  // FP32, reloaded per level in FP64
  T cS[kStencil], cST[kStencil], cB[kStencil], cK[kStencil];
  if constexpr (sizeof(T) == 4) {
#pragma unroll
    for (int d = 0; d < kStencil; ++d) {
      if (kP1 && !kuhn_offset(d)) continue;
      cS[d] = own ? c.S[(size_t)d * N + j] : (T)0;
      cST[d] = own ? c.ST[(size_t)d * N + j] : (T)0;
      if constexpr (kP1) {
        cB[d] = own ? c.B[(size_t)d * N + j] : (T)0;
        cK[d] = own ? c.K[(size_t)d * N + j] : (T)0;
      }
    }
  }
  prefetch(n0 - 1);
  prefetch(n0);
  prefetch(n0 + 1);
  cp_async_commit();
  prefetch(n0 + 2);
  cp_async_commit();
  for (int n = n0; n < n1; ++n) {
    cp_async_wait<1>();   // levels n-1, n, n+1 have landed
    __syncthreads();
    const T* Xm = Xs + (size_t)(((n - 1) % 4 + 4) % 4) * 3 * NH;
    const T* X0 = Xs + (size_t)(n % 4) * 3 * NH;
    const T* Xp = Xs + (size_t)((n + 1) % 4) * 3 * NH;
    const bool hasm = n > 0, hasp = n < M;
    // the weights of the six combinations at this level
    const T wt0 = W.wt0, wt1 = W.wt1;
    const T mtm = hasm ? W.mto : (T)0, mtp = hasp ? W.mto : (T)0;
    const T lm = hasm ? W.lo : (T)0, lp = hasp ? W.lo : (T)0;
    const T km = hasm ? W.ko : (T)0, kp = hasp ? W.ko : (T)0;
    const T mt0 = hasm && hasp ? W.mtd2 : (hasm || hasp ? W.mtd1 : (T)0);
    const T l0 = hasm && hasp ? W.ld2 : (hasm || hasp ? W.ld1 : (T)0);
    const T k0 = hasm && hasp ? W.kd2 : (hasm || hasp ? W.kd1 : (T)0);
    for (int h = t; h < NH; h += blockDim.x) {
      const T Cm = Xm[h], Gm = Xm[NH + h], Fm = Xm[2 * NH + h];
      const T C0 = X0[h], G0 = X0[NH + h], F0 = X0[2 * NH + h];
      const T Gp = Xp[NH + h], Fp = Xp[2 * NH + h];
      U[h] = (C0 - Cm) - (wt0 * F0 + wt1 * Fm);
      U[NH + h] = wt0 * C0 + wt1 * Cm;
      U[2 * NH + h] = G0 - Gp;
      U[3 * NH + h] = wt0 * G0 + wt1 * Gp;
      const T u5 = (lm * Fm + l0 * F0 + lp * Fp) - (mtm * Gm + mt0 * G0 + mtp * Gp);
      const T u6 = km * Fm + k0 * F0 + kp * Fp;
      // H1-L2: the beta2 term goes through B with u5 (B u5 + B u6), and K sees 0
      U[4 * NH + h] = kL2 ? u5 + u6 : u5;
      U[5 * NH + h] = kL2 ? (T)0 : u6;
    }
    __syncthreads();
    if (n + 3 <= n1) prefetch(n + 3);    // into the slot of level n - 1, no longer read
    cp_async_commit();
    if constexpr (kP1) {
      if (own) {
        T yc = (T)0, yg = (T)0, yf = (T)0;
#pragma unroll
        for (int d = 0; d < kStencil; ++d) {
          if (!kuhn_offset(d)) continue;
          const int dx = d % 3 - 1, dy = (d / 3) % 3 - 1, dz = d / 9 - 1;
          const int h = hc + dx + HX * (dy + HY * dz);
          T s_, st_, b_, k_;
          if constexpr (sizeof(T) == 4) {
            s_ = cS[d];
            st_ = cST[d];
            b_ = cB[d];
            k_ = cK[d];
          } else {
            s_ = c.S[(size_t)d * N + j];
            st_ = c.ST[(size_t)d * N + j];
            b_ = c.B[(size_t)d * N + j];
            k_ = kL2 ? (T)0 : c.K[(size_t)d * N + j];
          }
          yc += b_ * U[h] + s_ * U[NH + h];
          yg += b_ * U[2 * NH + h] + st_ * U[3 * NH + h];
          yf += b_ * U[4 * NH + h];
          if constexpr (!kL2) yf += k_ * U[5 * NH + h];
        }
        const bool dirj = p.dir[j] != 0;
        const T C0 = X0[hc], G0 = X0[NH + hc], Cp = Xp[hc];
        if (n == 0 || dirj) yc = C0;
        if (n == M || dirj) yg = G0;
        else yg += tau * (T)p.sens[j] * (th * Cp + th1 * C0);
        const long long o = 3 * ((long long)n * N + j);
        if (b != nullptr) {
          y[o] = (T)(b[o] - (double)yc);
          y[o + 1] = (T)(b[o + 1] - (double)yg);
          y[o + 2] = (T)(b[o + 2] - (double)yf);
        } else {
          y[o] = yc;
          y[o + 1] = yg;
          y[o + 2] = yf;
        }
      }
      continue;
    }
    // x pass: Mx on u1, u3, u5, u6 and Kx on u6
    for (int e = t; e < NXP; e += blockDim.x) {
      const int ex = e % TX, ey = (e / TX) % HY, ez = e / (TX * HY);
      const int h = (ex + 1) + HX * (ey + HY * ez);
      T m_, m0, mp, k_, k0, kp;
      ax.row(bx0 + ex, m_, m0, mp, k_, k0, kp);
      PX[e] = m_ * U[h - 1] + m0 * U[h] + mp * U[h + 1];
      PX[NXP + e] = m_ * U[2 * NH + h - 1] + m0 * U[2 * NH + h] + mp * U[2 * NH + h + 1];
      PX[2 * NXP + e] = m_ * U[4 * NH + h - 1] + m0 * U[4 * NH + h] + mp * U[4 * NH + h + 1];
      PX[3 * NXP + e] = m_ * U[5 * NH + h - 1] + m0 * U[5 * NH + h] + mp * U[5 * NH + h + 1];
      PX[4 * NXP + e] = k_ * U[5 * NH + h - 1] + k0 * U[5 * NH + h] + kp * U[5 * NH + h + 1];
    }
    __syncthreads();
    // y pass: My on the four Mx results; My (Kx u6) + Ky (Mx u6)
    for (int e = t; e < NYP; e += blockDim.x) {
      const int ex = e % TX, ey = (e / TX) % TY, ez = e / (TX * TY);
      const int q = ex + TX * ((ey + 1) + HY * ez);
      T m_, m0, mp, k_, k0, kp;
      ay.row(by0 + ey, m_, m0, mp, k_, k0, kp);
#pragma unroll
      for (int f = 0; f < 4; ++f)
        PY[f * NYP + e] = m_ * PX[f * NXP + q - TX] + m0 * PX[f * NXP + q] + mp * PX[f * NXP + q + TX];
      PY[4 * NYP + e] = m_ * PX[4 * NXP + q - TX] + m0 * PX[4 * NXP + q] + mp * PX[4 * NXP + q + TX] +
                        k_ * PX[3 * NXP + q - TX] + k0 * PX[3 * NXP + q] + kp * PX[3 * NXP + q + TX];
    }
    __syncthreads();
    if (own) {
      // z pass and the S, S^T stencils
      const int qz = tx + TX * (ty + TY * (tz + 1));
      T m_, m0, mp, k_, k0, kp;
      az.row(iz, m_, m0, mp, k_, k0, kp);
      constexpr int zs = TX * TY;
      T yc = m_ * PY[qz - zs] + m0 * PY[qz] + mp * PY[qz + zs];
      T yg = m_ * PY[NYP + qz - zs] + m0 * PY[NYP + qz] + mp * PY[NYP + qz + zs];
      T yf = m_ * PY[2 * NYP + qz - zs] + m0 * PY[2 * NYP + qz] + mp * PY[2 * NYP + qz + zs];
      yf += m_ * PY[4 * NYP + qz - zs] + m0 * PY[4 * NYP + qz] + mp * PY[4 * NYP + qz + zs];
      yf += k_ * PY[3 * NYP + qz - zs] + k0 * PY[3 * NYP + qz] + kp * PY[3 * NYP + qz + zs];
#pragma unroll
      for (int d = 0; d < kStencil; ++d) {
        const int dx = d % 3 - 1, dy = (d / 3) % 3 - 1, dz = d / 9 - 1;
        const int h = hc + dx + HX * (dy + HY * dz);
        T s_, st_;
        if constexpr (sizeof(T) == 4) {
          s_ = cS[d];
          st_ = cST[d];
        } else {
          s_ = c.S[(size_t)d * N + j];
          st_ = c.ST[(size_t)d * N + j];
        }
        yc += s_ * U[NH + h];
        yg += st_ * U[3 * NH + h];
      }
      const bool dirj = p.dir[j] != 0;
      const T C0 = X0[hc], G0 = X0[NH + hc], Cp = Xp[hc];
      if (n == 0 || dirj) yc = C0;
      if (n == M || dirj) yg = G0;
      else yg += tau * (T)p.sens[j] * (th * Cp + th1 * C0);
      const long long o = 3 * ((long long)n * N + j);
      if (b != nullptr) {
        y[o] = (T)(b[o] - (double)yc);
        y[o + 1] = (T)(b[o + 1] - (double)yg);
        y[o + 2] = (T)(b[o + 2] - (double)yf);
      } else {
        y[o] = yc;
        y[o + 1] = yg;
        y[o + 2] = yf;
      }
    }
  }
  cp_async_wait<0>();
}

// Estimated multiply-adds of one level over the grid with tile shape Tl: the
// six time combinations on every halo node, the x and y passes, and the z pass
// with the two 27-point stencils per tile node (ragged tiles count in full).
template <typename Tl>
double tile_work(const DevProblem& p) {
  const double tiles = (double)((p.nx + Tl::TX - 1) / Tl::TX) * ((p.ny + Tl::TY - 1) / Tl::TY) *
                       ((p.nz + Tl::TZ - 1) / Tl::TZ);
  return tiles * (25.0 * Tl::NH + 30.0 * Tl::NXP + 36.0 * Tl::NYP + 138.0 * Tl::kThreads);
}

template <typename T, typename Tl, bool kP1 = false>
void launch_shape(const DevProblem& p, const T* x, T* y, const double* b, cudaStream_t s) {
  const int tx = (p.nx + Tl::TX - 1) / Tl::TX, ty = (p.ny + Tl::TY - 1) / Tl::TY, tz = (p.nz + Tl::TZ - 1) / Tl::TZ;
  constexpr int NT = levels_per_cta<T>();
  dim3 grid(tx * ty * tz, (p.M + 1 + NT - 1) / NT);
  Axis1D<T> ax, ay, az;
  ax.init(p.nx, p.hx);
  ay.init(p.ny, p.hy);
  az.init(p.nz, p.hz);
  LevelW<T> w;
  w.init(p.tau, p.theta, p.beta1, p.beta2);
  // (the dynamic shared-memory limits are raised once, in matvec_prepare)
  constexpr size_t smem = mv_smem<T, Tl, kP1>();
  if (p.reg != 0)
    matvec_tiled<T, true, Tl, kP1><<<grid, Tl::kThreads, smem, s>>>(p, x, y, b, tx, ty, ax, ay, az, w);
  else
    matvec_tiled<T, false, Tl, kP1><<<grid, Tl::kThreads, smem, s>>>(p, x, y, b, tx, ty, ax, ay, az, w);
}

template <typename T>
void launch_tiled(const DevProblem& p, const T* x, T* y, const double* b, cudaStream_t s) {
  if (p.elem == KKT_ELEM_P1) launch_shape<T, TileA, true>(p, x, y, b, s);
  else if (tile_work<TileB>(p) < tile_work<TileA>(p)) launch_shape<T, TileB>(p, x, y, b, s);
  else launch_shape<T, TileA>(p, x, y, b, s);
}

__global__ void d2f(const double* __restrict__ x, float* __restrict__ y, long long n, const int* gate) {
  if (gated_off(gate)) return;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    y[i] = (float)x[i];
}

__global__ void f2d(const float* __restrict__ x, double* __restrict__ y, long long n, const int* gate) {
  if (gated_off(gate)) return;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    y[i] = (double)x[i];
}

__global__ void sub_f2d(const double* __restrict__ b, const float* __restrict__ y, double* __restrict__ r, long long n,
                        const int* gate) {
  if (gated_off(gate)) return;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    r[i] = b[i] - (double)y[i];
}

}  // namespace

template <typename T, typename Tl>
kkt_status prepare_shape() {
  KKT_TRY_CUDA(cudaFuncSetAttribute(matvec_tiled<T, false, Tl>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)mv_smem<T, Tl>()));
  KKT_TRY_CUDA(cudaFuncSetAttribute(matvec_tiled<T, true, Tl>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)mv_smem<T, Tl>()));
  return KKT_OK;
}

template <typename T>
kkt_status prepare_p1() {
  KKT_TRY_CUDA(cudaFuncSetAttribute(matvec_tiled<T, false, TileA, true>,
                                    cudaFuncAttributeMaxDynamicSharedMemorySize, (int)mv_smem<T, TileA, true>()));
  KKT_TRY_CUDA(cudaFuncSetAttribute(matvec_tiled<T, true, TileA, true>,
                                    cudaFuncAttributeMaxDynamicSharedMemorySize, (int)mv_smem<T, TileA, true>()));
  return KKT_OK;
}

kkt_status matvec_prepare() {
  KKT_TRY((prepare_shape<double, TileA>()));
  KKT_TRY((prepare_shape<double, TileB>()));
  KKT_TRY((prepare_shape<float, TileA>()));
  KKT_TRY((prepare_shape<float, TileB>()));
  KKT_TRY((prepare_p1<double>()));
  KKT_TRY((prepare_p1<float>()));
  return KKT_OK;
}

kkt_status launch_matvec64(const DevProblem& p, const double* x, double* y, cudaStream_t s) {
  launch_tiled<double>(p, x, y, nullptr, s);
  KKT_COUNT(1);
  KKT_TRY_CUDA(cudaGetLastError());
  return KKT_OK;
}

kkt_status launch_matvec32(const DevProblem& p, const float* x, float* y, cudaStream_t s) {
  launch_tiled<float>(p, x, y, nullptr, s);
  KKT_COUNT(1);
  KKT_TRY_CUDA(cudaGetLastError());
  return KKT_OK;
}

kkt_status launch_residual(const DevProblem& p, const double* b, const double* x, double* r, cudaStream_t s) {
  launch_tiled<double>(p, x, r, b, s);
  KKT_COUNT(1);
  KKT_TRY_CUDA(cudaGetLastError());
  return KKT_OK;
}

// r = b - F x with the product in FP32 (x32, y32: scratch of 3P floats).
kkt_status launch_residual32(const DevProblem& p, const double* b, const double* x, double* r, float* x32,
                             float* y32, cudaStream_t s) {
  const long long n = 3 * p.P;
  d2f<<<1216, 256, 0, s>>>(x, x32, n, p.gate);
  launch_tiled<float>(p, x32, y32, nullptr, s);
  sub_f2d<<<1216, 256, 0, s>>>(b, y32, r, n, p.gate);
  KKT_COUNT(3);
  KKT_TRY_CUDA(cudaGetLastError());
  return KKT_OK;
}

// y = F x for FP64 vectors with the product in FP32 (x32, y32: scratch of 3P floats).
kkt_status launch_matvec32_d(const DevProblem& p, const double* x, double* y, float* x32, float* y32,
                             cudaStream_t s) {
  const long long n = 3 * p.P;
  d2f<<<1216, 256, 0, s>>>(x, x32, n, p.gate);
  launch_tiled<float>(p, x32, y32, nullptr, s);
  f2d<<<1216, 256, 0, s>>>(y32, y, n, p.gate);
  KKT_COUNT(3);
  KKT_TRY_CUDA(cudaGetLastError());
  return KKT_OK;
}

extern "C" kkt_status kkt_apply(kkt_problem* p, const void* x, void* y, int precision, void* stream) {
  if (!p || !x || !y) {
    set_error("kkt_apply: null argument");
    return KKT_ERR_ARG;
  }
  if (x == y) {
    set_error("kkt_apply: x and y must not overlap");
    return KKT_ERR_ARG;
  }
  if (precision == 64) return launch_matvec64(p->dev(), (const double*)x, (double*)y, (cudaStream_t)stream);
  if (precision == 32) return launch_matvec32(p->dev(), (const float*)x, (float*)y, (cudaStream_t)stream);
  set_error("kkt_apply: precision must be 64 or 32");
  return KKT_ERR_ARG;
}

extern "C" kkt_status kkt_residual(kkt_problem* p, const double* b, const double* x, double* r, void* stream) {
  if (!p || !b || !x || !r) {
    set_error("kkt_residual: null argument");
    return KKT_ERR_ARG;
  }
  if (r == x) {
    set_error("kkt_residual: r and x must not overlap");
    return KKT_ERR_ARG;
  }
  return launch_residual(p->dev(), b, x, r, (cudaStream_t)stream);
}
