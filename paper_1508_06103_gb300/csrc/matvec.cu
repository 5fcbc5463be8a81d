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
// in one pass (the four spatial stencils applied to six time combinations).

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
// levels.  Three consecutive levels of x on the tile plus a one-node halo sit
// in a shared-memory ring; per level the six time combinations
//   u1 = (C^n - C^{n-1}) - tau (theta f^n + (1-theta) f^{n-1})   (C row, via B)
//   u2 = tau (theta C^n + (1-theta) C^{n-1})                        (C row, via S)
//   u3 = G^n - G^{n+1}                                              (G row, via B)
//   u4 = tau (theta G^n + (1-theta) G^{n+1})                        (G row, via S^T)
//   u5 = -(Mt G)_n + beta1 (Lt f)_n                                 (f row, via B)
//   u6 = beta2 (Mt f)_n                                             (f row, via K)
// are formed once per halo node, and each output node applies the four
// 27-point stencils to them.  Stencil coefficients outside the domain are 0,
// so the halo of a boundary tile is zero-filled and read without tests.
// ---------------------------------------------------------------------------
constexpr int TX = 8, TY = 8, TZ = 4, NT = 16;
constexpr int HX = TX + 2, HY = TY + 2, HZ = TZ + 2, NH = HX * HY * HZ;

template <typename T>
__global__ void __launch_bounds__(TX * TY * TZ, 2) matvec_tiled(DevProblem p, const T* __restrict__ x,
                                                              T* __restrict__ y, const double* __restrict__ b,
                                                              int tiles_x, int tiles_y) {
  __shared__ T X[3][3][NH];     // [level slot][component][halo node]
  __shared__ T U[6][NH];
  const int N = p.N, M = p.M;
  const int tile = blockIdx.x;
  const int bx0 = (tile % tiles_x) * TX, by0 = ((tile / tiles_x) % tiles_y) * TY, bz0 = (tile / (tiles_x * tiles_y)) * TZ;
  const int n0 = blockIdx.y * NT, n1 = min(n0 + NT, M + 1);
  const Coefs<T> c = coefs<T>(p);
  const T tau = (T)p.tau, th = (T)p.theta, th1 = (T)(1.0 - p.theta);
  const T b1 = (T)p.beta1, b2 = (T)p.beta2;
  const int t = threadIdx.x;
  const int tx = t % TX, ty = (t / TX) % TY, tz = t / (TX * TY);
  const int ix = bx0 + tx, iy = by0 + ty, iz = bz0 + tz;
  const bool own = ix < p.nx && iy < p.ny && iz < p.nz;
  const int j = own ? ix + p.nx * (iy + p.ny * iz) : 0;
  const int hc = (tx + 1) + HX * ((ty + 1) + HY * (tz + 1));

  auto load_level = [&](int m) {   // level m of x on the halo into ring slot m mod 3
    const int slot = ((m % 3) + 3) % 3;
    for (int h = t; h < NH; h += blockDim.x) {
      const int hx = h % HX, hy = (h / HX) % HY, hz = h / (HX * HY);
      const int gx = bx0 - 1 + hx, gy = by0 - 1 + hy, gz = bz0 - 1 + hz;
      T vc = 0, vg = 0, vf = 0;
      if (m >= 0 && m <= M && gx >= 0 && gx < p.nx && gy >= 0 && gy < p.ny && gz >= 0 && gz < p.nz) {
        const T* src = x + 3 * ((long long)m * N + gx + (long long)p.nx * (gy + (long long)p.ny * gz));
        vc = src[0];
        vg = src[1];
        vf = src[2];
      }
      X[slot][0][h] = vc;
      X[slot][1][h] = vg;
      X[slot][2][h] = vf;
    }
  };
  load_level(n0 - 1);
  load_level(n0);
  for (int n = n0; n < n1; ++n) {
    load_level(n + 1);
    __syncthreads();
    const int sm = ((n - 1) % 3 + 3) % 3, s0 = n % 3, sp = (n + 1) % 3;
    const bool hasm = n > 0, hasp = n < M;
    const T mtm = hasm ? tau / (T)6 : (T)0, mtp = hasp ? tau / (T)6 : (T)0;
    const T mt0 = (hasm ? tau / (T)3 : (T)0) + (hasp ? tau / (T)3 : (T)0);
    const T ltm = hasm ? -(T)1 / tau : (T)0, ltp = hasp ? -(T)1 / tau : (T)0;
    const T lt0 = (hasm ? (T)1 / tau : (T)0) + (hasp ? (T)1 / tau : (T)0);
    for (int h = t; h < NH; h += blockDim.x) {
      const T Cm = X[sm][0][h], Gm = X[sm][1][h], Fm = X[sm][2][h];
      const T C0 = X[s0][0][h], G0 = X[s0][1][h], F0 = X[s0][2][h];
      const T Gp = X[sp][1][h], Fp = X[sp][2][h];
      U[0][h] = (C0 - Cm) - tau * (th * F0 + th1 * Fm);
      U[1][h] = tau * (th * C0 + th1 * Cm);
      U[2][h] = G0 - Gp;
      U[3][h] = tau * (th * G0 + th1 * Gp);
      U[4][h] = -(mtm * Gm + mt0 * G0 + mtp * Gp) + b1 * (ltm * Fm + lt0 * F0 + ltp * Fp);
      U[5][h] = b2 * (mtm * Fm + mt0 * F0 + mtp * Fp);
    }
    __syncthreads();
    if (own) {
      T yc = 0, yg = 0, yf = 0;
#pragma unroll
      for (int d = 0; d < kStencil; ++d) {
        const int dx = d % 3 - 1, dy = (d / 3) % 3 - 1, dz = d / 9 - 1;
        const int h = hc + dx + HX * (dy + HY * dz);
        const size_t ci = (size_t)d * N + j;
        const T Bd = c.B[ci];
        yc += Bd * U[0][h] + c.S[ci] * U[1][h];
        yg += Bd * U[2][h] + c.ST[ci] * U[3][h];
        yf += Bd * U[4][h] + c.K[ci] * U[5][h];
      }
      const bool dirj = p.dir[j] != 0;
      const T C0 = X[s0][0][hc], G0 = X[s0][1][hc], Cp = X[sp][0][hc];
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
}

template <typename T>
void launch_tiled(const DevProblem& p, const T* x, T* y, const double* b, cudaStream_t s) {
  const int tx = (p.nx + TX - 1) / TX, ty = (p.ny + TY - 1) / TY, tz = (p.nz + TZ - 1) / TZ;
  dim3 grid(tx * ty * tz, (p.M + 1 + NT - 1) / NT);
  matvec_tiled<T><<<grid, TX * TY * TZ, 0, s>>>(p, x, y, b, tx, ty);
}

__global__ void d2f(const double* __restrict__ x, float* __restrict__ y, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    y[i] = (float)x[i];
}

__global__ void f2d(const float* __restrict__ x, double* __restrict__ y, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    y[i] = (double)x[i];
}

__global__ void sub_f2d(const double* __restrict__ b, const float* __restrict__ y, double* __restrict__ r, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    r[i] = b[i] - (double)y[i];
}

}  // namespace

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
  d2f<<<1216, 256, 0, s>>>(x, x32, n);
  launch_tiled<float>(p, x32, y32, nullptr, s);
  sub_f2d<<<1216, 256, 0, s>>>(b, y32, r, n);
  KKT_COUNT(3);
  KKT_TRY_CUDA(cudaGetLastError());
  return KKT_OK;
}

// y = F x for FP64 vectors with the product in FP32 (x32, y32: scratch of 3P floats).
kkt_status launch_matvec32_d(const DevProblem& p, const double* x, double* y, float* x32, float* y32,
                             cudaStream_t s) {
  const long long n = 3 * p.P;
  d2f<<<1216, 256, 0, s>>>(x, x32, n);
  launch_tiled<float>(p, x32, y32, nullptr, s);
  f2d<<<1216, 256, 0, s>>>(y32, y, n);
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
