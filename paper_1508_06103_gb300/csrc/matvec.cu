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
// One thread per space-time point computes its three output slots; the time
// combinations are formed per neighbour, so each neighbour value is read
// from the three levels n-1, n, n+1 (cache hits).

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

// If b != nullptr the kernel writes b - F x instead of F x (FP64 only).
template <typename T>
__global__ void __launch_bounds__(256) matvec_kernel(DevProblem p, const T* __restrict__ x, T* __restrict__ y,
                                                     const double* __restrict__ b) {
  const long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (idx >= p.P) return;
  const int N = p.N, M = p.M;
  const int n = (int)(idx / N);
  const int j = (int)(idx - (long long)n * N);
  const int ix = j % p.nx, iy = (j / p.nx) % p.ny, iz = j / (p.nx * p.ny);
  const Coefs<T> c = coefs<T>(p);
  const T tau = (T)p.tau, th = (T)p.theta, th1 = (T)(1.0 - p.theta);
  const T b1 = (T)p.beta1, b2 = (T)p.beta2;
  const bool dirj = p.dir[j] != 0;
  const bool crow = n >= 1 && !dirj;
  const bool grow = n < M && !dirj;
  const bool hasm = n > 0, hasp = n < M;
  // time weights of the f row
  const T mtm = hasm ? tau / (T)6 : (T)0, mtp = hasp ? tau / (T)6 : (T)0;
  const T mt0 = (hasm ? tau / (T)3 : (T)0) + (hasp ? tau / (T)3 : (T)0);
  const T ltm = hasm ? -(T)1 / tau : (T)0, ltp = hasp ? -(T)1 / tau : (T)0;
  const T lt0 = (hasm ? (T)1 / tau : (T)0) + (hasp ? (T)1 / tau : (T)0);
  const T* x0 = x + 3 * idx;
  const T* xm = hasm ? x0 - 3LL * N : x0;
  const T* xp = hasp ? x0 + 3LL * N : x0;
  T yc = 0, yg = 0, yf = 0;
  const int zlo = iz > 0 ? -1 : 0, zhi = iz < p.nz - 1 ? 1 : 0;
  const int ylo = iy > 0 ? -1 : 0, yhi = iy < p.ny - 1 ? 1 : 0;
  const int xlo = ix > 0 ? -1 : 0, xhi = ix < p.nx - 1 ? 1 : 0;
  for (int dz = zlo; dz <= zhi; ++dz)
    for (int dy = ylo; dy <= yhi; ++dy)
      for (int dx = xlo; dx <= xhi; ++dx) {
        const int d = (dx + 1) + 3 * (dy + 1) + 9 * (dz + 1);
        const long long o = 3LL * (dx + p.nx * (dy + (long long)p.ny * dz));
        const T C0 = x0[o], G0 = x0[o + 1], F0 = x0[o + 2];
        const T Cm = hasm ? xm[o] : (T)0, Fm = hasm ? xm[o + 2] : (T)0, Gm = hasm ? xm[o + 1] : (T)0;
        const T Gp = hasp ? xp[o + 1] : (T)0, Fp = hasp ? xp[o + 2] : (T)0;
        const size_t ci = (size_t)d * N + j;
        const T Bd = c.B[ci];
        if (crow) {
          const T u1 = (C0 - Cm) - tau * (th * F0 + th1 * Fm);
          const T u2 = tau * (th * C0 + th1 * Cm);
          yc += Bd * u1 + c.S[ci] * u2;
        }
        if (grow) {
          const T u3 = G0 - Gp;
          const T u4 = tau * (th * G0 + th1 * Gp);
          yg += Bd * u3 + c.ST[ci] * u4;
        }
        const T u5 = -(mtm * Gm + mt0 * G0 + mtp * Gp) + b1 * (ltm * Fm + lt0 * F0 + ltp * Fp);
        const T u6 = b2 * (mtm * Fm + mt0 * F0 + mtp * Fp);
        yf += Bd * u5 + c.K[ci] * u6;
      }
  if (!crow) yc = x0[0];
  if (grow) {
    const T Cn = x0[0], Cp = xp[0];
    yg += tau * (T)p.sens[j] * (th * Cp + th1 * Cn);
  } else {
    yg = x0[1];
  }
  if (b != nullptr) {
    const double* bb = b + 3 * idx;
    y[3 * idx] = (T)(bb[0] - (double)yc);
    y[3 * idx + 1] = (T)(bb[1] - (double)yg);
    y[3 * idx + 2] = (T)(bb[2] - (double)yf);
  } else {
    y[3 * idx] = yc;
    y[3 * idx + 1] = yg;
    y[3 * idx + 2] = yf;
  }
}

__global__ void d2f(const double* __restrict__ x, float* __restrict__ y, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    y[i] = (float)x[i];
}

__global__ void sub_f2d(const double* __restrict__ b, const float* __restrict__ y, double* __restrict__ r, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    r[i] = b[i] - (double)y[i];
}

}  // namespace

kkt_status launch_matvec64(const DevProblem& p, const double* x, double* y, cudaStream_t s) {
  matvec_kernel<double><<<(unsigned)((p.P + 255) / 256), 256, 0, s>>>(p, x, y, nullptr);
  KKT_COUNT(1);
  KKT_TRY_CUDA(cudaGetLastError());
  return KKT_OK;
}

kkt_status launch_matvec32(const DevProblem& p, const float* x, float* y, cudaStream_t s) {
  matvec_kernel<float><<<(unsigned)((p.P + 255) / 256), 256, 0, s>>>(p, x, y, nullptr);
  KKT_COUNT(1);
  KKT_TRY_CUDA(cudaGetLastError());
  return KKT_OK;
}

kkt_status launch_residual(const DevProblem& p, const double* b, const double* x, double* r, cudaStream_t s) {
  matvec_kernel<double><<<(unsigned)((p.P + 255) / 256), 256, 0, s>>>(p, x, r, b);
  KKT_COUNT(1);
  KKT_TRY_CUDA(cudaGetLastError());
  return KKT_OK;
}

// r = b - F x with the product in FP32 (x32, y32: scratch of 3P floats).
kkt_status launch_residual32(const DevProblem& p, const double* b, const double* x, double* r, float* x32,
                             float* y32, cudaStream_t s) {
  const long long n = 3 * p.P;
  d2f<<<1216, 256, 0, s>>>(x, x32, n);
  matvec_kernel<float><<<(unsigned)((p.P + 255) / 256), 256, 0, s>>>(p, x32, y32, nullptr);
  sub_f2d<<<1216, 256, 0, s>>>(b, y32, r, n);
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
