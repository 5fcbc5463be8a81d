// Restarted right-preconditioned GMRES / flexible GMRES (Sec. 3.2 and 4;
// Saad 1993 for the flexible form) on device vectors.
//
// Arnoldi step j (all FP64, on the device):
//   z_j = M^{-1} v_j   (kept in Z for the flexible form)
//   w   = F z_j
//   h   = V_j^T w ;  w -= V_j h          classical Gram-Schmidt ...
//   h2  = V_j^T w ;  w -= V_j h2 ; h += h2   ... applied twice (CGS2)
//   v_{j+1} = w / ||w||
// The (j+2) Hessenberg entries are copied to the host once per step; the
// Givens rotations, the residual estimate and the back substitution run on
// the host in FP64.  Dot products are reduced in a fixed order (block
// partials, then one block per vector), so results are deterministic.

#include <cmath>
#include <vector>

#include "internal.cuh"

namespace {

constexpr int kDotBlocks = 304;   // 2 x 152 SMs (1216 measured slower: the coarse-level dots are short)
constexpr int kDotThreads = 256;

// partial[k * kDotBlocks + b] = sum over block b's part of V_k . w.  Block
// (k, b) runs with k fastest, so the m blocks that read the same part of w
// run together and w comes from L2 after its first read; V_k is read once,
// with evict-first loads that leave L2 to w.
__global__ void __launch_bounds__(kDotThreads) multidot_partial(const double* __restrict__ V, long long ldv,
                                                                const double* __restrict__ w, long long n,
                                                                double* __restrict__ part) {
  __shared__ double red[kDotThreads / 32];
  const int k = blockIdx.x, b = blockIdx.y, nb = gridDim.y;
  const double* v = V + (long long)k * ldv;
  double acc = 0.0;
  for (long long i = b * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)nb * blockDim.x)
    acc = fma(__ldcs(v + i), w[i], acc);
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int q = 0; q < kDotThreads / 32; ++q) s += red[q];
    part[k * nb + b] = s;
  }
}

// out[k] (+)= sum_b partial[k * nb + b], fixed order; one block per k
__global__ void multidot_final(const double* __restrict__ part, int nb, double* __restrict__ out, int accumulate) {
  __shared__ double red[32];
  const int k = blockIdx.x;
  double acc = 0.0;
  for (int b = threadIdx.x; b < nb; b += blockDim.x) acc += part[k * nb + b];
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int q = 0; q < (int)(blockDim.x + 31) / 32; ++q) s += red[q];
    out[k] = accumulate ? out[k] + s : s;
  }
}

// w -= sum_{k < m} V_k h[k]
__global__ void multi_axpy(double* __restrict__ w, const double* __restrict__ V, long long ldv,
                           const double* __restrict__ h, int m, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    double acc = w[i];
    for (int k = 0; k < m; ++k) acc = fma(-V[(long long)k * ldv + i], h[k], acc);
    w[i] = acc;
  }
}

// x += sum_{k < m} Z_k y[k]
__global__ void multi_update(double* __restrict__ x, const double* __restrict__ Z, long long ldz,
                             const double* __restrict__ y, int m, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    double acc = x[i];
    for (int k = 0; k < m; ++k) acc = fma(Z[(long long)k * ldz + i], y[k], acc);
    x[i] = acc;
  }
}

__global__ void scale_kernel(double* __restrict__ y, const double* __restrict__ x, double a, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    y[i] = a * x[i];
}

__global__ void axpby_kernel(double* __restrict__ y, double a, const double* __restrict__ x, double b, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    y[i] = a * x[i] + b * y[i];
}

__global__ void add_kernel(double* __restrict__ h, const double* __restrict__ h2, int m) {
  const int k = threadIdx.x;
  if (k < m) h[k] += h2[k];
}

constexpr unsigned kVecBlocks = 1216;   // 8 x 152 SMs

// out[0..m) = V_k . w  for k < m
kkt_status multidot(const double* V, long long ldv, int m, const double* w, long long n, double* part, double* out,
                    cudaStream_t s) {
  dim3 g(m, kDotBlocks);
  multidot_partial<<<g, kDotThreads, 0, s>>>(V, ldv, w, n, part);
  multidot_final<<<m, 256, 0, s>>>(part, kDotBlocks, out, 0);
  KKT_COUNT(2);
  KKT_TRY_CUDA(cudaGetLastError());
  return KKT_OK;
}

}  // namespace

kkt_status vec_copy(double* y, const double* x, long long n, cudaStream_t s) {
  KKT_TRY_CUDA(cudaMemcpyAsync(y, x, n * sizeof(double), cudaMemcpyDeviceToDevice, s));
  return KKT_OK;
}

kkt_status vec_zero(double* y, long long n, cudaStream_t s) {
  KKT_TRY_CUDA(cudaMemsetAsync(y, 0, n * sizeof(double), s));
  return KKT_OK;
}

kkt_status vec_axpby(double* y, double a, const double* x, double b, long long n, cudaStream_t s) {
  axpby_kernel<<<kVecBlocks, 256, 0, s>>>(y, a, x, b, n);
  KKT_COUNT(1);
  KKT_TRY_CUDA(cudaGetLastError());
  return KKT_OK;
}

kkt_status GmresWork::alloc(long long n_, int m_, bool flex) {
  if (n_ == n && m_ <= m && (!flex || flexible)) return KKT_OK;
  release();
  n = n_;
  m = m_;
  flexible = flex;
  nparts = kDotBlocks;
  if (cudaMalloc(&V, (size_t)(m + 1) * n * sizeof(double)) != cudaSuccess ||
      (flex && cudaMalloc(&Z, (size_t)m * n * sizeof(double)) != cudaSuccess) ||
      cudaMalloc(&w, n * sizeof(double)) != cudaSuccess || cudaMalloc(&r, n * sizeof(double)) != cudaSuccess ||
      cudaMalloc(&hbuf, 4 * (m + 2) * sizeof(double)) != cudaSuccess ||
      cudaMalloc(&part, (size_t)(m + 2) * kDotBlocks * sizeof(double)) != cudaSuccess ||
      cudaMallocHost(&hhost, 4 * (m + 2) * sizeof(double)) != cudaSuccess) {
    cudaGetLastError();
    release();
    set_error("gmres: workspace allocation failed");
    return KKT_ERR_NOMEM;
  }
  return KKT_OK;
}

void GmresWork::release() {
  cudaFree(V);
  cudaFree(Z);
  cudaFree(w);
  cudaFree(r);
  cudaFree(hbuf);
  cudaFree(part);
  if (hhost) cudaFreeHost(hhost);
  V = Z = w = r = hbuf = part = hhost = nullptr;
  n = 0;
  m = 0;
}

kkt_status gmres_run(Operator& A, Operator* M, const double* b, double* x, GmresWork& ws, int restart, double rtol,
                     int maxit, bool check_true, bool zero_guess, GmresResult* res, cudaStream_t s) {
  const long long n = ws.n;
  const int m = restart;
  double* hdev = ws.hbuf;                 // h (m+2)
  double* h2dev = ws.hbuf + (m + 2);      // second CGS pass
  double* ydev = ws.hbuf + 2 * (m + 2);   // solution coefficients
  double* hh = ws.hhost;
  res->iters = 0;
  res->relres = 0.0;
  res->status = KKT_OK;

  auto norm = [&](const double* v, double* out) -> kkt_status {
    KKT_TRY(multidot(v, 0, 1, v, n, ws.part, hdev, s));
    KKT_TRY_CUDA(cudaMemcpyAsync(hh, hdev, sizeof(double), cudaMemcpyDeviceToHost, s));
    KKT_TRY_CUDA(cudaStreamSynchronize(s));
    *out = std::sqrt(hh[0]);
    return KKT_OK;
  };

  double bnorm;
  KKT_TRY(norm(b, &bnorm));
  if (!std::isfinite(bnorm)) {
    set_error("gmres: right-hand side is not finite");
    res->status = KKT_ERR_NONFINITE;
    return KKT_ERR_NONFINITE;
  }
  if (bnorm == 0.0) {
    KKT_TRY(vec_zero(x, n, s));
    return KKT_OK;
  }
  // r = b - A x
  if (zero_guess) {
    KKT_TRY(vec_zero(x, n, s));
    KKT_TRY(vec_copy(ws.r, b, n, s));
  } else {
    KKT_TRY(A.apply(x, ws.w, s));
    KKT_TRY(vec_copy(ws.r, b, n, s));
    KKT_TRY(vec_axpby(ws.r, -1.0, ws.w, 1.0, n, s));
  }
  double beta;
  KKT_TRY(norm(ws.r, &beta));
  bool converged = beta <= rtol * bnorm;
  double est = beta / bnorm;
  int it = 0;
  bool breakdown = false;
  std::vector<double> H((size_t)(m + 1) * m), cs(m), sn(m), g(m + 1), y(m);
  auto Hij = [&](int i, int j) -> double& { return H[(size_t)i * m + j]; };

  while (!converged && it < maxit) {
    std::fill(H.begin(), H.end(), 0.0);
    std::fill(g.begin(), g.end(), 0.0);
    g[0] = beta;
    scale_kernel<<<kVecBlocks, 256, 0, s>>>(ws.V, ws.r, 1.0 / beta, n);
    KKT_COUNT(1);
    KKT_TRY_CUDA(cudaGetLastError());
    int k = 0;
    bool stop = false;
    for (int j = 0; j < m; ++j) {
      double* vj = ws.V + (size_t)j * n;
      double* zj = ws.flexible ? ws.Z + (size_t)j * n : ws.r;
      if (M) KKT_TRY(M->apply(vj, zj, s));
      else KKT_TRY(vec_copy(zj, vj, n, s));
      KKT_TRY(A.apply(zj, ws.w, s));
      // CGS2
      KKT_TRY(multidot(ws.V, n, j + 1, ws.w, n, ws.part, hdev, s));
      multi_axpy<<<kVecBlocks, 256, 0, s>>>(ws.w, ws.V, n, hdev, j + 1, n);
      KKT_TRY(multidot(ws.V, n, j + 1, ws.w, n, ws.part, h2dev, s));
      multi_axpy<<<kVecBlocks, 256, 0, s>>>(ws.w, ws.V, n, h2dev, j + 1, n);
      add_kernel<<<1, 64, 0, s>>>(hdev, h2dev, j + 1);
      KKT_COUNT(3);
      KKT_TRY_CUDA(cudaGetLastError());
      KKT_TRY(multidot(ws.w, 0, 1, ws.w, n, ws.part, hdev + j + 1, s));
      KKT_TRY_CUDA(cudaMemcpyAsync(hh, hdev, (j + 2) * sizeof(double), cudaMemcpyDeviceToHost, s));
      KKT_TRY_CUDA(cudaStreamSynchronize(s));
      for (int i = 0; i <= j; ++i) Hij(i, j) = hh[i];
      const double hn = std::sqrt(hh[j + 1]);
      Hij(j + 1, j) = hn;
      for (int i = 0; i <= j + 1; ++i)
        if (!std::isfinite(Hij(i, j))) {
          set_error("gmres: non-finite value in the Arnoldi process");
          res->status = KKT_ERR_NONFINITE;
          res->iters = it;
          return KKT_ERR_NONFINITE;
        }
      for (int i = 0; i < j; ++i) {
        const double t = cs[i] * Hij(i, j) + sn[i] * Hij(i + 1, j);
        Hij(i + 1, j) = -sn[i] * Hij(i, j) + cs[i] * Hij(i + 1, j);
        Hij(i, j) = t;
      }
      const double den = std::hypot(Hij(j, j), Hij(j + 1, j));
      if (den == 0.0) {
        // F M^{-1} v_j lies in span(v_0 .. v_{j-1}) with a zero rotated
        // diagonal: the least-squares problem gains nothing from column j,
        // so the cycle ends on columns 0 .. j-1 and reports a breakdown.
        ++it;
        k = j;
        stop = true;
        breakdown = true;
        break;
      }
      cs[j] = Hij(j, j) / den;
      sn[j] = Hij(j + 1, j) / den;
      Hij(j, j) = den;
      Hij(j + 1, j) = 0.0;
      g[j + 1] = -sn[j] * g[j];
      g[j] = cs[j] * g[j];
      ++it;
      k = j + 1;
      est = std::fabs(g[j + 1]) / bnorm;
      if (hn == 0.0 || est <= rtol || it >= maxit) {
        stop = true;
        breakdown = (hn == 0.0 && est > rtol);
        break;
      }
      scale_kernel<<<kVecBlocks, 256, 0, s>>>(ws.V + (size_t)(j + 1) * n, ws.w, 1.0 / hn, n);
      KKT_COUNT(1);
      KKT_TRY_CUDA(cudaGetLastError());
    }
    for (int i = k - 1; i >= 0; --i) {
      double acc = g[i];
      for (int q = i + 1; q < k; ++q) acc -= Hij(i, q) * y[q];
      y[i] = acc / Hij(i, i);
    }
    KKT_TRY_CUDA(cudaMemcpyAsync(ydev, y.data(), k * sizeof(double), cudaMemcpyHostToDevice, s));
    if (ws.flexible) {
      multi_update<<<kVecBlocks, 256, 0, s>>>(x, ws.Z, n, ydev, k, n);
      KKT_COUNT(1);
    } else {
      // x += M^{-1} (V y): form V y in w, precondition into r
      KKT_TRY(vec_zero(ws.w, n, s));
      multi_update<<<kVecBlocks, 256, 0, s>>>(ws.w, ws.V, n, ydev, k, n);
      KKT_COUNT(1);
      if (M) KKT_TRY(M->apply(ws.w, ws.r, s));
      else KKT_TRY(vec_copy(ws.r, ws.w, n, s));
      KKT_TRY(vec_axpby(x, 1.0, ws.r, 1.0, n, s));
    }
    KKT_TRY_CUDA(cudaGetLastError());
    if (stop && !check_true) {
      converged = est <= rtol;
      break;
    }
    // true residual
    KKT_TRY(A.apply(x, ws.w, s));
    KKT_TRY(vec_copy(ws.r, b, n, s));
    KKT_TRY(vec_axpby(ws.r, -1.0, ws.w, 1.0, n, s));
    KKT_TRY(norm(ws.r, &beta));
    converged = beta <= rtol * bnorm;
    if (breakdown && !converged) break;
  }
  res->iters = it;
  if (check_true) {
    res->relres = beta / bnorm;
  } else {
    res->relres = est;
  }
  if (converged) res->status = KKT_OK;
  else res->status = breakdown ? KKT_BREAKDOWN : KKT_NOT_CONVERGED;
  return KKT_OK;
}
