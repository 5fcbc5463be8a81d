// Subdomain ILU(0) factorisation in FP32 (the mixed-precision form), and the
// BF16-stored variant: factored in FP32, then rounded to BF16 for the solve.
#include <algorithm>

#include <cuda_bf16.h>

#include "factor.cuh"

namespace {

// b = round-to-nearest BF16 of a, four values per thread (n is a multiple of
// 4: chunk blocks are 326 x cp values with cp a multiple of 16, unit rows 328)
__global__ void store_bf16(const float4* __restrict__ a, __nv_bfloat162* __restrict__ b, long long n4) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n4; i += (long long)gridDim.x * blockDim.x) {
    const float4 v = a[i];
    b[2 * i] = __floats2bfloat162_rn(v.x, v.y);
    b[2 * i + 1] = __floats2bfloat162_rn(v.z, v.w);
  }
}

}  // namespace

kkt_status ras_factor_launch32(ras_precond* m, cudaStream_t s) { return factor_launch<float>(m, (float*)m->F, s); }

kkt_status ras_factor_launch16(ras_precond* m, cudaStream_t s) {
  if (m->fcount % 4 != 0) {
    set_error("ras_setup: internal error: BF16 factor count is not a multiple of 4");
    return KKT_ERR_ARG;
  }
  KKT_TRY(factor_launch<float>(m, (float*)m->Ffac, s));
  store_bf16<<<1216, 256, 0, s>>>((const float4*)m->Ffac, (__nv_bfloat162*)m->F, m->fcount / 4);
  KKT_COUNT(1);
  KKT_TRY_CUDA(cudaGetLastError());
  return KKT_OK;
}
