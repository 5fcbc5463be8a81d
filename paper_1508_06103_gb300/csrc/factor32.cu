// Subdomain ILU(0) factorisation in FP32 (the mixed-precision form).
#include <algorithm>

#include "factor.cuh"

kkt_status ras_factor_launch32(ras_precond* m, cudaStream_t s) { return factor_launch<float>(m, s); }
