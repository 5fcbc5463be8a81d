// Subdomain ILU(0) factorisation in FP64.
#include <algorithm>

#include "factor.cuh"

kkt_status ras_factor_launch64(ras_precond* m, cudaStream_t s) { return factor_launch<double>(m, (double*)m->F, s); }
