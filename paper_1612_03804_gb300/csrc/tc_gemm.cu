// tc_gemm.cu -- tensor-core slice products (3xTF32 / BF16); placeholder
// until the tcgen05 kernels land: the mixed modes report UNSUPPORTED.
#include <cuda_runtime.h>

#include "internal.h"

namespace sldqmc {
int tc_prepare(sldqmc_ctx *) { return SLDQMC_ERR_UNSUPPORTED; }
void tc_release(sldqmc_ctx *) {}
void tc_convert_E(sldqmc_ctx *) {}
void tc_chain_block(sldqmc_ctx *, const double *, const int8_t *, int, double, double, const int *, int,
                    double *, double *, double *)
{
}
}  // namespace sldqmc
