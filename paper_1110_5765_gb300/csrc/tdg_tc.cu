// Tensor-core form (placeholder until the tcgen05 kernel lands).
#include "tdg_common.cuh"
#include "tdg_internal.h"

namespace tdg {

cudaError_t launch_tc_gemm(int, const TcArgs &, const CUtensorMap &, const CUtensorMap &,
                           cudaStream_t) {
    return cudaErrorNotSupported;
}

void tc_gemm_boxes(int fp8, int *box_rows_a, int *box_rows_b, int *box_k) {
    *box_rows_a = 128;
    *box_rows_b = 128;
    *box_k = fp8 ? 128 : 64;
}

}  // namespace tdg
