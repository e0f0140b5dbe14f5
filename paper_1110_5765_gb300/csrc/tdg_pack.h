// Launchers of tdg_pack.cu beyond those every translation unit shares.
#pragma once

#include "tdg_internal.h"

namespace tdg {

// The symmetric form's A (eq. 6) and B (eq. 7) packs: one launch where the
// layouts allow (A k-contiguous, B x-contiguous), else B's pack and then A's.
template <typename T>
cudaError_t launch_pack_k_pair(const PackOperand<T> &a, const PackOperand<T> &b, int W,
                               const DevPlan *plan, int expectW, T *outA, long long ldoA,
                               long long rowsA, T *outB, long long ldoB, long long rowsB,
                               cudaStream_t st);

}  // namespace tdg
