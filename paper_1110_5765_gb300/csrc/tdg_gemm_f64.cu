// fp64 instantiations of the packed GEMM (dGEMM forms of Sec. 7), and the TMA
// box shapes every packed-GEMM launch needs.
#include "tdg_gemm.cuh"
#include "tdg_gemm_tiles.h"

namespace tdg {

template <int FORM, int W, typename C>
static cudaError_t go(const GemmArgs<double> &g, const GemmOperands &ops, cudaStream_t st) {
    return launch_cfg<double, FORM, W, C>(g, ops, st);
}

template <>
cudaError_t launch_packed_gemm<double>(int form, int W, const GemmArgs<double> &g,
                                       const GemmOperands &ops, cudaStream_t st) {
    using D = TilesF64;
    if (form == G_PLAIN) return go<G_PLAIN, 1, D>(g, ops, st);
    if (form == G_SYM) {
        switch (W) {
            case 1: return go<G_SYM, 1, D>(g, ops, st);
            case 2: return go<G_SYM, 2, D>(g, ops, st);
            case 3: return go<G_SYM, 3, D>(g, ops, st);
            case 4: return go<G_SYM, 4, D>(g, ops, st);
        }
    }
    if (form == G_ASYM) {
        switch (W) {
            case 1: return go<G_ASYM, 1, D>(g, ops, st);
            case 2: return go<G_ASYM, 2, D>(g, ops, st);
            case 3: return go<G_ASYM, 3, D>(g, ops, st);
            case 4: return go<G_ASYM, 4, D>(g, ops, st);
        }
    }
    return cudaErrorNotSupported;
}

// TMA boxes {BM, BK} for A and {BN, BK} for B, from the same tile table the
// launches use
void packed_gemm_boxes(int dtype, int form, int W, int *box_x_a, int *box_x_b, int *bk) {
    if (dtype == TDG_F64) {
        *box_x_a = TilesF64::BM; *box_x_b = TilesF64::BN; *bk = TilesF64::BK;
    } else if (form == G_ASYM && W <= 2) {
        *box_x_a = TilesF32AsymW2::BM; *box_x_b = TilesF32AsymW2::BN; *bk = TilesF32AsymW2::BK;
    } else if (form == G_ASYM) {
        *box_x_a = TilesF32Asym::BM; *box_x_b = TilesF32Asym::BN; *bk = TilesF32Asym::BK;
    } else {
        *box_x_a = TilesF32::BM; *box_x_b = TilesF32::BN; *bk = TilesF32::BK;
    }
}

}  // namespace tdg
