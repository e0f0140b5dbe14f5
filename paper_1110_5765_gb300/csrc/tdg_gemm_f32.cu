// fp32 instantiations of the packed GEMM (sGEMM forms of Sec. 7).
#include "tdg_gemm.cuh"
#include "tdg_gemm_tiles.h"

namespace tdg {

template <int FORM, int W, typename C>
static cudaError_t go(const GemmArgs<float> &g, const GemmOperands &ops, cudaStream_t st) {
    return launch_cfg<float, FORM, W, C>(g, ops, st);
}

template <>
cudaError_t launch_packed_gemm<float>(int form, int W, const GemmArgs<float> &g,
                                      const GemmOperands &ops, cudaStream_t st) {
    using S = TilesF32;
    using A = TilesF32Asym;
    using A2 = TilesF32AsymW2;
    if (form == G_PLAIN) {
        const long long tiles = ((g.Mrows + S::BM - 1) / S::BM) * ((g.N + S::BN - 1) / S::BN);
        if (2 * tiles <= device_sms()) return go<G_PLAIN, 1, TilesF32Small>(g, ops, st);
        return go<G_PLAIN, 1, S>(g, ops, st);
    }
    if (form == G_SYM) {
        switch (W) {
            case 1: return go<G_SYM, 1, S>(g, ops, st);
            case 2: return go<G_SYM, 2, S>(g, ops, st);
            case 3: return go<G_SYM, 3, S>(g, ops, st);
            case 4: return go<G_SYM, 4, S>(g, ops, st);
        }
    }
    if (form == G_ASYM) {
        switch (W) {
            case 1: return go<G_ASYM, 1, A2>(g, ops, st);
            case 2: return go<G_ASYM, 2, A2>(g, ops, st);
            case 3: return go<G_ASYM, 3, A>(g, ops, st);
            case 4: return go<G_ASYM, 4, A>(g, ops, st);
        }
    }
    return cudaErrorNotSupported;
}

}  // namespace tdg
