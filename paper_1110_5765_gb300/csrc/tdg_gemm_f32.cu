// fp32 instantiations of the packed GEMM (sGEMM forms of Sec. 7).
#include "tdg_gemm.cuh"

namespace tdg {

template <>
cudaError_t launch_packed_gemm<float>(int form, int W, const GemmArgs<float> &g,
                                      const CUtensorMap &mapA, const CUtensorMap &mapB,
                                      cudaStream_t st) {
    // plain / symmetric: 128 x 128 tiles, 8 x 8 per thread
    // asymmetric: 64 packed rows x 128 columns, 4 x 8 per thread (W result rows each)
    if (form == G_PLAIN) return launch_cfg<float, G_PLAIN, 1, 128, 128, 8, 8, 16, 6>(g, mapA, mapB, st);
    if (form == G_SYM) {
        switch (W) {
            case 1: return launch_cfg<float, G_SYM, 1, 128, 128, 8, 8, 16, 6>(g, mapA, mapB, st);
            case 2: return launch_cfg<float, G_SYM, 2, 128, 128, 8, 8, 16, 6>(g, mapA, mapB, st);
            case 3: return launch_cfg<float, G_SYM, 3, 128, 128, 8, 8, 16, 6>(g, mapA, mapB, st);
            case 4: return launch_cfg<float, G_SYM, 4, 128, 128, 8, 8, 16, 6>(g, mapA, mapB, st);
        }
    }
    if (form == G_ASYM) {
        switch (W) {
            case 1: return launch_cfg<float, G_ASYM, 1, 64, 128, 4, 8, 16, 6>(g, mapA, mapB, st);
            case 2: return launch_cfg<float, G_ASYM, 2, 64, 128, 4, 8, 16, 6>(g, mapA, mapB, st);
            case 3: return launch_cfg<float, G_ASYM, 3, 64, 128, 4, 8, 16, 6>(g, mapA, mapB, st);
            case 4: return launch_cfg<float, G_ASYM, 4, 64, 128, 4, 8, 16, 6>(g, mapA, mapB, st);
        }
    }
    return cudaErrorNotSupported;
}

}  // namespace tdg
