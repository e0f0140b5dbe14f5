// fp64 instantiations of the packed GEMM (dGEMM forms of Sec. 7).
#include "tdg_gemm.cuh"

namespace tdg {

template <>
cudaError_t launch_packed_gemm<double>(int form, int W, const GemmArgs<double> &g,
                                       const CUtensorMap &mapA, const CUtensorMap &mapB,
                                       cudaStream_t st) {
    // 64 x 64 tiles, 4 x 4 per thread (asymmetric: 64 packed rows, W result rows each)
    if (form == G_PLAIN) return launch_cfg<double, G_PLAIN, 1, 64, 64, 4, 4, 16, 4>(g, mapA, mapB, st);
    if (form == G_SYM) {
        switch (W) {
            case 1: return launch_cfg<double, G_SYM, 1, 64, 64, 4, 4, 16, 4>(g, mapA, mapB, st);
            case 2: return launch_cfg<double, G_SYM, 2, 64, 64, 4, 4, 16, 4>(g, mapA, mapB, st);
            case 3: return launch_cfg<double, G_SYM, 3, 64, 64, 4, 4, 16, 4>(g, mapA, mapB, st);
            case 4: return launch_cfg<double, G_SYM, 4, 64, 64, 4, 4, 16, 4>(g, mapA, mapB, st);
        }
    }
    if (form == G_ASYM) {
        switch (W) {
            case 1: return launch_cfg<double, G_ASYM, 1, 64, 64, 4, 4, 16, 4>(g, mapA, mapB, st);
            case 2: return launch_cfg<double, G_ASYM, 2, 64, 64, 4, 4, 16, 4>(g, mapA, mapB, st);
            case 3: return launch_cfg<double, G_ASYM, 3, 64, 64, 4, 4, 16, 4>(g, mapA, mapB, st);
            case 4: return launch_cfg<double, G_ASYM, 4, 64, 64, 4, 4, 16, 4>(g, mapA, mapB, st);
        }
    }
    return cudaErrorNotSupported;
}

void packed_gemm_boxes(int dtype, int form, int *box_x_a, int *box_x_b, int *bk) {
    *bk = 16;
    if (dtype == TDG_F64) { *box_x_a = 64; *box_x_b = 64; return; }
    *box_x_a = form == G_ASYM ? 64 : 128;
    *box_x_b = 128;
}

}  // namespace tdg
