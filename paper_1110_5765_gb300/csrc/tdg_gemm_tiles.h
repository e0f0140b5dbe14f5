// Tile shapes of the packed GEMM: the one table both the kernel launches and
// the host-side TMA boxes read (a box that disagrees with the kernel's stage
// size would leave each stage's mbarrier short of its expected bytes).
#pragma once

namespace tdg {

template <int BM_, int BN_, int TM_, int TN_, int BK_, int STAGES_>
struct Tiles {
    static constexpr int BM = BM_, BN = BN_, TM = TM_, TN = TN_, BK = BK_, STAGES = STAGES_;
};

// fp32 plain / symmetric: 128 x 128 CTA tile, 8 x 8 per thread, 32-k stages x 3
// (the best of a sweep of k-tile, ring depth and thread tile on GB300 with the
// packed f32x2 main loop; 96 KB of ring keeps two CTAs per SM)
using TilesF32 = Tiles<128, 128, 8, 8, 32, 3>;
// fp32 plain product with few output tiles (at most half as many 128 x 128 tiles
// as SMs, e.g. 288 x 288 x 21600): 64 x 64 tiles, 4 x 4 per thread, so that four
// times as many SMs share the work (the conventional product does not split k,
// which would change its summation order)
using TilesF32Small = Tiles<64, 64, 4, 4, 32, 4>;
// fp32 asymmetric: 64 packed rows (W result rows each) x 128 columns
using TilesF32Asym = Tiles<64, 128, 4, 8, 16, 6>;     // W >= 3: W x 32 running sums per thread
using TilesF32AsymW2 = Tiles<128, 128, 8, 8, 32, 3>;  // W <= 2: W x 64 sums fit TMEM, 2.6 % faster
// fp64: 64 x 64, 4 x 4 per thread
using TilesF64 = Tiles<64, 64, 4, 4, 16, 4>;

}  // namespace tdg
