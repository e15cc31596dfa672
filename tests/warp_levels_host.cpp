// Host run of the one-warp coarse levels of the forward transform
// (paper_2005_08713_gb300/csrc/isx_warp_levels.cuh): 32 host threads play the
// 32 lanes, a std::barrier plays the warp barrier.  Reads cases until end of
// input, each "w h L" and h*w samples (row-major); runs levels 0 .. L-1 on a
// plane of pitch w + 3 (the in-place interleaved layout of the fused
// kernels), allocated to its exact size so that an address sanitizer sees
// any access outside it; prints the h*w results and a line "--" per case.
// Built and checked against the oracle by tests/test_host_warp_levels.py.
#include <algorithm>
#include <barrier>
#include <cstdint>
#include <cstdio>
#include <thread>
#include <vector>

static thread_local std::barrier<>* g_warp_barrier;
#define ISX_WL_FN inline
#define ISX_WL_SYNC() g_warp_barrier->arrive_and_wait()
#define ISX_WL_MIN(a, b) std::min<int>(a, b)
namespace isx {
inline int level_dim(int n, int l) { return ((n - 1) >> l) + 1; }
}  // namespace isx
#include "../paper_2005_08713_gb300/csrc/isx_warp_levels.cuh"

static int run_case(int w, int h, int L) {
  if (w < 1 || h < 1 || w > 32 || h > 32 || L < 0) return 2;
  const int pitch = w + 3;
  std::vector<int16_t> P((size_t)pitch * h, 0);
  for (int y = 0; y < h; ++y)
    for (int x = 0; x < w; ++x) {
      int v;
      if (std::scanf("%d", &v) != 1) return 2;
      P[(size_t)y * pitch + x] = (int16_t)v;
    }
  std::vector<int32_t> T(32 * isx::kWlPitch);
  if (L > 0) {
    std::barrier<> bar(32);
    std::vector<std::thread> lanes;
    for (int lane = 0; lane < 32; ++lane)
      lanes.emplace_back([&, lane] {
        g_warp_barrier = &bar;
        isx::warp_levels_fwd(P.data(), pitch, w, h, 0, L, T.data(), lane);
      });
    for (auto& t : lanes) t.join();
  }
  for (int y = 0; y < h; ++y) {
    for (int x = 0; x < w; ++x) std::printf("%d ", (int)P[(size_t)y * pitch + x]);
    std::printf("\n");
  }
  std::printf("--\n");
  return 0;
}

int main() {
  int w, h, L;
  while (std::scanf("%d %d %d", &w, &h, &L) == 3) {
    const int rc = run_case(w, h, L);
    if (rc != 0) return rc;
  }
  return 0;
}
