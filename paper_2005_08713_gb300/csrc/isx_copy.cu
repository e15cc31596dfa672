// Rectangle copies of isx_copy_rects: a viewport server assembles its
// requests' outputs from decoded cells and resident levels with one launch.
// No counterpart in the paper.
#include <cstdint>

#include "isx_kernels.h"

namespace isx {

// One CTA per piece; each warp copies whole rows.  A row is written as the
// 4-byte words of its destination (the unaligned head and tail bytes one by
// one), each word taken from the two aligned source words it straddles with
// a funnel shift, so that any byte offsets of source and destination (pixel
// offsets of 3-channel images) run at word width without divisions.  Every
// source word loaded holds at least one byte of the row.
__global__ void __launch_bounds__(256) k_copy_rects(const isx_rect_copy* __restrict__ pieces) {
  const isx_rect_copy j = pieces[blockIdx.x];
  const int lane = threadIdx.x & 31;
  const int nb = j.row_bytes;
  for (int r = threadIdx.x >> 5; r < j.rows; r += blockDim.x >> 5) {
    const uint8_t* s = static_cast<const uint8_t*>(j.src) + (int64_t)r * j.src_pitch;
    uint8_t* d = static_cast<uint8_t*>(j.dst) + (int64_t)r * j.dst_pitch;
    const int head = min((int)((4 - (reinterpret_cast<uintptr_t>(d) & 3)) & 3), nb);
    const int words = (nb - head) >> 2;
    const int tail = head + 4 * words;
    if (lane < head) d[lane] = s[lane];
    if (lane < nb - tail) d[tail + lane] = s[tail + lane];
    const uint8_t* sh = s + head;
    uint32_t* dw = reinterpret_cast<uint32_t*>(d + head);
    const int sa = (int)(reinterpret_cast<uintptr_t>(sh) & 3);
    const uint32_t* sw = reinterpret_cast<const uint32_t*>(sh - sa);
    if (sa == 0) {
      for (int k = lane; k < words; k += 32) dw[k] = __ldg(sw + k);
    } else {
      // word k of the row is bytes sa..3 of sw[k] and 0..sa-1 of sw[k+1]; sw[k+1] holds byte 4k+3
      for (int k = lane; k < words; k += 32) dw[k] = __funnelshift_r(__ldg(sw + k), __ldg(sw + k + 1), 8 * sa);
    }
  }
}

int launch_copy_rects(const isx_rect_copy* pieces, int n, cudaStream_t s) {
  k_copy_rects<<<n, 256, 0, s>>>(pieces);
  return 1;
}

}  // namespace isx
