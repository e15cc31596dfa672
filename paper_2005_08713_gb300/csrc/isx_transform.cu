// isx_transform.cu — planning, scans, colour transform and the recursive
// 5/3 lifting wavelet (forward and inverse), quantisation and the
// area-ordered coefficient layout used by the block coder.
//
// Wavelet (Sec. 4, "MATLAB's 5/3 Le Gall integer lifting"): per level the
// current LL region is lifted down every column, then along every row
// (predict d[n] = x[2n+1] - floor((x[2n]+x[2n+2])/2), update
// s[n] = x[2n] + floor((d[n-1]+d[n]+2)/4), mirrored at both ends); low
// outputs go to the first ceil(N/2) positions, high outputs after them
// (Mallat layout).  Floors are arithmetic right shifts.
#include <algorithm>

#include "isx_internal.cuh"
#include "isx_fused.cuh"
#include "isx_kernels.h"

namespace isx {

// ------------------------------------------------------------ planning
// One thread per tile: enumerate its blocks in stream order (per channel:
// LL cells, then the high-pass cells of levels L..1, raster order) and
// give each its slice of the area-ordered coefficient buffer.
// min_level > 0 keeps only LL blocks and levels > min_level (decode at a
// coarser resolution); out_index then counts the kept blocks only.
__global__ void k_plan_blocks(const TileDev* __restrict__ tiles, int n_tiles, int min_level, BlockDev* __restrict__ out) {
  int ti = blockIdx.x * blockDim.x + threadIdx.x;
  if (ti >= n_tiles) return;
  plan_tile_blocks(ti, tiles[ti], min_level, out);
}

// --------------------------------------------------------------- scans
// Exclusive prefix sum of int64 values, three phases; n up to 2^31.
constexpr int kScanItems = 8;
constexpr int kScanChunk = 256 * kScanItems;

__global__ void __launch_bounds__(256) k_scan_reduce(const int64_t* __restrict__ in, int64_t n, int64_t* __restrict__ part) {
  __shared__ int64_t tmp[33];
  int64_t base = (int64_t)blockIdx.x * kScanChunk;
  int64_t s = 0;
  for (int i = 0; i < kScanItems; ++i) {
    int64_t k = base + (int64_t)i * 256 + threadIdx.x;
    if (k < n) s += in[k];
  }
  int64_t total;
  cta_exclusive_sum<int64_t>(s, tmp, &total);
  if (threadIdx.x == 0) part[blockIdx.x] = total;
}

__global__ void __launch_bounds__(256) k_scan_partials(int64_t* __restrict__ part, int64_t np, int64_t* __restrict__ total_out) {
  __shared__ int64_t tmp[33];
  int64_t carry = 0;
  for (int64_t base = 0; base < np; base += 256) {
    int64_t k = base + threadIdx.x;
    int64_t v = k < np ? part[k] : 0;
    int64_t tot;
    int64_t ex = cta_exclusive_sum<int64_t>(v, tmp, &tot);
    if (k < np) part[k] = carry + ex;
    carry += tot;
  }
  if (threadIdx.x == 0 && total_out) *total_out = carry;
}

__global__ void __launch_bounds__(256) k_scan_final(const int64_t* __restrict__ in, int64_t n, const int64_t* __restrict__ part,
                                                    int64_t* __restrict__ out) {
  __shared__ int64_t tmp[33];
  int64_t base = (int64_t)blockIdx.x * kScanChunk;
  // each thread owns kScanItems consecutive elements
  int64_t v[kScanItems];
  int64_t s = 0;
  for (int i = 0; i < kScanItems; ++i) {
    int64_t k = base + (int64_t)threadIdx.x * kScanItems + i;
    v[i] = k < n ? in[k] : 0;
    s += v[i];
  }
  int64_t ex = cta_exclusive_sum<int64_t>(s, tmp, nullptr) + part[blockIdx.x];
  for (int i = 0; i < kScanItems; ++i) {
    int64_t k = base + (int64_t)threadIdx.x * kScanItems + i;
    if (k < n) out[k] = ex;
    ex += v[i];
  }
}

int launch_exclusive_scan(const int64_t* in, int64_t n, int64_t* out, int64_t* part, int64_t* total, cudaStream_t s) {
  int64_t nb = (n + kScanChunk - 1) / kScanChunk;
  if (nb == 0) nb = 1;
  k_scan_reduce<<<(unsigned)nb, 256, 0, s>>>(in, n, part);
  k_scan_partials<<<1, 256, 0, s>>>(part, nb, total);
  k_scan_final<<<(unsigned)nb, 256, 0, s>>>(in, n, part, out);
  return 3;
}

// Pixels -> C int32 planes (Mallat plane 0 .. C-1 of the tile), channels
// 0..2 through the tile's colour transform, the others as they are.
__global__ void k_load_pixels(const TileDev* __restrict__ tiles, int32_t* __restrict__ planes, int* __restrict__ status) {
  const TileDev& t = tiles[blockIdx.x];
  if (t.fused) return;
  if (threadIdx.x == 0 && blockIdx.y == 0) stamp_tile(t, kStampEncStart);
  const int64_t np = (int64_t)t.w * t.h;
  int32_t* out = planes + t.plane_base;
  uint32_t over = 0;   // bits of samples above the tile's bit depth
  for (int64_t e = (int64_t)blockIdx.y * blockDim.x + threadIdx.x; e < np; e += (int64_t)gridDim.y * blockDim.x) {
    int y = (int)(e / t.w), x = (int)(e - (int64_t)y * t.w);
    const uint8_t* row = t.pixels + (int64_t)y * t.pitch;
    int32_t v[3] = {0, 0, 0};
    for (int c = 0; c < t.C; ++c) {
      const int32_t s = sample_at(row, x, t.C, c, t.bits);
      over |= (uint32_t)s >> t.bits;
      if (t.ct && c < 3) v[c] = s;
      else out[c * np + e] = s;
    }
    if (t.ct)
      for (int c = 0; c < 3; ++c) out[c * np + e] = ct_forward(t.ct, c, v[0], v[1], v[2]);
  }
  if (over) set_status(status, kStRange);
}

// -------------------------------------------------------------- lifting
// Forward 1-D lifting of n samples read with `stride`, low outputs to
// out[0 .. nl), high outputs to out[nl .. n) (same stride).
__device__ void lift_fwd(const int32_t* x, int32_t* out, int n, int64_t stride) {
  if (n == 1) { out[0] = x[0]; return; }
  const int nl = (n + 1) >> 1;
  int32_t xe = x[0], dprev = 0;
  for (int k = 0; k < nl; ++k) {
    int32_t d, xe2;
    if (2 * k + 1 < n) {
      int32_t xo = x[(int64_t)(2 * k + 1) * stride];
      xe2 = (2 * k + 2 < n) ? x[(int64_t)(2 * k + 2) * stride] : xe;   // x[n] mirrors to x[n-2]
      d = xo - ((xe + xe2) >> 1);
      out[(int64_t)(nl + k) * stride] = d;
    } else {
      d = dprev;   // odd n, last even sample: d[nh] mirrors to d[nh-1]
      xe2 = xe;
    }
    int32_t dm1 = k == 0 ? d : dprev;   // d[-1] mirrors to d[0]
    out[(int64_t)k * stride] = xe + ((dm1 + d + 2) >> 2);
    dprev = d;
    xe = xe2;
  }
}

// Inverse of lift_fwd: in holds low [0, nl) and high [nl, n).
__device__ void lift_inv(const int32_t* in, int32_t* x, int n, int64_t stride) {
  if (n == 1) { x[0] = in[0]; return; }
  const int nl = (n + 1) >> 1, nh = n >> 1;
  int32_t dk = in[(int64_t)nl * stride];
  int32_t e = in[0] - ((dk + dk + 2) >> 2);
  for (int k = 0; k < nh; ++k) {
    int32_t en;
    int32_t dk1 = dk;
    if (k + 1 < nl) {
      if (k + 1 < nh) dk1 = in[(int64_t)(nl + k + 1) * stride];
      en = in[(int64_t)(k + 1) * stride] - ((dk + dk1 + 2) >> 2);
    } else {
      en = e;   // even n: x[n] mirrors to x[n-2]
    }
    x[(int64_t)(2 * k) * stride] = e;
    x[(int64_t)(2 * k + 1) * stride] = dk + ((e + en) >> 1);
    e = en;
    dk = dk1;
  }
  if (n & 1) x[(int64_t)(n - 1) * stride] = e;
}

// Task = tile in blockIdx.x, channel in blockIdx.z; blockIdx.y chunks the
// columns (vertical) or rows (horizontal) of the LL region.
// Plane geometry: stride = plane_w (the tile width for encode, the level-z
// width for decode); region cw x ch at level `lvl` of each tile.
struct PassGeom {
  int cw, ch, stride;
  int64_t base;
};

__device__ inline bool pass_geom(const TileDev& t, int c, int lvl, bool decode_plane, int z, PassGeom* g) {
  if (c >= t.C || lvl >= t.L || lvl < z || t.fused || t.win >= 0) return false;
  int pw = decode_plane ? level_dim(t.w, z) : t.w;
  int ph = decode_plane ? level_dim(t.h, z) : t.h;
  g->cw = level_dim(t.w, lvl);
  g->ch = level_dim(t.h, lvl);
  g->stride = pw;
  g->base = t.plane_base + (int64_t)c * pw * ph;
  return true;
}

__global__ void k_fwd_vpass(const TileDev* __restrict__ tiles, int lvl, const int32_t* __restrict__ A, int32_t* __restrict__ B) {
  const TileDev& t = tiles[blockIdx.x];
  PassGeom g;
  if (!pass_geom(t, blockIdx.z, lvl, false, 0, &g)) return;
  int col = blockIdx.y * blockDim.x + threadIdx.x;
  if (col >= g.cw) return;
  lift_fwd(A + g.base + col, B + g.base + col, g.ch, g.stride);
}

__global__ void k_fwd_hpass(const TileDev* __restrict__ tiles, int lvl, const int32_t* __restrict__ B, int32_t* __restrict__ A) {
  const TileDev& t = tiles[blockIdx.x];
  PassGeom g;
  if (!pass_geom(t, blockIdx.z, lvl, false, 0, &g)) return;
  int row = blockIdx.y * blockDim.x + threadIdx.x;
  if (row >= g.ch) return;
  lift_fwd(B + g.base + (int64_t)row * g.stride, A + g.base + (int64_t)row * g.stride, g.cw, 1);
}

// Inverse level lvl (0-based: undoes the transform of LL_lvl) on decode
// planes of size level_dim(w, z) x level_dim(h, z).
__global__ void k_inv_hpass(const TileDev* __restrict__ tiles, int lvl, int z, const int32_t* __restrict__ A, int32_t* __restrict__ B) {
  const TileDev& t = tiles[blockIdx.x];
  PassGeom g;
  if (!pass_geom(t, blockIdx.z, lvl, true, z, &g)) return;
  int row = blockIdx.y * blockDim.x + threadIdx.x;
  if (row >= g.ch) return;
  lift_inv(A + g.base + (int64_t)row * g.stride, B + g.base + (int64_t)row * g.stride, g.cw, 1);
}

__global__ void k_inv_vpass(const TileDev* __restrict__ tiles, int lvl, int z, const int32_t* __restrict__ B, int32_t* __restrict__ A) {
  const TileDev& t = tiles[blockIdx.x];
  PassGeom g;
  if (!pass_geom(t, blockIdx.z, lvl, true, z, &g)) return;
  int col = blockIdx.y * blockDim.x + threadIdx.x;
  if (col >= g.cw) return;
  lift_inv(B + g.base + col, A + g.base + col, g.ch, g.stride);
}

// --------------------------------------------------------- quantise + pack
// Per block: quantise (dead zone, q = sign(c) floor(|c| / 2^s)) and gather
// the coefficients of every 4x2 area (Eq. 1 order) into 8 consecutive
// int32 in Eq. 2 bit order (upper row then lower row, left to right).
// Positions outside the subband are the zero padding.
__global__ void __launch_bounds__(256) k_pack_blocks(const TileDev* __restrict__ tiles, const BlockDev* __restrict__ blocks,
                                                     const int32_t* __restrict__ planes, void* __restrict__ coef_buf) {
  const BlockDev b = blocks[blockIdx.x];
  const TileDev& t = tiles[b.tile];
  if (t.fused) return;   // packed by the fused kernel
  const int n = b.w * b.h / 8, na = b.p * n;
  const int q = qlog2_of(t, b.level);
  const int32_t* plane = planes + t.plane_base + (int64_t)b.c * t.w * t.h;
  for (int a = threadIdx.x; a < na; a += blockDim.x) {
    int type = a / n, k = a - type * n;
    int i, j;
    area_ij(k, b.w, &i, &j);
    int sx, sy, sw, sh;
    subband_rect(t.w, t.h, t.L, b.level, type, &sx, &sy, &sw, &sh);
    int32_t v[8];
#pragma unroll
    for (int e = 0; e < 8; ++e) {
      int yy = kCell * b.by + i + (e >> 2), xx = kCell * b.bx + j + (e & 3);
      int32_t c = 0;
      if (yy < sh && xx < sw) c = plane[(int64_t)(sy + yy) * t.w + sx + xx];
      int32_t m = c < 0 ? -c : c;
      m >>= q;
      v[e] = c < 0 ? -m : m;
    }
    if (b.coef16) {
      uint4 u;
      u.x = (uint16_t)v[0] | ((uint32_t)(uint16_t)v[1] << 16);
      u.y = (uint16_t)v[2] | ((uint32_t)(uint16_t)v[3] << 16);
      u.z = (uint16_t)v[4] | ((uint32_t)(uint16_t)v[5] << 16);
      u.w = (uint16_t)v[6] | ((uint32_t)(uint16_t)v[7] << 16);
      reinterpret_cast<uint4*>(reinterpret_cast<uint8_t*>(coef_buf) + b.coef)[a] = u;
    } else {
      int4* o = reinterpret_cast<int4*>(reinterpret_cast<uint8_t*>(coef_buf) + b.coef) + 2 * (int64_t)a;
      o[0] = make_int4(v[0], v[1], v[2], v[3]);
      o[1] = make_int4(v[4], v[5], v[6], v[7]);
    }
  }
}

// Copy quantised Mallat planes out (isx_forward_coefficients): the same
// quantiser applied in place over each subband.
__global__ void k_quantise_planes(const TileDev* __restrict__ tiles, const int32_t* __restrict__ planes, int32_t* __restrict__ out) {
  const TileDev& t = tiles[blockIdx.x];
  const int64_t np = (int64_t)t.w * t.h;
  for (int64_t e = (int64_t)blockIdx.y * blockDim.x + threadIdx.x; e < np * t.C; e += (int64_t)gridDim.y * blockDim.x) {
    int64_t pe = e % np;
    int y = (int)(pe / t.w), x = (int)(pe - (int64_t)y * t.w);
    // which subband holds (x, y): the finest level whose detail region contains it
    int level = 0;
    for (int l = 1; l <= t.L; ++l) {
      int lw = level_dim(t.w, l), lh = level_dim(t.h, l);
      if (x >= lw || y >= lh) { level = l; break; }
    }
    int q = qlog2_of(t, level);
    int32_t c = planes[t.plane_base + e];
    int32_t m = c < 0 ? -c : c;
    m >>= q;
    out[t.plane_base + e] = c < 0 ? -m : m;
  }
}

// ---------------------------------------------------------- decode output
// Inverse colour transform of channels 0..2 (ct_inverse), clamp to
// [0, 2^bits - 1] and write the part of the tile's level-z image that falls
// inside the requested rectangle.
__global__ void k_store_region(const TileDev* __restrict__ tiles, int z, const int32_t* __restrict__ planes) {
  const TileDev& t = tiles[blockIdx.x];
  if (t.fused || t.win >= 0) return;   // written by the fused inverse kernel / the windowed store
  uint8_t* __restrict__ out = t.dst;
  const int64_t pitch = t.dpitch;
  const int rx = t.rx, ry = t.ry, rw = t.rw, rh = t.rh;
  const int zw = level_dim(t.w, z), zh = level_dim(t.h, z);
  const int tx = t.x0 >> z, ty = t.y0 >> z;
  const int64_t np = (int64_t)zw * zh;
  const int32_t* pl = planes + t.plane_base;
  const int32_t maxv = (1 << t.bits) - 1;
  for (int64_t e = (int64_t)blockIdx.y * blockDim.x + threadIdx.x; e < np; e += (int64_t)gridDim.y * blockDim.x) {
    int y = (int)(e / zw), x = (int)(e - (int64_t)y * zw);
    int ox = tx + x - rx, oy = ty + y - ry;
    if (ox < 0 || oy < 0 || ox >= rw || oy >= rh) continue;
    int32_t v[3] = {0, 0, 0};
    if (t.ct) ct_inverse(t.ct, pl[e], pl[np + e], pl[2 * np + e], &v[0], &v[1], &v[2]);
    uint8_t* row = out + (int64_t)oy * pitch;
    for (int c = 0; c < t.C; ++c) {
      const int32_t s = t.ct && c < 3 ? v[c] : pl[c * np + e];
      int32_t q = min(max(s, 0), maxv);
      if (t.bits <= 8) row[ox * t.C + c] = (uint8_t)q;
      else reinterpret_cast<uint16_t*>(row)[ox * t.C + c] = (uint16_t)q;
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) stamp_tile(t, kStampDecEnd);
}

// ------------------------------------------------------- windowed inverse
// x[k], k in [a, b), of one inverse 5/3 level of a line of N samples (Sec. 4,
// the inverse of the lifting above): the low samples s[n] at
// lo[(n - l0) * ls], the high d[n] at hi[(n - h0) * hs].  The windows hold
// every index these outputs read (the host's inv_needs), so the line's own
// symmetric extension gives its end samples (d[-1] = d[0], d[nh] = d[nh-1],
// x[N] = x[N-2]) and nothing outside the line is read.
__device__ inline void lift_inv_window(const int32_t* lo, int l0, int64_t ls, const int32_t* hi, int h0, int64_t hs, int N, int a,
                                       int b, int32_t* out, int64_t os) {
  if (N == 1) {
    if (a == 0 && b > 0) out[0] = lo[(int64_t)(0 - l0) * ls];
    return;
  }
  const int nl = (N + 1) >> 1, nh = N >> 1;
  auto D = [&](int m) { return hi[(int64_t)(min(max(m, 0), nh - 1) - h0) * hs]; };
  auto XE = [&](int m) { return lo[(int64_t)(m - l0) * ls] - ((D(m - 1) + D(m) + 2) >> 2); };
  for (int k = a; k < b; ++k) {
    const int n = k >> 1;
    out[(int64_t)(k - a) * os] = (k & 1) ? D(n) + ((XE(n) + XE(min(n + 1, nl - 1))) >> 1) : XE(n);
  }
}

// Row pass of inverse level `lvl` of the windowed tiles: every row of W_l
// (its low rows, then its high rows) to the LL_{l-1} window's columns,
// into T_l; one thread per (row, run of 32 outputs).
__global__ void k_win_hpass(const TileDev* __restrict__ tiles, const WinDev* __restrict__ wins, int lvl, int32_t* __restrict__ planes) {
  const TileDev& t = tiles[blockIdx.x];
  if (t.win < 0 || (int)blockIdx.z >= t.C) return;
  const WinDev& W = wins[t.win];
  if (lvl <= W.z || lvl > W.L) return;
  const WinLevel& v = W.lev[lvl];
  const int c = blockIdx.z;
  const int nlx = v.lx1 - v.lx0, cols = nlx + (v.hx1 - v.hx0), rows = (v.ly1 - v.ly0) + (v.hy1 - v.hy0);
  const int ow = v.ox1 - v.ox0, runs = (ow + 31) >> 5;
  const int Nx = level_dim(t.w, lvl - 1);
  int32_t* base = planes + t.plane_base;
  const int32_t* in = base + v.buf + (int64_t)c * cols * rows;
  int32_t* out = base + v.tmp + (int64_t)c * ow * rows;
  for (int64_t e = (int64_t)blockIdx.y * blockDim.x + threadIdx.x; e < (int64_t)rows * runs; e += (int64_t)gridDim.y * blockDim.x) {
    const int r = (int)(e / runs), k = (int)(e - (int64_t)r * runs);
    const int a = v.ox0 + 32 * k, b = min(a + 32, v.ox1);
    const int32_t* row = in + (int64_t)r * cols;
    lift_inv_window(row, v.lx0, 1, row + nlx, v.hx0, 1, Nx, a, b, out + (int64_t)r * ow + (a - v.ox0), 1);
  }
}

// Column pass of inverse level `lvl`: every column of T_l to the LL_{l-1}
// window's rows, into the LL part of W_{l-1} (or F at level z); one thread
// per (column, run of 32 outputs), neighbouring threads on neighbouring
// columns.
__global__ void k_win_vpass(const TileDev* __restrict__ tiles, const WinDev* __restrict__ wins, int lvl, int32_t* __restrict__ planes) {
  const TileDev& t = tiles[blockIdx.x];
  if (t.win < 0 || (int)blockIdx.z >= t.C) return;
  const WinDev& W = wins[t.win];
  if (lvl <= W.z || lvl > W.L) return;
  const WinLevel& v = W.lev[lvl];
  const int c = blockIdx.z;
  const int nly = v.ly1 - v.ly0, rows = nly + (v.hy1 - v.hy0);
  const int ow = v.ox1 - v.ox0, oh = v.oy1 - v.oy0, runs = (oh + 31) >> 5;
  const int Ny = level_dim(t.h, lvl - 1);
  int32_t* base = planes + t.plane_base;
  const int32_t* in = base + v.tmp + (int64_t)c * ow * rows;
  int32_t* dst;
  int64_t pitch;
  if (lvl - 1 == W.z) {
    pitch = W.fx1 - W.fx0;
    dst = base + W.fbuf + (int64_t)c * pitch * (W.fy1 - W.fy0);
  } else {
    const WinLevel& u = W.lev[lvl - 1];
    pitch = (u.lx1 - u.lx0) + (u.hx1 - u.hx0);
    dst = base + u.buf + (int64_t)c * pitch * ((u.ly1 - u.ly0) + (u.hy1 - u.hy0));
  }
  for (int64_t e = (int64_t)blockIdx.y * blockDim.x + threadIdx.x; e < (int64_t)ow * runs; e += (int64_t)gridDim.y * blockDim.x) {
    const int k = (int)(e / ow), x = (int)(e - (int64_t)k * ow);
    const int a = v.oy0 + 32 * k, b = min(a + 32, v.oy1);
    lift_inv_window(in + x, v.ly0, ow, in + (int64_t)nly * ow + x, v.hy0, ow, Ny, a, b, dst + (int64_t)(a - v.oy0) * pitch + x, pitch);
  }
}

// The level-z window F of each windowed tile (inverse colour transform,
// clamp to [0, 2^bits - 1]) into its destination, as k_store_region.
__global__ void k_win_store(const TileDev* __restrict__ tiles, const WinDev* __restrict__ wins, const int32_t* __restrict__ planes) {
  const TileDev& t = tiles[blockIdx.x];
  if (t.win < 0) return;
  const WinDev& W = wins[t.win];
  const int fw = W.fx1 - W.fx0, fh = W.fy1 - W.fy0;
  const int64_t np = (int64_t)fw * fh;
  const int32_t* pl = planes + t.plane_base + W.fbuf;
  const int tx = (t.x0 >> W.z) - t.rx, ty = (t.y0 >> W.z) - t.ry;   // the tile's origin in the output
  const int32_t maxv = (1 << t.bits) - 1;
  for (int64_t e = (int64_t)blockIdx.y * blockDim.x + threadIdx.x; e < np; e += (int64_t)gridDim.y * blockDim.x) {
    const int y = (int)(e / fw), x = (int)(e - (int64_t)y * fw);
    const int ox = tx + W.fx0 + x, oy = ty + W.fy0 + y;
    if (ox < 0 || oy < 0 || ox >= t.rw || oy >= t.rh) continue;
    int32_t v[3] = {0, 0, 0};
    if (t.ct) ct_inverse(t.ct, pl[e], pl[np + e], pl[2 * np + e], &v[0], &v[1], &v[2]);
    uint8_t* row = t.dst + (int64_t)oy * t.dpitch;
    for (int c = 0; c < t.C; ++c) {
      const int32_t s = t.ct && c < 3 ? v[c] : pl[c * np + e];
      const int32_t q = min(max(s, 0), maxv);
      if (t.bits <= 8) row[ox * t.C + c] = (uint8_t)q;
      else reinterpret_cast<uint16_t*>(row)[ox * t.C + c] = (uint16_t)q;
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) stamp_tile(t, kStampDecEnd);
}

__global__ void __launch_bounds__(kFusedThreads) k_fwd_tile_smem(const TileDev* __restrict__ tiles, const int32_t* __restrict__ task_tile,
                                                                 int slots, const BlockDev* __restrict__ blocks, uint8_t* __restrict__ coef,
                                                                 int* __restrict__ status) {
  extern __shared__ __align__(16) int16_t P[];
  __shared__ FusedBlock s_fb[kMaxFusedBlocks];
  const int tt = task_tile[blockIdx.x / slots], c = blockIdx.x % slots;
  const TileDev& t = tiles[tt];
  if (c >= t.C) return;
  if (threadIdx.x == 0) stamp_tile(t, kStampEncStart);
  fused_forward_channel(t, c, blocks, coef, status, P, s_fb);
}

__global__ void __launch_bounds__(kFusedThreads) k_inv_tile_smem(const TileDev* __restrict__ tiles, const int32_t* __restrict__ task_tile,
                                                                 const BlockDev* __restrict__ blocks, const DecInfo* __restrict__ info,
                                                                 const int64_t* __restrict__ sym_off, const uint8_t* __restrict__ sym,
                                                                 const int64_t* __restrict__ sym_total, int64_t sym_cap, int z, int slots,
                                                                 int16_t* __restrict__ fplanes, uint32_t* __restrict__ tickets) {
  extern __shared__ __align__(16) int16_t P[];
  __shared__ FusedBlock s_fb[kMaxFusedBlocks];
  __shared__ int32_t s_po[kMaxFusedBlocks][kMaxFusedPlanes][3];   // (plane, type) symbols from the block's first; -1: not kept
  __shared__ bool s_last;
  const int tt = task_tile[blockIdx.x / slots], c = blockIdx.x % slots;
  const TileDev& t = tiles[tt];
  if (c >= t.C || *sym_total > sym_cap) return;
  const int zw = level_dim(t.w, z), zh = level_dim(t.h, z), pitch = smem_pitch(zw);
  fused_inverse_plane(t, c, z, blocks, info, sym_off, sym, P, s_fb, s_po);
  if (t.ct && c < 3) {
    // Every CTA of channels 0..2 leaves its channel plane (int16) in global
    // memory and takes a ticket; the tile's third CTA to finish inverts the
    // colour transform from its own plane and the other two (no CTA waits
    // for another).
    int16_t* gp = fplanes + t.plane_base;
    fused_handoff(P, pitch, zw, zh, gp + (int64_t)c * zw * zh);
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) s_last = (atomicAdd(&tickets[blockIdx.x / slots], 1u) % 3u) == 2u;
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    store_tile_ct(t, z, zw, zh, c, P, pitch, gp);
    __syncthreads();
    discard_handoff(gp, zw, zh);
  } else {
    store_tile_channel(t, z, zw, zh, c, P, pitch);
  }
  __syncthreads();
  if (threadIdx.x == 0) stamp_tile(t, kStampDecEnd);
}

// --------------------------------------------------------------- launches
int launch_forward_transform(const TileDev* d_tiles, int n_tiles, int max_levels, int max_dim, int max_c, int32_t* A, int32_t* B,
                             int* status, cudaStream_t s) {
  int launches = 0;
  dim3 g0(n_tiles, 64);
  k_load_pixels<<<g0, 256, 0, s>>>(d_tiles, A, status);
  ++launches;
  const int T = 128;
  for (int l = 0; l < max_levels; ++l) {
    int md = level_dim(max_dim, l);
    dim3 g(n_tiles, ceil_div(md, T), max_c);
    k_fwd_vpass<<<g, T, 0, s>>>(d_tiles, l, A, B);
    k_fwd_hpass<<<g, T, 0, s>>>(d_tiles, l, B, A);
    launches += 2;
  }
  return launches;
}

int launch_pack_blocks(const TileDev* d_tiles, const BlockDev* d_blocks, int64_t n_blocks, const int32_t* planes, void* coef,
                       cudaStream_t s) {
  k_pack_blocks<<<(unsigned)n_blocks, 256, 0, s>>>(d_tiles, d_blocks, planes, coef);
  return 1;
}

int launch_fused_forward(const TileDev* d_tiles, const int32_t* d_task_tile, int n_fused, int slots, int smem_bytes, int threads,
                         const BlockDev* d_blocks, void* coef, int* status, cudaStream_t s) {
  if (n_fused == 0) return 0;
  k_fwd_tile_smem<<<slots * n_fused, threads, smem_bytes, s>>>(d_tiles, d_task_tile, slots, d_blocks, (uint8_t*)coef, status);
  return 1;
}

int launch_fused_inverse(const TileDev* d_tiles, const int32_t* d_task_tile, int n_fused, int slots, int smem_bytes, int threads,
                         const DecodeBuffers& db, int16_t* planes16, uint32_t* tickets, cudaStream_t s) {
  if (n_fused == 0) return 0;
  k_inv_tile_smem<<<slots * n_fused, threads, smem_bytes, s>>>(d_tiles, d_task_tile, db.blocks, db.info, db.sym_off, db.sym, db.totals,
                                                               db.sym_cap, db.z, slots, planes16, tickets);
  return 1;
}

bool fused_tile(int w, int h) { return tile_uses_smem(w, h); }
int fused_plane_bytes(int w, int h) { return smem_pitch(w) * h * 2; }

cudaError_t transform_set_attributes() {
  cudaError_t e = cudaFuncSetAttribute(k_fwd_tile_smem, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemPlaneBytes);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_inv_tile_smem, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemPlaneBytes);
  return e;
}

int launch_plan_blocks(const TileDev* d_tiles, int n_tiles, int min_level, BlockDev* d_blocks, cudaStream_t s) {
  k_plan_blocks<<<ceil_div(n_tiles, 128), 128, 0, s>>>(d_tiles, n_tiles, min_level, d_blocks);
  return 1;
}

int launch_quantise_planes(const TileDev* d_tiles, int n_tiles, const int32_t* planes, int32_t* out, cudaStream_t s) {
  k_quantise_planes<<<dim3(n_tiles, 64), 256, 0, s>>>(d_tiles, planes, out);
  return 1;
}

int launch_inverse_transform(const TileDev* d_tiles, int n_tiles, int max_levels, int z, int max_dim, int max_c, int32_t* A,
                             int32_t* B, cudaStream_t s) {
  int launches = 0;
  const int T = 128;
  for (int l = max_levels - 1; l >= z; --l) {
    int md = level_dim(max_dim, l);
    dim3 g(n_tiles, ceil_div(md, T), max_c);
    k_inv_hpass<<<g, T, 0, s>>>(d_tiles, l, z, A, B);
    k_inv_vpass<<<g, T, 0, s>>>(d_tiles, l, z, B, A);
    launches += 2;
  }
  return launches;
}

int launch_window_inverse(const TileDev* d_tiles, int n_tiles, int max_levels, int z, int max_c, const WinDev* wins, int32_t* planes,
                          int max_win, cudaStream_t s) {
  int launches = 0;
  const int T = 256;
  // grid-stride loops: enough CTAs for the largest window's rows x runs, at most 4 per SM and tile
  const int64_t work = (int64_t)max_win * ((max_win + 31) / 32);
  const unsigned gy = (unsigned)std::max<int64_t>(1, std::min<int64_t>((work + T - 1) / T, 608));
  for (int l = max_levels; l > z; --l) {
    dim3 g(n_tiles, gy, max_c);
    k_win_hpass<<<g, T, 0, s>>>(d_tiles, wins, l, planes);
    k_win_vpass<<<g, T, 0, s>>>(d_tiles, wins, l, planes);
    launches += 2;
  }
  k_win_store<<<dim3(n_tiles, gy), T, 0, s>>>(d_tiles, wins, planes);
  return launches + 1;
}

int launch_store_region(const TileDev* d_tiles, int n_tiles, int z, const int32_t* planes, cudaStream_t s) {
  k_store_region<<<dim3(n_tiles, 32), 256, 0, s>>>(d_tiles, z, planes);
  return 1;
}

}  // namespace isx
