// isx_host_plan.h — host-side descriptor checks and per-tile counts shared
// by the context entry points (isx_api.cu) and the no-allocation encoder
// (isx_static.cu), so that both accept the same descriptors and size the
// same blocks.
#pragma once
#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>

#include "isx.h"
#include "isx_internal.cuh"

namespace isx {

inline bool tile_ok(const isx_tile_desc& t, std::string* why) {
  if (t.width < 1 || t.width > 65535 || t.height < 1 || t.height > 65535) { *why = "width/height out of 1..65535"; return false; }
  if (t.channels < 1 || t.channels > 16) { *why = "channels out of 1..16"; return false; }
  if (t.bits < 1 || t.bits > 16) { *why = "bits out of 1..16"; return false; }
  if (t.levels < 0 || t.levels > kMaxLevels) { *why = "levels out of 0..15"; return false; }
  if (t.x0 < 0 || t.y0 < 0) { *why = "negative tile origin"; return false; }
  if (t.transform < ISX_CT_DEFAULT || t.transform > ISX_CT_YCOCG_R) { *why = "transform out of 0..3"; return false; }
  if ((t.transform == ISX_CT_RCT || t.transform == ISX_CT_YCOCG_R) && t.channels < 3) {
    *why = "a colour transform needs 3 or more channels";
    return false;
  }
  if (t.reserved != 0) { *why = "reserved field must be 0"; return false; }
  for (int l = 0; l <= t.levels; ++l)
    if (t.qstep_log2[l] > 15) { *why = "qstep_log2 out of 0..15"; return false; }
  return true;
}

// Stored colour-transform id of a valid descriptor: 0 none, 1 RCT (JPEG 2000),
// 2 YCoCg-R, on channels 0..2.
inline int tile_ct(const isx_tile_desc& t) {
  if (t.transform == ISX_CT_DEFAULT) return t.channels == 3 ? 1 : 0;
  return t.transform == ISX_CT_RCT ? 1 : t.transform == ISX_CT_YCOCG_R ? 2 : 0;
}

// Bounds on the int16 range of the transforms.  Every state of the forward
// transform of samples in [0, M] (a plane coded as it is, or Y) or [-M, M]
// (RCT or YCoCg-R chroma: a range of 2M) stays within kGain2D * range plus
// the floors' rounding.  kGain2D comes from the L1 norms of the equivalent
// filters of up to 15 iterated 5/3 levels, taken on finite lines with
// symmetric extension at both ends (at most 1.720 for the low and 2.873 for
// the high cascades; the infinite line gives 1.716 and 2.867), rounded up to
// 1.73 and 2.885: 2.885^2 / 2 <= 4.17.  The floors of the integer lifting add
// at most 2 inside a level and 1.875 to each LL, carried on by the linear
// filters with a 2-D gain of at most 2.885^2 <= 8.33: kRoundPerLevel per
// level.
constexpr double kGain2D = 4.17;
constexpr double kRoundPerLevel = 16.0;   // >= 1.875 * 8.33
inline double forward_state_bound(const isx_tile_desc& t) {
  const double M = (double)((1 << t.bits) - 1) * (tile_ct(t) ? 2.0 : 1.0);
  return M * kGain2D + 2.0 + kRoundPerLevel * t.levels;
}

// Every value the inverse holds for a tile decoded at level z with `drop`
// least significant planes discarded (Sec. 4, "Decompression"), for streams
// written by the encoder.  Each state of the inverse is a state of the
// lossless inverse (= a state of the forward transform, by perfect
// reconstruction) plus a deviation caused by the dequantised coefficients:
// a band sample of step D = 2^q decoded with k planes dropped is off by at
// most 2^k D - 1 (and never by more than F + D/2); one inverse level maps
// deviations (LL, HL, LH, HH) to at most LL + HL + LH + HH + 6 (the 5/3
// synthesis has L-inf gain 1 on each band pair; three passes, each floor off
// by less than 1), and a level whose inputs are all exact adds nothing.
inline double inverse_state_bound(const isx_tile_desc& t, int z, int drop) {
  const double F = forward_state_bound(t);
  auto dev = [&](int q) {
    const double D = std::ldexp(1.0, q);
    return std::min(std::ldexp(D, std::min(drop, 40)) - 1.0, F + D / 2);
  };
  double E = dev(t.qstep_log2[t.levels]);
  for (int l = t.levels; l > z; --l) {
    const double e = dev(t.qstep_log2[l - 1]);
    if (E > 0 || e > 0) E += 3.0 * e + 6.0;
  }
  return F + E;
}

// blocks of a tile (all levels, or LL + levels > zmin) and padded coefficients
inline void tile_counts(const isx_tile_desc& t, int zmin, int64_t* nb, int64_t* ncoef) {
  int64_t b = 0, c = 0;
  int lw = level_dim(t.width, t.levels), lh = level_dim(t.height, t.levels);
  b += (int64_t)ceil_div(lw, kCell) * ceil_div(lh, kCell);
  c += (int64_t)pad4(lw) * pad4(lh);
  for (int l = t.levels; l >= 1 && l > zmin; --l) {
    int gw = level_dim(t.width, l), gh = level_dim(t.height, l);
    b += (int64_t)ceil_div(gw, kCell) * ceil_div(gh, kCell);
    c += 3LL * pad4(gw) * pad4(gh);
  }
  *nb = b * t.channels;
  *ncoef = c * t.channels;
}

// Blocks of each level of a tile (level 0 = LL) and the largest block of
// each level in area quads (4 areas of 8 coefficients), all channels.
inline void level_blocks(const isx_tile_desc& t, int64_t* count, int* quads) {
  for (int l = 0; l <= t.levels; ++l) {
    const int gw = level_dim(t.width, l == 0 ? t.levels : l), gh = level_dim(t.height, l == 0 ? t.levels : l);
    count[l] += (int64_t)ceil_div(gw, kCell) * ceil_div(gh, kCell) * t.channels;
    const int p = l == 0 ? 1 : 3;
    const int q = p * pad4(std::min(gw, kCell)) * pad4(std::min(gh, kCell)) / 32;
    quads[l] = std::max(quads[l], q);
  }
}

inline void fill_tiledev(TileDev& d, const isx_tile_desc& t) {
  std::memset(&d, 0, sizeof(d));
  d.pixels = (const uint8_t*)t.pixels;
  d.pitch = t.row_pitch_bytes;
  d.w = t.width; d.h = t.height; d.C = t.channels; d.bits = t.bits; d.L = t.levels;
  d.x0 = t.x0; d.y0 = t.y0;
  d.ct = tile_ct(t);
  d.coef16 = forward_state_bound(t) <= 32767.0 ? 1 : 0;
  d.win = -1;
  for (int k = 0; k < 16; ++k) d.q[k] = k <= t.levels ? t.qstep_log2[k] : 0;
}

// ---------------------------------------------------- windowed region decode
// Band index ranges that the inverse 5/3 outputs [a, b) of a line of N
// samples read: the low samples [*l0, *l1) and the high samples [*h0, *h1).
// Output 2n is s[n] - floor((d[n-1] + d[n] + 2) / 4) and output 2n+1 is
// d[n] + floor((x[2n] + x[2n+2]) / 2), with the line's symmetric extension:
// d[-1] = d[0], d[nh] = d[nh-1] (odd N) and x[N] = x[N-2] (even N).  A line
// of one sample passes through.
inline void inv_needs(int N, int a, int b, int32_t* l0, int32_t* l1, int32_t* h0, int32_t* h1) {
  if (N == 1) { *l0 = 0; *l1 = 1; *h0 = *h1 = 0; return; }
  const int nl = (N + 1) / 2, nh = N / 2;
  int lmin = N, lmax = -1, hmin = N, hmax = -1;
  auto hi = [&](int n) {
    n = std::min(std::max(n, 0), nh - 1);
    hmin = std::min(hmin, n); hmax = std::max(hmax, n);
  };
  auto xe = [&](int n) {   // the even sample x[2n]
    lmin = std::min(lmin, n); lmax = std::max(lmax, n);
    hi(n - 1); hi(n);
  };
  // every index is monotone in the output position: the ends of [a, b) suffice
  const int ks[4] = {a, std::min(a + 1, b - 1), std::max(b - 2, a), b - 1};
  for (int k : ks) {
    const int n = k >> 1;
    if (!(k & 1)) xe(n);
    else { hi(n); xe(n); xe(std::min(n + 1, nl - 1)); }
  }
  *l0 = lmin; *l1 = lmax + 1; *h0 = hmin; *h1 = hmax + 1;
}

// The windows of a decode of the level-z window [ax, bx) x [ay, by) (tile-
// local level-z pixels) of tile t, from level z + 1 up to the tile's LL;
// returns the int32 elements its planes take (all channels).
inline int64_t plan_window(const isx_tile_desc& t, int z, int ax, int bx, int ay, int by, WinDev& W) {
  std::memset(&W, 0, sizeof(W));
  W.z = z; W.L = t.levels;
  W.fx0 = ax; W.fx1 = bx; W.fy0 = ay; W.fy1 = by;
  const int64_t C = t.channels;
  int64_t off = 0;
  W.fbuf = off;
  off += C * (bx - ax) * (by - ay);
  int ox0 = ax, ox1 = bx, oy0 = ay, oy1 = by;
  for (int l = z + 1; l <= t.levels; ++l) {
    WinLevel& v = W.lev[l];
    inv_needs(level_dim(t.width, l - 1), ox0, ox1, &v.lx0, &v.lx1, &v.hx0, &v.hx1);
    inv_needs(level_dim(t.height, l - 1), oy0, oy1, &v.ly0, &v.ly1, &v.hy0, &v.hy1);
    v.ox0 = ox0; v.ox1 = ox1; v.oy0 = oy0; v.oy1 = oy1;
    const int64_t cols = (v.lx1 - v.lx0) + (v.hx1 - v.hx0), rows = (v.ly1 - v.ly0) + (v.hy1 - v.hy0);
    v.buf = off;
    off += C * cols * rows;
    v.tmp = off;
    off += C * (ox1 - ox0) * rows;
    ox0 = v.lx0; ox1 = v.lx1; oy0 = v.ly0; oy1 = v.ly1;
  }
  return off;
}

// Blocks a windowed decode reads (all channels) and their padded coefficients.
inline void window_counts(const isx_tile_desc& t, const WinDev& W, int64_t* nb, int64_t* ncoef) {
  int64_t b = 0, c = 0;
  for (int lv = 0; lv <= t.levels; ++lv) {
    const int level = lv == 0 ? 0 : t.levels + 1 - lv;
    if (level != 0 && level <= W.z) continue;
    const int gw = level_dim(t.width, level == 0 ? t.levels : level), gh = level_dim(t.height, level == 0 ? t.levels : level);
    const int p = level == 0 ? 1 : 3;
    for (int by = 0; by < ceil_div(gh, kCell); ++by)
      for (int bx = 0; bx < ceil_div(gw, kCell); ++bx)
        if (block_in_window(W, level, by, bx)) {
          ++b;
          c += (int64_t)p * pad4(std::min(kCell, gw - kCell * bx)) * pad4(std::min(kCell, gh - kCell * by));
        }
  }
  *nb = b * t.channels;
  *ncoef = c * t.channels;
}

}  // namespace isx
