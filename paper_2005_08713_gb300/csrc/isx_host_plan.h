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
  for (int k = 0; k < 16; ++k) d.q[k] = k <= t.levels ? t.qstep_log2[k] : 0;
}

}  // namespace isx
