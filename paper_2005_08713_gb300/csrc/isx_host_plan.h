// isx_host_plan.h — host-side descriptor checks and per-tile counts shared
// by the context entry points (isx_api.cu) and the no-allocation encoder
// (isx_static.cu), so that both accept the same descriptors and size the
// same blocks.
#pragma once
#include <algorithm>
#include <cstring>
#include <string>

#include "isx.h"
#include "isx_internal.cuh"

namespace isx {

inline bool tile_ok(const isx_tile_desc& t, std::string* why) {
  if (t.width < 1 || t.width > 65535 || t.height < 1 || t.height > 65535) { *why = "width/height out of 1..65535"; return false; }
  if (t.channels != 1 && t.channels != 3) { *why = "channels must be 1 or 3"; return false; }
  if (t.bits < 1 || t.bits > 16) { *why = "bits out of 1..16"; return false; }
  if (t.channels == 3 && t.bits > 8) { *why = "3-channel tiles take bits 1..8"; return false; }
  if (t.levels < 0 || t.levels > kMaxLevels) { *why = "levels out of 0..15"; return false; }
  if (t.x0 < 0 || t.y0 < 0) { *why = "negative tile origin"; return false; }
  for (int l = 0; l <= t.levels; ++l)
    if (t.qstep_log2[l] > 15) { *why = "qstep_log2 out of 0..15"; return false; }
  return true;
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
  for (int k = 0; k < 16; ++k) d.q[k] = k <= t.levels ? t.qstep_log2[k] : 0;
}

}  // namespace isx
