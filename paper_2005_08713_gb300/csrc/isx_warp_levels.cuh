// isx_warp_levels.cuh — the coarse levels of the fused forward 5/3
// transform on one warp, in registers.
//
// Once a level's grid is at most 32 x 32 samples (levels 3 .. L-1 of a
// 256 x 256 tile) the CTA has too few lines to share out, so the first warp
// finishes the transform alone while the other warps pack the blocks.
// Lifting those levels in place in the shared-memory plane costs a
// shared-memory round trip per sample and pass, at strides of 8 .. 128
// samples (4- to 16-way bank conflicts), queued behind the other warps'
// traffic.  Here the warp gathers the grid once into registers (lane j holds
// column j: v[i] = sample (i, j)), lifts the lines of one direction in
// registers, turns the grid through a 32 x 33-word scratch (conflict-free)
// for the other direction, and writes each level's detail samples (the ones
// with an odd row or column index, Sec. 3's subbands) to the plane once.
//
// A level (the 5/3 lifting: predict, then update, with the same
// whole-sample symmetric extension as the line sweeps): columns, then rows;
// the low band (even row and column) is compacted into the next level's
// columns through the scratch.  (The inverse was built the same way and
// measured slower inside the decode kernel, whose coarse levels stay
// in-place line sweeps.)
//
// The functions are written for one full warp (all 32 lanes call them);
// ISX_WL_FN, ISX_WL_SYNC and ISX_WL_MIN let the same source run lane by lane
// on the host.
#pragma once

#ifndef ISX_WL_FN
#define ISX_WL_FN __device__ __forceinline__
#define ISX_WL_SYNC() __syncwarp()
#define ISX_WL_MIN(a, b) min(a, b)
#endif

namespace isx {

constexpr int kWarpGrid = 32;   // grids up to 32 x 32 samples take the one-warp path
constexpr int kWlPitch = 33;    // scratch row pitch in words (32 x 33 int32)

// In-register forward lifting of v[0 .. n), 2 <= n <= N: predict the odd
// samples, then update the even ones (x[n] mirrors to x[n-2], d[-1] to d[0],
// d[nh] to d[nh-1] for odd n).  Indices are static; n only selects.
template <int N>
ISX_WL_FN void reg_lift_fwd(int32_t (&v)[32], int n) {
#pragma unroll
  for (int k = 0; 2 * k + 1 < N; ++k) {
    const int32_t right = (2 * k + 2 < n) ? v[ISX_WL_MIN(2 * k + 2, N - 1)] : v[2 * k];
    const int32_t d = v[2 * k + 1] - ((v[2 * k] + right) >> 1);
    v[2 * k + 1] = (2 * k + 1 < n) ? d : v[2 * k + 1];
  }
#pragma unroll
  for (int k = 0; 2 * k < N; ++k) {
    const int32_t dl = k > 0 ? v[2 * k - 1] : v[1];
    const int32_t dr = (2 * k + 1 < n) ? v[ISX_WL_MIN(2 * k + 1, N - 1)] : dl;
    const int32_t s = v[2 * k] + ((dl + dr + 2) >> 2);
    v[2 * k] = (2 * k < n) ? s : v[2 * k];
  }
}

// Lane l holds v[i] = M[i][l] (i, l < N); afterwards v[i] = M[l][i].
template <int N>
ISX_WL_FN void reg_transpose(int32_t (&v)[32], int32_t* T, int lane) {
  if (lane < N) {
#pragma unroll
    for (int i = 0; i < N; ++i) T[i * kWlPitch + lane] = v[i];
  }
  ISX_WL_SYNC();
  if (lane < N) {
#pragma unroll
    for (int i = 0; i < N; ++i) v[i] = T[lane * kWlPitch + i];
  }
  ISX_WL_SYNC();
}

// Forward level m = l0 + R of a grid of at most N = 32 >> R samples a side
// (cw x ch, `s` = 2^m elements apart in the plane); v holds the columns on
// entry and the next level's columns (its low band, compacted) on return.
template <int R>
ISX_WL_FN void wl_fwd_level(int32_t (&v)[32], int16_t* P, int pitch, int32_t* T, int lane, int s, int cw, int ch) {
  constexpr int N = 32 >> R;
  if (ch >= 2) reg_lift_fwd<N>(v, ch);   // columns (lane j: column j)
  reg_transpose<N>(v, T, lane);
  if (cw >= 2) reg_lift_fwd<N>(v, cw);   // rows (lane r: row r)
  // the samples with an odd row or column index are final: store them
  if (lane < ch) {
    int16_t* row = P + (lane * s) * pitch;
#pragma unroll
    for (int c = 0; c < N; ++c)
      if (c < cw && ((lane | c) & 1)) row[c * s] = (int16_t)v[c];
  }
  // low band (2r', 2c') -> lane c', v[r']
  constexpr int H = N / 2;
  if (lane < N && !(lane & 1)) {
#pragma unroll
    for (int c = 0; c < H; ++c) T[c * kWlPitch + (lane >> 1)] = v[2 * c];
  }
  ISX_WL_SYNC();
  if (lane < H) {
#pragma unroll
    for (int r = 0; r < H; ++r) v[r] = T[lane * kWlPitch + r];
  }
  ISX_WL_SYNC();
}

// Levels l0 .. L-1 of the forward transform, the level-l0 grid (of a w x h
// plane, samples 2^l0 apart) being at most 32 x 32.  After five levels the
// grid is one sample and further levels change nothing.
ISX_WL_FN void warp_levels_fwd(int16_t* P, int pitch, int w, int h, int l0, int L, int32_t* T, int lane) {
  int32_t v[32];
  int cw = level_dim(w, l0), ch = level_dim(h, l0);
  {
    const int s = 1 << l0;
    const int jc = ISX_WL_MIN(lane, cw - 1);   // lanes past the grid read a valid sample and never store it
#pragma unroll
    for (int i = 0; i < 32; ++i) v[i] = P[(ISX_WL_MIN(i, ch - 1) * s) * pitch + jc * s];
  }
  int m = l0;
#define ISX_WL_FWD_STEP(R)                                           \
  if (m < L) {                                                       \
    wl_fwd_level<R>(v, P, pitch, T, lane, 1 << m, cw, ch);           \
    cw = (cw + 1) >> 1;                                              \
    ch = (ch + 1) >> 1;                                              \
    ++m;                                                             \
  }
  ISX_WL_FWD_STEP(0)
  ISX_WL_FWD_STEP(1)
  ISX_WL_FWD_STEP(2)
  ISX_WL_FWD_STEP(3)
  ISX_WL_FWD_STEP(4)
#undef ISX_WL_FWD_STEP
  // the low band left (cw x ch, samples 2^m apart; one sample once five levels ran)
  if (m > l0 && lane < cw) {
    const int s = 1 << m;
#pragma unroll
    for (int r = 0; r < 16; ++r)
      if (r < ch) P[(r * s) * pitch + lane * s] = (int16_t)v[r];
  }
}

}  // namespace isx
