// isx_fused.cuh — the fused shared-memory transforms (Sec. 3: colour
// transform and 5/3 lifting; Sec. 4: quantisation and the area order of the
// coefficient blocks), as device functions over one (tile, channel) run by a
// whole CTA.  Used by the per-stage kernels (isx_transform.cu) and by the
// persistent per-tile kernels (isx_persist.cu).
#pragma once
#include <cstdint>

#include "isx_internal.cuh"
#include "isx_warp_levels.cuh"

namespace isx {

// --------------------------------------------------- colour transform
// Colour transforms of channels 0..2 (Fig. 1, "optional colorspace
// transformation"), component c of (R, G, B):
//  ct 1, the RCT of JPEG 2000: Y = floor((R+2G+B)/4), Cb = B-G, Cr = R-G;
//  ct 2, YCoCg-R: Co = R-B, t = B + floor(Co/2), Cg = G-t, Y = t + floor(Cg/2).
__device__ __forceinline__ int32_t ct_forward(int ct, int c, int32_t R, int32_t G, int32_t B) {
  if (ct == 1) return c == 0 ? (R + 2 * G + B) >> 2 : c == 1 ? B - G : R - G;
  const int32_t Co = R - B, t = B + (Co >> 1), Cg = G - t;
  return c == 0 ? t + (Cg >> 1) : c == 1 ? Co : Cg;
}
// Inverse of ct_forward: (Y, Cb, Cr) or (Y, Co, Cg) -> (R, G, B).
__device__ __forceinline__ void ct_inverse(int ct, int32_t a, int32_t b, int32_t c, int32_t* R, int32_t* G, int32_t* B) {
  if (ct == 1) {
    *G = a - ((b + c) >> 2);
    *R = c + *G;
    *B = b + *G;
  } else {
    const int32_t t = a - (c >> 1);
    *G = c + t;
    *B = t - (b >> 1);
    *R = *B + b;
  }
}
// Sample x of channel c of an interleaved row (uint8 when bits <= 8, else uint16).
__device__ __forceinline__ int32_t sample_at(const uint8_t* row, int x, int C, int c, int bits) {
  return bits <= 8 ? (int32_t)row[x * C + c] : (int32_t)reinterpret_cast<const uint16_t*>(row)[x * C + c];
}

// The coefficient blocks of tile ti (one thread), in stream order from
// t.block_base: per channel the LL, then levels L .. 1 (levels 1 ..
// min_level left out), each level's 128 x 128 cells row by row, with the
// byte offsets of their coefficients and symbol regions.
__device__ inline void plan_tile_blocks(int ti, const TileDev& t, int min_level, BlockDev* __restrict__ out) {
  int64_t idx = t.block_base;
  int64_t coef = t.coef_base;
  int64_t sym = t.sym_base;
  int64_t pst = t.pst_base;
  const int dmax = dmax_of_bits(t.bits);
  for (int c = 0; c < t.C; ++c) {
    for (int lv = 0; lv <= t.L; ++lv) {
      int level = lv == 0 ? 0 : t.L + 1 - lv;   // 0 (LL), then L, L-1, ..., 1
      if (level != 0 && level <= min_level) continue;
      int gw = level_dim(t.w, level == 0 ? t.L : level), gh = level_dim(t.h, level == 0 ? t.L : level);
      int p = level == 0 ? 1 : 3;
      for (int by = 0; by < ceil_div(gh, kCell); ++by)
        for (int bx = 0; bx < ceil_div(gw, kCell); ++bx) {
          BlockDev b;
          b.tile = ti; b.c = c; b.level = level; b.by = by; b.bx = bx; b.p = p;
          b.w = pad4(min(kCell, gw - kCell * bx));
          b.h = pad4(min(kCell, gh - kCell * by));
          b.coef = coef;
          b.coef16 = t.coef16;
          b.dmax = dmax;
          b.sym = sym;
          b.pst = pst;
          pst += dmax;
          coef += (int64_t)p * b.w * b.h * (b.coef16 ? 2 : 4);
          sym += (int64_t)dmax * (((int64_t)p * b.w * b.h / 8 + 15) & ~15LL);
          out[idx++] = b;
        }
    }
  }
}

// ------------------------------------------------- fused shared-memory path
// Tiles whose channel plane fits in shared memory as int16 (the host checks
// that the worst-case gain of the iterated 5/3 filters keeps every state of
// the tile's transform below 2^15: TileDev::coef16 for the forward, the
// deviation bound of the decode for the inverse) are transformed by one CTA
// per (tile, channel), in place on the
// interleaved layout: after level l the LL samples sit at multiples of 2^l,
// and the high-pass samples of level l at odd multiples of 2^(l-1).
constexpr int kFusedThreads = 1024;   // most threads of a fused CTA (launches use 256, 512 or 1024)

__host__ __device__ inline int smem_pitch(int w);
__host__ __device__ inline bool tile_uses_smem(int w, int h) {
  // up to 1024 x 1024 a channel has at most 20 coefficient blocks (LL and
  // every level) within this plane budget: the block table below holds 32
  return w <= 1024 && h <= 1024 && (int64_t)smem_pitch(w) * h * 2 <= kSmemPlaneBytes;
}

// Interleaved position of subband sample (y, x) of `type` at `level`
// (level 0 = LL_L) relative to a grid whose LL is level `z`.
__device__ inline void ilv_pos(int L, int level, int type, int y, int x, int z, int* py, int* px) {
  if (level == 0) {
    *py = y << (L - z);
    *px = x << (L - z);
    return;
  }
  const int s = 1 << (level - 1 - z), s2 = s << 1;
  *py = y * s2 + (type >= 1 ? s : 0);
  *px = x * s2 + (type != 1 ? s : 0);
}

// Shared-memory row pitch (int16 elements): an odd number of 32-bit words,
// so that threads sweeping different rows hit different banks.
__host__ __device__ inline int smem_pitch(int w) { return ((w + 1) & ~1) | 2; }

// In-place forward 5/3 lifting of the sample pairs k0 .. k1-1 of a line of
// n samples `st` elements apart (pair k: x[2k], x[2k+1]; the last pair of an
// odd line has only its even sample): afterwards the low-pass samples sit at
// even and the high-pass samples at odd positions.  Predict and update run
// in one sweep with a small register window (x[2k+2] is read before
// position 2k+2 is overwritten).  The body runs in chunks of kSweepChunk
// pairs whose reads all lie inside the run: the chunk's loads are issued
// together, the lifting runs in registers, then the chunk is stored (a chunk
// reads x[2k+1 .. 2k+2K] and writes x[2k .. 2k+2K-1]).  The run's last
// pairs (at most kSweepChunk) take the same straight-line code in chunks of
// kTailChunk pairs: loads past the run are clamped to the run's last sample
// and the stores past it are predicated off, so no load waits behind a
// branch (a scalar tail loop cost a shared-memory round trip per pair, which
// dominated the short lines of the coarse levels).
// A run that does not start the line takes the two samples before it
// (pe = x[2k0-2], pd = x[2k0-1]) and one that does not end it the sample
// after it (ne = x[2k1]), all as they were before the sweep: the caller
// reads them before any thread of the line writes.
constexpr int kSweepChunk = 8, kTailChunk = 2;

template <typename T>
__device__ inline void sweep_fwd_range(T* x, int n, int st, int k0, int k1, int32_t pe, int32_t pd, int32_t ne) {
  constexpr int K = kSweepChunk;
  int32_t xe = x[(2 * k0) * st], dprev = 0;
  if (k0 > 0) dprev = pd - ((pe + xe) >> 1);   // d[k0-1], from the samples before the run
  int k = k0;
  for (; k + K < k1; k += K) {
    int32_t v[2 * K], o[2 * K];
#pragma unroll
    for (int i = 0; i < 2 * K; ++i) v[i] = x[(2 * k + 1 + i) * st];
#pragma unroll
    for (int i = 0; i < K; ++i) {
      const int32_t xe2 = v[2 * i + 1];
      const int32_t d = v[2 * i] - ((xe + xe2) >> 1);
      const int32_t dm1 = (k + i == 0) ? d : dprev;   // d[-1] mirrors to d[0]
      o[2 * i] = xe + ((dm1 + d + 2) >> 2);
      o[2 * i + 1] = d;
      dprev = d;
      xe = xe2;
    }
#pragma unroll
    for (int i = 0; i < 2 * K; ++i) x[(2 * k + i) * st] = (T)o[i];
  }
  // last pairs k .. k1-1 (at most K), in predicated chunks of kTailChunk
  // pairs; the sample after the run is ne, or x[n-2] at the end of an even
  // line (mirror)
  const int lim = min(2 * k1, n);   // samples of the run: x[2k .. lim-1]
  for (; k < k1; k += kTailChunk) {
    constexpr int J = kTailChunk;
    int32_t v[2 * J], o[2 * J];
#pragma unroll
    for (int i = 0; i < 2 * J; ++i) v[i] = x[min(2 * k + 1 + i, lim - 1) * st];
#pragma unroll
    for (int i = 0; i < J; ++i) {
      // even sample after pair k+i: own, the next run's, or x[n-2] (mirror) at the end of an even line
      const int32_t xe2 = (2 * (k + i) + 2 < lim) ? v[2 * i + 1] : (2 * k1 < n ? ne : xe);
      const int32_t d = (2 * (k + i) + 1 < n) ? v[2 * i] - ((xe + xe2) >> 1) : dprev;   // odd n: d[nh] mirrors to d[nh-1]
      const int32_t dm1 = (k + i == 0) ? d : dprev;
      o[2 * i] = xe + ((dm1 + d + 2) >> 2);
      o[2 * i + 1] = d;
      dprev = d;
      xe = xe2;
    }
#pragma unroll
    for (int i = 0; i < 2 * J; ++i) {
      if (2 * k + i < lim) x[(2 * k + i) * st] = (T)o[i];
    }
  }
}

template <typename T>
__device__ inline void sweep_fwd(T* x, int n, int st) {
  if (n >= 2) sweep_fwd_range(x, n, st, 0, (n + 1) >> 1, 0, 0, 0);
}

// In-place inverse of sweep_fwd_range over pairs k0 .. k1-1, chunked the same
// way (a chunk reads x[2k+2 .. 2k+2K+1] and writes x[2k .. 2k+2K-1]).  A run
// that does not start the line takes pd = x[2k0-1], one that does not end it
// ns = x[2k1] and nd = x[2k1+1], all as they were before the sweep.
template <typename T>
__device__ inline void sweep_inv_range(T* x, int n, int st, int k0, int k1, int32_t pd, int32_t ns, int32_t nd) {
  constexpr int K = kSweepChunk;
  const int nl = (n + 1) >> 1, nh = n >> 1;
  int32_t dk = k0 < nh ? (int32_t)x[(2 * k0 + 1) * st] : pd;   // d[nh] mirrors to d[nh-1]
  int32_t e = x[(2 * k0) * st] - (((k0 > 0 ? pd : dk) + dk + 2) >> 2);   // d[-1] mirrors to d[0]
  int k = k0;
  for (; k + K < k1 && k + K < nh; k += K) {
    int32_t v[2 * K], o[2 * K];
#pragma unroll
    for (int i = 0; i < 2 * K; ++i) v[i] = x[(2 * k + 2 + i) * st];
#pragma unroll
    for (int i = 0; i < K; ++i) {
      const int32_t dk1 = v[2 * i + 1];
      const int32_t en = v[2 * i] - ((dk + dk1 + 2) >> 2);
      o[2 * i] = e;
      o[2 * i + 1] = dk + ((e + en) >> 1);
      e = en;
      dk = dk1;
    }
#pragma unroll
    for (int i = 0; i < 2 * K; ++i) x[(2 * k + i) * st] = (T)o[i];
  }
  // last pairs k .. k1-1, in predicated chunks of kTailChunk pairs; v holds
  // s[k+1..], d[k+1..] of the run, then the next run's ns, nd
  const int lim = min(2 * k1, n);
  for (; k < k1; k += kTailChunk) {
    constexpr int J = kTailChunk;
    int32_t v[2 * J], o[2 * J];
#pragma unroll
    for (int i = 0; i < 2 * J; ++i) {
      const int idx = 2 * k + 2 + i;
      const int32_t xv = x[min(idx, lim - 1) * st];
      v[i] = idx < lim ? xv : (idx == 2 * k1 ? ns : nd);
    }
#pragma unroll
    for (int i = 0; i < J; ++i) {
      const int kk = k + i;
      const int32_t dk1 = (kk + 1 < nh) ? v[2 * i + 1] : dk;   // d[nh] mirrors to d[nh-1]
      const int32_t en = (kk + 1 < nl) ? v[2 * i] - ((dk + dk1 + 2) >> 2) : e;   // x[n] mirrors to x[n-2]
      o[2 * i] = e;
      o[2 * i + 1] = dk + ((e + en) >> 1);
      // pairs past the line's last odd sample leave e (the last even sample of an odd line) alone
      const bool live = kk < nh;
      e = live ? en : e;
      dk = live ? dk1 : dk;
    }
#pragma unroll
    for (int i = 0; i < 2 * J; ++i) {
      if (2 * k + i < lim && k + i / 2 < nh) x[(2 * k + i) * st] = (T)o[i];
    }
  }
  if (k1 == nl && (n & 1)) x[(n - 1) * st] = (T)e;
}

template <typename T>
__device__ inline void sweep_inv(T* x, int n, int st) {
  if (n >= 2) sweep_inv_range(x, n, st, 0, (n + 1) >> 1, 0, 0, 0);
}

// Named barrier over the first n threads of the CTA (warps 0 .. n/32-1),
// id 1 or 2 (0 is __syncthreads).
__device__ __forceinline__ void group_sync(int id, int n) { asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(n) : "memory"); }

struct CtaSync {
  __device__ void operator()() const { __syncthreads(); }
};
struct GroupSync {   // the first n threads, barrier 1
  int n;
  __device__ void operator()() const { group_sync(1, n); }
};

// One lifting pass over `nlines` lines of `len` samples (line i starts at
// P + i * lstep, its samples `st` elements apart) by threads tid < n, ending
// with sync().  When there are at least twice as many threads as lines
// (rounded up to whole warps) and the lines are long, each line may be cut
// into S <= smax runs of pairs, run j lifted by the threads of warp group j
// (so the warps keep the one-line-per-lane access pattern): every thread
// first reads the samples next to its run that a neighbouring run
// overwrites, the group synchronises, then the runs are lifted.  Splitting
// pays only where a few warps lift while the rest of the CTA does other
// work: with the whole CTA lifting, shared-memory bandwidth bounds the pass
// and the extra barrier costs more than the shorter runs save.
template <bool kFwd, class Sync>
__device__ inline void lift_pass(int16_t* P, int nlines, int len, int lstep, int st, int tid, int n, int smax, Sync sync) {
  const int G = (nlines + 31) & ~31;
  const int npairs = (len + 1) >> 1;
  const int S = min(min(n / G, smax), npairs >> 4);
  if (S <= 1) {
    for (int i = tid; i < nlines; i += n) {
      if (kFwd) sweep_fwd(P + i * lstep, len, st);
      else sweep_inv(P + i * lstep, len, st);
    }
    sync();
    return;
  }
  const int line = tid % G, run = tid / G;
  const bool act = run < S && line < nlines;
  int16_t* x = P + line * lstep;
  const int k0 = run * npairs / S, k1 = (run + 1) * npairs / S;
  int32_t h0 = 0, h1 = 0, h2 = 0;
  if (act) {
    if (kFwd) {
      if (k0 > 0) { h0 = x[(2 * k0 - 2) * st]; h1 = x[(2 * k0 - 1) * st]; }
      if (2 * k1 < len) h2 = x[(2 * k1) * st];
    } else {
      if (k0 > 0) h0 = x[(2 * k0 - 1) * st];
      if (2 * k1 < len) h1 = x[(2 * k1) * st];
      if (2 * k1 + 1 < len) h2 = x[(2 * k1 + 1) * st];
    }
  }
  sync();
  if (act) {
    if (kFwd) sweep_fwd_range(x, len, st, k0, k1, h0, h1, h2);
    else sweep_inv_range(x, len, st, k0, k1, h0, h1, h2);
  }
  sync();
}

// One level of the in-place 2-D transform on the grid at stride s
// (cw x ch samples): columns then rows (forward), rows then columns (inverse);
// one thread sweeps one line.
__device__ inline void level_fwd(int16_t* P, int pitch, int cw, int ch, int s) {
  lift_pass<true>(P, cw, ch, s, s * pitch, threadIdx.x, blockDim.x, 1, CtaSync());
  lift_pass<true>(P, ch, cw, s * pitch, s, threadIdx.x, blockDim.x, 1, CtaSync());
}

__device__ inline void level_inv(int16_t* P, int pitch, int cw, int ch, int s) {
  lift_pass<false>(P, ch, cw, s * pitch, s, threadIdx.x, blockDim.x, 1, CtaSync());
  lift_pass<false>(P, cw, ch, s, s * pitch, threadIdx.x, blockDim.x, 1, CtaSync());
}

// The decode's one-warp coarse levels (grids of at most 32 x 32 samples):
// in-place line sweeps, one lane per line.  The register version
// (isx_warp_levels.cuh) measured slower here: beside the block rebuild's
// conflicted shared-memory stores, its transposes and plane reads wait
// longer in the shared-memory queue than these sweeps.
__device__ inline void level_inv_warp(int16_t* P, int pitch, int cw, int ch, int s) {
  const int lane = threadIdx.x & 31;
  if (cw >= 2)
    for (int r = lane; r < ch; r += 32) sweep_inv(P + (r * s) * pitch, cw, s);
  __syncwarp();
  if (ch >= 2)
    for (int c = lane; c < cw; c += 32) sweep_inv(P + c * s, ch, s * pitch);
  __syncwarp();
}

// Scratch of the encode's one-warp coarse levels (isx_warp_levels.cuh): 32 x 33 words.
static __shared__ int32_t s_wl_scratch[32 * kWlPitch];

// Warps that lift the levels coarser than the finest while the rest of the
// CTA packs (encode) or rebuilds (decode) the finest level's blocks: the
// lines of the level (cw x ch grid) rounded up to whole warps, times up to
// `split` runs per line, leaving at least half of the warps to the blocks
// (0: no overlap).  Measured per phase: two runs per line shorten the
// encode's lifting; the decode's lifting is fastest on one run per line.
constexpr int kOverlapSplitFwd = 2, kOverlapSplitInv = 1;
// Warps that pack (encode) or rebuild (decode) the finest level's blocks
// meanwhile, at most: the lifting warps are the critical path, and every
// further block warp takes issue slots and shared-memory bandwidth from
// them.  The block warps are taken among those that share no warp scheduler
// with warp 0 (warp w issues on scheduler w % 4), which lifts the coarse
// levels alone.
constexpr int kOverlapBlockWarpsFwd = 8, kOverlapBlockWarpsInv = 12;

// Rank of warp w among the block warps (w >= W, w % 4 != 0), or -1.
__device__ inline int block_warp_rank(int w, int W) {
  if (w < W || (w & 3) == 0) return -1;
  return (w - W) - (((w - 1) >> 2) - ((W - 1) >> 2));
}
// Block warps available in a CTA of nwarps warps after W lifting warps (W >= 1).
__device__ inline int block_warps(int nwarps, int W, int cap) {
  return min(cap, (nwarps - W) - (((nwarps - 1) >> 2) - ((W - 1) >> 2)));
}
__device__ inline int overlap_warps(int cw, int ch, int nwarps, int split) {
  const int base = (max(cw, ch) + 31) >> 5;
  int sp = split;
  while (sp > 1 && 2 * base * sp > nwarps) --sp;
  const int W = base * sp;
  return W < nwarps ? W : 0;
}

// Levels 0 .. L-1 of the forward transform of a w x h plane.
__device__ inline void transform_fwd_levels(int16_t* P, int pitch, int w, int h, int L) {
  int l = 0;
  for (; l < L; ++l) {
    const int cw = level_dim(w, l), ch = level_dim(h, l);
    if (cw <= kWarpGrid && ch <= kWarpGrid) break;
    level_fwd(P, pitch, cw, ch, 1 << l);
  }
  if (l < L) {
    if (threadIdx.x < 32) warp_levels_fwd(P, pitch, w, h, l, L, s_wl_scratch, threadIdx.x);
    __syncthreads();
  }
}

// Inverse levels L-1 .. z, the plane's LL being level z.
__device__ inline void transform_inv_levels(int16_t* P, int pitch, int w, int h, int L, int z) {
  int l = L - 1;
  if (l >= z && level_dim(w, l) <= kWarpGrid && level_dim(h, l) <= kWarpGrid) {
    while (l >= z && level_dim(w, l) <= kWarpGrid && level_dim(h, l) <= kWarpGrid) --l;
    if (threadIdx.x < 32)
      for (int m = L - 1; m > l; --m) level_inv_warp(P, pitch, level_dim(w, m), level_dim(h, m), 1 << (m - z));
    __syncthreads();
  }
  for (; l >= z; --l) level_inv(P, pitch, level_dim(w, l), level_dim(h, l), 1 << (l - z));
}

// Forward levels lmin .. L-1 done by the first n threads only (barrier 1):
// after level 0 at most half the lines remain, and the rest of the CTA can
// pack the finished level-1 blocks meanwhile.
__device__ inline void transform_fwd_levels_group(int16_t* P, int pitch, int w, int h, int lmin, int L, int n) {
  int l = lmin;
  for (; l < L; ++l) {
    const int cw = level_dim(w, l), ch = level_dim(h, l), s = 1 << l;
    if (cw <= kWarpGrid && ch <= kWarpGrid) break;
    lift_pass<true>(P, cw, ch, s, s * pitch, threadIdx.x, n, 4, GroupSync{n});
    lift_pass<true>(P, ch, cw, s * pitch, s, threadIdx.x, n, 4, GroupSync{n});
  }
  if (l < L) {
    if (threadIdx.x < 32) warp_levels_fwd(P, pitch, w, h, l, L, s_wl_scratch, threadIdx.x);
    group_sync(1, n);
  }
}

// Inverse levels L-1 .. lmin (the plane's LL being level z) by the first n threads (barrier 1).
__device__ inline void transform_inv_levels_group(int16_t* P, int pitch, int w, int h, int L, int lmin, int z, int n) {
  int l = L - 1;
  if (l >= lmin && level_dim(w, l) <= kWarpGrid && level_dim(h, l) <= kWarpGrid) {
    while (l >= lmin && level_dim(w, l) <= kWarpGrid && level_dim(h, l) <= kWarpGrid) --l;
    if (threadIdx.x < 32)
      for (int m = L - 1; m > l; --m) level_inv_warp(P, pitch, level_dim(w, m), level_dim(h, m), 1 << (m - z));
    group_sync(1, n);
  }
  for (; l >= lmin; --l) {
    const int cw = level_dim(w, l), ch = level_dim(h, l), s = 1 << (l - z);
    lift_pass<false>(P, ch, cw, s * pitch, s, threadIdx.x, n, 4, GroupSync{n});
    lift_pass<false>(P, cw, ch, s, s * pitch, threadIdx.x, n, 4, GroupSync{n});
  }
}

// The coefficient blocks of the CTA's tile channel, as its single area loop
// sees them: area index g of the channel lies in the first block whose
// `end` exceeds it.
constexpr int kMaxFusedBlocks = 32;
constexpr int kMaxFusedPlanes = 20;   // planes of a fused block: at most 12 + 6

struct FusedBlock {
  int32_t end;                 // inclusive prefix sum of the blocks' loop units (areas, or area quads)
  int32_t n, w, nlog, wlog;    // AreaMap of the block
  int32_t q, step;             // quantiser step (log2); distance of neighbouring subband samples
  int32_t d, keep;             // decode: bit depth and planes kept
  int32_t quad;                // the loop's units are 4 consecutive areas of a type (n % 4 == 0)
  int32_t level;               // 0 = LL
  int64_t base;                // byte offset of its coefficients (encode) or symbols (decode)
  int4 geo[3];                 // per type: valid width, valid height, interleaved row and column of sample (0, 0)
};

// One warp fills fb[0 .. nbc) from blocks[b0 ..] for a plane whose LL is
// level z0 (lane i: block i); decode passes its DecInfo (else nullptr) and
// gets the symbol offset of every kept (plane, type) in po (a warp scan over
// the planes per block).  Blocks a decode could not read (p = 0 or d = 0;
// status already set) get no units.  The caller synchronises the CTA
// before use.
__device__ inline void fused_block_table(const TileDev& t, const BlockDev* __restrict__ blocks, const DecInfo* __restrict__ info,
                                         const int64_t* __restrict__ sym_off, int64_t b0, int nbc, int z0, FusedBlock* fb,
                                         int32_t (*po)[kMaxFusedPlanes][3]) {
  const int lane = threadIdx.x & 31;
  FusedBlock f;
  f.quad = 0;
  f.keep = 0;
  f.n = 0;
  int na = 0;
  uint32_t rem[3] = {~0u, ~0u, ~0u};   // decode: removed planes per type
  int p_types = 0;
  if (lane < nbc) {
    const BlockDev b = blocks[b0 + lane];
    f.n = b.w * b.h / 8;
    f.w = b.w;
    f.nlog = (f.n & (f.n - 1)) == 0 ? 31 - __clz(f.n) : -1;
    f.wlog = (f.w & (f.w - 1)) == 0 ? 31 - __clz(f.w) : -1;
    f.q = qlog2_of(t, b.level);
    f.step = b.level == 0 ? 1 << (t.L - z0) : 2 << (b.level - 1 - z0);
    f.d = f.keep = 0;
    f.quad = 0;
    f.level = b.level;
    f.base = b.coef;
    for (int ty = 0; ty < 3; ++ty) {
      int sx, sy, sw, sh, py, px;
      subband_rect(t.w, t.h, t.L, b.level, ty < b.p ? ty : 0, &sx, &sy, &sw, &sh);
      ilv_pos(t.L, b.level, ty < b.p ? ty : 0, kCell * b.by, kCell * b.bx, z0, &py, &px);
      f.geo[ty] = make_int4(min(sw - kCell * b.bx, b.w), min(sh - kCell * b.by, b.h), py, px);
    }
    na = b.p * f.n;
    f.quad = (f.n & 3) == 0;   // encode and decode loop over quads of areas where the block allows
    if (info) {
      const DecInfo di = info[b0 + lane];
      f.d = di.d;
      f.keep = min(di.keep, kMaxFusedPlanes);
      f.base = sym_off[b0 + lane];
      if (b.p == 0 || di.d == 0) na = 0;
      rem[0] = di.removed[0]; rem[1] = di.removed[1]; rem[2] = di.removed[2];
      p_types = b.p;
    }
  }
  if (f.quad) na >>= 2;
  int incl = na;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int y = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += y;
  }
  f.end = incl;
  if (lane < nbc) fb[lane] = f;
  if (!info) return;
  // Symbol offsets of each (plane, type) from the block's first symbol: the
  // kept types of a plane are stored back to back, planes 16-byte aligned.
  // Per block, lane pl sizes plane pl and a warp scan places the planes.
  for (int blk = 0; blk < nbc; ++blk) {
    const int keep = __shfl_sync(0xffffffffu, f.keep, blk), n = __shfl_sync(0xffffffffu, f.n, blk);
    const int pt = __shfl_sync(0xffffffffu, p_types, blk);
    uint32_t r[3];
#pragma unroll
    for (int ty = 0; ty < 3; ++ty) r[ty] = __shfl_sync(0xffffffffu, rem[ty], blk);
    const int pl = lane;
    uint32_t km = 0;
#pragma unroll
    for (int ty = 0; ty < 3; ++ty)
      if (ty < pt && !((r[ty] >> pl) & 1u)) km |= 1u << ty;
    const int bytes = pl < keep ? ((__popc(km) * n + 15) & ~15) : 0;
    int end = bytes;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, end, o);
      if (lane >= o) end += y;
    }
    if (pl < keep) {
      int32_t o = end - bytes;
#pragma unroll
      for (int ty = 0; ty < 3; ++ty) {
        const bool kept = (km >> ty) & 1u;
        po[blk][pl][ty] = kept ? o : -1;
        if (kept) o += n;
      }
    }
  }
}

// Rotates eight int16 held in pairs (w[k] = slots 2k, 2k+1) so that slot t
// takes slot (t + rot) & 7.
__device__ __forceinline__ void rotate8x16(const uint32_t (&w)[4], int rot, uint32_t (&o)[4]) {
  const int qw = rot >> 1, sh = (rot & 1) << 4;
  uint32_t y[4];
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const uint32_t t0 = (qw & 1) ? w[(k + 1) & 3] : w[k];
    const uint32_t t2 = (qw & 1) ? w[(k + 3) & 3] : w[(k + 2) & 3];
    y[k] = (qw & 2) ? t2 : t0;   // y[k] = w[(k + qw) & 3]
  }
#pragma unroll
  for (int k = 0; k < 4; ++k) o[k] = __funnelshift_r(y[k], y[(k + 1) & 3], sh);
}

__device__ __forceinline__ uint32_t quantise16(int32_t c, int q) {
  int32_t m = (c < 0 ? -c : c) >> q;
  return (uint32_t)(uint16_t)(c < 0 ? -m : m);
}

// Quantise + pack of 4 consecutive areas a0 .. a0+3 of one type (the quad
// of the decode's rebuild_quad): with a block width of 8 or more they tile
// a 4 x 8 region, read row by row in lane-rotated column order (lane l reads
// column (t + rho) & 7 in read t, rho = (l >> 2) & 7: neighbouring lanes'
// regions start 8 columns apart, so unrotated reads hit four banks).
__device__ inline void pack_quad(const FusedBlock& f, const AreaMap& am, int a0, const int16_t* P, int pitch,
                                 uint8_t* __restrict__ coef) {
  int type, k0;
  am.split(a0, &type, &k0);
  const int4 gm = f.geo[type];
  const int step = f.step, q = f.q;
  uint32_t R[4][4];   // region row r, columns 2k, 2k+1
  int i0, j0;
  am.ij(k0, &i0, &j0);
  if (am.wlog >= 3 && i0 + 3 < gm.y && j0 + 7 < gm.x) {
    const int rho = (threadIdx.x >> 2) & 7;
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      const int16_t* row = P + (gm.z + (i0 + r) * step) * pitch + gm.w + j0 * step;
      uint32_t O[4] = {0u, 0u, 0u, 0u};
#pragma unroll
      for (int t = 0; t < 8; ++t) O[t >> 1] |= quantise16(row[((t + rho) & 7) * step], q) << (16 * (t & 1));
      rotate8x16(O, (8 - rho) & 7, R[r]);   // slot c = column c
    }
  } else {
#pragma unroll
    for (int r = 0; r < 4; ++r)
#pragma unroll
      for (int k = 0; k < 4; ++k) R[r][k] = 0;
#pragma unroll
    for (int a = 0; a < 4; ++a) {
      int i, j;
      am.ij(k0 + a, &i, &j);
      const int16_t* src = P + (gm.z + i * step) * pitch + gm.w + j * step;
#pragma unroll
      for (int e = 0; e < 8; ++e) {
        const int rr = e >> 2, cc = e & 3;
        int32_t cval = 0;
        if (i + rr < gm.y && j + cc < gm.x) cval = src[(rr * step) * pitch + cc * step];
        const int r = 2 * (a & 1) + rr, c = 4 * (a >> 1) + cc;
        R[r][c >> 1] |= quantise16(cval, q) << (16 * (c & 1));
      }
    }
  }
  uint4* dst = reinterpret_cast<uint4*>(coef + f.base) + a0;
#pragma unroll
  for (int a = 0; a < 4; ++a) {
    const int r0 = 2 * (a & 1), k = 2 * (a >> 1);
    dst[a] = make_uint4(R[r0][k], R[r0][k + 1], R[r0 + 1][k], R[r0 + 1][k + 1]);
  }
}

// Quantise + area-ordered pack of the loop units [u0, u1) of the block table
// (an area quad where the block's type rows hold a multiple of 4 areas, else
// one area), by threads tid = first .. of n.
__device__ inline void pack_units(const FusedBlock* s_fb, int u0, int u1, int tid, int n, const int16_t* P, int pitch,
                                  uint8_t* __restrict__ coef) {
  int blk = 0;
  for (int g = u0 + tid; g < u1; g += n) {
    while (g >= s_fb[blk].end) ++blk;
    const FusedBlock& f = s_fb[blk];
    const int a = g - (blk ? s_fb[blk - 1].end : 0);
    AreaMap am;
    am.n = f.n; am.w = f.w; am.nlog = f.nlog; am.wlog = f.wlog;
    if (f.quad) {
      pack_quad(f, am, 4 * a, P, pitch, coef);
      continue;
    }
    int type, k, i, j;
    am.split(a, &type, &k);
    am.ij(k, &i, &j);
    const int4 gm = f.geo[type];
    const int step = f.step, q = f.q;
    const int16_t* src = P + (gm.z + i * step) * pitch + gm.w + j * step;
    int16_t v[8];
#pragma unroll
    for (int e = 0; e < 8; ++e) {
      const int r = e >> 2, cc = e & 3;
      int32_t cval = 0;
      if (i + r < gm.y && j + cc < gm.x) cval = src[(r * step) * pitch + cc * step];
      int32_t m = cval < 0 ? -cval : cval;
      m >>= q;
      v[e] = (int16_t)(cval < 0 ? -m : m);
    }
    uint4 u;
    u.x = (uint16_t)v[0] | ((uint32_t)(uint16_t)v[1] << 16);
    u.y = (uint16_t)v[2] | ((uint32_t)(uint16_t)v[3] << 16);
    u.z = (uint16_t)v[4] | ((uint32_t)(uint16_t)v[5] << 16);
    u.w = (uint16_t)v[6] | ((uint32_t)(uint16_t)v[7] << 16);
    reinterpret_cast<uint4*>(coef + f.base)[a] = u;
  }
}


// Decoded channels 0..2 of one tile with a colour transform at level z into
// the region output, by the last of the tile's CTAs of those channels:
// channel `c` is its own shared-memory plane (P, `pitch` elements a row),
// the other two come from the int16 planes the other CTAs left in global
// memory (gp: three row-major zw x zh planes, read through L2).  Each thread
// converts four pixels of a row (inverse colour transform, clamp to
// [0, 2^bits - 1]); samples are uint8 (bits <= 8) or uint16, C to a pixel.
__device__ inline void store_tile_ct(const TileDev& t, int z, int zw, int zh, int c, const int16_t* P, int pitch,
                                     const int16_t* __restrict__ gp) {
  uint8_t* __restrict__ out = t.dst;
  const int64_t opitch = t.dpitch;
  const int rx = t.rx, ry = t.ry, rw = t.rw, rh = t.rh;
  const int tx = (t.x0 >> z) - rx, ty = (t.y0 >> z) - ry;   // tile origin in the output
  const int32_t maxv = (1 << t.bits) - 1;
  const int qw = (zw + 3) >> 2;
  const int rows_per_pass = blockDim.x / qw;
  const int r0 = threadIdx.x / qw, x4 = (threadIdx.x - r0 * qw) << 2;
  if (r0 >= rows_per_pass) return;
  const int64_t np = (int64_t)zw * zh;
  // whole quads of a plane with rows of a multiple of 4 samples load 8-byte aligned
  const bool vec = (zw & 3) == 0 && (reinterpret_cast<uintptr_t>(gp) & 7) == 0;
  // whole quads of RGB8 inside the region with 4-byte aligned destinations take three word stores
  const bool words = t.C == 3 && t.bits <= 8 && ((reinterpret_cast<uintptr_t>(out) | (uintptr_t)opitch) & 3) == 0 &&
                     ((tx + x4) & 3) == 0 && x4 + 3 < zw && tx + x4 >= 0 && tx + x4 + 3 < rw;
  const int C = t.C;
  for (int y = r0; y < zh; y += rows_per_pass) {
    const int oy = ty + y;
    if (oy < 0 || oy >= rh) continue;
    int32_t ch[3][4];
    if (vec) {
      // whole quad: one 8-byte load per global plane, two word loads from shared memory
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        uint32_t lo, hi;
        if (k == c) {
          const uint32_t* sp = reinterpret_cast<const uint32_t*>(P + y * pitch + x4);
          lo = sp[0]; hi = sp[1];
        } else {
          const uint2 g2 = __ldcg(reinterpret_cast<const uint2*>(gp + k * np + (int64_t)y * zw + x4));
          lo = g2.x; hi = g2.y;
        }
        ch[k][0] = (int32_t)(int16_t)(lo & 0xFFFFu); ch[k][1] = (int32_t)lo >> 16;
        ch[k][2] = (int32_t)(int16_t)(hi & 0xFFFFu); ch[k][3] = (int32_t)hi >> 16;
      }
    } else {
#pragma unroll
      for (int k = 0; k < 3; ++k)
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int x = min(x4 + u, zw - 1);
          ch[k][u] = k == c ? (int32_t)P[y * pitch + x] : (int32_t)__ldcg(gp + k * np + (int64_t)y * zw + x);
        }
    }
    int32_t R[4], G[4], B[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      int32_t r, g, b;
      ct_inverse(t.ct, ch[0][u], ch[1][u], ch[2][u], &r, &g, &b);
      R[u] = min(max(r, 0), maxv);
      G[u] = min(max(g, 0), maxv);
      B[u] = min(max(b, 0), maxv);
    }
    uint8_t* row = out + (int64_t)oy * opitch;
    if (words) {
      uint32_t* d = reinterpret_cast<uint32_t*>(row + 3 * (tx + x4));
      d[0] = (uint32_t)R[0] | ((uint32_t)G[0] << 8) | ((uint32_t)B[0] << 16) | ((uint32_t)R[1] << 24);
      d[1] = (uint32_t)G[1] | ((uint32_t)B[1] << 8) | ((uint32_t)R[2] << 16) | ((uint32_t)G[2] << 24);
      d[2] = (uint32_t)B[2] | ((uint32_t)R[3] << 8) | ((uint32_t)G[3] << 16) | ((uint32_t)B[3] << 24);
    } else {
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int ox = tx + x4 + u;
        if (x4 + u >= zw || ox < 0 || ox >= rw) continue;
        if (t.bits <= 8) {
          row[C * ox] = (uint8_t)R[u];
          row[C * ox + 1] = (uint8_t)G[u];
          row[C * ox + 2] = (uint8_t)B[u];
        } else {
          uint16_t* r16 = reinterpret_cast<uint16_t*>(row);
          r16[C * ox] = (uint16_t)R[u];
          r16[C * ox + 1] = (uint16_t)G[u];
          r16[C * ox + 2] = (uint16_t)B[u];
        }
      }
    }
  }
}

// Channel c of a tile coded without a colour transform on it: samples
// clamped to [0, 2^bits - 1], uint8 (bits <= 8) or uint16, C to a pixel.
__device__ inline void store_tile_channel(const TileDev& t, int z, int zw, int zh, int c, const int16_t* P, int pitch) {
  uint8_t* __restrict__ out = t.dst;
  const int64_t opitch = t.dpitch;
  const int rx = t.rx, ry = t.ry, rw = t.rw, rh = t.rh;
  const int tx = (t.x0 >> z) - rx, ty = (t.y0 >> z) - ry;
  const int32_t maxv = (1 << t.bits) - 1;
  for (int e = threadIdx.x; e < zw * zh; e += blockDim.x) {
    const int y = e / zw, x = e - y * zw;
    const int ox = tx + x, oy = ty + y;
    if (ox < 0 || oy < 0 || ox >= rw || oy >= rh) continue;
    const int32_t v = min(max((int32_t)P[y * pitch + x], 0), maxv);
    uint8_t* row = out + (int64_t)oy * opitch;
    if (t.bits <= 8) row[ox * t.C + c] = (uint8_t)v;
    else reinterpret_cast<uint16_t*>(row)[ox * t.C + c] = (uint16_t)v;
  }
}

// 8 x 8 bit-matrix transpose of the bytes of (lo, hi): bit e of byte j moves
// to bit j of byte e (bytes 0-3 in lo, 4-7 in hi).  Three rounds swap the
// off-diagonal 1 x 1, 2 x 2 and 4 x 4 sub-blocks.
__device__ __forceinline__ void transpose8x8(uint32_t& lo, uint32_t& hi) {
  uint32_t t;
  t = (lo ^ (lo >> 7)) & 0x00AA00AAu; lo ^= t ^ (t << 7);
  t = (hi ^ (hi >> 7)) & 0x00AA00AAu; hi ^= t ^ (t << 7);
  t = (lo ^ (lo >> 14)) & 0x0000CCCCu; lo ^= t ^ (t << 14);
  t = (hi ^ (hi >> 14)) & 0x0000CCCCu; hi ^= t ^ (t << 14);
  t = ((lo >> 4) ^ hi) & 0x0F0F0F0Fu; hi ^= t; lo ^= t << 4;
}

// Decode side, fused with the coefficient rebuild: every block of the tile
// channel needed at level z (the LL and the levels above z) is rebuilt from
// its decoded symbol planes (sign plane, magnitude bits d-2 .. 0),
// dequantised at the bin midpoint and placed into the interleaved int16
// layout; the CTA then lifts back from level L to level z and writes the
// LL_z image row-major (int32) for the colour store.
// Rebuild of four consecutive areas (k0 .. k0+3, one type) of a block whose
// plane rows are multiples of 4 bytes: one word load per plane for the four
// areas, a 4 x 4 byte transpose per four planes, then per area the 8 x 8
// bit transposes of the single-area path.  Planes 0 .. 15 (sign and 15
// magnitude planes: every plane of int16 coefficients).
__device__ inline void rebuild_quad(const FusedBlock& f, const AreaMap& am, const int32_t (*po)[3], const uint8_t* __restrict__ sym,
                                    int a0, int16_t* P, int pitch) {
  int type, k0;
  am.split(a0, &type, &k0);
  const int d = f.d, keep = f.keep;
  const uint32_t* sk = reinterpret_cast<const uint32_t*>(sym + f.base + k0);   // 4-byte aligned: planes 16, n and k0 multiples of 4
  uint32_t pw[16];
#pragma unroll
  for (int pl = 0; pl < 16; ++pl) {
    pw[pl] = 0;
    if (pl < keep) {
      const int32_t o = po[pl][type];
      if (o >= 0) pw[pl] = __ldg(sk + (o >> 2));
    }
  }
  // aw[G][a]: bytes = planes 4G+1 .. 4G+4 of area a (plane 16 reads as 0)
  uint32_t aw[4][4];
#pragma unroll
  for (int G = 0; G < 4; ++G) {
    const uint32_t A = pw[4 * G + 1], B = pw[4 * G + 2], C = pw[4 * G + 3], D = G < 3 ? pw[4 * G + 4] : 0u;
    const uint32_t t0 = __byte_perm(A, B, 0x5140), t1 = __byte_perm(C, D, 0x5140);
    const uint32_t t2 = __byte_perm(A, B, 0x7362), t3 = __byte_perm(C, D, 0x7362);
    aw[G][0] = __byte_perm(t0, t1, 0x5410);
    aw[G][1] = __byte_perm(t0, t1, 0x7632);
    aw[G][2] = __byte_perm(t2, t3, 0x5410);
    aw[G][3] = __byte_perm(t2, t3, 0x7632);
  }
  const int4 gm = f.geo[type];
  const int step = f.step, q = f.q;
  const int32_t half = (1 << q) >> 1;
  const int rowstep = step * pitch;
  const int shift = 33 - d;
  // With a block width of 8 or more (a power of two) the quad's areas tile a
  // 4 x 8 region: area a covers rows 2 (a & 1) .., columns 4 (a >> 1) ..
  // The 32 coefficients are packed in pairs, R[r][k] = columns 2k, 2k+1 of
  // region row r.
  uint32_t R[4][4];
#pragma unroll
  for (int r = 0; r < 4; ++r)
#pragma unroll
    for (int k = 0; k < 4; ++k) R[r][k] = 0;
#pragma unroll
  for (int a = 0; a < 4; ++a) {
    uint32_t w0 = aw[0][a], w1 = aw[1][a], w2 = aw[2][a], w3 = aw[3][a];
    transpose8x8(w0, w1);
    transpose8x8(w2, w3);
    const uint32_t neg = (pw[0] >> (8 * a)) & 255u;
#pragma unroll
    for (int e = 0; e < 8; ++e) {
      const int cc = e & 3;
      // magnitude bits, most significant plane first (bit j of the pair = plane j + 1); with d <= 16
      // the two unrelated upper bytes of the permute end below bit 33 - d and are shifted out
      const uint32_t rb = __byte_perm(e < 4 ? w0 : w1, e < 4 ? w2 : w3, cc | ((4 + cc) << 4));
      const int32_t m = d >= 2 ? (int32_t)(__brev(rb) >> shift) : 0;
      const int32_t v = m == 0 ? 0 : (m << q) + half;
      const uint32_t h16 = (uint32_t)(uint16_t)(((neg >> e) & 1u) ? -v : v);
      const int r = 2 * (a & 1) + (e >> 2), c = 4 * (a >> 1) + cc;
      R[r][c >> 1] |= h16 << (16 * (c & 1));
    }
  }
  int i0, j0;
  am.ij(k0, &i0, &j0);
  int16_t* base = P + (gm.z + i0 * step) * pitch + gm.w + j0 * step;
  if (am.wlog >= 3 && i0 + 3 < gm.y && j0 + 7 < gm.x) {
    // Rotated stores: in store t of a row, lane l writes column (t + rho) & 7
    // with rho = (l >> 2) & 7.  Neighbouring lanes' regions start 8 columns
    // apart, so without rotation every store of a warp hits only four banks
    // (8- to 32-way conflicts at steps 2 .. 8); rotated, the 32 lanes spread
    // over all banks.
    const int rho = (threadIdx.x >> 2) & 7;
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      uint32_t O[4];
      rotate8x16(R[r], rho, O);   // slot t = column (t + rho) & 7
      int16_t* row = base + r * rowstep;
#pragma unroll
      for (int t = 0; t < 8; ++t) row[((t + rho) & 7) * step] = (int16_t)(O[t >> 1] >> (16 * (t & 1)));
    }
    return;
  }
#pragma unroll
  for (int a = 0; a < 4; ++a) {
    int i, j;
    am.ij(k0 + a, &i, &j);
    int16_t* dst = P + (gm.z + i * step) * pitch + gm.w + j * step;
#pragma unroll
    for (int e = 0; e < 8; ++e) {
      const int rr = e >> 2, cc = e & 3;
      if (i + rr >= gm.y || j + cc >= gm.x) continue;
      const int r = 2 * (a & 1) + rr, c = 4 * (a >> 1) + cc;
      dst[rr * rowstep + cc * step] = (int16_t)(R[r][c >> 1] >> (16 * (c & 1)));
    }
  }
}

// Rebuild of the loop units [u0, u1) of the block table (areas or area
// quads) into the interleaved plane, by threads tid = first .. of n.
__device__ inline void rebuild_units(const FusedBlock* s_fb, const int32_t (*s_po)[kMaxFusedPlanes][3], const uint8_t* __restrict__ sym,
                                     int u0, int u1, int tid, int n, int16_t* P, int pitch) {
  int blk = 0;
  for (int g = u0 + tid; g < u1; g += n) {
    while (g >= s_fb[blk].end) ++blk;
    const FusedBlock& f = s_fb[blk];
    const int u = g - (blk ? s_fb[blk - 1].end : 0);
    AreaMap am;
    am.n = f.n; am.w = f.w; am.nlog = f.nlog; am.wlog = f.wlog;
    if (f.quad) {
      rebuild_quad(f, am, s_po[blk], sym, 4 * u, P, pitch);
      continue;
    }
    const int a = u;
    int type, k;
    am.split(a, &type, &k);
    const int d = f.d, keep = f.keep;
    // symbols of the sign plane and of magnitude planes 1..16 (plane j+1 in byte j of w[]),
    // loaded together before use; planes not kept (removed or dropped) read as 0
    const uint8_t* sk = sym + f.base + k;
    uint32_t sv[17];
#pragma unroll
    for (int pl = 0; pl < 17; ++pl) {
      sv[pl] = 0;
      if (pl < keep) {
        const int32_t o = s_po[blk][pl][type];
        if (o >= 0) sv[pl] = __ldg(sk + o);
      }
    }
    const uint32_t neg = sv[0];
    uint32_t w[6];
#pragma unroll
    for (int u = 0; u < 4; ++u)
      w[u] = __byte_perm(__byte_perm(sv[4 * u + 1], sv[4 * u + 2], 0x0040), __byte_perm(sv[4 * u + 3], sv[4 * u + 4], 0x0040), 0x5410);
    w[4] = w[5] = 0;
    if (keep > 17) {   // magnitude planes 17..19 (data of more than 10 bits only)
      uint32_t e4[3];
#pragma unroll
      for (int u = 0; u < 3; ++u) {
        const int pl = 17 + u;
        e4[u] = 0;
        if (pl < keep) {
          const int32_t o = s_po[blk][pl][type];
          if (o >= 0) e4[u] = __ldg(sk + o);
        }
      }
      w[4] = __byte_perm(__byte_perm(e4[0], e4[1], 0x0040), e4[2], 0x0410) & 0x00FFFFFFu;
    }
    // bit transposes: afterwards byte e of each pair holds, in bit j, bit e of plane j+1
    transpose8x8(w[0], w[1]);
    transpose8x8(w[2], w[3]);
    if (keep > 17) transpose8x8(w[4], w[5]);
    int i, j;
    am.ij(k, &i, &j);
    const int4 gm = f.geo[type];
    const int step = f.step, q = f.q;
    const int32_t half = (1 << q) >> 1;
    int16_t* dst = P + (gm.z + i * step) * pitch + gm.w + j * step;
#pragma unroll
    for (int e = 0; e < 8; ++e) {
      const int r = e >> 2, cc = e & 3;
      if (i + r >= gm.y || j + cc >= gm.x) continue;
      const uint32_t lo = e < 4 ? w[0] : w[1], mid = e < 4 ? w[2] : w[3], hi = e < 4 ? w[4] : w[5];
      const int sel = e & 3;
      // magnitude bits, most significant plane first: reverse the d-1 plane bits
      const uint32_t rbits = (__byte_perm(lo, mid, sel | ((4 + sel) << 4)) & 0xFFFFu) | (((hi >> (8 * sel)) & 255u) << 16);
      const int32_t m = d >= 2 ? (int32_t)(__brev(rbits) >> (33 - d)) : 0;
      const int32_t v = m == 0 ? 0 : (m << q) + half;
      dst[(r * step) * pitch + cc * step] = (int16_t)(((neg >> e) & 1u) ? -v : v);
    }
  }
}

// Forward of channel c of fused tile t by every thread of the CTA (256, 512
// or 1024; barriers 0, 1 and 2): pixels through the colour transform into
// the interleaved int16 plane P, levels 0 .. L-1 in place, then the
// quantised, area-ordered coefficients of the channel's blocks into `coef`.
// The caller synchronises the CTA before P or s_fb is used again.
__device__ inline void fused_forward_channel(const TileDev& t, int c, const BlockDev* __restrict__ blocks, uint8_t* __restrict__ coef,
                                             int* __restrict__ status, int16_t* P, FusedBlock* s_fb) {
  const int w = t.w, h = t.h, pitch = smem_pitch(w);
  // load + colour transform of channel c
  uint32_t over = 0;   // bits of samples above the tile's bit depth
  const bool quad = t.C == 3 && t.ct == 1 && t.bits <= 8 && (w & 3) == 0 && (t.pitch & 3) == 0 &&
                    ((reinterpret_cast<uintptr_t>(t.pixels) & 3) == 0);
  if (quad) {
    // four pixels (12 bytes, three aligned words) per thread and row; a
    // thread keeps its column quad and steps over rows, loading four rows'
    // words before converting them
    const int qw = w >> 2;
    const int dy = blockDim.x / qw;
    const int y0 = threadIdx.x / qw, x4 = (threadIdx.x - y0 * qw) << 2;
    if (y0 < dy) {
      const uint8_t* base = t.pixels + 3 * x4;
      for (int yb = y0; yb < h; yb += 4 * dy) {
        uint32_t wv[4][3];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int y = yb + u * dy;
          if (y < h) {
            const uint32_t* src = reinterpret_cast<const uint32_t*>(base + (int64_t)y * t.pitch);
            wv[u][0] = __ldg(src);
            wv[u][1] = __ldg(src + 1);
            wv[u][2] = __ldg(src + 2);
          }
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int y = yb + u * dy;
          if (y >= h) continue;
          const uint32_t w0 = wv[u][0], w1 = wv[u][1], w2 = wv[u][2];
          const int32_t R[4] = {(int32_t)(w0 & 255), (int32_t)((w0 >> 24) & 255), (int32_t)((w1 >> 16) & 255), (int32_t)((w2 >> 8) & 255)};
          const int32_t G[4] = {(int32_t)((w0 >> 8) & 255), (int32_t)(w1 & 255), (int32_t)((w1 >> 24) & 255), (int32_t)((w2 >> 16) & 255)};
          const int32_t B[4] = {(int32_t)((w0 >> 16) & 255), (int32_t)((w1 >> 8) & 255), (int32_t)(w2 & 255), (int32_t)((w2 >> 24) & 255)};
          int32_t v[4];
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            over |= (uint32_t)(R[q] | G[q] | B[q]) >> t.bits;
            v[q] = c == 0 ? (R[q] + 2 * G[q] + B[q]) >> 2 : c == 1 ? B[q] - G[q] : R[q] - G[q];
          }
          uint32_t* dst = reinterpret_cast<uint32_t*>(P + y * pitch + x4);   // 4-byte aligned: pitch and x4 are even
          dst[0] = (uint32_t)(uint16_t)v[0] | ((uint32_t)(uint16_t)v[1] << 16);
          dst[1] = (uint32_t)(uint16_t)v[2] | ((uint32_t)(uint16_t)v[3] << 16);
        }
      }
    }
  } else
  for (int e = threadIdx.x; e < w * h; e += blockDim.x) {
    const int y = e / w, x = e - y * w;
    const uint8_t* row = t.pixels + (int64_t)y * t.pitch;
    int32_t v;
    if (t.ct && c < 3) {
      const int32_t R = sample_at(row, x, t.C, 0, t.bits), G = sample_at(row, x, t.C, 1, t.bits), B = sample_at(row, x, t.C, 2, t.bits);
      over |= (uint32_t)(R | G | B) >> t.bits;
      v = ct_forward(t.ct, c, R, G, B);
    } else {
      v = sample_at(row, x, t.C, c, t.bits);
      over |= (uint32_t)v >> t.bits;
    }
    P[y * pitch + x] = (int16_t)v;
  }
  // samples above the tile's bit depth void the int16 range bound of the transform
  if (__any_sync(0xffffffffu, over != 0) && (threadIdx.x & 31) == 0) set_status(status, kStRange);
  __syncthreads();
  // quantise + area-ordered pack of this channel's blocks (one loop over the areas of a range of blocks)
  const int nbc = t.nb / t.C;
  const int nwarps = blockDim.x >> 5, warp = threadIdx.x >> 5;
  // After level 0 the level-1 blocks (3/4 of the coefficients) are final and
  // at most half of the lines are left to lift: the first W warps lift levels
  // 1.. while the others build the block table and pack the level-1 blocks.
  const int W = t.L >= 2 && level_dim(w, 0) > kWarpGrid ? overlap_warps(level_dim(w, 1), level_dim(h, 1), nwarps, kOverlapSplitFwd) : 0;
  if (W == 0) {
    transform_fwd_levels(P, pitch, w, h, t.L);
    if (threadIdx.x < 32) fused_block_table(t, blocks, nullptr, nullptr, t.block_base + (int64_t)c * nbc, nbc, 0, s_fb, nullptr);
    __syncthreads();
    pack_units(s_fb, 0, s_fb[nbc - 1].end, threadIdx.x, blockDim.x, P, pitch, coef);
    return;
  }
  level_fwd(P, pitch, level_dim(w, 0), level_dim(h, 0), 1);
  // table order: LL, levels L .. 1 (stream order), so the level-1 blocks come last
  if (warp < W) {
    transform_fwd_levels_group(P, pitch, w, h, 1, t.L, W * 32);
  } else {
    const int gt = threadIdx.x - W * 32, gn = blockDim.x - W * 32;
    if (gt < 32) fused_block_table(t, blocks, nullptr, nullptr, t.block_base + (int64_t)c * nbc, nbc, 0, s_fb, nullptr);
    group_sync(2, gn);
    int k1 = nbc;
    while (k1 > 0 && s_fb[k1 - 1].level == 1) --k1;
    const int rank = block_warp_rank(warp, W), K = block_warps(nwarps, W, kOverlapBlockWarpsFwd);
    if (rank >= 0 && rank < K)
      pack_units(s_fb, k1 ? s_fb[k1 - 1].end : 0, s_fb[nbc - 1].end, rank * 32 + (threadIdx.x & 31), K * 32, P, pitch, coef);
  }
  __syncthreads();
  int k1 = nbc;
  while (k1 > 0 && s_fb[k1 - 1].level == 1) --k1;
  pack_units(s_fb, 0, k1 ? s_fb[k1 - 1].end : 0, threadIdx.x, blockDim.x, P, pitch, coef);
}

// Inverse of channel c of fused tile t at level z by every thread of the
// CTA: every block of the channel needed at level z rebuilt from its symbol
// planes into P, then levels L-1 .. z in place; on return (the CTA
// synchronised) P holds the channel's LL_z (level_dim(w, z) x
// level_dim(h, z) samples, row pitch smem_pitch of its width).
__device__ inline void fused_inverse_plane(const TileDev& t, int c, int z, const BlockDev* __restrict__ blocks,
                                           const DecInfo* __restrict__ info, const int64_t* __restrict__ sym_off,
                                           const uint8_t* __restrict__ sym, int16_t* P, FusedBlock* s_fb,
                                           int32_t (*s_po)[kMaxFusedPlanes][3]) {
  const int zw = level_dim(t.w, z), zh = level_dim(t.h, z), pitch = smem_pitch(zw);
  // rebuild of every block of the channel needed at level z, one loop over all their areas
  const int nbc = t.nb / t.C;
  if (threadIdx.x < 32) fused_block_table(t, blocks, info, sym_off, t.block_base + (int64_t)c * nbc, nbc, z, s_fb, s_po);
  __syncthreads();
  const int total = s_fb[nbc - 1].end;
  const int nwarps = blockDim.x >> 5, warp = threadIdx.x >> 5;
  // The blocks of the finest level decoded (z + 1) come last in the table and
  // hold 3/4 of the coefficients; the inverse levels above it touch only the
  // coarser grid.  So: rebuild the coarser blocks, then the first W warps
  // invert levels L-1 .. z+1 while the others rebuild the finest blocks,
  // then the CTA inverts level z+1 into the level-z image.
  int kf = nbc;
  while (kf > 0 && s_fb[kf - 1].level == z + 1) --kf;
  const int uF = kf ? s_fb[kf - 1].end : 0;
  const int W = t.L - 1 >= z + 1 && kf < nbc && level_dim(t.w, z) > kWarpGrid
                    ? overlap_warps(level_dim(t.w, z + 1), level_dim(t.h, z + 1), nwarps, kOverlapSplitInv)
                    : 0;
  if (W == 0) {
    rebuild_units(s_fb, s_po, sym, 0, total, threadIdx.x, blockDim.x, P, pitch);
    __syncthreads();
    transform_inv_levels(P, pitch, t.w, t.h, t.L, z);
  } else {
    rebuild_units(s_fb, s_po, sym, 0, uF, threadIdx.x, blockDim.x, P, pitch);
    __syncthreads();
    const int rank = block_warp_rank(warp, W), K = block_warps(nwarps, W, kOverlapBlockWarpsInv);
    if (warp < W) transform_inv_levels_group(P, pitch, t.w, t.h, t.L, z + 1, z, W * 32);
    else if (rank >= 0 && rank < K) rebuild_units(s_fb, s_po, sym, uF, total, rank * 32 + (threadIdx.x & 31), K * 32, P, pitch);
    __syncthreads();
    level_inv(P, pitch, level_dim(t.w, z), level_dim(t.h, z), 1);
  }
}

// A colour tile's channel plane (LL_z in P) to its int16 hand-off plane
// `mine` in global memory (zw x zh, row-major), for the CTA that inverts
// the colour transform.
__device__ inline void fused_handoff(const int16_t* P, int pitch, int zw, int zh, int16_t* mine) {
  if ((zw & 7) == 0 && ((reinterpret_cast<uintptr_t>(mine) & 15) == 0)) {
    // rows of eight-sample chunks: four word loads from shared memory, one 16-byte store
    const int cw = zw >> 3;
    for (int e = threadIdx.x; e < cw * zh; e += blockDim.x) {
      const int y = e / cw, x8 = (e - y * cw) << 3;
      const uint32_t* src = reinterpret_cast<const uint32_t*>(P + y * pitch + x8);   // pitch and x8 even: 4-byte aligned
      uint4 v;
      v.x = src[0]; v.y = src[1]; v.z = src[2]; v.w = src[3];
      reinterpret_cast<uint4*>(mine + (int64_t)y * zw)[x8 >> 3] = v;
    }
  } else {
    for (int e = threadIdx.x; e < zw * zh; e += blockDim.x) {
      const int y = e / zw, x = e - y * zw;
      mine[e] = P[y * pitch + x];
    }
  }
}

// The hand-off planes of a colour tile (3 x zw x zh int16 from gp) are dead
// once the colour store has read them: drop their L2 lines without a
// write-back to DRAM (only whole 128-byte lines inside the tile's planes; a
// line shared with a neighbouring tile's region is left alone).  The caller
// synchronises the CTA first.
__device__ inline void discard_handoff(const int16_t* gp, int zw, int zh) {
  const uintptr_t lo = (reinterpret_cast<uintptr_t>(gp) + 127) & ~(uintptr_t)127;
  const uintptr_t hi = (reinterpret_cast<uintptr_t>(gp + 3 * (int64_t)zw * zh)) & ~(uintptr_t)127;
  for (uintptr_t a = lo + 128 * (uintptr_t)threadIdx.x; a < hi; a += 128 * (uintptr_t)blockDim.x)
    asm volatile("discard.global.L2 [%0], 128;" ::"l"(a) : "memory");
}

}  // namespace isx
