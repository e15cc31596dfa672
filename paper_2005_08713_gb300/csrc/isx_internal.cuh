// isx_internal.cuh — device-side data structures and primitives of the
// GB300 codec library.  Not part of the public ABI (include/isx.h).
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace isx {

constexpr int kCell = 128;          // coefficient block edge (Sec. 4: "partitioned in 128*128 blocks")
constexpr int kMaxLevels = 15;
constexpr int kMaxD = 31;           // block bit depth field is 5 bits
constexpr int kMaxW = 18;           // largest zero-run counter width considered (w in [2, b], b <= 18)
constexpr int kCtaThreads = 256;    // CTA size of the per-block coding kernels
constexpr int kMaxDConst = 31;
constexpr int kSmemPlaneBytes = 160 * 1024;   // largest int16 channel plane of a tile on the fused shared-memory path

enum DevStatus : int { kStOk = 0, kStCapacity = 2, kStCorrupt = 3, kStTimeout = 6, kStInternal = 7, kStRange = 8 };

// One tile as the kernels see it (copied from isx_tile_desc plus its plan).
struct TileDev {
  const uint8_t* pixels;    // device, HWC
  int64_t pitch;            // bytes
  int32_t w, h, C, bits, L, x0, y0;
  int32_t ct;               // colour transform of channels 0..2: 0 none, 1 RCT, 2 YCoCg-R (the stored id)
  int32_t coef16;           // every coefficient (and every state of the transforms) fits int16
  uint8_t q[16];
  int32_t nb;               // number of coefficient blocks
  int32_t fused;            // 1: transformed by the fused shared-memory kernels
  int64_t block_base;       // index of its first block
  int64_t plane_base;       // element offset of its first Mallat plane
  int64_t coef_base;        // byte offset of its first area-ordered coefficient block
  int64_t sym_base;         // byte offset of its first block's symbol region (encode)
  int64_t pst_base;         // index of its first block's first plane-statistics slot (encode)
  // decode destination: the part of the tile inside the rectangle (rx, ry,
  // rw, rh) of level-z pixels goes to dst, whose first byte is pixel
  // (rx, ry); rows dpitch bytes apart, the tile's own sample format
  uint8_t* dst;
  int64_t dpitch;
  int32_t rx, ry, rw, rh;
  // optional per-tile %globaltimer stamps (isx_set_tile_stamps): four arrays
  // of stamp_n entries, this tile at index stamp_i
  uint64_t* stamps;
  int32_t stamp_n, stamp_i;
  int32_t win;              // decode: index of its WinDev (windowed region decode), -1: the whole tile
};

// Windowed region decode of a tile (an untiled image or any large tile):
// only the samples the requested window depends on are decoded and
// inverted.  Inverse level l maps the level-l bands restricted to band
// ranges [lx0, lx1) (low, along x), [hx0, hx1) (high, along x), and the
// same along y, to the window [ox0, ox1) x [oy0, oy1) of LL_{l-1}.  Its
// input W_l is a compact plane per channel: (nlx + nhx) columns, the low
// part first, by (nly + nhy) rows, the low rows first; the row pass writes
// T_l ((ox1 - ox0) x (nly + nhy) per channel), the column pass the LL part
// of W_{l-1} (or F, the level-z window, when l - 1 = z).  Element offsets
// are relative to the tile's plane_base.
struct WinLevel {
  int32_t lx0, lx1, hx0, hx1, ly0, ly1, hy0, hy1;
  int32_t ox0, ox1, oy0, oy1;
  int64_t buf, tmp;
};
struct WinDev {
  int32_t z, L;
  int32_t fx0, fx1, fy0, fy1;   // the level-z window (tile-local level-z coordinates)
  int64_t fbuf;                 // F: C planes of (fx1 - fx0) x (fy1 - fy0)
  WinLevel lev[kMaxLevels + 1]; // [l] for z < l <= L
};
__host__ __device__ inline bool ranges_meet(int a0, int a1, int b0, int b1) { return a0 < b1 && b0 < a1 && a0 < a1 && b0 < b1; }
// Cells [*x0, *x1) x [*y0, *y1) of `level` (0 = the LL of level L) that
// bound the windows' band ranges: the only cells a windowed decode visits.
__host__ __device__ inline void window_cells(const WinDev& W, int level, int* x0, int* x1, int* y0, int* y1) {
  int a0, a1, b0, b1;
  if (level == 0) {
    if (W.z == W.L) { a0 = W.fx0; a1 = W.fx1; b0 = W.fy0; b1 = W.fy1; }
    else { const WinLevel& v = W.lev[W.L]; a0 = v.lx0; a1 = v.lx1; b0 = v.ly0; b1 = v.ly1; }
  } else {
    const WinLevel& v = W.lev[level];
    a0 = v.hx1 > v.hx0 ? min(v.lx0, v.hx0) : v.lx0;
    a1 = v.hx1 > v.hx0 ? max(v.lx1, v.hx1) : v.lx1;
    b0 = v.hy1 > v.hy0 ? min(v.ly0, v.hy0) : v.ly0;
    b1 = v.hy1 > v.hy0 ? max(v.ly1, v.hy1) : v.ly1;
  }
  *x0 = a0 / kCell; *x1 = (a1 + kCell - 1) / kCell;
  *y0 = b0 / kCell; *y1 = (b1 + kCell - 1) / kCell;
}

// Does block (level, by, bx) of a windowed tile hold a coefficient inside its windows?
// level 0 = the LL band of level L.
__host__ __device__ inline bool block_in_window(const WinDev& W, int level, int by, int bx) {
  const int x0 = kCell * bx, x1 = x0 + kCell, y0 = kCell * by, y1 = y0 + kCell;
  if (level == 0) {
    if (W.z == W.L) return ranges_meet(x0, x1, W.fx0, W.fx1) && ranges_meet(y0, y1, W.fy0, W.fy1);
    const WinLevel& v = W.lev[W.L];
    return ranges_meet(x0, x1, v.lx0, v.lx1) && ranges_meet(y0, y1, v.ly0, v.ly1);
  }
  if (level <= W.z) return false;
  const WinLevel& v = W.lev[level];
  const bool xl = ranges_meet(x0, x1, v.lx0, v.lx1), xh = ranges_meet(x0, x1, v.hx0, v.hx1);
  const bool yl = ranges_meet(y0, y1, v.ly0, v.ly1), yh = ranges_meet(y0, y1, v.hy0, v.hy1);
  return (xh && yl) || (xl && yh) || (xh && yh);   // HL, LH, HH
}

// One coefficient block (Fig. 3): LL (p = 1) or HL, LH, HH (p = 3).
struct BlockDev {
  int32_t tile, c, level;   // level 0 = the LL band of the tile
  int32_t by, bx;           // cell position within the subband grid
  int32_t p, w, h;          // types and padded size (multiples of 4)
  int32_t coef16;           // coefficients stored as int16 (TileDev::coef16) or int32
  int32_t dmax;             // largest bit depth its coefficients can reach (bits + 6, at most 31)
  int64_t coef;             // byte offset of its coefficients: [type][area][8]
  int64_t sym;              // byte offset of its symbol region (encode)
  int64_t pst;              // index of its plane-statistics slots, dmax of them (encode)
};

__host__ __device__ inline int dmax_of_bits(int bits) { return bits + 6 < kMaxD ? bits + 6 : kMaxD; }

// Per-block statistics gathered from the symbol stream (encode, pass 1).
struct BlockStats {
  uint32_t hist[256];       // literal counts; [0] = isolated zero symbols, [s] = raw count of s
  uint32_t extra[kMaxW + 1];// sum over runs of (ceil(L / (2^w - 1)) - 1), w = 2..18
  uint32_t n_runs;          // zero runs of length >= 2
  uint32_t n_sym;           // kept symbols
  uint32_t removed[3];      // bit pl set: plane pl of that type removed
  int32_t d;
};

// Per-(block, plane) statistics of one plane segment (encode, pass 1): the
// counts of BlockStats restricted to the segment, from which the Huffman
// pass finds the segment's exact bit length.  hist (with hist[0] = zeros) is
// filled only for segments of more than 512 symbols; the zero-run counts
// always.  A segment holds at most 3 * 128 * 128 / 8 = 6144 symbols:
// 16-bit counts.
struct __align__(16) PlaneStats {
  uint16_t hist[256];
  uint16_t extra[kMaxW + 1];
  uint16_t runs;
  uint16_t zeros;           // isolated zero symbols (the literal 0)
  uint16_t pad[3];
};
static_assert(sizeof(PlaneStats) == 560, "PlaneStats is 35 16-byte words");
static_assert(3 * kCell * kCell / 8 < 65536, "a plane segment's counts fit 16 bits");

// Per-block code (encode, pass 2); 16-byte aligned so that the code and
// length arrays copy as 16-byte words.
struct __align__(16) BlockCode {
  uint32_t code[256];
  uint8_t len[256];
  uint32_t tree[80];        // preorder tree, MSB-first bit string (<= 2559 bits)
  int32_t tree_bits;
  int32_t czr, wbits, t0;   // zero-run symbol, counter width, default seektable width
  int32_t d, p, any_kept;
  uint32_t removed[3];
  uint64_t token_bits;      // sum of all segment lengths
  uint64_t slot_bytes;      // upper bound of the block size (t at its largest)
};

// Per-block decode information found by the header pass.
struct DecInfo {
  int32_t d, keep;           // bit depth, planes decoded (d minus dropped LSB planes, at least 1)
  uint32_t removed[3];
};

// Samples along one axis after l halvings with rounding up: ceil(n / 2^l)
// (nested ceilings of halves compose); 0 stays 0.
__host__ __device__ inline int level_dim(int n, int l) { return ((n - 1) >> l) + 1; }
__host__ __device__ inline int pad4(int n) { return (n + 3) & ~3; }
__host__ __device__ inline int ceil_div(int a, int b) { return (a + b - 1) / b; }
__device__ inline int bitlen_u32(uint32_t v) { return 32 - __clz(v); }
__device__ inline int bitlen_u64(uint64_t v) { return 64 - __clzll(v); }

// Area order of Eq. 1 (reading: i = 4 floor(2k'/w) + 2 (k' mod 2),
// j = 4 (floor(k'/2) mod (w/4))) for the within-plane index k'.
__device__ inline void area_ij(int k, int w, int* i, int* j) {
  *i = 4 * ((2 * k) / w) + 2 * (k & 1);
  *j = 4 * ((k >> 1) % (w >> 2));
}

// Area index -> (type, k') and k' -> (i, j) for one block, with shifts when
// the block's sizes are powers of two (the common case) instead of divisions.
struct AreaMap {
  int n, w, nlog, wlog;
  __device__ void init(int bw, int bh) {
    w = bw;
    n = bw * bh / 8;
    nlog = (n & (n - 1)) == 0 ? 31 - __clz(n) : -1;
    wlog = (w & (w - 1)) == 0 ? 31 - __clz(w) : -1;
  }
  __device__ void split(int a, int* type, int* k) const {
    if (nlog >= 0) { *type = a >> nlog; *k = a & (n - 1); }
    else { *type = a / n; *k = a - *type * n; }
  }
  __device__ void ij(int k, int* i, int* j) const {
    if (wlog >= 0) {
      *i = 4 * ((2 * k) >> wlog) + 2 * (k & 1);
      *j = 4 * ((k >> 1) & ((w >> 2) - 1));
    } else {
      area_ij(k, w, i, j);
    }
  }
};

// Subband rectangle of a block's type within the tile's Mallat plane.
__device__ inline void subband_rect(int tw, int th, int L, int level, int type, int* x, int* y, int* sw, int* sh) {
  if (level == 0) {
    *x = 0; *y = 0; *sw = level_dim(tw, L); *sh = level_dim(th, L);
    return;
  }
  int pw = level_dim(tw, level - 1), ph = level_dim(th, level - 1);
  int lw = (pw + 1) >> 1, lh = (ph + 1) >> 1;
  if (type == 0) { *x = lw; *y = 0; *sw = pw >> 1; *sh = lh; }
  else if (type == 1) { *x = 0; *y = lh; *sw = lw; *sh = ph >> 1; }
  else { *x = lw; *y = lh; *sw = pw >> 1; *sh = ph >> 1; }
}

__device__ inline int qlog2_of(const TileDev& t, int level) { return level == 0 ? t.q[t.L] : t.q[level - 1]; }

// --------------------------------------------------------- CTA primitives
// Exclusive sum scan over the CTA (blockDim.x a multiple of 32, <= 1024).
template <typename T>
__device__ T cta_exclusive_sum(T v, T* warp_tmp /* >= 33 */, T* total) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  T x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    T y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) warp_tmp[wid] = x;
  __syncthreads();
  if (wid == 0) {
    T s = lane < nw ? warp_tmp[lane] : T(0);
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      T y = __shfl_up_sync(0xffffffffu, s, o);
      if (lane >= o) s += y;
    }
    if (lane < nw) warp_tmp[lane] = s;   // inclusive warp prefixes
    if (lane == nw - 1) warp_tmp[32] = s;
  }
  __syncthreads();
  T base = wid ? warp_tmp[wid - 1] : T(0);
  T res = base + x - v;
  if (total) *total = warp_tmp[32];
  __syncthreads();
  return res;
}

// Zero-carry scan element: bit 31 = "all symbols so far are zero",
// low bits = number of zeros at the end of the covered range.
__device__ inline uint32_t carry_combine(uint32_t a, uint32_t b) {
  const uint32_t AZ = 0x80000000u;
  if (b & AZ) return (a & AZ) | ((a & ~AZ) + (b & ~AZ));
  return b;
}

__device__ inline uint32_t cta_exclusive_carry(uint32_t v, uint32_t* warp_tmp /* >= 33 */) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const uint32_t ID = 0x80000000u;
  uint32_t x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x = carry_combine(y, x);
  }
  if (lane == 31) warp_tmp[wid] = x;
  __syncthreads();
  if (wid == 0) {
    uint32_t s = lane < nw ? warp_tmp[lane] : ID;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      uint32_t y = __shfl_up_sync(0xffffffffu, s, o);
      if (lane >= o) s = carry_combine(y, s);
    }
    if (lane < nw) warp_tmp[lane] = s;
  }
  __syncthreads();
  uint32_t prev_in_warp = __shfl_up_sync(0xffffffffu, x, 1);
  if (lane == 0) prev_in_warp = ID;
  uint32_t base = wid ? warp_tmp[wid - 1] : ID;
  uint32_t res = carry_combine(base, prev_in_warp);
  __syncthreads();
  return res;
}

template <typename T>
__device__ T cta_reduce_max(T v, T* tmp /* >= 32 */) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    T y = __shfl_xor_sync(0xffffffffu, v, o);
    v = v > y ? v : y;
  }
  if (lane == 0) tmp[wid] = v;
  __syncthreads();
  if (wid == 0) {
    T s = lane < nw ? tmp[lane] : T(0);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      T y = __shfl_xor_sync(0xffffffffu, s, o);
      s = s > y ? s : y;
    }
    if (lane == 0) tmp[0] = s;
  }
  __syncthreads();
  T r = tmp[0];
  __syncthreads();
  return r;
}

__device__ inline void set_status(int* status, int code) { atomicCAS(status, 0, code); }

// Barriers of device code run by a whole CTA (CtaBarrier) or by a group of
// whole warps of it (NamedBarrier: the n threads that use barrier id, 3..15;
// 0 is __syncthreads, 1 and 2 belong to the fused transforms).
struct CtaBarrier {
  __device__ void operator()() const { __syncthreads(); }
};
struct NamedBarrier {
  int id, n;
  __device__ void operator()() const { asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(n) : "memory"); }
};

// Per-tile timestamps (ns of the GPU's global timer): the earliest start and
// the latest end of a tile's work in an encode or a decode.
enum StampKind { kStampEncStart = 0, kStampEncEnd = 1, kStampDecStart = 2, kStampDecEnd = 3 };
__device__ inline uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
__device__ inline void stamp_tile(const TileDev& t, int kind) {
  if (!t.stamps) return;
  unsigned long long* p = reinterpret_cast<unsigned long long*>(t.stamps + (int64_t)kind * t.stamp_n + t.stamp_i);
  if (kind == kStampEncStart || kind == kStampDecStart) atomicMin(p, (unsigned long long)global_ns());
  else atomicMax(p, (unsigned long long)global_ns());
}

}  // namespace isx
