// isx_coder_enc.cuh — device code of the block coder (Sec. 4, Fig. 2 c-e,
// Fig. 3): the symbol pass, the per-block Huffman construction, the exact
// segment sizes and the bit-exact emission, as functions over one block or
// one group of blocks.  Used by the per-stage kernels (isx_encode.cu) and by
// the persistent per-tile encoder (isx_persist.cu).
#pragma once
#include <cstdint>

#include "isx_internal.cuh"

namespace isx {
constexpr uint32_t kAllZero = 0x80000000u;

// The coefficients of one block: 8 per area in Eq. 2 bit order, int16 or int32.
struct CoefRef {
  const uint8_t* base;
  int is16;
  __device__ void load(int a, int32_t* c) const {
    if (is16) {
      const uint4 u = reinterpret_cast<const uint4*>(base)[a];
      const uint32_t w[4] = {u.x, u.y, u.z, u.w};
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        c[2 * k] = (int32_t)(int16_t)(w[k] & 0xffffu);
        c[2 * k + 1] = (int32_t)(int16_t)(w[k] >> 16);
      }
    } else {
      const int4* p4 = reinterpret_cast<const int4*>(base) + 2 * (int64_t)a;
      const int4 u = p4[0], v = p4[1];
      c[0] = u.x; c[1] = u.y; c[2] = u.z; c[3] = u.w; c[4] = v.x; c[5] = v.y; c[6] = v.z; c[7] = v.w;
    }
  }
};

__device__ inline uint32_t kept_types(const uint32_t* removed, int p, int pl) {
  uint32_t km = 0;
#pragma unroll
  for (int t = 0; t < 3; ++t)   // fixed trip count: removed[] stays in registers
    if (t < p && !((removed[t] >> pl) & 1u)) km |= 1u << t;
  return km;
}

__device__ inline int64_t region16(uint32_t km, int n) { return ((int64_t)__popc(km) * n + 15) & ~15LL; }

// ------------------------------------------------------------ warp runs
// A zero-run carry element: bit 31 = every symbol covered is zero, low bits
// = zeros at the end of the covered range.  Lanes cover 16 symbols each.
__device__ inline uint32_t warp_carry_exclusive(uint32_t v, uint32_t* inclusive_of_lane, uint32_t* total) {
  const int lane = threadIdx.x & 31;
  uint32_t x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x = carry_combine(y, x);
  }
  uint32_t ex = __shfl_up_sync(0xffffffffu, x, 1);
  if (lane == 0) ex = kAllZero;
  *inclusive_of_lane = x;
  *total = __shfl_sync(0xffffffffu, x, 31);
  return ex;
}

// Summary of a lane's symbols: leading zeros, trailing zeros, any nonzero.
struct LaneSyms {
  uint32_t w[4];
  int cnt;
  __device__ uint32_t at(int k) const {   // selects, not an indexed array: w[] stays in registers
    const uint32_t lo = (k & 4) ? w[1] : w[0], hi = (k & 4) ? w[3] : w[2];
    return (((k & 8) ? hi : lo) >> (8 * (k & 3))) & 0xffu;
  }
};

__device__ inline LaneSyms load_lane(const uint8_t* seg, int len, int base) {
  const int lane = threadIdx.x & 31;
  LaneSyms L;
  const int my0 = base + lane * 16;
  L.cnt = max(0, min(16, len - my0));
  L.w[0] = L.w[1] = L.w[2] = L.w[3] = 0;
  if (L.cnt > 0) {
    const uint4 u = *reinterpret_cast<const uint4*>(seg + my0);
    L.w[0] = u.x; L.w[1] = u.y; L.w[2] = u.z; L.w[3] = u.w;
  }
  return L;
}

// Bit k set: symbol k of the lane is nonzero (k < cnt).  Four byte
// compares per word; the multiply gathers the four flags into bits 24..27
// (the partial products never overlap, so there are no carries).
__device__ inline uint32_t nonzero_mask(const LaneSyms& L) {
  uint32_t Z = 0;
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const uint32_t t = __vcmpeq4(L.w[q], 0u) & 0x01010101u;
    Z |= ((t * 0x01020408u) >> 24) << (4 * q);
  }
  const uint32_t valid = (1u << L.cnt) - 1u;   // cnt <= 16
  return ~Z & valid;
}

// ------------------------------------------------------------- pass 1
// Plane histograms in shared memory hold two 16-bit counts per word: symbol
// s in the half (s & 1) of word s >> 1, the little-endian layout of
// PlaneStats::hist.
__device__ inline void count_symbol(uint32_t* ph, uint32_t s) { atomicAdd(&ph[s >> 1], 1u << ((s & 1u) << 4)); }

__device__ inline void record_run(uint32_t L, uint32_t* zeros, uint32_t* runs, uint32_t* extra) {
  if (L == 1) {
    atomicAdd(zeros, 1u);   // an isolated zero is the literal symbol 0
    return;
  }
  atomicAdd(runs, 1u);
  for (int w = 2; w <= kMaxW; ++w) {
    const uint32_t M = (1u << w) - 1u;
    if (M >= L) break;
    atomicAdd(&extra[w], (L + M - 1) / M - 1);
  }
}

// Every kept plane segment gets its zero-run statistics (PlaneStats: runs,
// extra[w], isolated zeros).  A segment of more than kRawMax symbols also
// gets its literal histogram, from which the Huffman pass finds its length;
// for a shorter one that pass sums the literal costs over its symbols (at
// most one 16-byte word per lane).
constexpr int kRawMax = 512;
__device__ inline bool plane_has_hist(uint32_t km, int n) { return __popc(km) * n > kRawMax; }

// Shared memory of one block's symbol pass: the literal histograms of the
// plane segments with one (kPlanes: slot pl for plane pl; one warp fills a
// plane's at a time), one slot, kRest, that every other segment adds to
// (the block's histogram is the sum over all slots), and every plane's
// zero-run statistics.
template <bool kPlanes>
struct SymShared {
  static constexpr int kRest = kPlanes ? kMaxD : 0;
  uint32_t ph[kRest + 1][128];
  uint32_t pextra[kMaxD][kMaxW + 1];
  uint32_t pruns[kMaxD], pzero[kMaxD];
  uint32_t orv[3], neg[3];
  uint32_t km[32];
  int64_t poff[32];
};

// Symbol pass of block bi by threads tid = 0 .. nthr-1 (whole warps; sync()
// synchronises exactly them): bit depth d, removed planes, the kept
// symbols written once to the block's symbol region, then its histogram and
// zero runs (BlockStats) and those of every kept plane segment (PlaneStats;
// the histogram part only for segments of more than kRawMax symbols, which
// need kPlanes).
template <bool kPlanes, class Sync>
__device__ inline void enc_symbols_block(int64_t bi, const BlockDev* __restrict__ blocks, const uint8_t* __restrict__ coef,
                                         uint8_t* __restrict__ sym, BlockStats* __restrict__ stats, PlaneStats* __restrict__ pst,
                                         int* __restrict__ status, SymShared<kPlanes>& SH, int tid, int nthr, Sync sync) {
  constexpr int kRest = SymShared<kPlanes>::kRest;
  // a launch without plane statistics must only meet blocks that need none
  if (!kPlanes && tid == 0 && blocks[bi].p * (blocks[bi].w * blocks[bi].h / 8) > kRawMax) set_status(status, kStInternal);
  const BlockDev b = blocks[bi];
  const int n = b.w * b.h / 8, na = b.p * n;
  AreaMap am;
  am.init(b.w, b.h);
  const CoefRef cf{coef + b.coef, b.coef16};
  const int lane = tid & 31, wid = tid >> 5, nw = nthr >> 5;
  if (tid < 3) { SH.orv[tid] = 0; SH.neg[tid] = 0; }
  sync();
  // int16 blocks whose type rows hold a multiple of 4 areas go 4 consecutive areas (64 bytes) per thread
  const bool quads = b.coef16 && (n & 3) == 0;
  {
    uint32_t o[3] = {0, 0, 0}, ng[3] = {0, 0, 0};
    if (quads) {
      const uint4* q4 = reinterpret_cast<const uint4*>(coef + b.coef);
      for (int u = tid; u < (na >> 2); u += nthr) {
        uint4 v[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) v[i] = q4[4 * u + i];
        uint32_t x = 0, g = 0;
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          const uint32_t w[4] = {v[i].x, v[i].y, v[i].z, v[i].w};
#pragma unroll
          for (int k = 0; k < 4; ++k) {
            const int32_t lo = (int32_t)(int16_t)(w[k] & 0xffffu), hi = (int32_t)w[k] >> 16;
            x |= (uint32_t)abs(lo) | (uint32_t)abs(hi);
            g |= w[k] & 0x80008000u;
          }
        }
        const int t = (4 * u) / n;
        o[0] |= t == 0 ? x : 0u; o[1] |= t == 1 ? x : 0u; o[2] |= t == 2 ? x : 0u;
        const uint32_t gn = g ? 1u : 0u;
        ng[0] |= t == 0 ? gn : 0u; ng[1] |= t == 1 ? gn : 0u; ng[2] |= t == 2 ? gn : 0u;
      }
    } else {
      for (int a = tid; a < na; a += nthr) {
        int t, kk;
        am.split(a, &t, &kk);
        int32_t c[8];
        cf.load(a, c);
        uint32_t x = 0, g = 0;
#pragma unroll
        for (int e = 0; e < 8; ++e) {
          x |= (uint32_t)abs(c[e]);
          g |= (uint32_t)(c[e] < 0);
        }
        o[0] |= t == 0 ? x : 0u; o[1] |= t == 1 ? x : 0u; o[2] |= t == 2 ? x : 0u;
        ng[0] |= t == 0 ? g : 0u; ng[1] |= t == 1 ? g : 0u; ng[2] |= t == 2 ? g : 0u;
      }
    }
    for (int t = 0; t < 3; ++t) {
      const uint32_t ro = __reduce_or_sync(0xffffffffu, o[t]);
      const uint32_t rn = __reduce_or_sync(0xffffffffu, ng[t]);
      if (lane == 0) {
        if (ro) atomicOr(&SH.orv[t], ro);
        if (rn) atomicOr(&SH.neg[t], rn);
      }
    }
  }
  sync();
  const uint32_t all_or = SH.orv[0] | SH.orv[1] | SH.orv[2];
  const int d = 1 + (all_or ? bitlen_u32(all_or) : 0);
  uint32_t removed[3];
#pragma unroll
  for (int t = 0; t < 3; ++t) {
    uint32_t r = 0;
    for (int pl = 0; pl < d; ++pl) {
      const bool empty = t >= b.p || (pl == 0 ? SH.neg[t] == 0 : ((SH.orv[t] >> (d - 1 - pl)) & 1u) == 0);
      if (empty) r |= 1u << pl;
    }
    removed[t] = r;
  }
  if (d > b.dmax) {
    // only samples above the stated bit depth get here: record an empty block
    // (every plane removed, no symbols) so that the later passes stay within
    // the block's buffers, and report the input error
    BlockStats* st = stats + bi;
    for (int i = tid; i < 256; i += nthr) st->hist[i] = 0;
    if (tid <= kMaxW) st->extra[tid] = 0;
    if (tid == 0) {
      st->n_runs = 0;
      st->n_sym = 0;
      st->removed[0] = st->removed[1] = st->removed[2] = 1u;
      st->d = 1;
      set_status(status, kStRange);
    }
    return;
  }
  uint32_t n_sym = 0;
  {
    int64_t off = 0;
    for (int pl = 0; pl < d; ++pl) {
      const uint32_t km = kept_types(removed, b.p, pl);
      if (tid == 0) { SH.km[pl] = km; SH.poff[pl] = off; }
      off += km ? region16(km, n) : 0;
      n_sym += (uint32_t)__popc(km) * n;
    }
  }
  // slots 0 .. d-1 (kPlanes) and kRest
  const int nslot = kPlanes ? d + 1 : 1;
  for (int i = tid; i < nslot * 128; i += nthr) {
    const int k = i >> 7;
    SH.ph[k == nslot - 1 ? kRest : k][i & 127] = 0;
  }
  for (int i = tid; i < d * (kMaxW + 1); i += nthr) SH.pextra[i / (kMaxW + 1)][i % (kMaxW + 1)] = 0;
  if (tid < d) { SH.pruns[tid] = 0; SH.pzero[tid] = 0; }
  sync();
  // symbols of every kept (plane, type), written once
  uint8_t* S = sym + b.sym;
  if (quads) {
    // four areas per thread: one word of four symbols per kept plane
    const uint4* q4 = reinterpret_cast<const uint4*>(coef + b.coef);
    for (int u = tid; u < (na >> 2); u += nthr) {
      const int t = (4 * u) / n, k0 = 4 * u - t * n;
      uint4 v[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) v[i] = q4[4 * u + i];
      uint32_t negw = 0, mp[4][4];
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const uint32_t w[4] = {v[i].x, v[i].y, v[i].z, v[i].w};
        int32_t c[8];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          c[2 * k] = (int32_t)(int16_t)(w[k] & 0xffffu);
          c[2 * k + 1] = (int32_t)w[k] >> 16;
        }
        uint32_t negm = 0;
#pragma unroll
        for (int e = 0; e < 8; ++e) negm |= (uint32_t)(c[e] < 0) << e;
        negw |= negm << (8 * i);
        // magnitudes packed in pairs (e, e + 4) so one shift serves both rows of the area
        mp[i][0] = (uint32_t)abs(c[0]) | ((uint32_t)abs(c[4]) << 16);
        mp[i][1] = (uint32_t)abs(c[1]) | ((uint32_t)abs(c[5]) << 16);
        mp[i][2] = (uint32_t)abs(c[2]) | ((uint32_t)abs(c[6]) << 16);
        mp[i][3] = (uint32_t)abs(c[3]) | ((uint32_t)abs(c[7]) << 16);
      }
      for (int pl = 0; pl < d; ++pl) {
        const uint32_t km = SH.km[pl];
        if (!((km >> t) & 1u)) continue;
        uint32_t sw;
        if (pl == 0) {
          sw = negw;
        } else {
          const int sh = d - 1 - pl;
          sw = 0;
#pragma unroll
          for (int i = 0; i < 4; ++i) {
            const uint32_t x = ((mp[i][0] >> sh) & 0x10001u) | (((mp[i][1] >> sh) & 0x10001u) << 1) |
                               (((mp[i][2] >> sh) & 0x10001u) << 2) | (((mp[i][3] >> sh) & 0x10001u) << 3);
            sw |= ((x & 0xfu) | ((x >> 12) & 0xf0u)) << (8 * i);
          }
        }
        const int ki = __popc(km & ((1u << t) - 1u));
        // plane rows start 16-byte aligned and n, k0 are multiples of 4: an aligned word
        *reinterpret_cast<uint32_t*>(S + SH.poff[pl] + (int64_t)ki * n + k0) = sw;
      }
    }
  } else
  for (int a = tid; a < na; a += nthr) {
    int t, k;
    am.split(a, &t, &k);
    int32_t c[8];
    cf.load(a, c);
    uint32_t negm = 0, m01 = 0, m23 = 0, m45 = 0, m67 = 0;
#pragma unroll
    for (int e = 0; e < 8; ++e) negm |= (uint32_t)(c[e] < 0) << e;
    // magnitudes packed in pairs (e, e + 4) so one shift serves both rows of the area
    m01 = (uint32_t)abs(c[0]) | ((uint32_t)abs(c[4]) << 16);
    m23 = (uint32_t)abs(c[1]) | ((uint32_t)abs(c[5]) << 16);
    m45 = (uint32_t)abs(c[2]) | ((uint32_t)abs(c[6]) << 16);
    m67 = (uint32_t)abs(c[3]) | ((uint32_t)abs(c[7]) << 16);
    const bool wide = !b.coef16;
    for (int pl = 0; pl < d; ++pl) {
      const uint32_t km = SH.km[pl];
      if (!((km >> t) & 1u)) continue;
      uint32_t s;
      if (pl == 0) {
        s = negm;
      } else {
        const int sh = d - 1 - pl;
        if (!wide) {
          const uint32_t x = ((m01 >> sh) & 0x10001u) | (((m23 >> sh) & 0x10001u) << 1) | (((m45 >> sh) & 0x10001u) << 2) |
                             (((m67 >> sh) & 0x10001u) << 3);
          s = (x & 0xfu) | ((x >> 12) & 0xf0u);
        } else {
          s = 0;
#pragma unroll
          for (int e = 0; e < 8; ++e) s |= (((uint32_t)abs(c[e]) >> sh) & 1u) << e;
        }
      }
      const int ki = __popc(km & ((1u << t) - 1u));
      S[SH.poff[pl] + (int64_t)ki * n + k] = (uint8_t)s;
    }
  }
  sync();
  // histogram and zero runs, one warp per plane segment
  for (int pl = wid; pl < d; pl += nw) {
    const uint32_t km = SH.km[pl];
    if (!km) continue;
    const int len = __popc(km) * n;
    const uint8_t* seg = S + SH.poff[pl];
    uint32_t* ph = SH.ph[kPlanes && plane_has_hist(km, n) ? pl : kRest];
    uint32_t* pextra = SH.pextra[pl];
    uint32_t* pruns = &SH.pruns[pl];
    uint32_t* pzero = &SH.pzero[pl];
    uint32_t carry = kAllZero;
    for (int base = 0; base < len; base += 512) {
      const LaneSyms L = load_lane(seg, len, base);
      const uint32_t NZ = nonzero_mask(L);
      const uint32_t Z = ~NZ & ((1u << L.cnt) - 1u);   // the lane's zero symbols
      const bool seen = NZ != 0;
      uint32_t lz = 0, zeros = 0;
      if (seen) {
        for (uint32_t m = NZ; m; m &= m - 1u) count_symbol(ph, L.at(__ffs(m) - 1));
        const int first = __ffs(NZ) - 1, last = 31 - __clz(NZ);
        lz = (uint32_t)first;
        zeros = (uint32_t)(L.cnt - 1 - last);
        // zero runs between the lane's first and last nonzero symbols
        const uint32_t Zi = Z & ((last >= 31 ? 0xffffffffu : (2u << last) - 1u) & ~((2u << first) - 1u));
        for (uint32_t st = Zi & ~(Zi << 1); st; st &= st - 1u) {
          const int s0 = __ffs(st) - 1;
          record_run((uint32_t)(__ffs(~(Zi >> s0)) - 1), pzero, pruns, pextra);
        }
      }
      const uint32_t elem = seen ? zeros : (kAllZero | (uint32_t)L.cnt);
      uint32_t incl, tot;
      const uint32_t ex = warp_carry_exclusive(elem, &incl, &tot);
      const uint32_t cin = carry_combine(carry, ex) & ~kAllZero;
      if (seen && cin + lz > 0) record_run(cin + lz, pzero, pruns, pextra);
      carry = carry_combine(carry, tot);
    }
    const uint32_t fin = carry & ~kAllZero;
    if (lane == 0 && fin) record_run(fin, pzero, pruns, pextra);
  }
  sync();
  // the plane statistics (35 16-byte words; without a histogram only the
  // last 3), then the block's totals
  uint4* dst = reinterpret_cast<uint4*>(pst + b.pst);
  const int per = kPlanes ? 35 : 3;
  for (int i = tid; i < d * per; i += nthr) {
    const int pl = i / per, q = i - pl * per + (35 - per);
    const uint32_t km = SH.km[pl];
    if (!km || (q < 32 && !plane_has_hist(km, n))) continue;
    uint4 v;
    if (q < 32) {
      v = *reinterpret_cast<const uint4*>(&SH.ph[pl][4 * q]);
      if (q == 0) v.x |= SH.pzero[pl];   // symbol 0: the isolated zeros
    } else {
      // 16-bit extra[0..18], runs, isolated zeros, then zero padding:
      // halves 8 (q - 32) .. 8 (q - 32) + 7 of the 24 in words 32..34
      uint32_t h[4];
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const int e0 = 8 * (q - 32) + 2 * k, e1 = e0 + 1;
        const uint32_t lo = e0 <= kMaxW ? SH.pextra[pl][e0] : (e0 == kMaxW + 1 ? SH.pruns[pl] : (e0 == kMaxW + 2 ? SH.pzero[pl] : 0u));
        const uint32_t hi = e1 <= kMaxW ? SH.pextra[pl][e1] : (e1 == kMaxW + 1 ? SH.pruns[pl] : (e1 == kMaxW + 2 ? SH.pzero[pl] : 0u));
        h[k] = lo | (hi << 16);
      }
      v = make_uint4(h[0], h[1], h[2], h[3]);
    }
    dst[(int64_t)pl * 35 + q] = v;
  }
  BlockStats* st = stats + bi;
  for (int i = tid; i < 256; i += nthr) {
    uint32_t c = (SH.ph[kRest][i >> 1] >> ((i & 1) << 4)) & 0xffffu;
    for (int pl = 0; kPlanes && pl < d; ++pl) c += (SH.ph[pl][i >> 1] >> ((i & 1) << 4)) & 0xffffu;
    if (i == 0)
      for (int pl = 0; pl < d; ++pl) c += SH.pzero[pl];
    st->hist[i] = c;
  }
  if (tid <= kMaxW) {
    uint32_t c = 0;
    for (int pl = 0; pl < d; ++pl) c += SH.pextra[pl][tid];
    st->extra[tid] = c;
  }
  if (tid == 0) {
    uint32_t r = 0;
    for (int pl = 0; pl < d; ++pl) r += SH.pruns[pl];
    st->n_runs = r;
    st->n_sym = n_sym;
    st->removed[0] = removed[0]; st->removed[1] = removed[1]; st->removed[2] = removed[2];
    st->d = d;
  }
}


// ------------------------------------------------- token costs and writer
// Code of a block: codewords and lengths by symbol, and the bits of a
// nonzero literal (lit[s] = len[s], plus w for C_zr's zero counter;
// lit[0] = 0: a zero symbol is always part of a run).
struct CodeTab {
  const uint32_t* code;
  const uint8_t* len;
  const uint8_t* lit;
  int czr, wbits;
  uint32_t M;
};

__device__ inline uint32_t run_bits(const CodeTab& ct, uint32_t L) {
  if (L == 1) return ct.len[0];
  if (ct.M == 0) return 0;
  const uint32_t tokens = L <= ct.M ? 1u : (L + ct.M - 1) / ct.M;
  return tokens * (uint32_t)(ct.len[ct.czr] + ct.wbits);
}

// MSB-first writer of one lane's contiguous bit range straight into the
// stream (32-bit words, big endian).  Words strictly inside the range are
// stored; the first and last (shared with neighbouring ranges) are OR-ed
// into the zero-initialised stream.
struct LaneWriter {
  uint32_t* out;
  int64_t w0, wcur;
  uint64_t acc;
  int nacc;
  __device__ void begin(uint32_t* o, int64_t bitpos) {
    out = o;
    wcur = w0 = bitpos >> 5;
    acc = 0;
    nacc = (int)(bitpos & 31);
  }
  __device__ void word(uint32_t x) {
    const uint32_t be = __byte_perm(x, 0, 0x0123);
    if (wcur == w0) atomicOr(&out[wcur], be);
    else out[wcur] = be;
    ++wcur;
  }
  // v < 2^nb (codewords and counters have no bits above their length),
  // 0 <= nb <= 32; the two shifts place it at bit 64 - nacc - nb.
  __device__ void put(uint32_t v, int nb) {
    acc |= ((uint64_t)v << (32 - nb)) << (32 - nacc);
    nacc += nb;
    if (nacc >= 32) {
      word((uint32_t)(acc >> 32));
      acc <<= 32;
      nacc -= 32;
    }
  }
  __device__ void end() {
    if (nacc > 0) atomicOr(&out[wcur], __byte_perm((uint32_t)(acc >> 32), 0, 0x0123));
  }
};

__device__ inline void put_run(const CodeTab& ct, LaneWriter& W, uint32_t L) {
  if (L == 1) {
    W.put(ct.code[0], ct.len[0]);
    return;
  }
  if (ct.M == 0) return;   // counter width is always >= 2
  const int lc = ct.len[ct.czr];
  const uint32_t cz = ct.code[ct.czr];
  while (L > 0) {
    const uint32_t k = L >= ct.M ? ct.M : L;
    W.put(cz, lc);
    W.put(k, ct.wbits);
    L -= k;
  }
}

__device__ inline void put_literal(const CodeTab& ct, LaneWriter& W, uint32_t s) {
  W.put(ct.code[s], ct.len[s]);
  if ((int)s == ct.czr) W.put(0, ct.wbits);   // counter 0: a literal C_zr
}

// One warp walks plane segment `seg` (len symbols) in chunks of 512,
// writes its tokens from absolute bit position `pos` and returns its bit
// length.  A chunk that would end beyond `limit` bits (the length the
// statistics gave) is not written: the walk stops there and returns more
// than `limit`, so nothing is written outside the segment's span.
__device__ uint64_t warp_segment(const uint8_t* seg, int len, const CodeTab& ct, uint32_t* out, int64_t pos, uint64_t limit) {
  const int lane = threadIdx.x & 31;
  uint32_t carry = kAllZero;
  uint64_t total = 0;
  for (int base = 0; base < len; base += 512) {
    const LaneSyms L = load_lane(seg, len, base);
    // nonzero symbols of the lane as a bit mask: the loops visit only those;
    // the zeros between two of them form one run
    const uint32_t NZ = nonzero_mask(L);
    const bool seen = NZ != 0;
    uint32_t zeros = 0, lz = 0, bits = 0;
    if (seen) {
      const int first = __ffs(NZ) - 1, last = 31 - __clz(NZ);
      lz = (uint32_t)first;
      zeros = (uint32_t)(L.cnt - 1 - last);
      // the literals' bits: lit[] over all 16 positions (zero symbols cost
      // 0 there; positions past the segment are cleared first)
      uint32_t wv[4] = {L.w[0], L.w[1], L.w[2], L.w[3]};
      if (L.cnt < 16) {
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const int nb = min(max(L.cnt - 4 * q, 0), 4);
          wv[q] &= nb >= 4 ? 0xffffffffu : ((1u << (8 * nb)) - 1u);
        }
      }
#pragma unroll
      for (int k = 0; k < 16; ++k) bits += ct.lit[__byte_perm(wv[k >> 2], 0, 0x4440 | (k & 3))];
      // the zero runs between the lane's first and last nonzero symbols
      const uint32_t Zi = ~NZ & ((2u << last) - 1u) & ~((2u << first) - 1u);
      for (uint32_t st = Zi & ~(Zi << 1); st; st &= st - 1u) {
        const int s0 = __ffs(st) - 1;
        bits += run_bits(ct, (uint32_t)(__ffs(~(Zi >> s0)) - 1));
      }
    }
    const uint32_t elem = seen ? zeros : (kAllZero | (uint32_t)L.cnt);
    uint32_t incl, tot;
    const uint32_t ex = warp_carry_exclusive(elem, &incl, &tot);
    const uint32_t cin = carry_combine(carry, ex) & ~kAllZero;
    const uint32_t lead = seen ? cin + lz : 0;
    if (lead) bits += run_bits(ct, lead);
    // the lane holding the segment's last symbol closes the final run
    const bool last_lane = base + 512 >= len && lane == (len - 1 - base) / 16;
    const uint32_t fin = last_lane ? (carry_combine(carry, incl) & ~kAllZero) : 0;
    if (fin) bits += run_bits(ct, fin);
    // bit offsets of the lanes within the chunk
    uint32_t x = bits;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += y;
    }
    const uint32_t chunk_bits = __shfl_sync(0xffffffffu, x, 31);
    if (total + chunk_bits > limit) return total + chunk_bits;   // warp-uniform
    if (bits) {
      LaneWriter W;
      W.begin(out, pos + (int64_t)total + (x - bits));
      if (lead) put_run(ct, W, lead);
      int prev = __ffs(NZ) - 1;
      for (uint32_t m = NZ; m; m &= m - 1u) {
        const int k = __ffs(m) - 1;
        if (k - prev > 1) put_run(ct, W, (uint32_t)(k - prev - 1));
        put_literal(ct, W, L.at(k));
        prev = k;
      }
      if (fin) put_run(ct, W, fin);
      W.end();
    }
    total += chunk_bits;
    carry = carry_combine(carry, tot);
  }
  return total;
}

// Symbol offset of plane pl inside a block's region.
__device__ inline int64_t plane_offset(const uint32_t* removed, int p, int n, int pl) {
  int64_t off = 0;
  for (int q = 0; q < pl; ++q) {
    const uint32_t km = kept_types(removed, p, q);
    if (km) off += region16(km, n);
  }
  return off;
}


// ------------------------------------------------------------- pass 2
// Per-block layout: seektable width t, header bits and the exact bit length
// of every plane segment (0 for a removed plane), found by the Huffman pass
// from the plane statistics.
struct BlockHdr {
  int32_t t, pad;
  int64_t hdr_bits;
  uint32_t seglen[32];
};

// Two-queue Huffman construction (one warp per block): leaves with f > 0
// sorted ascending by (f, symbol) (warp bitonic sort in registers); each
// merge takes the lighter queue front twice, the leaf queue first on equal
// weight; the first taken becomes the left child (bit 0).
constexpr int kHuffWarps = 8;
constexpr uint32_t kInf = 0xffffffffu;

struct __align__(16) HuffWarp {
  uint32_t f[256];        // frequencies
  uint32_t leaf[256];     // sorted leaves: (f << 8) | symbol
  uint32_t iw[256];       // internal node weights in creation order
  uint16_t parent[512];   // parent node id | 0x8000 for a right child
  uint32_t tree[81];
};

// Sorts 8 keys per lane (element lane*8 + r) ascending across the warp.
__device__ inline void warp_bitonic_256(uint32_t (&k)[8]) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int size = 2; size <= 256; size <<= 1) {
#pragma unroll
    for (int stride = size >> 1; stride > 0; stride >>= 1) {
      if (stride >= 8) {
        const int lstride = stride >> 3;
#pragma unroll
        for (int r = 0; r < 8; ++r) {
          const int i = lane * 8 + r;
          const bool up = (i & size) == 0;
          const uint32_t other = __shfl_xor_sync(0xffffffffu, k[r], lstride);
          const bool lower = (lane & lstride) == 0;
          const uint32_t mn = min(k[r], other), mx = max(k[r], other);
          k[r] = (lower == up) ? mn : mx;
        }
      } else {
#pragma unroll
        for (int r = 0; r < 8; ++r) {
          const int pr = r ^ stride;
          if (pr > r) {
            const int i = lane * 8 + r;
            const bool up = (i & size) == 0;
            const uint32_t a = k[r], b = k[pr];
            k[r] = up ? min(a, b) : max(a, b);
            k[pr] = up ? max(a, b) : min(a, b);
          }
        }
      }
    }
  }
}

// Sorted leaves of the frequencies in H.f, by one warp: H.leaf holds
// (f << 8) | symbol ascending for every symbol with f > 0 (then kInf);
// returns their count.
__device__ inline int huff_leaves_warp(HuffWarp& H) {
  const int lane = threadIdx.x & 31;
  uint32_t k[8];
#pragma unroll
  for (int r = 0; r < 8; ++r) {
    const int sym = lane * 8 + r;
    const uint32_t fr = H.f[sym];
    k[r] = fr ? ((fr << 8) | (uint32_t)sym) : kInf;
  }
  // symbols with a nonzero count
  int present = 0;
#pragma unroll
  for (int r = 0; r < 8; ++r) present += __popc(__ballot_sync(0xffffffffu, k[r] != kInf));
  if (present <= 32) {
    // small alphabet (the coarse levels' blocks): gather the keys, one per
    // lane, and sort 32 instead of 256
    int base = 0;
#pragma unroll
    for (int r = 0; r < 8; ++r) {
      const uint32_t m = __ballot_sync(0xffffffffu, k[r] != kInf);
      if (k[r] != kInf) H.leaf[base + __popc(m & ((1u << lane) - 1u))] = k[r];
      base += __popc(m);
    }
    __syncwarp();
    uint32_t x = lane < present ? H.leaf[lane] : kInf;
#pragma unroll
    for (int size = 2; size <= 32; size <<= 1) {
#pragma unroll
      for (int stride = size >> 1; stride > 0; stride >>= 1) {
        const uint32_t other = __shfl_xor_sync(0xffffffffu, x, stride);
        const bool up = (lane & size) == 0, lower = (lane & stride) == 0;
        x = (lower == up) ? min(x, other) : max(x, other);
      }
    }
    __syncwarp();
    H.leaf[lane] = x;   // key of rank `lane` (lanes >= present: none)
  } else {
    warp_bitonic_256(k);
#pragma unroll
    for (int r = 0; r < 8; ++r) H.leaf[lane * 8 + r] = k[r];
  }
  __syncwarp();
  return present;
}

// Two-queue merge of the nl >= 2 sorted leaves of H by ONE thread: each
// step takes the lighter queue front twice, the leaf queue first on equal
// weight, and the first taken becomes the left child.  Writes the internal
// weights in creation order (H.iw) and the parent links (H.parent); node
// nl + i is the i-th internal node, the root 2 nl - 2.  The refills are
// loads under a condition and selects, not branches: the eight threads of a
// warp that run it run different blocks' merges side by side.
__device__ inline void huff_merge_thread(HuffWarp& H, int nl) {
  int qa = 0, qb = 0;
  uint32_t wl = H.leaf[0] >> 8, wi = kInf;
  for (int ni = 0; ni < nl - 1; ++ni) {
    const bool ta = wl <= wi;
    const int a = ta ? qa : nl + qb;
    const uint32_t wa = ta ? wl : wi;
    qa += ta;
    qb += !ta;
    uint32_t x = kInf, y = kInf;
    if (qa < nl) x = H.leaf[qa] >> 8;
    if (qb < ni) y = H.iw[qb];
    wl = ta ? x : wl;
    wi = ta ? wi : y;
    const bool tb = wl <= wi;
    const int b = tb ? qa : nl + qb;
    const uint32_t wb = tb ? wl : wi;
    qa += tb;
    qb += !tb;
    x = kInf;
    y = kInf;
    if (qa < nl) x = H.leaf[qa] >> 8;
    if (qb < ni) y = H.iw[qb];
    wl = tb ? x : wl;
    wi = tb ? wi : y;
    const uint32_t wn = wa + wb;
    H.iw[ni] = wn;
    H.parent[a] = (uint16_t)(nl + ni);
    H.parent[b] = (uint16_t)((nl + ni) | 0x8000);
    if (qb == ni) wi = wn;   // the internal queue was empty: the new node is its front
  }
}

// The merges of a CTA's blocks: thread j of warp 0 merges the leaves of
// warp j's block (s_nl[j] of them; fewer than 2: nothing to merge).
// Called by every thread of the CTA between two barriers.
__device__ inline void huff_merge_cta(HuffWarp* HW, const int* s_nl) {
  const int t = threadIdx.x;
  if (t < kHuffWarps && s_nl[t] > 1) huff_merge_thread(HW[t], s_nl[t]);
}

// Huffman code of block bi (C_zr, counter width w by Eq. 3, provisional
// and final trees, codes, preorder tree bits): warp w of the CTA takes
// block bi (-1: none) with HW[w] its shared-memory workspace; the CTA's
// tree merges run side by side (huff_merge_cta).  Every thread of the CTA
// calls it; sync() is the CTA barrier.
template <class Sync>
__device__ inline void cta_block_huffman(int64_t bi, const BlockDev* __restrict__ blocks, const BlockStats* __restrict__ stats,
                                         BlockCode* __restrict__ codes, HuffWarp* HW, int* s_nl, Sync sync) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  HuffWarp& H = HW[wid];
  // a block with no kept symbol is coded by its header alone
  bool active = bi >= 0;
  const BlockStats* st = active ? stats + bi : stats;
  BlockCode* bc = active ? codes + bi : codes;
  int d = 0, p = 0;
  uint32_t n_sym = 0;
  if (active) {
    const BlockDev b = blocks[bi];
    d = st->d;
    p = b.p;
    n_sym = st->n_sym;
    if (lane == 0) {
      bc->d = d;
      bc->p = p;
      for (int t = 0; t < 3; ++t) bc->removed[t] = st->removed[t];
      bc->t0 = bitlen_u32((uint32_t)(p * b.w * b.h / 8)) - 1 + 5;
    }
    if (n_sym == 0) {
      if (lane == 0) {
        bc->any_kept = 0;
        bc->token_bits = 0;
        bc->tree_bits = 0;
        bc->czr = 0;
        bc->wbits = 0;
      }
      active = false;
    }
  }
  // C_zr: least frequent of 1..255, smallest on ties
  int czr = 0, nl = 0;
  uint32_t lit_czr = 0;
  if (active) {
    uint32_t best = kInf;
    for (int s = lane; s < 256; s += 32) {
      const uint32_t fr = st->hist[s];
      H.f[s] = fr;
      if (s >= 1) best = min(best, (fr << 8) | (uint32_t)s);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) best = min(best, __shfl_xor_sync(0xffffffffu, best, o));
    czr = (int)(best & 0xffu);
    lit_czr = best >> 8;
    __syncwarp();
    // provisional code: every run counts once for C_zr; l = C_zr's code length
    if (lane == 0) H.f[czr] = lit_czr + st->n_runs;
    __syncwarp();
    nl = huff_leaves_warp(H);
  }
  // The provisional tree is built with its parent links: when the chosen
  // width needs no extra run tokens, the final counts equal these and the
  // tree is reused as is.
  if (lane == 0) s_nl[wid] = active ? nl : 0;
  sync();
  huff_merge_cta(HW, s_nl);
  sync();
  int wbest = 2;
  bool rebuild = false;
  if (active) {
    const int root = nl <= 1 ? 0 : 2 * nl - 2;
    int l = 0, io = 0;   // C_zr's code length and the place of its leaf in the sorted order
    if (H.f[czr] > 0 && nl > 1) {
      int leaf = -1;
#pragma unroll
      for (int m = 0; m < 8; ++m) {
        const int i = lane + 32 * m;
        if (i < nl && (int)(H.leaf[i] & 0xffu) == czr) leaf = i;
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) leaf = max(leaf, __shfl_xor_sync(0xffffffffu, leaf, o));
      int dep = 0;
      for (int v = leaf; v != root && dep < 64; ++dep) v = H.parent[v] & 0x7fff;   // the leaf's depth
      l = dep;
      io = leaf;
    }
    // Eq. 3 (reading): w minimises (w + l) * (#C_zr tokens at width w) over [2, b]
    int bmax = n_sym > 1 ? bitlen_u32(n_sym - 1) : 0;
    if (bmax < 2) bmax = 2;
    uint64_t bestc = ~0ull;
    for (int w = 2; w <= bmax; ++w) {
      const uint64_t pairs = (uint64_t)lit_czr + st->n_runs + st->extra[w];
      const uint64_t cost = (uint64_t)(w + l) * pairs;
      if (cost < bestc) { bestc = cost; wbest = w; }
    }
    if (st->extra[wbest] != 0) {
      // C_zr's count grows (it had runs, so it is a leaf: the only one when
      // nl = 1): the final tree's sorted leaves are the provisional ones with
      // C_zr's key moved right to its new place, the keys between shifting
      // left by one
      const uint32_t fz = lit_czr + st->n_runs + st->extra[wbest];
      const uint32_t knew = (fz << 8) | (uint32_t)czr;
      int below = 0;   // keys below the new one, the old C_zr key among them
#pragma unroll
      for (int m = 0; m < 8; ++m) {
        const int i = lane + 32 * m;
        below += i < nl && H.leaf[i] < knew;
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) below += __shfl_xor_sync(0xffffffffu, below, o);
      const int jn = below - 1;
      // two halves of 128 places: each reads only places the other half has
      // not written yet (the first writes below 128, the second reads above)
#pragma unroll
      for (int half = 0; half < 2; ++half) {
        uint32_t nxt[4];
#pragma unroll
        for (int m = 0; m < 4; ++m) {
          const int i = lane + 32 * (4 * half + m);
          nxt[m] = i >= io && i < jn ? H.leaf[i + 1] : knew;
        }
        __syncwarp();
#pragma unroll
        for (int m = 0; m < 4; ++m) {
          const int i = lane + 32 * (4 * half + m);
          if (i >= io && i <= jn) H.leaf[i] = nxt[m];
        }
        __syncwarp();
      }
      if (lane == 0) H.f[czr] = fz;
      __syncwarp();
      rebuild = true;
    }
  }
  if (lane == 0) s_nl[wid] = rebuild ? nl : 0;
  sync();
  huff_merge_cta(HW, s_nl);
  sync();
  if (!active) return;
  const int root = nl <= 1 ? 0 : 2 * nl - 2;
  // codes: every leaf walks up to the root; a lane walks its (up to) 8 leaves together
  for (int s2 = lane; s2 < 256; s2 += 32) { bc->code[s2] = 0; bc->len[s2] = 0; }
  for (int k = lane; k < 81; k += 32) H.tree[k] = 0;
  int v[8], len[8];
  uint32_t code[8];
#pragma unroll
  for (int m = 0; m < 8; ++m) {
    v[m] = lane + 32 * m;
    code[m] = 0;
    len[m] = 0;
  }
  for (int depth = 0; depth < 40; ++depth) {
    bool more = false;
#pragma unroll
    for (int m = 0; m < 8; ++m) {
      if (lane + 32 * m < nl && v[m] != root) {
        const uint32_t p = H.parent[v[m]];
        code[m] |= (p >> 15) << len[m];
        ++len[m];
        v[m] = p & 0x7fff;
        more = true;
      }
    }
    if (!__any_sync(0xffffffffu, more)) break;
  }
  // Preorder tree (Fig. 3: 0 = internal node, 1 + 8-bit symbol = leaf).  Leaves
  // appear in preorder in the lexicographic order of their codes, and the
  // record of a leaf with code c of length l and rank r in that order starts
  // at bit l + 10 r - popcount(c): its l ancestors' 0 bits, plus, for each
  // right turn on its path, the left sibling subtree (10 bits per leaf less
  // one).  Ranks by counting smaller left-aligned codes.
  uint32_t* K = H.iw;   // the merge's weights are no longer needed
  uint64_t tb = 0;
#pragma unroll
  for (int m = 0; m < 8; ++m) {
    const int i = lane + 32 * m;
    if (i < nl) {
      K[i] = len[m] ? code[m] << (31 - len[m]) : 0u;   // codes are at most 31 bits (Fibonacci bound)
      const int sym = (int)(H.leaf[i] & 0xffu);
      bc->code[sym] = code[m];
      bc->len[sym] = (uint8_t)len[m];
      tb += (uint64_t)H.f[sym] * len[m];
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) tb += __shfl_xor_sync(0xffffffffu, tb, o);
  __syncwarp();
  int rank[8];
#pragma unroll
  for (int m = 0; m < 8; ++m) rank[m] = 0;
  uint32_t key[8];
#pragma unroll
  for (int m = 0; m < 8; ++m) key[m] = lane + 32 * m < nl ? K[lane + 32 * m] : 0u;
  if (lane < 3 && nl + lane < ((nl + 3) & ~3)) K[nl + lane] = kInf;   // pad to whole words of four: never smaller
  __syncwarp();
  for (int j = 0; j < nl; j += 4) {
    const uint4 kq = *reinterpret_cast<const uint4*>(K + j);
#pragma unroll
    for (int m = 0; m < 8; ++m) rank[m] += (kq.x < key[m]) + (kq.y < key[m]) + (kq.z < key[m]) + (kq.w < key[m]);
  }
#pragma unroll
  for (int m = 0; m < 8; ++m) {
    const int i = lane + 32 * m;
    if (i < nl) {
      const int pos = len[m] + 10 * rank[m] - __popc(code[m]);
      const uint32_t val = 0x100u | (H.leaf[i] & 0xffu);
      const int wi = pos >> 5, off = pos & 31;
      const uint64_t vv = (uint64_t)val << (64 - off - 9);
      atomicOr(&H.tree[wi], (uint32_t)(vv >> 32));
      if ((uint32_t)vv) atomicOr(&H.tree[wi + 1], (uint32_t)vv);
    }
  }
  if (lane == 0) bc->tree_bits = 10 * nl - 1;
  __syncwarp();
  for (int k = lane; k < 80; k += 32) bc->tree[k] = H.tree[k];
  if (lane == 0) {
    bc->any_kept = 1;
    bc->czr = czr;
    bc->wbits = wbest;
    bc->token_bits = tb + (uint64_t)wbest * H.f[czr];
  }
}

// Layout of block bi by one warp (pass 2b): the exact bit length of every
// plane segment, the seektable width t, the header bits and the block's
// bytes in the stream (item_size; a tile's first block also carries the
// tile header).  s_len: 256 bytes of shared memory for the warp.
__device__ inline void enc_block_layout(int64_t bi, const TileDev* __restrict__ tiles, const BlockDev* __restrict__ blocks,
                                        const PlaneStats* __restrict__ pst, const uint8_t* __restrict__ sym,
                                        const BlockCode* __restrict__ codes, BlockHdr* __restrict__ hdrs,
                                        int64_t* __restrict__ item_size, int* __restrict__ status, uint8_t* s_len) {
  const int lane = threadIdx.x & 31;
  const BlockDev b = blocks[bi];
  const BlockCode& bc = codes[bi];
  BlockHdr& BH = hdrs[bi];
  const int d = bc.d, p = b.p;
  const TileDev& tile = tiles[b.tile];
  const int64_t extra_bytes = bi == tile.block_base ? 32 + 4 * (int64_t)tile.nb : 0;
  if (!bc.any_kept) {
    if (lane == 0) {
      BH.t = 0;
      BH.hdr_bits = 5 + (int64_t)p * d;
      item_size[bi] = (5 + (int64_t)p * d + 7) / 8 + extra_bytes;
    }
    return;
  }
  const int czr = bc.czr, wbest = bc.wbits;
  const uint2 lq = reinterpret_cast<const uint2*>(bc.len)[lane];
  reinterpret_cast<uint2*>(s_len)[lane] = lq;
  __syncwarp();
  // Plane segment lengths: a literal s costs len[s] bits, plus w for C_zr
  // (its zero counter); every zero-run token C_zr plus a w-bit counter; an
  // isolated zero is the literal 0.  Literals of a segment with a histogram:
  // lane k takes symbols 8k .. 8k + 7 of it; of a shorter segment: lane k
  // takes its symbols 16k .. 16k + 15.  Either is one 16-byte load per lane,
  // two planes' loads in flight.
  const int n = b.w * b.h / 8;
  uint32_t keptm = 0;
  for (int pl = 0; pl < d; ++pl)
    if (kept_types(bc.removed, p, pl)) keptm |= 1u << pl;
  if (lane == 0)
    for (int pl = 0; pl < d; ++pl)
      if (!((keptm >> pl) & 1u)) BH.seglen[pl] = 0;
  const uint32_t lczr = (uint32_t)s_len[czr] + (uint32_t)wbest;   // a run token, or a literal C_zr
  const uint32_t lzero = s_len[0];
  const PlaneStats* ps = pst + b.pst;
  const uint8_t* S = sym + b.sym;
  uint64_t sum = 0;
  uint32_t mx = 0;
  int64_t off = 0;   // symbol offset of the next kept plane
  uint32_t m = keptm;
  while (m) {
    int pls[2], cnt[2];
    uint4 q[2];
    uint32_t tok[2], zc[2];
#pragma unroll
    for (int k = 0; k < 2; ++k) {
      pls[k] = m ? __ffs(m) - 1 : -1;
      m &= m - 1u;
      cnt[k] = -1;   // a histogram
      q[k] = make_uint4(0, 0, 0, 0);
      tok[k] = zc[k] = 0;
      if (pls[k] >= 0) {   // warp-uniform
        const PlaneStats& P = ps[pls[k]];
        const uint32_t km = kept_types(bc.removed, p, pls[k]);
        if (plane_has_hist(km, n)) {
          q[k] = reinterpret_cast<const uint4*>(P.hist)[lane];
          zc[k] = P.hist[czr];
        } else {
          cnt[k] = max(0, min(16, __popc(km) * n - 16 * lane));
          if (cnt[k] > 0) q[k] = *reinterpret_cast<const uint4*>(S + off + 16 * lane);
          zc[k] = P.zeros;
        }
        tok[k] = (uint32_t)P.runs + P.extra[wbest];
        off += region16(km, n);
      }
    }
#pragma unroll
    for (int k = 0; k < 2; ++k) {
      if (pls[k] < 0) break;   // warp-uniform
      const uint4 h = q[k];
      uint32_t a;
      if (cnt[k] < 0) {
        a = (h.x & 0xffffu) * (lq.x & 0xffu) + (h.x >> 16) * ((lq.x >> 8) & 0xffu) + (h.y & 0xffffu) * ((lq.x >> 16) & 0xffu) +
            (h.y >> 16) * (lq.x >> 24) + (h.z & 0xffffu) * (lq.y & 0xffu) + (h.z >> 16) * ((lq.y >> 8) & 0xffu) +
            (h.w & 0xffffu) * ((lq.y >> 16) & 0xffu) + (h.w >> 16) * (lq.y >> 24);
      } else {
        LaneSyms L;
        L.w[0] = h.x; L.w[1] = h.y; L.w[2] = h.z; L.w[3] = h.w;
        L.cnt = cnt[k];
        a = 0;
        for (uint32_t nz = nonzero_mask(L); nz; nz &= nz - 1u) {
          const uint32_t s = L.at(__ffs(nz) - 1);
          a += (uint32_t)s_len[s] + ((int)s == czr ? (uint32_t)wbest : 0u);
        }
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
      // with a histogram, zc counts the C_zr literals (isolated zeros are in
      // it); without, the isolated zeros (the C_zr literals are in the sum)
      const uint32_t v = a + (cnt[k] < 0 ? zc[k] * (uint32_t)wbest : zc[k] * lzero) + tok[k] * lczr;
      if (lane == 0) BH.seglen[pls[k]] = v;
      sum += v;
      mx = max(mx, v);
    }
  }
  if (lane == 0) {
    // seektable width: t0, raised only when a segment length needs more bits
    const int t = max(bc.t0, mx ? bitlen_u32(mx) : 0);
    const int64_t hdr = 5 + (int64_t)p * d + 18 + (int64_t)d * t + bc.tree_bits;
    BH.t = t;
    BH.hdr_bits = hdr;
    item_size[bi] = (hdr + (int64_t)sum + 7) / 8 + extra_bytes;
    // the segments must add up to the bit count of the Huffman pass
    if (sum != bc.token_bits) set_status(status, kStInternal);
  }
}


constexpr int kEmitWarps = 8;
constexpr int kEncGroup = 16;
constexpr int kEncSmem = kEncGroup * (256 * 4 + 256 + 256) + kEncGroup * 32 * 2;

__device__ inline int64_t block_bit_start(const TileDev& t, const int64_t* final_pos, int64_t bi) {
  return 8 * (final_pos[bi] + (bi == t.block_base ? 32 + 4 * (int64_t)t.nb : 0));
}

// Group of kEncGroup level-sorted blocks: their code tables in shared
// memory and their (block, plane) segments listed plane-major.
struct EncGroup {
  uint32_t (*code)[256];
  uint8_t (*len)[256];
  uint8_t (*lit)[256];
  uint16_t* item;
  int nitem;
};

// Block i of a group: perm[g0 + i], or g0 + i without a permutation.
__device__ inline int64_t group_block(const int64_t* perm, int64_t g0, int i) { return perm ? perm[g0 + i] : g0 + i; }

// Loads the code tables of the ng (<= kEncGroup) blocks g0 .. of a group
// into shared memory (dyn) and lists their (block, plane) segments, by
// threads tid = 0 .. nthr-1 (sync() synchronises them).
template <class Sync>
__device__ void load_group(const int64_t* perm, int64_t g0, int ng, const BlockDev* blocks, const BlockCode* codes, uint8_t* dyn,
                           EncGroup& G, int* s_nitem, int tid, int nthr, Sync sync) {
  G.code = reinterpret_cast<uint32_t (*)[256]>(dyn);
  G.len = reinterpret_cast<uint8_t (*)[256]>(dyn + kEncGroup * 256 * 4);
  G.lit = reinterpret_cast<uint8_t (*)[256]>(dyn + kEncGroup * (256 * 4 + 256));
  G.item = reinterpret_cast<uint16_t*>(dyn + kEncGroup * (256 * 4 + 256 + 256));
  // code and length tables of the group's blocks, all copies in flight at
  // once: per block 64 16-byte words of codes and 16 of lengths (each also
  // gives 16 entries of lit[])
  for (int idx = tid; idx < ng * 80; idx += nthr) {
    const int j = idx / 80, q = idx - j * 80;
    const BlockCode& bc = codes[group_block(perm, g0, j)];
    if (!bc.any_kept) continue;
    if (q < 64) {
      reinterpret_cast<uint4*>(G.code[j])[q] = reinterpret_cast<const uint4*>(bc.code)[q];
    } else {
      uint4 v = reinterpret_cast<const uint4*>(bc.len)[q - 64];
      reinterpret_cast<uint4*>(G.len[j])[q - 64] = v;
      const int s0 = 16 * (q - 64), cz = bc.czr - s0;
      if (s0 == 0) v.x &= ~0xffu;   // symbol 0
      if (cz >= 0 && cz < 16) {     // C_zr: plus its counter (lengths stay below 256: no carry between bytes)
        const uint32_t add = (uint32_t)bc.wbits << (8 * (cz & 3));
        v.x += cz >> 2 == 0 ? add : 0u;
        v.y += cz >> 2 == 1 ? add : 0u;
        v.z += cz >> 2 == 2 ? add : 0u;
        v.w += cz >> 2 == 3 ? add : 0u;
      }
      reinterpret_cast<uint4*>(G.lit[j])[q - 64] = v;
    }
  }
  if (tid < 32) {
    const int j = tid;
    uint32_t planes = 0;
    if (j < ng) {
      const BlockCode& bc = codes[group_block(perm, g0, j)];
      if (bc.any_kept)
        for (int pl = 0; pl < bc.d; ++pl)
          if (kept_types(bc.removed, bc.p, pl)) planes |= 1u << pl;
    }
    int base = 0;
    for (int pl = 0; pl < 32; ++pl) {
      const uint32_t m = __ballot_sync(0xffffffffu, (planes >> pl) & 1u);
      if ((planes >> pl) & 1u) G.item[base + __popc(m & ((1u << j) - 1u))] = (uint16_t)((j << 5) | pl);
      base += __popc(m);
    }
    if (j == 0) *s_nitem = base;
  }
  sync();
  G.nitem = *s_nitem;
}

// The stream is written in whole 32-bit words: it needs its size rounded
// up to a multiple of 4 bytes of capacity.
__device__ inline int64_t needed_capacity(int64_t total) { return (total + 3) & ~3LL; }


// Emit pass of a group of ng blocks (group_block(perm, g0, .)): warps
// write the blocks' headers (d, removed mask, C_zr, w, t, seektable, tree),
// then one warp per segment writes its tokens, at the blocks' final bit
// positions (final_pos) in the zero-initialised stream.  Threads tid = 0 ..
// nthr-1, whole warps; dyn holds kEncSmem bytes.
template <class Sync>
__device__ void enc_emit_group(const int64_t* perm, int64_t g0, int ng, const TileDev* __restrict__ tiles,
                               const BlockDev* __restrict__ blocks, const uint8_t* sym, const BlockCode* __restrict__ codes,
                               const BlockHdr* __restrict__ hdrs, const int64_t* __restrict__ final_pos, uint32_t* __restrict__ out,
                               int* __restrict__ status, uint8_t* dyn, int* s_nitem, int tid, int nthr, Sync sync) {
  EncGroup G;
  load_group(perm, g0, ng, blocks, codes, dyn, G, s_nitem, tid, nthr, sync);
  const int wid = tid >> 5, lane = tid & 31, nw = nthr >> 5;
  for (int j = wid; j < ng; j += nw) {
    const int64_t bi = group_block(perm, g0, j);
    const BlockDev b = blocks[bi];
    const BlockCode& bc = codes[bi];
    const BlockHdr& H = hdrs[bi];
    const int d = bc.d, p = b.p;
    const int64_t B0 = block_bit_start(tiles[b.tile], final_pos, bi);
    if (lane == 0) {
      LaneWriter W;
      W.begin(out, B0);
      W.put((uint32_t)d, 5);
      for (int ty = 0; ty < p; ++ty)
        for (int pl = 0; pl < d; ++pl) W.put((bc.removed[ty] >> pl) & 1u, 1);
      if (bc.any_kept) {
        W.put((uint32_t)bc.czr, 8);
        W.put((uint32_t)bc.wbits, 5);
        W.put((uint32_t)H.t, 5);
      }
      W.end();
    }
    if (!bc.any_kept) continue;
    const int t = H.t;
    const int64_t seek = B0 + 5 + (int64_t)p * d + 18;
    if (lane < d) {
      LaneWriter W;
      W.begin(out, seek + (int64_t)lane * t);
      W.put(H.seglen[lane], t);
      W.end();
    }
    const int64_t tree_pos = seek + (int64_t)d * t;
    for (int k = lane; k * 32 < bc.tree_bits; k += 32) {
      const int nbk = min(32, bc.tree_bits - 32 * k);
      LaneWriter W;
      W.begin(out, tree_pos + 32 * k);
      W.put(bc.tree[k] >> (32 - nbk), nbk);
      W.end();
    }
  }
  for (int it = wid; it < G.nitem; it += nw) {
    const int j = G.item[it] >> 5, pl = G.item[it] & 31;
    const int64_t bi = group_block(perm, g0, j);
    const BlockDev b = blocks[bi];
    const BlockCode& bc = codes[bi];
    const BlockHdr& H = hdrs[bi];
    const int n = b.w * b.h / 8;
    const CodeTab ct{G.code[j], G.len[j], G.lit[j], bc.czr, bc.wbits, (1u << bc.wbits) - 1u};
    int64_t pos = block_bit_start(tiles[b.tile], final_pos, bi) + H.hdr_bits;
    for (int q = 0; q < pl; ++q) pos += H.seglen[q];
    const uint32_t km = kept_types(bc.removed, b.p, pl);
    const uint64_t bits =
        warp_segment(sym + b.sym + plane_offset(bc.removed, b.p, n, pl), __popc(km) * n, ct, out, pos, H.seglen[pl]);
    // the symbols must give the length the plane statistics gave
    if (lane == 0 && bits != H.seglen[pl]) set_status(status, kStInternal);
  }
}


// Header of tile t (little endian: magic, size, channels, bits, levels,
// colour transform, block count, quantiser steps, then the block end
// offsets) at out + toff, by threads tid = 0 .. nthr-1.
__device__ inline void write_tile_header(const TileDev& t, int64_t toff, const int64_t* __restrict__ final_pos,
                                         const int64_t* __restrict__ item_size, uint8_t* __restrict__ out, int tid, int nthr) {
  uint8_t* o = out + toff;
  const int64_t hdr = 32 + 4 * (int64_t)t.nb;
  if (tid == 0) {
    o[0] = 'I'; o[1] = 'S'; o[2] = 'X'; o[3] = '1';
    o[4] = (uint8_t)t.w; o[5] = (uint8_t)(t.w >> 8);
    o[6] = (uint8_t)t.h; o[7] = (uint8_t)(t.h >> 8);
    o[8] = (uint8_t)t.C; o[9] = (uint8_t)t.bits; o[10] = (uint8_t)t.L; o[11] = (uint8_t)t.ct;
    for (int k = 0; k < 4; ++k) o[12 + k] = (uint8_t)((uint32_t)t.nb >> (8 * k));
    for (int k = 0; k < 16; ++k) o[16 + k] = k <= t.L ? t.q[k] : 0;
  }
  for (int j = tid; j < t.nb; j += nthr) {
    const int64_t bi = t.block_base + j;
    const int64_t end = final_pos[bi] + item_size[bi] - (toff + hdr);   // the first item includes the header
    for (int k = 0; k < 4; ++k) o[32 + 4 * j + k] = (uint8_t)((uint64_t)end >> (8 * k));
  }
}

}  // namespace isx
