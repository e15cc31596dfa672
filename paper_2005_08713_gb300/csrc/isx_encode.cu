// isx_encode.cu — the block coder (Sec. 4, Fig. 2 c-e, Fig. 3):
//   pass 1  k_block_stats    per block: bit depth d, removed planes, symbol
//                            histogram, zero runs (one CTA per block);
//   pass 2  k_block_huffman  per block: zero-run symbol C_zr, counter width
//                            w (Eq. 3), provisional and final Huffman codes,
//                            tree bits, exact token bits (one thread per block:
//                            32 blocks' trees are built side by side in a warp);
//   pass 3  k_block_emit     per block: header, seektable, tree and plane
//                            segments written bit-exactly into a slot;
//   pass 4  k_finalize_tiles / k_copy_blocks: tile headers and a compacted,
//                            contiguous stream.
// Symbols: every 4x2 area (8 coefficients stored consecutively in Eq. 2
// bit order) gives one byte per bitplane; plane 0 is the sign plane, plane
// pl >= 1 magnitude bit d-1-pl (signed-magnitude representation, Sec. 4).
#include "isx_internal.cuh"
#include "isx_kernels.h"

namespace isx {

constexpr uint32_t kAllZero = 0x80000000u;
constexpr int kStageWords = 12288;   // 48 KB output window per CTA

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

__device__ inline uint32_t area_symbol(const CoefRef& cf, int a, int pl, int d) {
  int32_t c[8];
  cf.load(a, c);
  uint32_t s = 0;
  if (pl == 0) {
#pragma unroll
    for (int e = 0; e < 8; ++e) s |= (uint32_t)(c[e] < 0) << e;
  } else {
    const int sh = d - 1 - pl;
#pragma unroll
    for (int e = 0; e < 8; ++e) s |= ((uint32_t)(abs(c[e]) >> sh) & 1u) << e;
  }
  return s;
}

// Removed-plane masks and depth from the OR of the magnitudes of each type.
__device__ inline void block_masks(const uint32_t* s_or, const uint32_t* s_neg, int p, int d, uint32_t* removed) {
  for (int t = 0; t < 3; ++t) {
    uint32_t r = 0;
    for (int pl = 0; pl < d; ++pl) {
      bool empty = t >= p || (pl == 0 ? s_neg[t] == 0 : ((s_or[t] >> (d - 1 - pl)) & 1u) == 0);
      if (empty) r |= 1u << pl;
    }
    removed[t] = r;
  }
}

__device__ inline uint32_t kept_types(const uint32_t* removed, int p, int pl) {
  uint32_t km = 0;
  for (int t = 0; t < p; ++t)
    if (!((removed[t] >> pl) & 1u)) km |= 1u << t;
  return km;
}

// ------------------------------------------------------------- pass 1
__device__ inline void record_run(uint32_t L, uint32_t* s_hist, uint32_t* s_runs, uint32_t* s_extra) {
  if (L == 1) {
    atomicAdd(&s_hist[0], 1u);   // an isolated zero is the literal symbol 0
    return;
  }
  atomicAdd(s_runs, 1u);
  for (int w = 2; w <= kMaxW; ++w) {
    uint32_t M = (1u << w) - 1u;
    if (M >= L) break;
    atomicAdd(&s_extra[w], (L + M - 1) / M - 1);
  }
}

__global__ void __launch_bounds__(kCtaThreads) k_block_stats(const BlockDev* __restrict__ blocks, const uint8_t* __restrict__ coef,
                                                            BlockStats* __restrict__ stats) {
  __shared__ uint32_t s_hist[256];
  __shared__ uint32_t s_extra[kMaxW + 1];
  __shared__ uint32_t s_runs;
  __shared__ uint32_t s_or[3], s_neg[3];
  __shared__ uint32_t s_tmp[33];
  const BlockDev b = blocks[blockIdx.x];
  const int n = b.w * b.h / 8, na = b.p * n;
  const CoefRef cf{coef + b.coef, b.coef16};
  const int tid = threadIdx.x;
  for (int i = tid; i < 256; i += blockDim.x) s_hist[i] = 0;
  if (tid <= kMaxW) s_extra[tid] = 0;
  if (tid < 3) { s_or[tid] = 0; s_neg[tid] = 0; }
  if (tid == 0) s_runs = 0;
  __syncthreads();
  {
    uint32_t o[3] = {0, 0, 0}, ng[3] = {0, 0, 0};
    for (int a = tid; a < na; a += blockDim.x) {
      const int t = a / n;
      int32_t c[8];
      cf.load(a, c);
#pragma unroll
      for (int e = 0; e < 8; ++e) {
        o[t] |= (uint32_t)abs(c[e]);
        ng[t] |= (uint32_t)(c[e] < 0);
      }
    }
    for (int t = 0; t < 3; ++t) {
      uint32_t ro = __reduce_or_sync(0xffffffffu, o[t]);
      uint32_t rn = __reduce_or_sync(0xffffffffu, ng[t]);
      if ((tid & 31) == 0) {
        if (ro) atomicOr(&s_or[t], ro);
        if (rn) atomicOr(&s_neg[t], rn);
      }
    }
  }
  __syncthreads();
  const uint32_t all_or = s_or[0] | s_or[1] | s_or[2];
  const int d = 1 + (all_or ? bitlen_u32(all_or) : 0);
  uint32_t removed[3];
  block_masks(s_or, s_neg, b.p, d, removed);
  const int m = (na + blockDim.x - 1) / blockDim.x;
  const int a0 = tid * m, a1 = min(a0 + m, na);
  uint32_t n_sym = 0;
  for (int pl = 0; pl < d; ++pl) {
    const uint32_t km = kept_types(removed, b.p, pl);
    if (!km) continue;
    n_sym += (uint32_t)__popc(km) * n;
    const int t_last = 31 - __clz(km);
    const int end_owner = (t_last * n + n - 1) / m;
    uint32_t cnt = 0, zeros = 0, lz = 0;
    bool seen = false;
    for (int a = a0; a < a1; ++a) {
      if (!((km >> (a / n)) & 1u)) continue;
      uint32_t s = area_symbol(cf, a, pl, d);
      ++cnt;
      if (s == 0) {
        ++zeros;
      } else {
        atomicAdd(&s_hist[s], 1u);
        if (!seen) { lz = zeros; seen = true; }
        else if (zeros) record_run(zeros, s_hist, &s_runs, s_extra);
        zeros = 0;
      }
    }
    const uint32_t elem = seen ? zeros : (kAllZero | cnt);
    const uint32_t cin = cta_exclusive_carry(elem, s_tmp) & ~kAllZero;
    if (seen && cin + lz > 0) record_run(cin + lz, s_hist, &s_runs, s_extra);
    if (tid == end_owner) {
      uint32_t Lf = seen ? zeros : cin + cnt;
      if (Lf) record_run(Lf, s_hist, &s_runs, s_extra);
    }
  }
  __syncthreads();
  BlockStats* st = stats + blockIdx.x;
  for (int i = tid; i < 256; i += blockDim.x) st->hist[i] = s_hist[i];
  if (tid <= kMaxW) st->extra[tid] = s_extra[tid];
  if (tid == 0) {
    st->n_runs = s_runs;
    st->n_sym = n_sym;
    st->removed[0] = removed[0]; st->removed[1] = removed[1]; st->removed[2] = removed[2];
    st->d = d;
  }
}

// ------------------------------------------------------------- pass 2
// Two-queue Huffman construction: leaves with f > 0 sorted ascending by
// (f, symbol); each merge takes the lighter queue front twice, the leaf
// queue first on equal weight; first taken = left child (bit 0).
struct Huff {
  uint32_t key[256];     // sorted leaves: (f << 8) | symbol
  uint32_t wgt[511];
  uint16_t kid[255][2];
  uint16_t parent[511];
  int nl, root;
};

__device__ void sort_keys(uint32_t* a, uint32_t* tmp, int n) {
  // bottom-up merge sort, ascending
  uint32_t* src = a;
  uint32_t* dst = tmp;
  for (int width = 1; width < n; width <<= 1) {
    for (int lo = 0; lo < n; lo += 2 * width) {
      int mid = min(lo + width, n), hi = min(lo + 2 * width, n);
      int i = lo, j = mid, k = lo;
      while (i < mid && j < hi) dst[k++] = src[i] <= src[j] ? src[i++] : src[j++];
      while (i < mid) dst[k++] = src[i++];
      while (j < hi) dst[k++] = src[j++];
    }
    uint32_t* t = src; src = dst; dst = t;
  }
  if (src != a)
    for (int i = 0; i < n; ++i) a[i] = src[i];
}

__device__ void huff_merge(Huff& H, const uint32_t* f) {
  int nl = 0;
  for (int s = 0; s < 256; ++s)
    if (f[s]) H.key[nl++] = (f[s] << 8) | (uint32_t)s;
  sort_keys(H.key, H.wgt, nl);
  for (int i = 0; i < nl; ++i) H.wgt[i] = H.key[i] >> 8;
  int qa = 0, qb = nl, nxt = nl;
  for (int st = 0; st < nl - 1; ++st) {
    int a, b;
    if (qa < nl && (qb >= nxt || H.wgt[qa] <= H.wgt[qb])) a = qa++; else a = qb++;
    if (qa < nl && (qb >= nxt || H.wgt[qa] <= H.wgt[qb])) b = qa++; else b = qb++;
    H.wgt[nxt] = H.wgt[a] + H.wgt[b];
    H.kid[nxt - nl][0] = (uint16_t)a;
    H.kid[nxt - nl][1] = (uint16_t)b;
    H.parent[a] = (uint16_t)nxt;
    H.parent[b] = (uint16_t)nxt;
    ++nxt;
  }
  H.nl = nl;
  H.root = nl <= 1 ? 0 : nxt - 1;
}

__device__ int huff_depth_of(const Huff& H, int sym) {
  if (H.nl <= 1) return 0;
  int leaf = -1;
  for (int i = 0; i < H.nl; ++i)
    if ((int)(H.key[i] & 255u) == sym) { leaf = i; break; }
  if (leaf < 0) return 0;
  int dep = 0;
  for (int v = leaf; v != H.root; v = H.parent[v]) ++dep;
  return dep;
}

__device__ inline void put_bits_local(uint32_t* words, int pos, uint32_t v, int nb) {
  if (nb <= 0) return;
  int wi = pos >> 5, off = pos & 31;
  uint64_t vv = (uint64_t)(v & (nb == 32 ? 0xffffffffu : ((1u << nb) - 1u))) << (64 - off - nb);
  words[wi] |= (uint32_t)(vv >> 32);
  if ((uint32_t)vv) words[wi + 1] |= (uint32_t)vv;
}

__global__ void __launch_bounds__(64) k_block_huffman(const BlockDev* __restrict__ blocks, const BlockStats* __restrict__ stats,
                                                      BlockCode* __restrict__ codes, int64_t* __restrict__ slot_size, int64_t nb) {
  const int64_t bi = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (bi >= nb) return;
  const BlockStats& st = stats[bi];
  const BlockDev b = blocks[bi];
  BlockCode& bc = codes[bi];
  const int d = st.d, p = b.p;
  const uint32_t n_sym = st.n_sym;
  bc.d = d;
  bc.p = p;
  for (int t = 0; t < 3; ++t) bc.removed[t] = st.removed[t];
  const int t0 = bitlen_u32((uint32_t)(p * b.w * b.h / 8)) - 1 + 5;
  bc.t0 = t0;
  if (n_sym == 0) {
    bc.any_kept = 0;
    bc.token_bits = 0;
    bc.tree_bits = 0;
    bc.czr = 0; bc.wbits = 0;
    int64_t bytes = (5 + p * d + 7) / 8;
    slot_size[bi] = (bytes + 15) & ~15LL;
    return;
  }
  bc.any_kept = 1;
  uint32_t f[256];
  for (int s = 0; s < 256; ++s) f[s] = st.hist[s];
  int czr = 1;
  for (int s = 2; s < 256; ++s)
    if (f[s] < f[czr]) czr = s;
  const uint32_t lit_czr = f[czr];
  // provisional code: every run counts once for C_zr
  f[czr] = lit_czr + st.n_runs;
  Huff H;
  huff_merge(H, f);
  const int l = f[czr] > 0 ? huff_depth_of(H, czr) : 0;
  // Eq. 3 (reading): w minimises (w + l) * (#C_zr tokens at width w) over [2, b]
  int bmax = n_sym > 1 ? bitlen_u32(n_sym - 1) : 0;
  if (bmax < 2) bmax = 2;
  int wbest = 2;
  uint64_t best = ~0ull;
  for (int w = 2; w <= bmax; ++w) {
    uint64_t pairs = (uint64_t)lit_czr + st.n_runs + st.extra[w];
    uint64_t cost = (uint64_t)(w + l) * pairs;
    if (cost < best) { best = cost; wbest = w; }
  }
  f[czr] = lit_czr + st.n_runs + st.extra[wbest];
  huff_merge(H, f);
  // codes, top down (children were created before their parents)
  uint32_t ncode[511];
  uint8_t ndep[511];
  const int nl = H.nl, nn = nl > 1 ? 2 * nl - 1 : 1;
  ncode[H.root] = 0;
  ndep[H.root] = 0;
  for (int i = nn - 1; i >= nl; --i) {
    for (int side = 0; side < 2; ++side) {
      int c = H.kid[i - nl][side];
      ncode[c] = (ncode[i] << 1) | (uint32_t)side;
      ndep[c] = (uint8_t)(ndep[i] + 1);
    }
  }
  for (int s = 0; s < 256; ++s) { bc.code[s] = 0; bc.len[s] = 0; }
  uint64_t token_bits = 0;
  for (int i = 0; i < nl; ++i) {
    int s = H.key[i] & 255u;
    bc.code[s] = ncode[i];
    bc.len[s] = ndep[i];
    token_bits += (uint64_t)f[s] * ndep[i];
  }
  token_bits += (uint64_t)wbest * f[czr];
  // preorder tree (Fig. 3): subtree sizes bottom up, offsets top down
  uint16_t* sz = H.parent;            // reuse: parents are no longer needed
  uint16_t off[511];
  for (int i = 0; i < nl; ++i) sz[i] = 9;
  for (int i = nl; i < nn; ++i) sz[i] = (uint16_t)(1 + sz[H.kid[i - nl][0]] + sz[H.kid[i - nl][1]]);
  off[H.root] = 0;
  for (int i = nn - 1; i >= nl; --i) {
    int a = H.kid[i - nl][0], c = H.kid[i - nl][1];
    off[a] = (uint16_t)(off[i] + 1);
    off[c] = (uint16_t)(off[i] + 1 + sz[a]);
  }
  uint32_t tw[81];
  for (int k = 0; k < 81; ++k) tw[k] = 0;
  for (int i = 0; i < nl; ++i) put_bits_local(tw, off[i], 0x100u | (H.key[i] & 255u), 9);
  for (int k = 0; k < 80; ++k) bc.tree[k] = tw[k];
  const int tree_bits = sz[H.root];
  bc.tree_bits = tree_bits;
  bc.czr = czr;
  bc.wbits = wbest;
  bc.token_bits = token_bits;
  const int tmax = max(t0, bitlen_u64(token_bits));
  const uint64_t hdr = 5 + (uint64_t)p * d + 18 + (uint64_t)d * tmax + tree_bits;
  const int64_t bytes = (int64_t)((hdr + token_bits + 7) / 8);
  slot_size[bi] = (bytes + 15) & ~15LL;
}

// ------------------------------------------------------------- pass 3
// MSB-first bit writer into a shared-memory window of the block's output
// (words hold the stream big-endian: stream bit q is bit 31 - q%32).
struct Window {
  uint32_t* w;
  int64_t lo;   // first bit of the window (multiple of 32)
  int64_t hi;   // one past its last bit
};

__device__ inline void put_bits(const Window& win, int64_t pos, uint32_t v, int nb) {
  if (nb <= 0 || pos + nb <= win.lo || pos >= win.hi) return;
  const int64_t rel = pos - win.lo;
  const int64_t wi = rel >= 0 ? rel >> 5 : -((-rel + 31) >> 5);
  const int off = (int)(rel - wi * 32);
  const uint64_t vv = (uint64_t)(v & (nb == 32 ? 0xffffffffu : ((1u << nb) - 1u))) << (64 - off - nb);
  const int64_t nw = (win.hi - win.lo) >> 5;
  const uint32_t hi = (uint32_t)(vv >> 32), lo = (uint32_t)vv;
  if (hi && wi >= 0 && wi < nw) atomicOr(&win.w[wi], hi);
  if (lo && wi + 1 >= 0 && wi + 1 < nw) atomicOr(&win.w[wi + 1], lo);
}

struct CodeTab {
  const uint32_t* code;
  const uint8_t* len;
  int czr, wbits;
  uint32_t M;
};

__device__ inline uint64_t run_bits(const CodeTab& ct, uint32_t L) {
  if (L == 1) return ct.len[0];
  if (ct.M == 0) return 0;
  uint32_t pairs = (L + ct.M - 1) / ct.M;
  return (uint64_t)pairs * (ct.len[ct.czr] + ct.wbits);
}

__device__ inline int64_t put_run(const CodeTab& ct, const Window& win, int64_t pos, uint32_t L) {
  if (L == 1) {
    put_bits(win, pos, ct.code[0], ct.len[0]);
    return pos + ct.len[0];
  }
  const int lc = ct.len[ct.czr];
  const uint32_t cz = ct.code[ct.czr];
  if (ct.M == 0) return pos;   // counter width is always >= 2; never loop on a bad table
  while (L > 0) {
    uint32_t k = L >= ct.M ? ct.M : L;
    put_bits(win, pos, cz, lc);
    pos += lc;
    put_bits(win, pos, k, ct.wbits);
    pos += ct.wbits;
    L -= k;
  }
  return pos;
}

__device__ inline int64_t put_literal(const CodeTab& ct, const Window& win, int64_t pos, uint32_t s) {
  put_bits(win, pos, ct.code[s], ct.len[s]);
  pos += ct.len[s];
  if ((int)s == ct.czr) pos += ct.wbits;   // counter 0: a literal C_zr
  return pos;
}

// One pass over all planes: writes the tokens that fall in the window and
// records the segment lengths.  All threads of the CTA call it.
__device__ void emit_planes(const CoefRef& cf, int n, int p, int d, const uint32_t* removed, const CodeTab& ct,
                            const Window& win, int64_t seg_start, uint32_t* s_seglen, uint32_t* s_tmp32, uint64_t* s_tmp64) {
  const int na = p * n;
  const int m = (na + blockDim.x - 1) / blockDim.x;
  const int a0 = threadIdx.x * m, a1 = min(a0 + m, na);
  for (int pl = 0; pl < d; ++pl) {
    const uint32_t km = kept_types(removed, p, pl);
    if (!km) {
      if (threadIdx.x == 0) s_seglen[pl] = 0;
      continue;
    }
    const int t_last = 31 - __clz(km);
    const bool is_end = (int)threadIdx.x == (t_last * n + n - 1) / m;
    // count
    uint32_t cnt = 0, zeros = 0, lz = 0;
    bool seen = false;
    uint64_t bits = 0;
    for (int a = a0; a < a1; ++a) {
      if (!((km >> (a / n)) & 1u)) continue;
      uint32_t s = area_symbol(cf, a, pl, d);
      ++cnt;
      if (s == 0) {
        ++zeros;
      } else {
        if (!seen) { lz = zeros; seen = true; }
        else if (zeros) bits += run_bits(ct, zeros);
        bits += ct.len[s] + ((int)s == ct.czr ? ct.wbits : 0);
        zeros = 0;
      }
    }
    const uint32_t elem = seen ? zeros : (kAllZero | cnt);
    const uint32_t cin = cta_exclusive_carry(elem, s_tmp32) & ~kAllZero;
    const uint32_t lead = seen ? cin + lz : 0;
    if (lead) bits += run_bits(ct, lead);
    uint32_t fin = 0;
    if (is_end) fin = seen ? zeros : cin + cnt;
    if (fin) bits += run_bits(ct, fin);
    uint64_t seg_total;
    const uint64_t myoff = cta_exclusive_sum<uint64_t>(bits, s_tmp64, &seg_total);
    // write
    int64_t pos = seg_start + (int64_t)myoff;
    if (lead) pos = put_run(ct, win, pos, lead);
    zeros = 0;
    bool first = true;
    for (int a = a0; a < a1; ++a) {
      if (!((km >> (a / n)) & 1u)) continue;
      uint32_t s = area_symbol(cf, a, pl, d);
      if (s == 0) {
        ++zeros;
      } else {
        if (!first && zeros) pos = put_run(ct, win, pos, zeros);
        first = false;
        pos = put_literal(ct, win, pos, s);
        zeros = 0;
      }
    }
    if (fin) pos = put_run(ct, win, pos, fin);
    if (threadIdx.x == 0) s_seglen[pl] = (uint32_t)seg_total;
    seg_start += (int64_t)seg_total;
    __syncthreads();
  }
  __syncthreads();
}

__global__ void __launch_bounds__(kCtaThreads) k_block_emit(const TileDev* __restrict__ tiles, const BlockDev* __restrict__ blocks,
                                                           const uint8_t* __restrict__ coef, const BlockCode* __restrict__ codes,
                                                           const int64_t* __restrict__ slot_off, const int64_t* __restrict__ slot_size,
                                                           uint8_t* __restrict__ slots, int64_t slot_cap, const int64_t* __restrict__ totals,
                                                           int64_t* __restrict__ item_size, int* __restrict__ status) {
  extern __shared__ uint32_t stage[];
  __shared__ uint32_t s_code[256];
  __shared__ uint8_t s_len[256];
  __shared__ uint32_t s_seglen[32];
  __shared__ uint32_t s_tmp32[33];
  __shared__ uint64_t s_tmp64[33];
  __shared__ int s_t;
  const int64_t bi = blockIdx.x;
  if (totals[0] > slot_cap) return;   // not enough scratch: reported by k_finalize_tiles
  const BlockDev b = blocks[bi];
  const BlockCode& bc = codes[bi];
  const TileDev& tile = tiles[b.tile];
  const int n = b.w * b.h / 8, p = b.p, d = bc.d;
  const int tid = threadIdx.x;
  uint32_t removed[3] = {bc.removed[0], bc.removed[1], bc.removed[2]};
  uint8_t* out = slots + slot_off[bi];
  const int64_t cap_bytes = slot_size[bi];
  const int64_t stage_bits = (int64_t)kStageWords * 32;
  const int64_t first_item_extra = (bi == tile.block_base) ? 32 + 4 * (int64_t)tile.nb : 0;
  if (!bc.any_kept) {
    // d and the all-ones removed mask only
    if (tid == 0) {
      uint32_t w[5] = {0, 0, 0, 0, 0};
      put_bits_local(w, 0, (uint32_t)d, 5);
      for (int t = 0; t < p; ++t)
        for (int pl = 0; pl < d; ++pl) put_bits_local(w, 5 + t * d + pl, 1u, 1);
      int bytes = (5 + p * d + 7) / 8;
      for (int k = 0; k < bytes; ++k) out[k] = (uint8_t)(w[k >> 2] >> (24 - 8 * (k & 3)));
      item_size[bi] = bytes + first_item_extra;
    }
    return;
  }
  for (int s = tid; s < 256; s += blockDim.x) { s_code[s] = bc.code[s]; s_len[s] = bc.len[s]; }
  if (tid == 0) s_t = bc.t0;
  __syncthreads();
  CodeTab ct{s_code, s_len, bc.czr, bc.wbits, (1u << bc.wbits) - 1u};
  const int tree_bits = bc.tree_bits;
  const int64_t hm = 5 + (int64_t)p * d;
  int t = s_t;
  int64_t total_bits = 0;
  for (int64_t wlo = 0;; wlo += stage_bits) {
    Window win{stage, wlo, wlo + stage_bits};
    for (int attempt = 0; attempt < 2; ++attempt) {
      for (int k = tid; k < kStageWords; k += blockDim.x) stage[k] = 0;
      __syncthreads();
      const int64_t hdr = hm + 18 + (int64_t)d * t + tree_bits;
      emit_planes(CoefRef{coef + b.coef, b.coef16}, n, p, d, removed, ct, win, hdr, s_seglen, s_tmp32, s_tmp64);
      if (wlo > 0) break;
      // first window: fix t (raised only when a segment length needs more bits)
      uint32_t mx = 0;
      uint64_t sum = 0;
      for (int pl = 0; pl < d; ++pl) { mx = max(mx, s_seglen[pl]); sum += s_seglen[pl]; }
      if (sum != bc.token_bits) {
        if (tid == 0) set_status(status, 7);
        return;
      }
      const int need = mx ? bitlen_u32(mx) : 0;
      if (need <= t) break;
      t = need;
      __syncthreads();
    }
    const int64_t hdr = hm + 18 + (int64_t)d * t + tree_bits;
    total_bits = hdr + (int64_t)bc.token_bits;
    if (wlo == 0) {
      // header: d, removed mask, C_zr, w, t, seektable, tree
      if (tid == 0) {
        put_bits(win, 0, (uint32_t)d, 5);
        for (int ty = 0; ty < p; ++ty)
          for (int pl = 0; pl < d; ++pl)
            if ((removed[ty] >> pl) & 1u) put_bits(win, 5 + ty * d + pl, 1u, 1);
        put_bits(win, hm, (uint32_t)bc.czr, 8);
        put_bits(win, hm + 8, (uint32_t)bc.wbits, 5);
        put_bits(win, hm + 13, (uint32_t)t, 5);
      }
      if (tid < d) put_bits(win, hm + 18 + (int64_t)tid * t, s_seglen[tid], t);
      const int64_t tree_pos = hm + 18 + (int64_t)d * t;
      for (int k = tid; k * 32 < tree_bits; k += blockDim.x) {
        int nbk = min(32, tree_bits - 32 * k);
        put_bits(win, tree_pos + 32 * k, bc.tree[k] >> (32 - nbk), nbk);
      }
      if (tid == 0) {
        int64_t bytes = (total_bits + 7) / 8;
        if (bytes > cap_bytes) set_status(status, 7);
        item_size[bi] = bytes + first_item_extra;
      }
    }
    __syncthreads();
    // flush the window (bytes beyond the block end are zero padding inside the slot)
    const int64_t total_bytes = (total_bits + 7) / 8;
    const int64_t wbyte = wlo / 8;
    const int64_t nbytes = min((int64_t)kStageWords * 4, total_bytes - wbyte);
    const int64_t nwords = (nbytes + 3) / 4;
    if (wbyte + nwords * 4 <= cap_bytes) {
      uint32_t* o32 = reinterpret_cast<uint32_t*>(out + wbyte);
      for (int64_t k = tid; k < nwords; k += blockDim.x) o32[k] = __byte_perm(stage[k], 0, 0x0123);
    } else if (tid == 0) {
      set_status(status, 7);
    }
    __syncthreads();
    if (wlo + stage_bits >= total_bits) break;
  }
}

// ------------------------------------------------------------- pass 4
// One CTA per tile: its stream offset, its header (little endian) and its
// blocks copied from their slots into the contiguous output.  Every output
// byte of a tile is written by that tile's CTA only.
__global__ void __launch_bounds__(256) k_assemble_tiles(const TileDev* tiles, int n_tiles, const int64_t* final_pos,
                                                       const int64_t* item_size, const int64_t* slot_off, const int64_t* totals,
                                                       int64_t slot_cap, int64_t header_total, const uint8_t* slots, uint8_t* out,
                                                       int64_t out_cap, uint64_t* tile_offsets, int* status) {
  const int ti = blockIdx.x;
  const TileDev& t = tiles[ti];
  const int64_t tot_slots = totals[0], tot_stream = totals[1];
  const bool scratch_ok = tot_slots <= slot_cap;
  const int64_t total = scratch_ok ? tot_stream : tot_slots + header_total;
  if (ti == n_tiles - 1 && threadIdx.x == 0) {
    tile_offsets[n_tiles] = (uint64_t)total;
    if (!scratch_ok || total > out_cap) set_status(status, kStCapacity);
  }
  const int64_t toff = final_pos[t.block_base];
  if (threadIdx.x == 0) tile_offsets[ti] = (uint64_t)toff;
  if (!scratch_ok || total > out_cap) return;
  uint8_t* o = out + toff;
  const int64_t hdr = 32 + 4 * (int64_t)t.nb;
  if (threadIdx.x == 0) {
    o[0] = 'I'; o[1] = 'S'; o[2] = 'X'; o[3] = '1';
    o[4] = (uint8_t)t.w; o[5] = (uint8_t)(t.w >> 8);
    o[6] = (uint8_t)t.h; o[7] = (uint8_t)(t.h >> 8);
    o[8] = (uint8_t)t.C; o[9] = (uint8_t)t.bits; o[10] = (uint8_t)t.L; o[11] = t.C == 3 ? 1 : 0;
    for (int k = 0; k < 4; ++k) o[12 + k] = (uint8_t)((uint32_t)t.nb >> (8 * k));
    for (int k = 0; k < 16; ++k) o[16 + k] = k <= t.L ? t.q[k] : 0;
  }
  for (int j = threadIdx.x; j < t.nb; j += blockDim.x) {
    const int64_t bi = t.block_base + j;
    const int64_t end = final_pos[bi] + item_size[bi] - (toff + hdr);   // the first item includes the header
    for (int k = 0; k < 4; ++k) o[32 + 4 * j + k] = (uint8_t)((uint64_t)end >> (8 * k));
  }
  for (int j = 0; j < t.nb; ++j) {
    const int64_t bi = t.block_base + j;
    const int64_t extra = j == 0 ? hdr : 0;
    const int64_t size = item_size[bi] - extra;
    const uint8_t* src = slots + slot_off[bi];
    uint8_t* dst = out + final_pos[bi] + extra;
    for (int64_t k = threadIdx.x; k < size; k += blockDim.x) dst[k] = src[k];
  }
}

int launch_encode_coding(const EncodeBuffers& eb, cudaStream_t s, StageMarks* T) {
  int launches = 0;
  const unsigned nb = (unsigned)eb.n_blocks;
  T->mark("encode.stats", s);
  k_block_stats<<<nb, kCtaThreads, 0, s>>>(eb.blocks, (const uint8_t*)eb.coef, eb.stats);
  T->mark("encode.huffman", s);
  k_block_huffman<<<(unsigned)((eb.n_blocks + 63) / 64), 64, 0, s>>>(eb.blocks, eb.stats, eb.codes, eb.slot_size, eb.n_blocks);
  launches += 2;
  T->mark("encode.scan", s);
  launches += launch_exclusive_scan(eb.slot_size, eb.n_blocks, eb.slot_off, eb.scan_part, eb.totals + 0, s);
  const size_t smem = (size_t)kStageWords * 4;
  T->mark("encode.emit", s);
  k_block_emit<<<nb, kCtaThreads, smem, s>>>(eb.tiles, eb.blocks, (const uint8_t*)eb.coef, eb.codes, eb.slot_off, eb.slot_size, eb.slots,
                                             eb.slot_capacity, eb.totals, eb.exact_size, eb.status);
  ++launches;
  T->mark("encode.scan", s);
  launches += launch_exclusive_scan(eb.exact_size, eb.n_blocks, eb.final_pos, eb.scan_part, eb.totals + 1, s);
  return launches;
}

int launch_encode_finalize(const EncodeBuffers& eb, int64_t header_total, cudaStream_t s) {
  k_assemble_tiles<<<eb.n_tiles, 256, 0, s>>>(eb.tiles, eb.n_tiles, eb.final_pos, eb.exact_size, eb.slot_off, eb.totals, eb.slot_capacity,
                                              header_total, eb.slots, eb.out, eb.out_capacity, eb.tile_offsets, eb.status);
  return 1;
}

void encode_set_attributes() {
  cudaFuncSetAttribute(k_block_emit, cudaFuncAttributeMaxDynamicSharedMemorySize, kStageWords * 4);
}

}  // namespace isx
