// isx_coder_dec.cuh — device code of the block decoder (Sec. 4, Fig. 3):
// parsing the tile and block headers, the per-block lookup tables, the
// plane segment decoders and the symbol writers, as functions over one
// block or one segment.  Used by the per-stage kernels (isx_decode.cu) and
// by the persistent per-tile decoder (isx_persist.cu).
#pragma once
#include <cstdint>

#include "isx_internal.cuh"

namespace isx {
constexpr int kTabBits = 9;

// Index of the ki-th (0-based) set bit of a 3-bit type mask.
__device__ inline int nth_type(uint32_t km, int ki) {
  for (int t = 0; t < 3; ++t)
    if ((km >> t) & 1u) {
      if (ki == 0) return t;
      --ki;
    }
  return 0;
}

__device__ inline uint32_t rd_u32le(const uint8_t* p) {
  return (uint32_t)p[0] | ((uint32_t)p[1] << 8) | ((uint32_t)p[2] << 16) | ((uint32_t)p[3] << 24);
}


__device__ inline uint32_t kept_mask(const uint32_t* removed, int p, int pl) {
  uint32_t km = 0;
#pragma unroll
  for (int t = 0; t < 3; ++t)   // fixed trip count: removed[] stays in registers
    if (t < p && !((removed[t] >> pl) & 1u)) km |= 1u << t;
  return km;
}

// Symbol buffer layout of one block: for every decoded plane pl in order,
// its kept types' symbols (n each, types in order HL, LH, HH), the plane's
// region rounded up to 16 bytes.
__device__ inline int64_t plane_region(uint32_t km, int n) { return ((int64_t)__popc(km) * n + 15) & ~15LL; }

// Decode table of one block, built once by k_dec_tables and read by every
// segment decoder of the block: codes up to kTabBits bits resolve with one
// lookup, longer ones walk the tree from the node reached after kTabBits bits.
struct DecTab {
  uint16_t tab[1 << kTabBits];   // (len << 8) | symbol, or 0x8000 | node
  uint32_t node[512];            // internal: kid0 | kid1 << 16; leaf: 0x80000000 | symbol
  int64_t segpos[32];            // bit position of plane segment pl from the block start
  uint32_t seglen[32];
  int32_t czr, wbits, nnodes, pad;
};

// Double-buffered MSB-first reader: 16-byte chunks are requested one chunk
// ahead of use; bytes outside the block read as 0.
struct BitPf {
  const uint8_t* p;
  int64_t nbytes;
  int64_t cbyte;       // block offset of the next chunk to request (16-byte aligned in memory)
  uint4 nxt;
  uint32_t a0, a1, a2, a3;
  int avail;
  uint64_t buf;
  int nbuf;
  int64_t wend;        // bit position just past the last bit in buf
  __device__ int64_t pos() const { return wend - nbuf; }   // bit position of the next bit
  __device__ uint4 chunk(int64_t off) const {
    if (off >= 0 && off + 16 <= nbytes) return __ldg(reinterpret_cast<const uint4*>(p + off));
    uint32_t w[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      uint32_t v = 0;
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const int64_t o = off + 4 * q + k;
        v |= (uint32_t)(o >= 0 && o < nbytes ? p[o] : 0) << (8 * k);
      }
      w[q] = v;
    }
    return make_uint4(w[0], w[1], w[2], w[3]);
  }
  __device__ uint32_t next_word() {
    if (avail == 0) {
      a0 = __byte_perm(nxt.x, 0, 0x0123);
      a1 = __byte_perm(nxt.y, 0, 0x0123);
      a2 = __byte_perm(nxt.z, 0, 0x0123);
      a3 = __byte_perm(nxt.w, 0, 0x0123);
      avail = 4;
      nxt = chunk(cbyte);
      cbyte += 16;
    }
    const uint32_t w = a0;
    a0 = a1; a1 = a2; a2 = a3;
    --avail;
    return w;
  }
  __device__ void seek(const uint8_t* base, int64_t n, int64_t bitpos) {
    p = base;
    nbytes = n;
    const int64_t byte = bitpos >> 3;
    const int mis = (int)(reinterpret_cast<uintptr_t>(p + byte) & 15);
    cbyte = byte - mis;
    nxt = chunk(cbyte);
    cbyte += 16;
    avail = 0;
    buf = (uint64_t)next_word() << 32;
    buf |= next_word();
    nbuf = 64;
    int drop = mis * 8 + (int)(bitpos & 7);
    while (drop >= 32) {   // skip whole words of the first chunk
      buf = (buf << 32) | next_word();
      drop -= 32;
    }
    buf <<= drop;
    nbuf = 64 - drop;
    wend = bitpos + nbuf;
  }
  __device__ uint32_t peek(int n) const { return n ? (uint32_t)(buf >> (64 - n)) : 0u; }
  __device__ void skip(int n) {   // n <= 32
    buf <<= n;
    nbuf -= n;
    if (nbuf <= 32) {
      buf |= (uint64_t)next_word() << (32 - nbuf);
      nbuf += 32;
      wend += 32;
    }
  }
  __device__ uint32_t get(int n) {
    const uint32_t v = peek(n);
    skip(n);
    return v;
  }
};

// Header pass: one thread per block parses the Fig. 3 header (d, removed
// mask, C_zr, w, t, seektable, preorder tree), builds the block's decode
// table and sizes its symbol region.
__device__ inline void dec_tables_block(int64_t bi, const BlockDev* __restrict__ blocks, const uint8_t* __restrict__ stream,
                                        const int64_t* __restrict__ bbyte, const int32_t* __restrict__ blen, int drop,
                                        DecInfo* __restrict__ info, DecTab* __restrict__ tabs, int64_t* __restrict__ sym_bytes,
                                        int* __restrict__ status) {
  const BlockDev b = blocks[bi];
  DecInfo di;
  di.d = 0; di.keep = 0; di.removed[0] = di.removed[1] = di.removed[2] = ~0u;
  int64_t bytes = 0;
  DecTab& T = tabs[bi];
  T.nnodes = 0;
  if (b.p > 0) {
    const int nbytes = blen[bi];
    const int64_t nbits = (int64_t)nbytes * 8;
    BitPf in;
    in.seek(stream + bbyte[bi], nbytes, 0);
    int d = (int)in.get(5);
    bool any = false;
    for (int t = 0; t < 3; ++t) {
      uint32_t r = 0;
      for (int pl = 0; pl < d; ++pl) {
        if (t >= b.p || in.get(1)) r |= 1u << pl;
        else any = true;
      }
      di.removed[t] = r;
    }
    bool ok = d >= 1 && in.pos() <= nbits;
    if (ok && any) {
      T.czr = (int)in.get(8);
      T.wbits = (int)in.get(5);
      const int t = (int)in.get(5);
      ok = t >= 1 && T.wbits >= 1;
      for (int pl = 0; ok && pl < d; ++pl) T.seglen[pl] = in.get(t);
      // Preorder tree: 0 = internal node (its left subtree, then its right
      // subtree, follow), 1 + 8 bits = leaf.  The walk keeps the current
      // node's code and depth only: a left child is the node read right after
      // its parent (kid0 = parent + 1); after a leaf the walk climbs while
      // the node is a right child (odd code) and moves to the sibling.  The
      // internal node entered at each depth is remembered, and its node word
      // (kid0 | kid1 << 16) is stored once, when its right child starts: no
      // read-modify-write of global memory.
      int path[33];
      uint32_t code = 0;
      int dep = 0, nn = 0;
      while (ok) {
        if (nn >= 511 || in.pos() >= nbits) { ok = false; break; }
        const int v = nn++;
        if (dep > 0 && (code & 1u)) T.node[path[dep - 1]] = (uint32_t)(path[dep - 1] + 1) | ((uint32_t)v << 16);
        if (in.get(1)) {
          const uint32_t sym = in.get(8);
          T.node[v] = 0x80000000u | sym;
          if (dep <= kTabBits) {
            const uint32_t lo = code << (kTabBits - dep), cnt = 1u << (kTabBits - dep);
            const uint32_t e = ((uint32_t)dep << 8) | sym;
            if (cnt >= 8) {   // whole 8-entry groups, 16-byte aligned
              const uint32_t e2 = e | (e << 16);
              uint4* t4 = reinterpret_cast<uint4*>(T.tab + lo);
              for (uint32_t k = 0; k < (cnt >> 3); ++k) t4[k] = make_uint4(e2, e2, e2, e2);
            } else {
              for (uint32_t k = 0; k < cnt; ++k) T.tab[lo + k] = (uint16_t)e;
            }
          }
          while (dep > 0 && (code & 1u)) {
            code >>= 1;
            --dep;
          }
          if (dep == 0) break;   // back at the root: the tree is complete
          code |= 1u;            // the right sibling
        } else {
          if (dep >= 32) { ok = false; break; }   // codes longer than 32 bits
          if (dep == kTabBits) T.tab[code] = (uint16_t)(0x8000 | v);
          path[dep] = v;
          code <<= 1;
          ++dep;
        }
      }
      if (ok) {
        int64_t pos = in.pos();
        for (int pl = 0; pl < d; ++pl) {
          T.segpos[pl] = pos;
          pos += T.seglen[pl];
        }
        ok = pos <= nbits;
        T.nnodes = nn;
      }
    }
    if (!ok) {
      set_status(status, kStCorrupt);
      d = 0;
      T.nnodes = 0;
    }
    di.d = d;
    di.keep = d ? max(1, d - drop) : 0;
    const int n = b.w * b.h / 8;
    for (int pl = 0; pl < di.keep; ++pl) bytes += plane_region(kept_mask(di.removed, b.p, pl), n);
  }
  info[bi] = di;
  sym_bytes[bi] = bytes;
}


// Blocks ordered by level (counting sort): neighbouring blocks in the order
// have the same size.
constexpr int kLevels = 16;



// 8-byte symbol writer of one thread over a cleared region: a word is
// stored only if it holds a nonzero symbol.
struct SymOut {
  uint64_t* dst;       // the word being filled
  uint64_t cur;
  int c;               // position of the next symbol in the word
  __device__ void flush() {
    if (cur) *dst = cur;
    ++dst;
    cur = 0;
    c = 0;
  }
  __device__ void put(uint32_t s) {
    cur |= (uint64_t)s << (8 * c);
    if (++c == 8) flush();
  }
  // The region was cleared beforehand: a run of zeros only moves the position.
  __device__ void zeros(uint32_t cnt) {
    const uint32_t p = (uint32_t)c + cnt;
    if (p < 8) {
      c = (int)p;
      return;
    }
    flush();
    dst += (p >> 3) - 1;
    c = (int)(p & 7);
  }
};
// Segment items (block << 5 | plane) in block-major order: blocks by level
// (neighbouring blocks have the same size), each block's kept planes in
// order, so that the 32 lanes of a warp decode the planes of a few blocks
// whose lookup tables the warp keeps in shared memory.  In a latency-bound
// decode (few blocks: ml_min_bits > 0) the segments of at least ml_min_bits
// bits go instead to the list `big`, each decoded by a whole warp
// (k_dec_segments_ml); a block whose tree is a single leaf (0-bit codes)
// keeps all its segments on one lane each.
__device__ inline uint32_t block_item_planes(const BlockDev& b, const DecInfo& di, const DecTab& T, int64_t ml_min_bits,
                                             uint32_t* big_planes) {
  uint32_t planes = 0, big = 0;
  if (b.p > 0 && di.d > 0 && T.nnodes > 0)
    for (int pl = 0; pl < di.keep; ++pl)
      if (kept_mask(di.removed, b.p, pl)) {
        // (chunks of at most 65535 bits: the warp decoder records token starts as 16-bit offsets)
        if (ml_min_bits > 0 && T.nnodes > 1 && (int64_t)T.seglen[pl] >= ml_min_bits && T.seglen[pl] <= 32u * 65535u)
          big |= 1u << pl;
        else planes |= 1u << pl;
      }
  *big_planes = big;
  return planes;
}




// One-warp CTAs: a CTA holds its registers and shared memory until its
// slowest lane is done, and the lanes decode segments of unequal lengths,
// so small CTAs let each SM replace finished warps sooner (measured: 1 %
// faster decode than 8-warp CTAs; more table slots per warp measured
// slower: the copies cost more than the global-memory lookups they save).
constexpr int kSegWarps = 1, kSegSlots = 4;   // lookup tables in shared memory per warp

// Decodes plane segment pl of block bi (one thread) into the block's symbol
// region: tokens through `tab` (the block's lookup table, a shared-memory or
// the global copy) and its tree, zero runs skipped in the cleared region.
__device__ inline void dec_segment(int64_t bi, int pl, const uint16_t* tab, const BlockDev* __restrict__ blocks,
                                   const uint8_t* __restrict__ stream, const int64_t* __restrict__ bbyte, const int32_t* __restrict__ blen,
                                   const DecInfo* __restrict__ info, const DecTab* __restrict__ tabs, const int64_t* __restrict__ sym_off,
                                   uint8_t* __restrict__ sym, int* __restrict__ status) {
  const BlockDev b = blocks[bi];
  const DecInfo di = info[bi];
  const DecTab* T = tabs + bi;
  const int n = b.w * b.h / 8;
  const uint32_t km = kept_mask(di.removed, b.p, pl);
  int64_t off = sym_off[bi];
  for (int q = 0; q < pl; ++q) off += plane_region(kept_mask(di.removed, b.p, q), n);
  const int need = __popc(km) * n;
  const int64_t start = T->segpos[pl];
  const int64_t limit = start + T->seglen[pl];
  const int czr = T->czr, wb = T->wbits;
  const uint32_t* node = T->node;
  BitPf in;
  in.seek(stream + bbyte[bi], blen[bi], start);
  SymOut out{reinterpret_cast<uint64_t*>(sym + off), 0, 0};
  int pos = 0;
  bool bad = false;
  while (pos < need) {
    const uint32_t e = tab[in.peek(kTabBits)];
    int s;
    if (e & 0x8000u) {
      uint32_t nd = __ldg(&node[e & 0x1ff]);
      in.skip(kTabBits);
      int guard = 0;
      while (!(nd & 0x80000000u)) {
        const uint32_t kid = in.get(1) ? (nd >> 16) : (nd & 0xffffu);
        nd = __ldg(&node[kid & 0x1ff]);
        if (++guard > 32) { bad = true; break; }
      }
      if (bad) break;
      s = (int)(nd & 0xff);
    } else {
      s = (int)(e & 0xff);
      in.skip((int)(e >> 8));
    }
    if (s == czr) {
      const uint32_t cnt = in.get(wb);
      if (cnt == 0) {
        out.put((uint32_t)s);
        ++pos;
      } else {
        if (pos + (int)cnt > need) { bad = true; break; }
        out.zeros(cnt);
        pos += (int)cnt;
      }
    } else {
      out.put((uint32_t)s);
      ++pos;
    }
  }
  // a corrupt segment that reads past its end (or stops short) is caught
  // here: the loop ends after `need` symbols whatever the bits say
  if (out.c) out.flush();
  if (bad || in.pos() != limit) set_status(status, kStCorrupt);
}


// ------------------------------------------ one warp per segment (latency)
// One token (a codeword, and its w-bit counter when the codeword is C_zr):
// sym = the literal symbol (0 for a run), cnt = the symbols it stands for.
// false for a code the tree does not hold (a wrong path or a corrupt stream).
// The lanes of a warp decode different chunks, so every branch here would
// split the warp: a code of at most kTabBits bits (all but the rarest
// symbols) and its counter are decoded with selects, one lookup and one
// skip; only a longer code walks the tree.  The counter is read from the
// same 64-bit buffer: at a token's start it holds at least 33 bits, and a
// code of at most 9 bits plus a counter of at most 18 bits (kMaxW, the
// widest the encoder writes) fit; a wider counter field takes the tree-walk
// path's separate read.
__device__ __forceinline__ bool ml_token(BitPf& in, const uint16_t* tab, const uint32_t* __restrict__ node, int czr, int wb,
                                         uint32_t* sym, uint32_t* cnt) {
  const uint32_t e = tab[in.peek(kTabBits)];
  if (!(e & 0x8000u) && wb <= kMaxW) {
    const uint32_t len = e >> 8, s = e & 0xffu;
    const bool run = (int)s == czr;
    const uint32_t c = (uint32_t)((in.buf << len) >> (64 - wb));   // the counter, if this is C_zr
    in.skip((int)(len + (run ? (uint32_t)wb : 0u)));
    *sym = run ? (c ? 0u : s) : s;
    *cnt = run && c ? c : 1u;
    return len != 0;   // every code of a tree with two or more leaves has a bit
  }
  uint32_t s;
  if (e & 0x8000u) {
    uint32_t nd = __ldg(&node[e & 0x1ff]);
    in.skip(kTabBits);
    int guard = 0;
    while (!(nd & 0x80000000u)) {
      const uint32_t kid = in.get(1) ? (nd >> 16) : (nd & 0xffffu);
      nd = __ldg(&node[kid & 0x1ff]);
      if (++guard > 32) return false;
    }
    s = nd & 0xffu;
  } else {
    if ((e >> 8) == 0) return false;
    s = e & 0xffu;
    in.skip((int)(e >> 8));
  }
  if ((int)s == czr) {
    const uint32_t c = in.get(wb);
    if (c) {
      *sym = 0;
      *cnt = c;
      return true;
    }
  }
  *sym = s;
  *cnt = 1;
  return true;
}

// Writer of one lane's range [s0, s1) of a segment's symbols (the region
// was cleared beforehand): 16-symbol chunks wholly inside the range are
// stored, the chunks it shares with a neighbouring lane are OR-ed word by
// word.
struct SymOutShared {
  uint8_t* base;
  int64_t s0, s1, pos;
  uint32_t w[4];
  bool dirty;
  __device__ void flush_at(int64_t c0) {   // c0: first symbol of the chunk
    if (dirty) {
      uint32_t* dst = reinterpret_cast<uint32_t*>(base + c0);
      if (c0 >= s0 && c0 + 16 <= s1) {
        *reinterpret_cast<uint4*>(dst) = make_uint4(w[0], w[1], w[2], w[3]);
      } else {
#pragma unroll
        for (int k = 0; k < 4; ++k)
          if (w[k]) atomicOr(dst + k, w[k]);
      }
    }
    w[0] = w[1] = w[2] = w[3] = 0;
    dirty = false;
  }
  __device__ void put(uint32_t s) {
    if (s) {
      const int q = (int)(pos & 15);
      const uint32_t v = s << (8 * (q & 3));
      // selects instead of an indexed array: w stays in registers
      if ((q >> 2) == 0) w[0] |= v;
      else if ((q >> 2) == 1) w[1] |= v;
      else if ((q >> 2) == 2) w[2] |= v;
      else w[3] |= v;
      dirty = true;
    }
    ++pos;
    if ((pos & 15) == 0) flush_at(pos - 16);
  }
  __device__ void zeros(uint32_t c) {   // the cleared region already holds them: only the position moves
    const int64_t end = pos + c;
    if ((end >> 4) != (pos >> 4)) flush_at((pos >> 4) << 4);
    pos = end;
  }
  __device__ void finish() {
    if (pos & 15) flush_at((pos >> 4) << 4);
  }
  // A token: cnt symbols, all zero but a literal's (cnt = 1).  Selects set the
  // byte; the chunk is flushed only when the token leaves it.
  __device__ void token(uint32_t s, uint32_t c) {
    const int q = (int)(pos & 15);
    const uint32_t v = s << (8 * (q & 3));
    w[0] |= (q >> 2) == 0 ? v : 0u;
    w[1] |= (q >> 2) == 1 ? v : 0u;
    w[2] |= (q >> 2) == 2 ? v : 0u;
    w[3] |= (q >> 2) == 3 ? v : 0u;
    dirty = dirty || s != 0;
    const int64_t end = pos + c;
    if ((end >> 4) != (pos >> 4)) flush_at((pos >> 4) << 4);
    pos = end;
  }
};

// Self-synchronising decode of one plane segment per warp, for decodes of
// few blocks (one tile, a viewport), where a segment decoded serially by one
// lane would set the call's latency (Sec. 4: the seektable gives every plane
// segment its own start).  The segment is cut into at most 32 chunks of C
// bits, one per lane.
//  1. Each lane decodes its chunk from the chunk's first bit, recording the
//     bit offsets of the first kMlMarks tokens it starts there, and counts
//     the symbols.  Only chunk 0 starts on a true token boundary; the other
//     lanes may start inside a token, but Huffman codes resynchronise: once
//     two decodes reach the same bit as a token start they agree from then
//     on.
//  2. Each lane continues past its chunk's end, token by token, until it
//     reaches a bit that a later chunk's lane recorded as a token start (or
//     the segment's end); a chunk it crosses without landing is covered by
//     it.
//  3. Following the landings from chunk 0 gives the true token boundary
//     where each lane's valid decode starts: by induction every lane on that
//     chain decodes the true token sequence from its boundary on.
//  4. A lane's valid symbol count is its count from the chunk start plus the
//     continuation, minus the count of the (short) stretch before its
//     boundary, decoded again; a warp scan places the lanes.
//  5. Each valid lane decodes its range again and writes its symbols.
// The bytes are those of the one-lane decoder.  A stream the true path
// cannot decode exactly (a bad code, a wrong symbol count, a segment that
// does not end on its last bit) sets ISX_ERR_CORRUPT.  It costs about twice
// the one-lane decoder's instructions, so throughput-bound calls (many
// blocks) keep one lane per segment.
constexpr int kMlMarks = 64;        // token starts recorded per chunk: the window a landing is searched in
constexpr int kMlMinChunk = 64;     // bits
constexpr int64_t kMlMinBits = 2048;
constexpr int kMlCtas = 152 * 8;


// Rebuild pass: per block, every area's 8 coefficients from the decoded
// planes (sign plane, then magnitude bits d-2 .. 0), dequantised at the bin
// midpoint, stored into the level-z Mallat plane (padding cropped).
// Element (relative to the tile's plane_base) that band sample (x, y) of
// `type` at `level` (0 = the LL of level L) of channel c takes in a windowed
// decode, or -1 when the windows do not need it.
__device__ inline int64_t window_slot(const WinDev& W, int C, int c, int level, int type, int x, int y) {
  if (level == 0) {
    if (W.z == W.L) {
      if (x < W.fx0 || x >= W.fx1 || y < W.fy0 || y >= W.fy1) return -1;
      const int64_t fw = W.fx1 - W.fx0, fh = W.fy1 - W.fy0;
      return W.fbuf + (int64_t)c * fw * fh + (int64_t)(y - W.fy0) * fw + (x - W.fx0);
    }
    const WinLevel& v = W.lev[W.L];
    if (x < v.lx0 || x >= v.lx1 || y < v.ly0 || y >= v.ly1) return -1;
    const int64_t cols = (v.lx1 - v.lx0) + (v.hx1 - v.hx0), rows = (v.ly1 - v.ly0) + (v.hy1 - v.hy0);
    return v.buf + (int64_t)c * cols * rows + (int64_t)(y - v.ly0) * cols + (x - v.lx0);
  }
  const WinLevel& v = W.lev[level];
  const bool hx = type != 1, hy = type >= 1;   // HL: high x; LH: high y; HH: both
  const int x0 = hx ? v.hx0 : v.lx0, x1 = hx ? v.hx1 : v.lx1, y0 = hy ? v.hy0 : v.ly0, y1 = hy ? v.hy1 : v.ly1;
  if (x < x0 || x >= x1 || y < y0 || y >= y1) return -1;
  const int64_t cols = (v.lx1 - v.lx0) + (v.hx1 - v.hx0), rows = (v.ly1 - v.ly0) + (v.hy1 - v.hy0);
  const int64_t col = (hx ? (v.lx1 - v.lx0) : 0) + (x - x0), row = (hy ? (v.ly1 - v.ly0) : 0) + (y - y0);
  return v.buf + (int64_t)c * cols * rows + row * cols + col;
}

// Tile ti of a decode (one thread): check its stream header against the
// descriptor, then list the blocks needed at level z (LL and levels > z)
// with their byte ranges, from t.block_base on.
__device__ inline void decode_plan_tile(int ti, const TileDev* __restrict__ tiles, const int64_t* __restrict__ tile_index,
                                        const uint8_t* __restrict__ stream, const uint64_t* __restrict__ offs, int z,
                                        const WinDev* __restrict__ wins, BlockDev* __restrict__ blocks, int64_t* __restrict__ bbyte,
                                        int32_t* __restrict__ blen, int* __restrict__ status) {
  const TileDev t = tiles[ti];
  const int64_t src = tile_index[ti];
  const int64_t toff = (int64_t)offs[src], tend = (int64_t)offs[src + 1];
  const uint8_t* s = stream + toff;
  // expected number of blocks in the whole tile
  int nb_all = 0;
  for (int lv = 0; lv <= t.L; ++lv) {
    int level = lv == 0 ? 0 : lv;
    int gw = level_dim(t.w, level == 0 ? t.L : level), gh = level_dim(t.h, level == 0 ? t.L : level);
    nb_all += ceil_div(gw, kCell) * ceil_div(gh, kCell);
  }
  nb_all *= t.C;
  bool ok = tend - toff >= 32 && s[0] == 'I' && s[1] == 'S' && s[2] == 'X' && s[3] == '1';
  if (ok) {
    ok = (int)(s[4] | (s[5] << 8)) == t.w && (int)(s[6] | (s[7] << 8)) == t.h && s[8] == t.C && s[9] == t.bits &&
         s[10] == t.L && s[11] == t.ct && (int)rd_u32le(s + 12) == nb_all && tend - toff >= 32 + 4 * (int64_t)nb_all;
    for (int k = 0; ok && k <= t.L; ++k) ok = s[16 + k] == t.q[k];
  }
  // Each block's bytes are [end[j-1], end[j]) of the cumulative end table; only the blocks the decode
  // needs are visited (for a windowed decode, the cells bounding its windows), each checked on its own.
  int64_t idx = t.block_base;
  const int64_t data = toff + 32 + 4 * (int64_t)nb_all;
  const WinDev* W = t.win >= 0 ? wins + t.win : nullptr;
  bool bad = !ok;
  int jbase = 0;
  for (int c = 0; c < t.C; ++c) {
    for (int lv = 0; lv <= t.L; ++lv) {
      const int level = lv == 0 ? 0 : t.L + 1 - lv;
      const int gw = level_dim(t.w, level == 0 ? t.L : level), gh = level_dim(t.h, level == 0 ? t.L : level);
      const int p = level == 0 ? 1 : 3;
      const int gwc = ceil_div(gw, kCell), ghc = ceil_div(gh, kCell);
      int bx0 = 0, bx1 = gwc, by0 = 0, by1 = ghc;
      if (level != 0 && level <= z) {
        bx1 = 0;   // the z finest levels are not needed at level z
      } else if (W) {
        window_cells(*W, level, &bx0, &bx1, &by0, &by1);
        bx1 = min(bx1, gwc);
        by1 = min(by1, ghc);
      }
      for (int by = by0; by < by1; ++by)
        for (int bx = bx0; bx < bx1; ++bx) {
          // a windowed decode lists only the blocks its windows meet (the host counted the same ones)
          if (W && !block_in_window(*W, level, by, bx)) continue;
          const int j = jbase + by * gwc + bx;
          uint32_t st = 0, en = 0;
          bool bok = ok;
          if (ok) {
            en = rd_u32le(s + 32 + 4 * j);
            st = j ? rd_u32le(s + 32 + 4 * (j - 1)) : 0u;
            bok = st <= en && data + (int64_t)en <= tend;
          }
          if (!bok) bad = true;
          BlockDev b;
          b.tile = ti; b.c = c; b.level = level; b.by = by; b.bx = bx;
          b.p = bok ? p : 0;
          b.w = pad4(min(kCell, gw - kCell * bx));
          b.h = pad4(min(kCell, gh - kCell * by));
          b.coef = 0;
          blocks[idx] = b;
          bbyte[idx] = data + st;
          blen[idx] = bok ? (int32_t)(en - st) : 0;
          ++idx;
        }
      jbase += gwc * ghc;
    }
  }
  if (bad) set_status(status, kStCorrupt);
}

}  // namespace isx
