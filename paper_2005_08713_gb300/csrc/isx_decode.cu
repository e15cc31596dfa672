// isx_decode.cu — block decoder (Sec. 4, "Decompression is simply
// traversing the pipeline ... in reverse"): tile stream headers -> block
// list; per block the Fig. 3 header (d, removed mask, C_zr, w, t,
// seektable, preorder Huffman tree), then every plane segment decoded on
// its own from its seektable start (one thread per plane), zero runs
// expanded, symbols turned back into sign and magnitude bits (Eq. 1, 2),
// dequantised (bin midpoint) and stored into the level-z Mallat plane.
// Every loop is bounded by the known symbol counts; malformed input sets
// the device status to ISX_ERR_CORRUPT and the block is skipped.
#include "isx_internal.cuh"
#include "isx_kernels.h"

namespace isx {

constexpr int kTabBits = 10;
constexpr int kSymBytes = 96 * 1024;   // symbol planes per pass, shared memory

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

// One thread per selected tile: check its header against the descriptor,
// then list the blocks needed at level z (LL and levels > z) with their
// byte ranges.
__global__ void k_decode_plan(const TileDev* __restrict__ tiles, int n_tiles, const int64_t* __restrict__ tile_index,
                              const uint8_t* __restrict__ stream, const uint64_t* __restrict__ offs, int z, BlockDev* __restrict__ blocks,
                              int64_t* __restrict__ bbyte, int32_t* __restrict__ blen, int* __restrict__ status) {
  const int ti = blockIdx.x * blockDim.x + threadIdx.x;
  if (ti >= n_tiles) return;
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
         s[10] == t.L && (int)rd_u32le(s + 12) == nb_all && tend - toff >= 32 + 4 * (int64_t)nb_all;
    for (int k = 0; ok && k <= t.L; ++k) ok = s[16 + k] == t.q[k];
  }
  int64_t idx = t.block_base;
  const int64_t data = toff + 32 + 4 * (int64_t)nb_all;
  int j = 0;
  uint32_t prev = 0;
  for (int c = 0; c < t.C; ++c) {
    for (int lv = 0; lv <= t.L; ++lv) {
      int level = lv == 0 ? 0 : t.L + 1 - lv;
      int gw = level_dim(t.w, level == 0 ? t.L : level), gh = level_dim(t.h, level == 0 ? t.L : level);
      int p = level == 0 ? 1 : 3;
      for (int by = 0; by < ceil_div(gh, kCell); ++by)
        for (int bx = 0; bx < ceil_div(gw, kCell); ++bx, ++j) {
          uint32_t end = ok ? rd_u32le(s + 32 + 4 * j) : 0;
          bool bok = ok && end >= prev && data + (int64_t)end <= tend;
          if (level == 0 || level > z) {
            BlockDev b;
            b.tile = ti; b.c = c; b.level = level; b.by = by; b.bx = bx;
            b.p = bok ? p : 0;
            b.w = pad4(min(kCell, gw - kCell * bx));
            b.h = pad4(min(kCell, gh - kCell * by));
            b.coef = 0;
            blocks[idx] = b;
            bbyte[idx] = data + prev;
            blen[idx] = bok ? (int32_t)(end - prev) : 0;
            ++idx;
          }
          if (bok) prev = end;
          else ok = false;
        }
    }
  }
  if (!ok) set_status(status, kStCorrupt);
}

// MSB-first bit reader over a block's bytes (reads past the end give 0).
struct BitIn {
  const uint8_t* p;
  int64_t nbytes;
  int64_t next;    // next byte to load
  uint64_t buf;    // left aligned
  int nbuf;
  int64_t pos;     // bits consumed from the block start
  __device__ void seek(int64_t bitpos) {
    next = bitpos >> 3;
    buf = 0;
    nbuf = 0;
    pos = next * 8;
    refill();
    skip((int)(bitpos & 7));
  }
  __device__ void refill() {
    while (nbuf <= 56) {
      uint64_t b = next < nbytes ? p[next] : 0;
      ++next;
      buf |= b << (56 - nbuf);
      nbuf += 8;
    }
  }
  __device__ uint32_t peek(int n) const { return n ? (uint32_t)(buf >> (64 - n)) : 0u; }
  __device__ void skip(int n) {
    buf <<= n;
    nbuf -= n;
    pos += n;
    if (nbuf < 32) refill();
  }
  __device__ uint32_t get(int n) {
    uint32_t v = peek(n);
    skip(n);
    return v;
  }
};

struct DecShared {
  uint16_t tab[1 << kTabBits];     // (len << 8) | sym, or 0x8000 | node for longer codes
  uint16_t kid[512][2];
  int16_t sym[512];                // leaf symbol or -1
  uint32_t code[512];
  uint8_t dep[512];
  uint32_t seglen[32];
  int64_t segpos[32];
  uint32_t removed[3];
  int nnodes, d, czr, wbits, ok, keep;
};

__device__ bool parse_block_header(DecShared& S, const uint8_t* bp, int blen, int p) {
  BitIn in{bp, blen, 0, 0, 0, 0};
  in.seek(0);
  const int64_t nbits = (int64_t)blen * 8;
  int d = (int)in.get(5);
  if (d < 1) return false;
  S.d = d;
  bool any = false;
  for (int t = 0; t < 3; ++t) S.removed[t] = 0;
  for (int t = 0; t < 3; ++t)
    for (int pl = 0; pl < d; ++pl) {
      uint32_t bit = t < p ? in.get(1) : 1u;
      if (bit) S.removed[t] |= 1u << pl;
      else any = true;
    }
  if (in.pos > nbits) return false;
  if (!any) {
    S.nnodes = 0;
    return true;
  }
  S.czr = (int)in.get(8);
  S.wbits = (int)in.get(5);
  int t = (int)in.get(5);
  if (t < 1 || S.wbits < 1) return false;
  for (int pl = 0; pl < d; ++pl) S.seglen[pl] = in.get(t);
  // preorder tree: 0 = internal node, 1 + 8 bits = leaf
  int stack[34];
  int filled[34];
  int sp = 0, nn = 0;
  for (;;) {
    if (nn >= 511 || in.pos >= nbits) return false;
    int v = nn++;
    uint32_t bit = in.get(1);
    S.kid[v][0] = S.kid[v][1] = 0;
    if (sp == 0) {
      S.code[v] = 0;
      S.dep[v] = 0;
    } else {
      int par = stack[sp - 1];
      int side = filled[sp - 1]++;
      S.kid[par][side] = (uint16_t)v;
      S.code[v] = (S.code[par] << 1) | (uint32_t)side;
      S.dep[v] = (uint8_t)(S.dep[par] + 1);
    }
    if (bit) {
      S.sym[v] = (int16_t)in.get(8);
      while (sp > 0 && filled[sp - 1] == 2) --sp;
      if (sp == 0) break;
    } else {
      S.sym[v] = -1;
      if (sp >= 32) return false;   // codes longer than 32 bits
      stack[sp] = v;
      filled[sp] = 0;
      ++sp;
    }
  }
  S.nnodes = nn;
  int64_t pos = in.pos;
  for (int pl = 0; pl < d; ++pl) {
    S.segpos[pl] = pos;
    pos += S.seglen[pl];
  }
  return pos <= nbits;
}

__global__ void __launch_bounds__(kCtaThreads) k_decode_block(const TileDev* __restrict__ tiles, const BlockDev* __restrict__ blocks,
                                                             const uint8_t* __restrict__ stream, const int64_t* __restrict__ bbyte,
                                                             const int32_t* __restrict__ blen, int z, int drop, int32_t* __restrict__ planes,
                                                             int* __restrict__ status) {
  extern __shared__ uint8_t s_sym[];
  __shared__ DecShared S;
  const BlockDev b = blocks[blockIdx.x];
  if (b.p == 0) return;   // unreadable tile (status already set)
  const TileDev& t = tiles[b.tile];
  const int tid = threadIdx.x;
  const uint8_t* bp = stream + bbyte[blockIdx.x];
  const int nbytes = blen[blockIdx.x];
  const int n = b.w * b.h / 8, na = b.p * n;
  if (tid == 0) {
    S.ok = parse_block_header(S, bp, nbytes, b.p) ? 1 : 0;
    if (!S.ok) set_status(status, kStCorrupt);
    S.keep = S.ok ? max(1, S.d - drop) : 0;
  }
  __syncthreads();
  if (!S.ok) return;
  const int d = S.d;
  const int keep = S.keep;
  // plane geometry of the destination
  const int zw = level_dim(t.w, z), zh = level_dim(t.h, z);
  int32_t* plane = planes + t.plane_base + (int64_t)b.c * zw * zh;
  const int q = qlog2_of(t, b.level);
  const int32_t delta = 1 << q;
  if (S.nnodes > 0) {
    // decode table: codes up to kTabBits bits resolve in one lookup
    for (int v = tid; v < S.nnodes; v += blockDim.x) {
      int dep = S.dep[v];
      if (S.sym[v] >= 0 && dep <= kTabBits) {
        uint32_t lo = S.code[v] << (kTabBits - dep), cnt = 1u << (kTabBits - dep);
        for (uint32_t k = 0; k < cnt; ++k) S.tab[lo + k] = (uint16_t)((dep << 8) | S.sym[v]);
      } else if (S.sym[v] < 0 && dep == kTabBits) {
        S.tab[S.code[v]] = (uint16_t)(0x8000 | v);
      }
    }
  }
  const int planes_per_pass = max(1, kSymBytes / na);
  const bool single = planes_per_pass >= keep;
  for (int pb = 0; pb < keep; pb += planes_per_pass) {
    const int pe = min(keep, pb + planes_per_pass);
    for (int k = tid; k < (pe - pb) * na; k += blockDim.x) s_sym[k] = 0;
    __syncthreads();
    // one thread per plane segment
    if (tid < pe - pb && S.nnodes > 0) {
      const int pl = pb + tid;
      uint32_t km = 0;
      for (int ty = 0; ty < b.p; ++ty)
        if (!((S.removed[ty] >> pl) & 1u)) km |= 1u << ty;
      if (km) {
        const int need = __popc(km) * n;
        BitIn in{bp, nbytes, 0, 0, 0, 0};
        in.seek(S.segpos[pl]);
        const int64_t limit = S.segpos[pl] + S.seglen[pl];
        uint8_t* dst = s_sym + (int64_t)(pl - pb) * na;
        int pos = 0;
        bool bad = false;
        while (pos < need) {
          uint32_t e = S.tab[in.peek(kTabBits)];
          int sym;
          if (e & 0x8000u) {
            int v = e & 0x1ff;
            in.skip(kTabBits);
            int guard = 0;
            while (S.sym[v] < 0) {
              v = S.kid[v][in.get(1)];
              if (++guard > 32) { bad = true; break; }
            }
            if (bad) break;
            sym = S.sym[v];
          } else {
            sym = e & 0xff;
            in.skip((int)(e >> 8));
          }
          if (sym == S.czr) {
            uint32_t cnt = in.get(S.wbits);
            if (cnt == 0) {
              int ki = pos / n;
              int ty = nth_type(km, ki);
              dst[ty * n + pos - ki * n] = (uint8_t)sym;
              ++pos;
            } else {
              pos += (int)cnt;   // zeros: the buffer is already clear
              if (pos > need) { bad = true; break; }
            }
          } else {
            int ki = pos / n;
            int ty = nth_type(km, ki);
            dst[ty * n + pos - ki * n] = (uint8_t)sym;
            ++pos;
          }
          if (in.pos > limit) { bad = true; break; }
        }
        if (bad || in.pos != limit) set_status(status, kStCorrupt);
      }
    }
    __syncthreads();
    // rebuild the coefficients of each area
    for (int a = tid; a < na; a += blockDim.x) {
      const int type = a / n, k = a - type * n;
      int i, j;
      area_ij(k, b.w, &i, &j);
      int sx, sy, sw, sh;
      subband_rect(t.w, t.h, t.L, b.level, type, &sx, &sy, &sw, &sh);
      uint32_t mag[8], neg[8];
#pragma unroll
      for (int e = 0; e < 8; ++e) { mag[e] = 0; neg[e] = 0; }
      for (int pl = pb; pl < pe; ++pl) {
        uint32_t s = s_sym[(int64_t)(pl - pb) * na + a];
        if (!s) continue;
#pragma unroll
        for (int e = 0; e < 8; ++e) {
          uint32_t bit = (s >> e) & 1u;
          if (pl == 0) neg[e] = bit;
          else mag[e] |= bit << (d - 1 - pl);
        }
      }
#pragma unroll
      for (int e = 0; e < 8; ++e) {
        int yy = kCell * b.by + i + (e >> 2), xx = kCell * b.bx + j + (e & 3);
        if (yy >= sh || xx >= sw) continue;
        int32_t* dst = plane + (int64_t)(sy + yy) * zw + sx + xx;
        if (!single) {
          // several passes: accumulate sign (bit 31) and magnitude, convert at the end
          uint32_t acc = (pb == 0) ? 0u : (uint32_t)*dst;
          acc |= (neg[e] << 31) | mag[e];
          if (pe < keep) { *dst = (int32_t)acc; continue; }
          neg[e] = acc >> 31;
          mag[e] = acc & 0x7fffffffu;
        }
        int32_t m = (int32_t)mag[e];
        int32_t v = m == 0 ? 0 : m * delta + (delta >> 1);
        *dst = neg[e] ? -v : v;
      }
    }
    __syncthreads();
  }
}

int launch_decode_blocks(const DecodeBuffers& db, cudaStream_t s, StageMarks* T) {
  T->mark("decode.plan", s);
  k_decode_plan<<<ceil_div(db.n_tiles, 128), 128, 0, s>>>(db.tiles, db.n_tiles, db.tile_index, db.stream, db.stream_offsets, db.z,
                                                         db.blocks, db.block_byte, db.block_len, db.status);
  T->mark("decode.blocks", s);
  if (db.n_blocks > 0)
    k_decode_block<<<(unsigned)db.n_blocks, kCtaThreads, kSymBytes, s>>>(db.tiles, db.blocks, db.stream, db.block_byte, db.block_len,
                                                                          db.z, db.drop, db.planes, db.status);
  return 2;
}

void decode_set_attributes() {
  cudaFuncSetAttribute(k_decode_block, cudaFuncAttributeMaxDynamicSharedMemorySize, kSymBytes);
}

}  // namespace isx
