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
#include "isx_coder_dec.cuh"
#include "isx_kernels.h"

namespace isx {
// One thread per selected tile: check its header against the descriptor,
// then list the blocks needed at level z (LL and levels > z) with their
// byte ranges.
__global__ void k_decode_plan(const TileDev* __restrict__ tiles, int n_tiles, const int64_t* __restrict__ tile_index,
                              const uint8_t* __restrict__ stream, const uint64_t* __restrict__ offs, int z, const WinDev* __restrict__ wins,
                              BlockDev* __restrict__ blocks, int64_t* __restrict__ bbyte, int32_t* __restrict__ blen,
                              int* __restrict__ status) {
  const int ti = blockIdx.x * blockDim.x + threadIdx.x;
  if (ti >= n_tiles) return;
  stamp_tile(tiles[ti], kStampDecStart);
  decode_plan_tile(ti, tiles, tile_index, stream, offs, z, wins, blocks, bbyte, blen, status);
}

__global__ void k_dec_tables(const BlockDev* __restrict__ blocks, int64_t nb, const uint8_t* __restrict__ stream,
                             const int64_t* __restrict__ bbyte, const int32_t* __restrict__ blen, int drop, DecInfo* __restrict__ info,
                             DecTab* __restrict__ tabs, int64_t* __restrict__ sym_bytes, int* __restrict__ status) {
  const int64_t bi = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (bi < nb) dec_tables_block(bi, blocks, stream, bbyte, blen, drop, info, tabs, sym_bytes, status);
}

__global__ void k_dec_level_count(const BlockDev* __restrict__ blocks, int64_t nb, int64_t* __restrict__ cnt) {
  const int64_t bi = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (bi >= nb) return;
  atomicAdd(reinterpret_cast<unsigned long long*>(&cnt[blocks[bi].level]), 1ull);
}

__global__ void k_dec_level_fill(const BlockDev* __restrict__ blocks, int64_t nb, const int64_t* __restrict__ off, int64_t* __restrict__ fill,
                                 int64_t* __restrict__ perm) {
  const int64_t bi = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (bi >= nb) return;
  const int l = blocks[bi].level;
  perm[off[l] + (int64_t)atomicAdd(reinterpret_cast<unsigned long long*>(&fill[l]), 1ull)] = bi;
}

__global__ void __launch_bounds__(128) k_dec_item_count(const BlockDev* __restrict__ blocks, const int64_t* __restrict__ perm, int64_t nb,
                                                       const DecInfo* __restrict__ info, const DecTab* __restrict__ tabs,
                                                       int64_t ml_min_bits, int64_t* __restrict__ cnt, int64_t* __restrict__ big,
                                                       int64_t* __restrict__ n_big) {
  const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= nb) return;
  const int64_t bi = perm[j];
  uint32_t bigp;
  cnt[j] = __popc(block_item_planes(blocks[bi], info[bi], tabs[bi], ml_min_bits, &bigp));
  while (bigp) {
    const int pl = __ffs(bigp) - 1;
    bigp &= bigp - 1u;
    big[atomicAdd(reinterpret_cast<unsigned long long*>(n_big), 1ull)] = (bi << 5) | pl;
  }
}

__global__ void __launch_bounds__(128) k_dec_item_fill(const BlockDev* __restrict__ blocks, const int64_t* __restrict__ perm, int64_t nb,
                                                      const DecInfo* __restrict__ info, const DecTab* __restrict__ tabs,
                                                      int64_t ml_min_bits, const int64_t* __restrict__ base, int64_t* __restrict__ items) {
  const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= nb) return;
  const int64_t bi = perm[j];
  uint32_t bigp;
  uint32_t planes = block_item_planes(blocks[bi], info[bi], tabs[bi], ml_min_bits, &bigp);
  int64_t o = base[j];
  while (planes) {
    const int pl = __ffs(planes) - 1;
    planes &= planes - 1u;
    items[o++] = (bi << 5) | pl;
  }
}

// Clears the decode's symbol buffer (totals[0] bytes): zero runs are then
// skipped instead of written.
__global__ void k_dec_zero_sym(uint4* __restrict__ sym, const int64_t* __restrict__ total, int64_t cap) {
  const int64_t n = min(*total, cap) / 16;
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x)
    sym[k] = make_uint4(0, 0, 0, 0);
}

__global__ void __launch_bounds__(32 * kSegWarps) k_dec_segments(const BlockDev* __restrict__ blocks, const int64_t* __restrict__ items,
                                                     const int64_t* __restrict__ n_items_p, const uint8_t* __restrict__ stream,
                                                     const int64_t* __restrict__ bbyte, const int32_t* __restrict__ blen,
                                                     const DecInfo* __restrict__ info, const DecTab* __restrict__ tabs,
                                                     const int64_t* __restrict__ sym_off, uint8_t* __restrict__ sym,
                                                     const int64_t* __restrict__ sym_total, int64_t sym_cap, int* __restrict__ status) {
  __shared__ __align__(16) uint16_t s_tab[kSegWarps][kSegSlots][1 << kTabBits];
  const int64_t it = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (*sym_total > sym_cap) {   // a stream claiming more planes than its bit depth allows
    if (it == 0) set_status(status, kStCorrupt);
    return;
  }
  const bool active = it < *n_items_p;
  int64_t bi = -1;
  int pl = 0;
  if (active) {
    const int64_t item = items[it];
    bi = item >> 5;
    pl = (int)(item & 31);
  }
  // The items are block-major: the lanes of one block are neighbours.  The
  // first kSegSlots blocks of the warp get their 9-bit lookup table copied to
  // shared memory (the lookups are on every symbol's critical path); any
  // further block reads its table from global memory.
  const int64_t prev = __shfl_up_sync(0xffffffffu, bi, 1);
  const uint32_t heads = __ballot_sync(0xffffffffu, active && (lane == 0 || prev != bi));
  const int slot = __popc(heads & ((2u << lane) - 1u)) - 1;
  const int nslots = min(__popc(heads), kSegSlots);
  uint32_t h = heads;
  for (int sidx = 0; sidx < nslots; ++sidx) {
    const int64_t b = __shfl_sync(0xffffffffu, bi, __ffs(h) - 1);
    h &= h - 1u;
    const uint4* src = reinterpret_cast<const uint4*>(tabs[b].tab);
    uint4* dst = reinterpret_cast<uint4*>(s_tab[wid][sidx]);
    for (int k = lane; k < (1 << kTabBits) / 8; k += 32) dst[k] = __ldg(src + k);
  }
  __syncwarp();
  if (!active) return;
  dec_segment(bi, pl, slot < kSegSlots ? s_tab[wid][slot] : tabs[bi].tab, blocks, stream, bbyte, blen, info, tabs, sym_off, sym, status);
}

__global__ void __launch_bounds__(32) k_dec_segments_ml(const BlockDev* __restrict__ blocks, const int64_t* __restrict__ big,
                                                        const int64_t* __restrict__ n_big_p, int64_t* __restrict__ next,
                                                        const uint8_t* __restrict__ stream, const int64_t* __restrict__ bbyte,
                                                        const int32_t* __restrict__ blen, const DecInfo* __restrict__ info,
                                                        const DecTab* __restrict__ tabs, const int64_t* __restrict__ sym_off,
                                                        uint8_t* __restrict__ sym, const int64_t* __restrict__ sym_total, int64_t sym_cap,
                                                        int* __restrict__ status) {
  __shared__ __align__(16) uint16_t s_tab[1 << kTabBits];
  __shared__ uint16_t s_marks[kMlMarks][32];   // [mark][lane]: a warp's stores and loads of one mark index hit distinct banks
  __shared__ int s_nm[32];
  const int lane = threadIdx.x;
  const uint32_t FULL = 0xffffffffu;
  if (*sym_total > sym_cap) return;   // reported by the one-lane decoder
  const int64_t nbig = *n_big_p;
  for (;;) {
    int64_t g = 0;
    if (lane == 0) g = (int64_t)atomicAdd(reinterpret_cast<unsigned long long*>(next), 1ull);
    g = __shfl_sync(FULL, g, 0);
    if (g >= nbig) return;
    const int64_t item = big[g];
    const int64_t bi = item >> 5;
    const int pl = (int)(item & 31);
    const BlockDev b = blocks[bi];
    const DecInfo di = info[bi];
    const DecTab* T = tabs + bi;
    __syncwarp();   // the previous segment's shared-memory reads are done
    {
      const uint4* src = reinterpret_cast<const uint4*>(T->tab);
      uint4* dst = reinterpret_cast<uint4*>(s_tab);
      for (int k = lane; k < (1 << kTabBits) / 8; k += 32) dst[k] = __ldg(src + k);
    }
    const int n = b.w * b.h / 8;
    const uint32_t km = kept_mask(di.removed, b.p, pl);
    int64_t poff = sym_off[bi];
    for (int r = 0; r < pl; ++r) poff += plane_region(kept_mask(di.removed, b.p, r), n);
    const int need = __popc(km) * n;
    const int64_t seg0 = T->segpos[pl], send = seg0 + (int64_t)T->seglen[pl];
    const int64_t C = max((int64_t)kMlMinChunk, ((int64_t)T->seglen[pl] + 31) / 32);
    const int N = (int)(((int64_t)T->seglen[pl] + C - 1) / C);
    const bool act = lane < N;
    const int j = lane;
    const int64_t cst = seg0 + (int64_t)j * C, cen = min(cst + C, send);
    const int czr = T->czr, wb = T->wbits;
    const uint32_t* node = T->node;
    const uint8_t* bp = stream + bbyte[bi];
    const int64_t bl = blen[bi];
    __syncwarp();   // table in shared memory
    // 1. speculative decode of the own chunk
    BitPf in;
    uint32_t cnt_own = 0, cnt_cont = 0;
    int nm = 0;
    bool broken = false;
    if (act) {
      in.seek(bp, bl, cst);
      while (in.pos() < cen) {
        if (nm < kMlMarks) s_marks[nm++][lane] = (uint16_t)(in.pos() - cst);
        uint32_t sy, c;
        if (!ml_token(in, s_tab, node, czr, wb, &sy, &c)) { broken = true; break; }
        cnt_own += c;
      }
    }
    s_nm[lane] = nm;
    __syncwarp();
    // 2. continuation until a later chunk's recorded token start (or the segment's end)
    int land_k = N;
    int64_t land_p = act ? in.pos() : 0;
    if (act && !broken && j < N - 1) {
      int k = j + 1, ptr = 0;
      for (;;) {
        const int64_t p = in.pos();
        if (p >= send) { land_k = N; land_p = p; break; }
        while (k < N - 1 && p >= seg0 + (int64_t)(k + 1) * C) { ++k; ptr = 0; }
        const uint32_t rel = (uint32_t)(p - (seg0 + (int64_t)k * C));
        const int nmk = s_nm[k];
        while (ptr < nmk && s_marks[ptr][k] < rel) ++ptr;
        if (ptr < nmk && s_marks[ptr][k] == rel) { land_k = k; land_p = p; break; }
        uint32_t sy, c;
        if (!ml_token(in, s_tab, node, czr, wb, &sy, &c)) { broken = true; break; }
        cnt_cont += c;
      }
    }
    // 3. the chain of true token boundaries, from chunk 0
    bool valid = false, chain_bad = false;
    int64_t vstart = 0, vend = 0;
    {
      int cur = 0;
      int64_t cs = seg0;
      for (int it = 0; it < 32; ++it) {
        const int src = min(cur, N - 1) & 31;
        const int lk = __shfl_sync(FULL, land_k, src);
        const int64_t lp = __shfl_sync(FULL, land_p, src);
        const int lb = __shfl_sync(FULL, (int)broken, src);
        if (cur < N) {
          if (cur == j) { valid = true; vstart = cs; vend = lp; }
          if (lb) { chain_bad = true; cur = N; }
          else { cs = lp; cur = lk; }
        }
      }
    }
    bool bad = valid && (chain_bad || vend > send);
    // 4. valid symbol count: own count + continuation - count before the boundary
    uint32_t vc = 0;
    if (valid && !bad) {
      uint32_t prefix = 0;
      if (vstart > cst) {
        in.seek(bp, bl, cst);
        while (in.pos() < vstart) {
          uint32_t sy, c;
          if (!ml_token(in, s_tab, node, czr, wb, &sy, &c)) { bad = true; break; }
          prefix += c;
        }
        if (in.pos() != vstart) bad = true;
      }
      vc = cnt_own + cnt_cont - prefix;   // modular: a garbage prefix cancels
      if (vc > (uint32_t)need) bad = true;
    }
    if (!valid || bad) vc = 0;
    uint32_t incl = vc;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(FULL, incl, o);
      if (lane >= o) incl += y;
    }
    const uint32_t tot = __shfl_sync(FULL, incl, 31);
    // the segment is written only when every lane agrees that it decodes exactly
    if (__any_sync(FULL, bad) || tot != (uint32_t)need) {
      if (lane == 0) set_status(status, kStCorrupt);
      continue;
    }
    // 5. write the valid ranges
    if (valid && vc) {
      const int64_t s0 = incl - vc;
      SymOutShared out{sym + poff, s0, s0 + vc, s0, {0u, 0u, 0u, 0u}, false};
      in.seek(bp, bl, vstart);
      bool wbad = false;
      while (in.pos() < vend) {
        uint32_t sy, c;
        if (!ml_token(in, s_tab, node, czr, wb, &sy, &c) || out.pos + c > out.s1) { wbad = true; break; }
        out.token(sy, c);
      }
      out.finish();
      if (wbad || in.pos() != vend || out.pos != out.s1) set_status(status, kStCorrupt);
    }
  }
}

__global__ void __launch_bounds__(256) k_dec_rebuild(const TileDev* __restrict__ tiles, const BlockDev* __restrict__ blocks,
                                                    const DecInfo* __restrict__ info, const int64_t* __restrict__ sym_off,
                                                    const uint8_t* __restrict__ sym, const int64_t* __restrict__ sym_total,
                                                    int64_t sym_cap, int z, const WinDev* __restrict__ wins, int32_t* __restrict__ planes) {
  __shared__ int64_t s_poff[32];
  if (*sym_total > sym_cap) return;
  __shared__ uint32_t s_km[32];
  const BlockDev b = blocks[blockIdx.x];
  const DecInfo di = info[blockIdx.x];
  if (b.p == 0 || di.d == 0) return;
  const TileDev& t = tiles[b.tile];
  if (t.fused) return;   // rebuilt inside the fused inverse transform
  const int n = b.w * b.h / 8, na = b.p * n;
  if (threadIdx.x == 0) {
    int64_t off = sym_off[blockIdx.x];
    for (int pl = 0; pl < di.keep; ++pl) {
      s_km[pl] = kept_mask(di.removed, b.p, pl);
      s_poff[pl] = off;
      off += plane_region(s_km[pl], n);
    }
  }
  __syncthreads();
  const int zw = level_dim(t.w, z), zh = level_dim(t.h, z);
  int32_t* plane = planes + t.plane_base + (int64_t)b.c * zw * zh;
  const WinDev* W = t.win >= 0 ? wins + t.win : nullptr;
  const int q = qlog2_of(t, b.level);
  const int32_t delta = 1 << q;
  const int d = di.d;
  for (int a = threadIdx.x; a < na; a += blockDim.x) {
    const int type = a / n, k = a - type * n;
    uint32_t mag[8], neg = 0;
#pragma unroll
    for (int e = 0; e < 8; ++e) mag[e] = 0;
    for (int pl = 0; pl < di.keep; ++pl) {
      const uint32_t km = s_km[pl];
      if (!((km >> type) & 1u)) continue;
      const int ki = __popc(km & ((1u << type) - 1u));
      const uint32_t s = sym[s_poff[pl] + (int64_t)ki * n + k];
      if (!s) continue;
      if (pl == 0) {
        neg = s;
      } else {
        const int sh = d - 1 - pl;
#pragma unroll
        for (int e = 0; e < 8; ++e) mag[e] |= ((s >> e) & 1u) << sh;
      }
    }
    int i, j;
    area_ij(k, b.w, &i, &j);
    int sx, sy, sw, sh;
    subband_rect(t.w, t.h, t.L, b.level, type, &sx, &sy, &sw, &sh);
#pragma unroll
    for (int e = 0; e < 8; ++e) {
      const int yy = kCell * b.by + i + (e >> 2), xx = kCell * b.bx + j + (e & 3);
      if (yy >= sh || xx >= sw) continue;
      const int32_t m = (int32_t)mag[e];
      const int32_t v = m == 0 ? 0 : m * delta + (delta >> 1);
      const int32_t c = ((neg >> e) & 1u) ? -v : v;
      if (!W) {
        plane[(int64_t)(sy + yy) * zw + sx + xx] = c;
        continue;
      }
      const int64_t o = window_slot(*W, t.C, b.c, b.level, type, xx, yy);
      if (o >= 0) planes[t.plane_base + o] = c;
    }
  }
}

int launch_decode_blocks(const DecodeBuffers& db, cudaStream_t s, StageMarks* T) {
  int L = 0;
  T->mark("decode.plan", s);
  k_decode_plan<<<ceil_div(db.n_tiles, 128), 128, 0, s>>>(db.tiles, db.n_tiles, db.tile_index, db.stream, db.stream_offsets, db.z,
                                                         db.wins, db.blocks, db.block_byte, db.block_len, db.status);
  ++L;
  if (db.n_blocks == 0) return L;
  const unsigned g = (unsigned)((db.n_blocks + 127) / 128);
  T->mark("decode.tables", s);
  k_dec_tables<<<g, 128, 0, s>>>(db.blocks, db.n_blocks, db.stream, db.block_byte, db.block_len, db.drop, db.info,
                                 reinterpret_cast<DecTab*>(db.tables), db.sym_bytes, db.status);
  ++L;
  T->mark("decode.order", s);
  L += launch_exclusive_scan(db.sym_bytes, db.n_blocks, db.sym_off, db.scan_part, db.totals, s);
  L += launch_level_sort(db.blocks, db.n_blocks, db.bucket, db.perm, db.scan_part, db.totals + 2, s);
  // totals[3]: segments for the one-warp decoder, totals[4]: its work counter
  const int64_t ml_bits = db.latency_mode ? kMlMinBits : 0;
  cudaMemsetAsync(db.totals + 3, 0, 2 * sizeof(int64_t), s);
  k_dec_item_count<<<g, 128, 0, s>>>(db.blocks, db.perm, db.n_blocks, db.info, reinterpret_cast<const DecTab*>(db.tables), ml_bits,
                                     db.item_cnt, db.big, db.totals + 3);
  L += 1 + launch_exclusive_scan(db.item_cnt, db.n_blocks, db.item_base, db.scan_part, db.totals + 1, s);
  k_dec_item_fill<<<g, 128, 0, s>>>(db.blocks, db.perm, db.n_blocks, db.info, reinterpret_cast<const DecTab*>(db.tables), ml_bits, db.item_base,
                                    db.items);
  ++L;
  T->mark("decode.segments", s);
  k_dec_zero_sym<<<152 * 8, 256, 0, s>>>(reinterpret_cast<uint4*>(db.sym), db.totals, db.sym_cap);
  ++L;
  k_dec_segments<<<(unsigned)((db.max_items + 32 * kSegWarps - 1) / (32 * kSegWarps)), 32 * kSegWarps, 0, s>>>(
      db.blocks, db.items, db.totals + 1, db.stream, db.block_byte, db.block_len, db.info, reinterpret_cast<const DecTab*>(db.tables),
      db.sym_off, db.sym, db.totals, db.sym_cap, db.status);
  ++L;
  if (db.latency_mode) {
    k_dec_segments_ml<<<kMlCtas, 32, 0, s>>>(db.blocks, db.big, db.totals + 3, db.totals + 4, db.stream, db.block_byte, db.block_len,
                                             db.info, reinterpret_cast<const DecTab*>(db.tables), db.sym_off, db.sym, db.totals,
                                             db.sym_cap, db.status);
    ++L;
  }
  if (db.global_rebuild) {   // fused tiles rebuild their blocks inside the fused inverse
    T->mark("decode.rebuild", s);
    k_dec_rebuild<<<(unsigned)db.n_blocks, 256, 0, s>>>(db.tiles, db.blocks, db.info, db.sym_off, db.sym, db.totals, db.sym_cap, db.z,
                                                        db.wins, db.planes);
    ++L;
  }
  return L;
}

size_t dec_table_bytes() { return sizeof(DecTab); }

// Blocks ordered by level (counting sort; order inside a level arbitrary).
int launch_level_sort(const BlockDev* blocks, int64_t nb, int64_t* bucket /* 2 * kLevels */, int64_t* perm, int64_t* scan_part,
                      int64_t* total, cudaStream_t s) {
  const unsigned g = (unsigned)((nb + 127) / 128);
  cudaMemsetAsync(bucket, 0, 2 * sizeof(int64_t) * kLevels, s);
  k_dec_level_count<<<g, 128, 0, s>>>(blocks, nb, bucket);
  int L = 1 + launch_exclusive_scan(bucket, kLevels, bucket + kLevels, scan_part, total, s);
  cudaMemsetAsync(bucket, 0, sizeof(int64_t) * kLevels, s);
  k_dec_level_fill<<<g, 128, 0, s>>>(blocks, nb, bucket + kLevels, bucket, perm);
  return L + 1;
}

cudaError_t decode_set_attributes() { return cudaSuccess; }

}  // namespace isx
