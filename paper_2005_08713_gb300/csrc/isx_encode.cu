// isx_encode.cu — the block coder (Sec. 4, Fig. 2 c-e, Fig. 3):
//   pass 1  k_enc_symbols    per block: bit depth d, removed planes, the kept
//                            symbols written once to a flat symbol buffer,
//                            then every plane segment's histogram and zero
//                            runs from that buffer (and the block's totals);
//   pass 2  k_block_huffman  per block (one warp): zero-run symbol C_zr,
//                            counter width w (Eq. 3), provisional and final
//                            Huffman codes, tree bits;
//           k_enc_layout     per block (one warp): the exact plane segment
//                            lengths (from the plane statistics, or the
//                            symbols of short segments), seektable width t
//                            and the block's size;
//           scan             the blocks' final byte offsets;
//   pass 3  k_enc_emit       per group of blocks (one warp per segment):
//                            header, seektable, tree and segments written
//                            bit-exactly into their final place in the
//                            contiguous stream;
//           k_tile_headers   tile headers.
// Symbols: every 4x2 area (8 coefficients stored consecutively in Eq. 2
// bit order) gives one byte per bitplane; plane 0 is the sign plane, plane
// pl >= 1 magnitude bit d-1-pl (signed-magnitude representation, Sec. 4).
// A block's symbol region holds, for every plane with a kept type, the kept
// types' symbols (n = w*h/8 each, types in order HL, LH, HH) padded to 16
// bytes: the plane segments of Fig. 3 before zero-run and Huffman coding.
#include "isx_internal.cuh"
#include "isx_coder_enc.cuh"
#include "isx_kernels.h"

namespace isx {
// kPlanes: the launch may meet blocks with plane segments of more than
// kRawMax symbols (their literal histograms need kMaxD shared slots).
template <bool kPlanes>
__global__ void __launch_bounds__(256) k_enc_symbols(const BlockDev* __restrict__ blocks, const int64_t* __restrict__ perm,
                                                    const uint8_t* __restrict__ coef, uint8_t* __restrict__ sym,
                                                    BlockStats* __restrict__ stats, PlaneStats* __restrict__ pst,
                                                    int* __restrict__ status) {
  __shared__ SymShared<kPlanes> S;
  // blocks by level: neighbouring CTAs do similar work
  enc_symbols_block<kPlanes>(perm[blockIdx.x], blocks, coef, sym, stats, pst, status, S, threadIdx.x, blockDim.x, CtaBarrier());
}

__global__ void __launch_bounds__(32 * kHuffWarps, 4) k_block_huffman(const BlockDev* __restrict__ blocks, const int64_t* __restrict__ perm,
                                                                  const BlockStats* __restrict__ stats, BlockCode* __restrict__ codes,
                                                                  int64_t nb) {
  __shared__ HuffWarp hw[kHuffWarps];
  __shared__ int s_nl[kHuffWarps];
  const int wid = threadIdx.x >> 5;
  const int64_t gi = (int64_t)blockIdx.x * kHuffWarps + wid;
  // blocks by level: the warps of a CTA get blocks of similar size, whose
  // tree merges then take similar numbers of steps side by side
  cta_block_huffman(gi < nb ? perm[gi] : (int64_t)-1, blocks, stats, codes, hw, s_nl, CtaBarrier());
}

constexpr int kLayoutWarps = 8;
__global__ void __launch_bounds__(32 * kLayoutWarps) k_enc_layout(const TileDev* __restrict__ tiles, const BlockDev* __restrict__ blocks,
                                                                  const int64_t* __restrict__ perm, const PlaneStats* __restrict__ pst,
                                                                  const uint8_t* __restrict__ sym, const BlockCode* __restrict__ codes,
                                                                  BlockHdr* __restrict__ hdrs, int64_t* __restrict__ item_size,
                                                                  int* __restrict__ status, int64_t nb) {
  __shared__ __align__(16) uint8_t s_len[kLayoutWarps][256];
  const int wid = threadIdx.x >> 5;
  const int64_t gi = (int64_t)blockIdx.x * kLayoutWarps + wid;
  if (gi >= nb) return;
  enc_block_layout(perm[gi], tiles, blocks, pst, sym, codes, hdrs, item_size, status, s_len[wid]);
}

__global__ void k_zero_stream(uint32_t* __restrict__ out, const int64_t* __restrict__ totals, int64_t out_cap) {
  const int64_t total = totals[0];
  if (needed_capacity(total) > out_cap) return;
  const int64_t nw = (total + 3) / 4;
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < nw; k += (int64_t)gridDim.x * blockDim.x) out[k] = 0;
}

__global__ void __launch_bounds__(32 * kEmitWarps) k_enc_emit(const TileDev* __restrict__ tiles, const BlockDev* __restrict__ blocks,
                                                             const int64_t* __restrict__ perm, int64_t nb, const uint8_t* sym,
                                                             const BlockCode* __restrict__ codes, const BlockHdr* __restrict__ hdrs,
                                                             const int64_t* __restrict__ final_pos, const int64_t* __restrict__ totals,
                                                             int64_t out_cap, uint32_t* __restrict__ out, int* __restrict__ status) {
  extern __shared__ __align__(16) uint8_t dyn[];
  __shared__ int s_nitem;
  if (needed_capacity(totals[0]) > out_cap) return;
  const int64_t g0 = (int64_t)blockIdx.x * kEncGroup;
  enc_emit_group(perm, g0, (int)min((int64_t)kEncGroup, nb - g0), tiles, blocks, sym, codes, hdrs, final_pos, out, status, dyn,
                 &s_nitem, threadIdx.x, blockDim.x, CtaBarrier());
}

// Tile headers and the stream offsets; capacity check.
__global__ void k_tile_headers(const TileDev* __restrict__ tiles, int n_tiles, const int64_t* __restrict__ final_pos,
                               const int64_t* __restrict__ item_size, const int64_t* __restrict__ totals, uint8_t* __restrict__ out,
                               int64_t out_cap, uint64_t* __restrict__ tile_offsets, int* __restrict__ status) {
  const int ti = blockIdx.x;
  const TileDev& t = tiles[ti];
  const int64_t total = totals[0];
  const bool fits = needed_capacity(total) <= out_cap;
  if (ti == n_tiles - 1 && threadIdx.x == 0) {
    // the stream size, or the capacity it needs when it does not fit
    tile_offsets[n_tiles] = (uint64_t)(fits ? total : needed_capacity(total));
    if (!fits) set_status(status, kStCapacity);
  }
  const int64_t toff = final_pos[t.block_base];
  if (threadIdx.x == 0) tile_offsets[ti] = (uint64_t)toff;
  if (fits) write_tile_header(t, toff, final_pos, item_size, out, threadIdx.x, blockDim.x);
  __syncthreads();
  if (threadIdx.x == 0) stamp_tile(t, kStampEncEnd);   // the tile's stream is complete
}

int launch_encode_coding(const EncodeBuffers& eb, cudaStream_t s, StageMarks* T) {
  int L = 0;
  const unsigned nb = (unsigned)eb.n_blocks;
  T->mark("encode.order", s);
  L += launch_level_sort(eb.blocks, eb.n_blocks, eb.bucket, eb.perm, eb.scan_part, eb.totals + 1, s);
  T->mark("encode.symbols", s);
  int64_t listed = 0;
  for (int l = 0; l < 16; ++l) listed += eb.level_blocks[l];
  if (listed == eb.n_blocks) {
    // one launch per level (the level sort's order): CTAs no larger than the
    // level's blocks need (the small blocks of the coarse levels would leave
    // most of a 256-thread CTA idle through its barriers)
    int64_t off = 0;
    for (int l = 0; l < 16; ++l) {
      if (!eb.level_blocks[l]) continue;
      int threads = 32;
      while (threads < 256 && threads < eb.level_quads[l]) threads <<= 1;
      // a block of q quads (rounded down) has segments of at most 4 q + 3 symbols
      if (4 * (int64_t)eb.level_quads[l] + 3 > kRawMax)
        k_enc_symbols<true><<<(unsigned)eb.level_blocks[l], threads, 0, s>>>(eb.blocks, eb.perm + off, (const uint8_t*)eb.coef, eb.sym,
                                                                             eb.stats, eb.pst, eb.status);
      else
        k_enc_symbols<false><<<(unsigned)eb.level_blocks[l], threads, 0, s>>>(eb.blocks, eb.perm + off, (const uint8_t*)eb.coef, eb.sym,
                                                                              eb.stats, eb.pst, eb.status);
      off += eb.level_blocks[l];
      ++L;
    }
  } else {
    k_enc_symbols<true><<<nb, 256, 0, s>>>(eb.blocks, eb.perm, (const uint8_t*)eb.coef, eb.sym, eb.stats, eb.pst, eb.status);
    ++L;
  }
  T->mark("encode.huffman", s);
  k_block_huffman<<<(unsigned)((eb.n_blocks + kHuffWarps - 1) / kHuffWarps), 32 * kHuffWarps, 0, s>>>(eb.blocks, eb.perm, eb.stats,
                                                                                                    eb.codes, eb.n_blocks);
  T->mark("encode.layout", s);
  BlockHdr* hdrs = reinterpret_cast<BlockHdr*>(eb.hdrs);
  k_enc_layout<<<(unsigned)((eb.n_blocks + kLayoutWarps - 1) / kLayoutWarps), 32 * kLayoutWarps, 0, s>>>(
      eb.tiles, eb.blocks, eb.perm, eb.pst, eb.sym, eb.codes, hdrs, eb.item_size, eb.status, eb.n_blocks);
  L += 2;
  T->mark("encode.scan", s);
  L += launch_exclusive_scan(eb.item_size, eb.n_blocks, eb.final_pos, eb.scan_part, eb.totals, s);
  T->mark("encode.zero", s);
  k_zero_stream<<<152 * 8, 256, 0, s>>>(reinterpret_cast<uint32_t*>(eb.out), eb.totals, eb.out_capacity);
  T->mark("encode.emit", s);
  const unsigned gg = (unsigned)((eb.n_blocks + kEncGroup - 1) / kEncGroup);
  k_enc_emit<<<gg, 32 * kEmitWarps, kEncSmem, s>>>(eb.tiles, eb.blocks, eb.perm, eb.n_blocks, eb.sym, eb.codes, hdrs, eb.final_pos,
                                                   eb.totals, eb.out_capacity, reinterpret_cast<uint32_t*>(eb.out), eb.status);
  T->mark("encode.tile_headers", s);
  k_tile_headers<<<eb.n_tiles, 128, 0, s>>>(eb.tiles, eb.n_tiles, eb.final_pos, eb.item_size, eb.totals, eb.out, eb.out_capacity,
                                            eb.tile_offsets, eb.status);
  L += 3;
  return L;
}

size_t enc_hdr_bytes() { return sizeof(BlockHdr); }

cudaError_t encode_set_attributes() {
  return cudaFuncSetAttribute(k_enc_emit, cudaFuncAttributeMaxDynamicSharedMemorySize, kEncSmem);
}

}  // namespace isx
