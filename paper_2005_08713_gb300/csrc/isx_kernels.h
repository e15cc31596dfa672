// isx_kernels.h — host-callable launchers of the library's kernels.  Each
// returns the number of kernels it enqueued (counted for the benchmark).
#pragma once
#include <cstdint>
#include <cuda_runtime.h>
#include "isx.h"
#include "isx_internal.cuh"

namespace isx {

int launch_exclusive_scan(const int64_t* in, int64_t n, int64_t* out, int64_t* part, int64_t* total, cudaStream_t s);
int launch_plan_blocks(const TileDev* d_tiles, int n_tiles, int min_level, BlockDev* d_blocks, cudaStream_t s);
// status: kStRange when a sample exceeds its tile's bit depth
// Global (int32, HBM) path of the tiles with TileDev::fused = 0; max_c = the largest channel count.
int launch_forward_transform(const TileDev* d_tiles, int n_tiles, int max_levels, int max_dim, int max_c, int32_t* A, int32_t* B,
                             int* status, cudaStream_t s);
int launch_pack_blocks(const TileDev* d_tiles, const BlockDev* d_blocks, int64_t n_blocks, const int32_t* planes, void* coef,
                       cudaStream_t s);
// Fused forward transform of n_fused tiles of one size class (as above):
// `slots` CTAs per tile (the class's largest channel count; CTA c takes
// channel c).
int launch_fused_forward(const TileDev* d_tiles, const int32_t* d_task_tile, int n_fused, int slots, int smem_bytes, int threads,
                         const BlockDev* d_blocks, void* coef, int* status, cudaStream_t s);
bool fused_tile(int w, int h);   // geometry: the int16 channel plane fits in shared memory
int fused_plane_bytes(int w, int h);
cudaError_t transform_set_attributes();   // dynamic shared memory limits of the fused transforms (current device)
int launch_quantise_planes(const TileDev* d_tiles, int n_tiles, const int32_t* planes, int32_t* out, cudaStream_t s);
int launch_inverse_transform(const TileDev* d_tiles, int n_tiles, int max_levels, int z, int max_dim, int max_c, int32_t* A,
                             int32_t* B, cudaStream_t s);
// Pixels of the tiles not taken by the fused kernels (TileDev::fused = 0) into their destinations.
int launch_store_region(const TileDev* d_tiles, int n_tiles, int z, const int32_t* planes, cudaStream_t s);
// isx_copy_rects: one CTA per piece (a rectangle's rows split in runs of at most kCopyPieceRows; pieces
// on the device).
constexpr int kCopyPieceRows = 32;
int launch_copy_rects(const isx_rect_copy* pieces, int n, cudaStream_t s);
// Inverse transform and store of the windowed tiles (TileDev::win >= 0): levels max_levels .. z+1 on their
// window planes, then the level-z window into the destinations.
int launch_window_inverse(const TileDev* d_tiles, int n_tiles, int max_levels, int z, int max_c, const WinDev* wins,
                          int32_t* planes, int max_win, cudaStream_t s);

// encode coding stages
struct EncodeBuffers {
  const TileDev* tiles;
  int n_tiles;
  const BlockDev* blocks;
  int64_t n_blocks;
  const void* coef;          // int16 or int32 per block (BlockDev::coef16), byte offsets
  uint8_t* sym;              // symbol regions (BlockDev::sym)
  BlockStats* stats;
  PlaneStats* pst;           // dmax slots per block from BlockDev::pst
  BlockCode* codes;
  void* hdrs;                // [n_blocks] enc_hdr_bytes() each
  int64_t* item_size;        // [n_blocks] block bytes, plus its tile header for a tile's first block
  int64_t* final_pos;        // [n_blocks]
  int64_t* scan_part;
  int64_t* totals;           // [2]: stream size, scratch
  int64_t* bucket;           // [2 * 16]
  int64_t* perm;             // [n_blocks] blocks ordered by level
  uint8_t* out;              // 4-byte aligned
  int64_t out_capacity;
  uint64_t* tile_offsets;    // [n_tiles + 1]
  int* status;
  // Blocks per level (BlockDev::level; the level sort puts them in this order)
  // and the largest block of each level in area quads: the symbol pass then
  // launches per level with CTAs sized to the blocks (all zero: one launch).
  int64_t level_blocks[16] = {};
  int level_quads[16] = {};
};
size_t enc_hdr_bytes();
cudaError_t encode_set_attributes();   // dynamic shared memory limits of the coding kernels (current device)

// Records an event between kernel groups: closes the open stage and opens
// `name` (nullptr: none).  A no-op unless timing is enabled.
struct StageMarks {
  virtual void mark(const char* name, cudaStream_t s) = 0;
  virtual ~StageMarks() = default;
};
int launch_encode_coding(const EncodeBuffers& eb, cudaStream_t s, StageMarks* T);

// decode stages
struct DecodeBuffers {
  const TileDev* tiles;      // selected tiles (plane_base over level-z planes)
  int n_tiles;
  const int64_t* tile_index; // [n_tiles] index of each selected tile in the stream's offset table
  const uint8_t* stream;
  const uint64_t* stream_offsets;
  BlockDev* blocks;
  int64_t* block_byte;       // [n_blocks] byte offset of each block in the stream
  int32_t* block_len;        // [n_blocks]
  int64_t n_blocks;
  int z, drop;
  int32_t* planes;
  DecInfo* info;             // [n_blocks]
  int64_t* sym_bytes;        // [n_blocks]
  int64_t* sym_off;          // [n_blocks]
  int64_t* scan_part;
  int64_t* totals;           // [8]: symbol buffer bytes, segment items, level sort, one-warp segments, their work counter
  void* tables;              // [n_blocks] decode tables (dec_table_bytes() each)
  int64_t* bucket;           // [2 * 64] counts / offsets of the sort buckets
  int64_t* items;            // [max_items] (block << 5 | plane), blocks by level, planes in order
  int64_t max_items;
  int64_t* perm;             // [n_blocks] blocks by level
  int64_t* item_cnt;         // [n_blocks] kept plane segments of block perm[j]
  int64_t* item_base;        // [n_blocks] first item of block perm[j]
  int64_t* big;              // [max_items] segments decoded by a whole warp (latency mode; count in totals[3])
  bool latency_mode = false; // few blocks: long segments are decoded one warp each
  const WinDev* wins = nullptr;   // windows of the windowed tiles (TileDev::win)
  uint8_t* sym;              // symbol buffer
  int64_t sym_cap;           // its size: an upper bound from the tiles' bit depths
  int* status;
  bool global_rebuild = true;   // some selected tile takes the global (non-fused) inverse
};
int launch_decode_blocks(const DecodeBuffers& db, cudaStream_t s, StageMarks* T);
// Fused inverse (decode) of n_fused tiles of one size class, `slots` CTAs
// per tile of `threads` threads (256, 512 or 1024) with smem_bytes of
// plane: each tile's pixels go to its destination (TileDev::dst); tiles
// with a colour transform pass the int16 planes of channels 0..2 through
// planes16 (TileDev::plane_base) and the last of those three CTAs, found
// with tickets[n_fused] (zeroed beforehand), inverts the transform; other
// channels are written by their own CTA.
int launch_fused_inverse(const TileDev* d_tiles, const int32_t* d_task_tile, int n_fused, int slots, int smem_bytes, int threads,
                         const DecodeBuffers& db, int16_t* planes16, uint32_t* tickets, cudaStream_t s);
size_t dec_table_bytes();
int launch_level_sort(const BlockDev* blocks, int64_t nb, int64_t* bucket /* 2 * 16 */, int64_t* perm, int64_t* scan_part,
                      int64_t* total, cudaStream_t s);

}  // namespace isx
