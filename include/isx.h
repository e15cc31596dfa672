/* isx.h — C ABI of the GB300 codec library (libisx_gb300.so).
 *
 * The library implements, on one NVIDIA GB300 (sm_103a), the encoder and
 * decoder of Hulsken, "Fast Compression Method for Medical Images on the
 * Web" (2020):  reversible colour transform and recursive 5/3 integer
 * lifting wavelet (Sec. 3, Sec. 4), JPEG 2000-style quantisation (Sec. 3),
 * 128 x 128 coefficient blocks serialised into signed-magnitude bitplanes of
 * 4 x 2 areas (Eq. 1, Eq. 2), empty-plane removal, zero runs with an
 * optimised counter width (Eq. 3), per-block Huffman codes and the
 * compressed block layout of Fig. 3; decoding at any resolution level and
 * with dropped least significant planes (Sec. 4, "Decompression").
 *
 * Conventions for every entry point:
 *  - Pointers named d_* (and isx_tile_desc.pixels) are DEVICE pointers on
 *    the context's GPU; h_* pointers are host memory.  The caller owns all
 *    buffers it passes; the library owns only the scratch of its context.
 *  - `stream` is a cudaStream_t (NULL = legacy default stream).  Calls are
 *    stream ordered and asynchronous unless stated otherwise: results are
 *    valid once the stream has been synchronised.
 *  - Argument errors are returned synchronously and nothing is enqueued.
 *    Data errors found on the GPU (corrupt stream, output capacity) are
 *    recorded in the context's device status word; isx_sync_status()
 *    synchronises the stream and returns (and clears) them.  No kernel
 *    traps and no call aborts the process.
 *  - A context is used by one host thread at a time.
 */
#ifndef ISX_H_
#define ISX_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct isx_ctx isx_ctx;

typedef enum {
  ISX_OK = 0,
  ISX_ERR_ARG = 1,       /* invalid argument (nothing enqueued) */
  ISX_ERR_CAPACITY = 2,  /* output buffer too small; required size reported */
  ISX_ERR_CORRUPT = 3,   /* malformed compressed stream */
  ISX_ERR_OOM = 4,       /* scratch would exceed the context's HBM budget, or cudaMalloc failed */
  ISX_ERR_CUDA = 5,      /* a CUDA runtime call failed */
  ISX_ERR_TIMEOUT = 6,   /* a bounded device-side wait gave up */
  ISX_ERR_INTERNAL = 7   /* an internal consistency check failed: the encoder's plane segment sizes disagree
                            with the bits its Huffman pass counted or with the segments' symbols (the stream
                            is then invalid; nothing was written outside the output buffer) */
} isx_status;

/* Colour transform of a tile (the paper's "optional colorspace
 * transformation", Fig. 1; Sec. 3 allows any number of channels):
 * ISX_CT_DEFAULT applies the JPEG 2000 RCT to three-channel tiles and no
 * transform otherwise; ISX_CT_RCT and ISX_CT_YCOCG_R (Malvar and Sullivan's
 * reversible YCoCg-R) transform channels 0..2 of a tile of 3 or more
 * channels, the other channels are coded as they are. */
#define ISX_CT_DEFAULT 0
#define ISX_CT_NONE 1
#define ISX_CT_RCT 2
#define ISX_CT_YCOCG_R 3

/* One tile: an independent rectangle of an image, transformed on its own.
 * pixels: DEVICE pointer, interleaved HWC samples, uint8 when bits <= 8 and
 * uint16 otherwise, rows `row_pitch_bytes` apart.  `transform` selects the
 * colour transform (ISX_CT_*).  qstep_log2[l-1] is the quantiser step 2^q
 * of wavelet level l (l = 1 is the finest), qstep_log2[levels] the step of
 * the LL band; all 0 = lossless.  x0, y0 place the tile in the image
 * (level-0 pixels) for region decodes.  A field outside its stated range is
 * an argument error (ISX_ERR_ARG). */
typedef struct {
  int32_t width, height;   /* 1 .. 65535 */
  int32_t channels;        /* 1 .. 16 */
  int32_t bits;            /* significant bits per sample, 1 .. 16 */
  int32_t levels;          /* wavelet levels, 0 .. 15 */
  int32_t x0, y0;          /* tile origin in the image, >= 0 */
  uint8_t qstep_log2[16];  /* 0 .. 15 each */
  const void* pixels;      /* device pointer (ignored by decode calls) */
  int64_t row_pitch_bytes;
  int32_t transform;       /* ISX_CT_DEFAULT .. ISX_CT_YCOCG_R; RCT and YCoCg-R need channels >= 3 */
  int32_t reserved;        /* 0 */
} isx_tile_desc;

/* Creates a context on CUDA device `device`.  hbm_budget_bytes caps the
 * scratch the context may hold (0 = no cap). */
isx_status isx_create(isx_ctx** out, int device, size_t hbm_budget_bytes);

/* Frees the context and its scratch (synchronises the device first). */
void isx_destroy(isx_ctx* ctx);

/* Encode n_tiles tiles into one contiguous stream (Fig. 1 left to right,
 * Fig. 2 a-e, Fig. 3).
 *   tiles          HOST array of n_tiles descriptors (pixels on the device).
 *   d_out          DEVICE buffer of out_capacity bytes, 4-byte aligned,
 *                  receiving the tile streams back to back, tile i at
 *                  d_tile_offsets[i].  The stream is written in whole
 *                  32-bit words: it needs its size rounded up to a
 *                  multiple of 4 bytes of capacity.
 *   d_tile_offsets DEVICE array of n_tiles + 1 uint64; [n_tiles] is the
 *                  total size.  If the stream does not fit, nothing is
 *                  written to d_out, [n_tiles] receives the capacity it
 *                  needs and isx_sync_status returns ISX_ERR_CAPACITY.
 * Tile stream layout (little endian): "ISX1", u16 width, u16 height,
 * u8 channels, u8 bits, u8 levels, u8 colour transform of channels 0..2
 * (0 none, 1 RCT, 2 YCoCg-R),
 * u32 n_blocks, u8 qstep_log2[16], u32 block_end[n_blocks], block data.
 * Blocks: per channel the LL blocks, then the high-pass blocks of levels
 * L .. 1, each subband cut into 128 x 128 cells in raster order.  The bytes
 * are identical to those of the reference CPU codec. */
isx_status isx_encode_tiles(isx_ctx* ctx, const isx_tile_desc* tiles, int32_t n_tiles, void* d_out,
                            size_t out_capacity, uint64_t* d_tile_offsets, void* stream);

/* Decode the rectangle (rx, ry, rw, rh), given in pixels of resolution level
 * `level` (0 = full size; level z halves the size z times: the decoder
 * skips the high-pass blocks of the z finest levels and inverts the rest,
 * Sec. 4), from tiles encoded by isx_encode_tiles.
 *   d_stream, d_tile_offsets  DEVICE stream and its n_tiles + 1 offsets.
 *   tiles           HOST array describing the same tiles (pixels ignored).
 *   drop_lsb_planes discards that many least significant magnitude planes
 *                   of every block (Sec. 4, quality-progressive decode).
 *   d_out           DEVICE buffer, rh rows of rw * channels samples
 *                   (uint8 for bits <= 8, else uint16), out_pitch_bytes
 *                   apart.  Every tile must share channels and bits.
 * A tile covers [x0 >> level, (x0 >> level) + ceil(width / 2^level)) at
 * level `level`.  Pixels of the rectangle that no tile covers are left
 * unchanged.  level must not exceed the levels of any tile it touches. */
isx_status isx_decode_region(isx_ctx* ctx, const void* d_stream, const uint64_t* d_tile_offsets,
                             const isx_tile_desc* tiles, int32_t n_tiles, int32_t level, int32_t rx,
                             int32_t ry, int32_t rw, int32_t rh, int32_t drop_lsb_planes, void* d_out,
                             int64_t out_pitch_bytes, void* stream);

/* End-to-end encode of tiles held in HOST memory (pinned or pageable):
 * copies every tile's pixels to the device (tiles[i].pixels is a HOST
 * pointer here), encodes them, and copies the stream and the offsets back
 * into h_out (out_capacity bytes) and h_tile_offsets (n_tiles + 1).
 * Synchronous: returns once the host buffers hold the result. */
isx_status isx_encode_tiles_host(isx_ctx* ctx, const isx_tile_desc* tiles, int32_t n_tiles, void* h_out,
                                 size_t out_capacity, uint64_t* h_tile_offsets, void* stream);

/* End-to-end region decode from a HOST stream: copies the stream
 * (h_tile_offsets[n_tiles] bytes) and offsets to the device, decodes as
 * isx_decode_region and copies the rw x rh x channels result into h_out
 * (pixels that no tile covers are written as 0).  Synchronous.  A decode of
 * at least 64 MB of pixels and 32 tiles inverts its tiles in chunks and
 * copies each chunk's rows back on a stream of the context's own while the
 * next chunk is inverted (h_out pinned lets those copies overlap); the
 * result is the same. */
isx_status isx_decode_region_host(isx_ctx* ctx, const void* h_stream, const uint64_t* h_tile_offsets,
                                  const isx_tile_desc* tiles, int32_t n_tiles, int32_t level, int32_t rx,
                                  int32_t ry, int32_t rw, int32_t rh, int32_t drop_lsb_planes, void* h_out,
                                  int64_t out_pitch_bytes, void* stream);

/* Forward transform stage alone: colour transform (Fig. 1), 5/3 lifting
 * wavelet (Sec. 4) and quantisation (Sec. 3) of each tile, written as
 * int32 Mallat planes (per tile, channels planes of height x width, tiles
 * back to back; per level HL top-right, LH bottom-left, HH bottom-right) to
 * d_coef, a DEVICE buffer owned by the caller, which must hold
 * sum(channels * width * height) elements.  Asynchronous; argument errors
 * as isx_encode_tiles. */
isx_status isx_forward_coefficients(isx_ctx* ctx, const isx_tile_desc* tiles, int32_t n_tiles,
                                    int32_t* d_coef, void* stream);

/* Synchronises `stream` and returns the first data error recorded on the
 * device since the last call (ISX_OK if none), then clears it. */
isx_status isx_sync_status(isx_ctx* ctx, void* stream);

/* Stage timing for profiling: when enabled, CUDA events are recorded
 * between the kernel groups of every encode/decode call on its stream
 * (stage names such as "encode.emit" or "decode.blocks").  Enabling or
 * disabling clears the running totals. */
isx_status isx_set_timing(isx_ctx* ctx, int32_t enable);

/* Running totals of the stage timings: writes up to `cap` entries of total
 * milliseconds (ms) and call counts (counts), and the stage names, one per
 * line, into `names` (names_len bytes, NUL terminated).  Synchronises on the
 * recorded events.  Returns the number of stages, or -1 for a null ctx. */
int32_t isx_stage_times(isx_ctx* ctx, char* names, int64_t names_len, double* ms, int64_t* counts, int32_t cap);

/* Number of kernels the last encode/decode call enqueued. */
int32_t isx_last_launch_count(isx_ctx* ctx);

/* Message for the last error on this context (static storage). */
const char* isx_last_error(isx_ctx* ctx);

/* Which inverse transform a decode of `tile` at `level` with
 * `drop_lsb_planes` dropped planes (Sec. 4, "Decompression") takes:
 * 1 = the fused shared-memory inverse, which holds every sample of the
 * 5/3 synthesis (Sec. 4) in int16; 0 = the global inverse in int32
 * planes; -1 = an invalid descriptor, level or drop.  Host computation
 * only (no GPU needed).  h_bound (HOST, optional) receives the proven
 * bound on the magnitude of every value the inverse holds for streams the
 * encoder wrote: the forward transform's range for the tile's bit depth
 * and channel count (5/3 filter gains plus rounding) plus the largest
 * deviation the tile's quantiser steps and the dropped planes can carry
 * through the synthesis.  The fused inverse is taken only when the tile
 * fits its shared-memory plane (width and height at level `level` up to
 * 1024, plane <= 160 KB) and the bound is at most 32767. */
int32_t isx_decode_path(const isx_tile_desc* tile, int32_t level, int32_t drop_lsb_planes, double* h_bound);

/* Per-tile latency stamps: d_stamps is a DEVICE array of 4 * n_tiles uint64
 * (nanoseconds of the GPU's global timer, %globaltimer) owned by the
 * caller, or NULL to stop.  Later calls on the context (and plans created
 * while it is set) record, for tile i (its index in tiles[] for an encode,
 * its index in the stream's offset table for a decode):
 *   [i]            encode start: the earliest start of its first kernel,
 *   [n_tiles + i]  encode end: its tile header written, the last step of
 *                  its stream,
 *   [2 n_tiles + i] decode start: its stream header parsed,
 *   [3 n_tiles + i] decode end: its pixels stored.
 * Each encode (decode) clears its two arrays on its stream before its
 * kernels (start to ~0, end to 0), so tiles a call does not touch keep
 * those values.  A call with more tiles than n_tiles is an argument error.
 * No counterpart in the paper: this measures tile latency inside batches. */
isx_status isx_set_tile_stamps(isx_ctx* ctx, uint64_t* d_stamps, int32_t n_tiles);

/* ------------------------------------------------------------------------
 * Batching and serving.  These entry points have no counterpart in the
 * paper; they organise many tiles and many requests around the same coding
 * kernels.
 * ---------------------------------------------------------------------- */

/* One decode job: the part of tile `tile` (index into tiles[] and into the
 * stream's offset table) that lies inside the rectangle (rx, ry, rw, rh) of
 * level-`level` pixels is written to d_out, a DEVICE pointer to the
 * rectangle's pixel (rx, ry), rows out_pitch_bytes apart, in the tile's own
 * sample format (channels interleaved; uint8 for bits <= 8, else uint16).
 * Pixels of the rectangle outside the tile are left unchanged. */
typedef struct {
  int32_t tile;
  int32_t rx, ry, rw, rh;
  void* d_out;
  int64_t out_pitch_bytes;
} isx_decode_job;

/* Decode any number of jobs in one call (every job at the same level and
 * LSB drop; level and drop as in isx_decode_region, Sec. 4
 * "Decompression"): a region decode is the set of jobs of the tiles meeting the
 * region, all pointing into one image; a batch of tiles can be decoded each
 * into its own buffer; jobs of several requests can share the call.  Tiles
 * of different channel counts and bit depths may be mixed.  Asynchronous,
 * errors as isx_decode_region. */
isx_status isx_decode_jobs(isx_ctx* ctx, const void* d_stream, const uint64_t* d_tile_offsets,
                           const isx_tile_desc* tiles, int32_t n_tiles, const isx_decode_job* jobs,
                           int32_t n_jobs, int32_t level, int32_t drop_lsb_planes, void* stream);

/* Device scratch (bytes) that isx_decode_jobs would need for these jobs
 * (host computation only; d_out pointers are not read). */
isx_status isx_decode_jobs_scratch(isx_ctx* ctx, const isx_tile_desc* tiles, int32_t n_tiles,
                                   const isx_decode_job* jobs, int32_t n_jobs, int32_t level,
                                   int32_t drop_lsb_planes, size_t* bytes);

/* Grows the context's scratch to at least `bytes` now (synchronises the
 * device when it grows), so that later calls up to that size allocate
 * nothing; ISX_ERR_OOM beyond the context's HBM budget. */
isx_status isx_reserve_scratch(isx_ctx* ctx, size_t bytes);

/* Bytes of device scratch the context holds. */
size_t isx_scratch_bytes(isx_ctx* ctx);

/* Fused transform schedule.  Tiles whose int16 channel plane fits in shared
 * memory (width and height <= 1024, plane <= 160 KB) and whose samples keep
 * every coefficient inside int16 (see isx_decode_path) are transformed by
 * one CTA per tile and channel; they are grouped in
 * ISX_SIZE_CLASSES classes by plane size (<= 4 KB, 16 KB, 48 KB, 96 KB,
 * 160 KB) and each class launches with its own threads per CTA (256, 512
 * or 1024) for the forward and the inverse transform. */
#define ISX_SIZE_CLASSES 5
typedef struct {
  int32_t forward_threads[ISX_SIZE_CLASSES];
  int32_t inverse_threads[ISX_SIZE_CLASSES];
} isx_schedule;

isx_status isx_get_schedule(isx_ctx* ctx, isx_schedule* out);
/* Every entry must be 256, 512 or 1024 (ISX_ERR_ARG otherwise). */
isx_status isx_set_schedule(isx_ctx* ctx, const isx_schedule* schedule);

/* Autotuner: encodes and decodes `tiles` (device pixels) once, then times
 * the fused forward and inverse launches of every size class present with
 * each thread count, `reps` launches each (CUDA events on `stream`), and
 * keeps the fastest per class in the context's schedule, which later calls
 * and plans use.  Synchronous; allocates temporary device buffers. */
isx_status isx_autotune(isx_ctx* ctx, const isx_tile_desc* tiles, int32_t n_tiles, int32_t reps, void* stream);

/* Plans: an encode of a fixed set of tiles, or a decode of a fixed set of
 * jobs, prepared once (host planning, device memory of its own, descriptors
 * uploaded; uses the context's schedule at creation).  Launching a plan
 * enqueues only kernels and memsets on `stream`, with no host
 * synchronisation and no allocation, so a launch can be captured into a
 * CUDA graph and replayed.  A plan is used from one host thread at a time
 * and by one launch in flight at a time (its scratch is reused).  Data
 * errors go to the plan's own device status word (isx_plan_sync_status). */
typedef struct isx_plan isx_plan;
isx_status isx_plan_encode(isx_ctx* ctx, const isx_tile_desc* tiles, int32_t n_tiles, isx_plan** out);
isx_status isx_plan_decode(isx_ctx* ctx, const isx_tile_desc* tiles, int32_t n_tiles,
                           const isx_decode_job* jobs, int32_t n_jobs, int32_t level,
                           int32_t drop_lsb_planes, isx_plan** out);
/* Same output contract as isx_encode_tiles (the tiles' pixels are read at
 * launch time from the pointers given at creation). */
isx_status isx_plan_launch_encode(isx_plan* plan, void* d_out, size_t out_capacity,
                                  uint64_t* d_tile_offsets, void* stream);
/* Decodes the plan's jobs from d_stream / d_tile_offsets (same tiles). */
isx_status isx_plan_launch_decode(isx_plan* plan, const void* d_stream, const uint64_t* d_tile_offsets,
                                  void* stream);
/* Synchronises `stream`, returns and clears the first data error of the
 * plan's launches since the last call. */
isx_status isx_plan_sync_status(isx_plan* plan, void* stream);
/* Device memory the plan holds (bytes), for admission by memory budget. */
size_t isx_plan_device_bytes(const isx_plan* plan);
/* Kernels the last launch enqueued. */
int32_t isx_plan_launch_count(const isx_plan* plan);
const char* isx_plan_last_error(const isx_plan* plan);
/* Synchronises the device and frees the plan. */
void isx_plan_destroy(isx_plan* plan);

/* One rectangle copy of isx_copy_rects: `rows` rows of `row_bytes` bytes
 * from src (rows src_pitch bytes apart) to dst (dst_pitch apart); DEVICE
 * pointers. */
typedef struct {
  const void* src;
  int64_t src_pitch;
  void* dst;
  int64_t dst_pitch;
  int32_t row_bytes, rows;
} isx_rect_copy;

/* Copies n rectangles (HOST array of descriptors, device data) in one
 * launch on `stream`: a viewport server assembles many requests from
 * decoded tiles and resident levels with one call.  No counterpart in the
 * paper.  Any byte offsets, pitches and row lengths (rectangles with 0
 * rows or 0 row bytes are skipped); each rectangle runs as pieces of at
 * most 32 rows.  Asynchronous; the descriptors are staged in the
 * context's pinned memory before returning (the call waits for the copy
 * of the previous call's descriptors).  Rectangles must not overlap one
 * another's destinations, nor a destination a source.
 * Errors: ISX_ERR_ARG for a negative count, size or row count, or a null
 * pointer of a non-empty rectangle; ISX_ERR_CUDA from the runtime. */
isx_status isx_copy_rects(isx_ctx* ctx, const isx_rect_copy* copies, int32_t n, void* stream);

/* Size of the library's static device scratch array (16 MiB), the whole
 * working memory of isx_encode_tile_static. */
#define ISX_STATIC_SCRATCH_BYTES ((size_t)16 << 20)

/* Encodes ONE tile without allocating anything: no cudaMalloc, no
 * cudaFree, no pinned host buffer, no context.  The paper has no
 * counterpart; this is a service entry point for callers that may not
 * allocate device memory while they encode (a server whose HBM is all
 * handed out to its own pools; code that cannot afford the device-wide
 * synchronisation an allocation or a free may cause).  Its bytes are
 * identical to those of isx_encode_tiles for the same tile.
 *   tile      HOST pointer to one descriptor (pixels on the device).
 *   d_out     DEVICE buffer of out_capacity bytes, 4-byte aligned, as for
 *             isx_encode_tiles (capacity >= size rounded up to 4).
 *   h_size    HOST; receives the stream size, or on ISX_ERR_CAPACITY the
 *             capacity the stream needs (nothing is written to d_out).
 *   stream    cudaStream_t the work is enqueued on (NULL = legacy stream).
 *   h_err     optional HOST buffer of err_len bytes for an error message.
 * Runs on the calling thread's current CUDA device and is SYNCHRONOUS: it
 * returns after `stream` has finished the work.  All working memory (tile
 * descriptor, blocks, planes, coefficients, symbols, codes, offsets and the
 * status word) is carved from one file-scope __device__ array of
 * ISX_STATIC_SCRATCH_BYTES per device, reserved when the library's device
 * code is loaded.  A tile whose working set exceeds it is rejected before
 * anything is enqueued with ISX_ERR_OOM and a message giving both sizes;
 * every tile of at most 512 x 512 pixels and 4 channels fits, at any bit
 * depth, colour transform and level count.
 * The first call on each device does the set-up: it looks up the array's
 * device address (cudaGetSymbolAddress, with that device current) and sets
 * the kernels' shared-memory attributes; make that first call before any
 * stream capture begins.  A set-up that fails returns ISX_ERR_CUDA and is
 * tried again by the next call.  A CUDA error already pending on the
 * calling thread (left by earlier work) makes the call return ISX_ERR_CUDA
 * before anything is enqueued, leaving that error pending.  Every return,
 * errors included, happens after `stream` has finished the call's work.
 * All calls on one device share the one array.  Each call zeroes what must
 * start at zero (the status word; d_out is cleared by the encoder itself)
 * and writes every other scratch byte before reading it, so calls made one
 * after another need nothing in between; calls that overlap in time (from
 * several host threads on the same device) race on the array and corrupt
 * each other: the caller must serialise them. */
isx_status isx_encode_tile_static(const isx_tile_desc* tile, void* d_out, size_t out_capacity, size_t* h_size,
                                  void* stream, char* h_err, size_t err_len);

#ifdef __cplusplus
}
#endif
#endif /* ISX_H_ */
