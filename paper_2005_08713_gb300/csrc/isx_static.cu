// isx_static.cu — isx_encode_tile_static: the encoder of one tile, working
// entirely in one statically sized device array of this file.
//
// Who needs it: callers that must not allocate device memory at the moment
// they encode.  A serving process that has handed every byte of HBM to its
// own pools cannot let a library grow a scratch arena behind its back, and
// cudaMalloc / cudaFree may synchronise the whole device, stalling every
// other stream of the process.  The context entry points (isx_encode_tiles)
// grow their arena on demand; this one never allocates: its working set is
// the array below, reserved once when the library's module is loaded.
#include <mutex>
#include <string>
#include <cstring>
#include <algorithm>

#include "isx.h"
#include "isx_kernels.h"
#include "isx_host_plan.h"

namespace isx {
namespace {

constexpr size_t kStaticBytes = ISX_STATIC_SCRATCH_BYTES;
__device__ __align__(256) uint8_t g_static_scratch[kStaticBytes];

// Per-device set-up: the array's device address and the kernels' shared
// memory attributes, with that device current.  Recorded as done only when
// every call succeeded, so that a failed set-up is tried again by the next
// call instead of failing every later call on the device.
constexpr int kMaxDevices = 64;
struct StaticSetup {
  bool done = false;
  uint8_t* base = nullptr;
};
StaticSetup g_setup[kMaxDevices];
std::mutex g_setup_mutex;

cudaError_t setup_device(StaticSetup& S) {
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  if (S.done) return cudaSuccess;
  void* p = nullptr;
  cudaError_t e = cudaGetSymbolAddress(&p, g_static_scratch);
  if (e == cudaSuccess) e = encode_set_attributes();
  if (e == cudaSuccess) e = transform_set_attributes();
  if (e != cudaSuccess) return e;
  S.base = static_cast<uint8_t*>(p);
  S.done = true;
  return cudaSuccess;
}

// Writes the tile descriptor, the fused-task list and a zero status word into
// the scratch (kernel parameters instead of a host copy).
__global__ void k_static_begin(TileDev t, TileDev* d_tile, int32_t* d_task, int* d_status) {
  *d_tile = t;
  d_task[0] = 0;
  *d_status = 0;
}

isx_status fail(char* err, size_t err_len, isx_status st, const std::string& msg) {
  if (err && err_len) {
    size_t k = std::min(msg.size(), err_len - 1);
    std::memcpy(err, msg.data(), k);
    err[k] = 0;
  }
  return st;
}

size_t take(size_t* used, size_t bytes) {
  size_t off = *used;
  *used += (bytes + 255) & ~(size_t)255;
  return off;
}

}  // namespace
}  // namespace isx

using namespace isx;

extern "C" isx_status isx_encode_tile_static(const isx_tile_desc* tile, void* d_out, size_t out_capacity, size_t* h_size,
                                             void* stream, char* h_err, size_t err_len) {
  if (h_err && err_len) h_err[0] = 0;
  if (!tile || !h_size || (!d_out && out_capacity)) return fail(h_err, err_len, ISX_ERR_ARG, "bad arguments");
  if (reinterpret_cast<uintptr_t>(d_out) & 3) return fail(h_err, err_len, ISX_ERR_ARG, "d_out must be 4-byte aligned");
  const isx_tile_desc& t = *tile;
  std::string why;
  if (!tile_ok(t, &why)) return fail(h_err, err_len, ISX_ERR_ARG, why);
  if (!t.pixels || t.row_pitch_bytes < (int64_t)t.width * t.channels * (t.bits <= 8 ? 1 : 2))
    return fail(h_err, err_len, ISX_ERR_ARG, "missing pixels or row pitch too small");

  // Blocks and padded coefficients of the tile: the LL band, then three
  // subbands per level, each cut into 128 x 128 cells (Fig. 3).
  int64_t nb = 0, nc = 0;
  tile_counts(t, 0, &nb, &nc);
  TileDev td;
  fill_tiledev(td, t);
  const bool fused = fused_tile(t.width, t.height) && td.coef16;
  const int64_t plane_total = fused ? 0 : (int64_t)t.channels * t.width * t.height;
  const int64_t coef_bytes = nc * (td.coef16 ? 2 : 4);
  const int64_t sym_bytes = ((int64_t)dmax_of_bits(t.bits) * (nc / 8 + 16 * nb) + 15) & ~15LL;
  const int64_t n_part = nb / 2048 + 2;

  size_t used = 0;
  const size_t o_tile = take(&used, sizeof(TileDev));
  const size_t o_task = take(&used, sizeof(int32_t));
  const size_t o_status = take(&used, sizeof(int));
  const size_t o_offsets = take(&used, 2 * sizeof(uint64_t));
  const size_t o_blocks = take(&used, sizeof(BlockDev) * nb);
  const size_t o_A = take(&used, 4 * (size_t)plane_total);
  const size_t o_B = take(&used, 4 * (size_t)plane_total);
  const size_t o_coef = take(&used, (size_t)coef_bytes);
  const size_t o_sym = take(&used, (size_t)sym_bytes);
  const size_t o_stats = take(&used, sizeof(BlockStats) * nb);
  const size_t o_pst = take(&used, sizeof(PlaneStats) * (size_t)nb * dmax_of_bits(t.bits));
  const size_t o_codes = take(&used, sizeof(BlockCode) * nb);
  const size_t o_hdrs = take(&used, enc_hdr_bytes() * nb);
  const size_t o_is = take(&used, 8 * nb), o_fp = take(&used, 8 * nb), o_perm = take(&used, 8 * nb);
  const size_t o_bucket = take(&used, 8 * 64), o_part = take(&used, 8 * n_part), o_tot = take(&used, 64);
  if (used > kStaticBytes)
    return fail(h_err, err_len, ISX_ERR_OOM,
                "tile needs " + std::to_string(used) + " bytes of working memory; the static scratch holds " +
                    std::to_string(kStaticBytes));

  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return fail(h_err, err_len, ISX_ERR_CUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
  if (dev < 0 || dev >= kMaxDevices) return fail(h_err, err_len, ISX_ERR_ARG, "device ordinal beyond 63");
  StaticSetup& S = g_setup[dev];
  e = setup_device(S);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return fail(h_err, err_len, ISX_ERR_CUDA, std::string("static scratch set-up: ") + cudaGetErrorString(e));
  }
  // An error left pending by earlier work of the caller would surface at our
  // launch check below and be reported as ours: refuse the call instead (the
  // error stays pending for its owner), before anything is enqueued.
  e = cudaPeekAtLastError();
  if (e != cudaSuccess)
    return fail(h_err, err_len, ISX_ERR_CUDA, std::string("a CUDA error was pending before the call: ") + cudaGetErrorString(e));

  uint8_t* ar = S.base;
  cudaStream_t s = (cudaStream_t)stream;
  td.nb = (int32_t)nb;
  td.fused = fused ? 1 : 0;
  td.block_base = 0; td.plane_base = 0; td.coef_base = 0; td.sym_base = 0; td.pst_base = 0;

  TileDev* d_tile = (TileDev*)(ar + o_tile);
  int32_t* d_task = (int32_t*)(ar + o_task);
  int* d_status = (int*)(ar + o_status);
  uint64_t* d_offsets = (uint64_t*)(ar + o_offsets);
  BlockDev* d_blocks = (BlockDev*)(ar + o_blocks);
  uint8_t* coef = ar + o_coef;

  k_static_begin<<<1, 1, 0, s>>>(td, d_tile, d_task, d_status);
  launch_plan_blocks(d_tile, 1, 0, d_blocks, s);
  if (fused) {
    launch_fused_forward(d_tile, d_task, 1, t.channels, fused_plane_bytes(t.width, t.height), 1024, d_blocks, coef, d_status, s);
  } else {
    launch_forward_transform(d_tile, 1, t.levels, std::max(t.width, t.height), t.channels, (int32_t*)(ar + o_A), (int32_t*)(ar + o_B),
                             d_status, s);
    launch_pack_blocks(d_tile, d_blocks, nb, (int32_t*)(ar + o_A), coef, s);
  }
  EncodeBuffers eb;
  eb.tiles = d_tile; eb.n_tiles = 1; eb.blocks = d_blocks; eb.n_blocks = nb; eb.coef = coef;
  eb.sym = ar + o_sym;
  eb.stats = (BlockStats*)(ar + o_stats);
  eb.pst = (PlaneStats*)(ar + o_pst);
  eb.codes = (BlockCode*)(ar + o_codes);
  eb.hdrs = ar + o_hdrs;
  eb.item_size = (int64_t*)(ar + o_is); eb.final_pos = (int64_t*)(ar + o_fp);
  eb.scan_part = (int64_t*)(ar + o_part); eb.totals = (int64_t*)(ar + o_tot);
  eb.bucket = (int64_t*)(ar + o_bucket); eb.perm = (int64_t*)(ar + o_perm);
  eb.out = (uint8_t*)d_out; eb.out_capacity = (int64_t)out_capacity;
  eb.tile_offsets = d_offsets; eb.status = d_status;
  // the symbol pass launches per level with CTAs sized to the level's blocks, as for isx_encode_tiles
  level_blocks(t, eb.level_blocks, eb.level_quads);
  struct NoMarks : StageMarks {
    void mark(const char*, cudaStream_t) override {}
  } marks;
  launch_encode_coding(eb, s, &marks);
  e = cudaGetLastError();
  if (e != cudaSuccess) {
    // kernels may already be in flight on the shared scratch and on d_out: the call stays synchronous
    cudaStreamSynchronize(s);
    return fail(h_err, err_len, ISX_ERR_CUDA, std::string("kernel launch: ") + cudaGetErrorString(e));
  }

  // offsets [0, size] and the status word sit next to each other in the scratch
  uint8_t res[32];
  e = cudaMemcpyAsync(res, ar + o_offsets, 16, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(res + 16, ar + o_status, sizeof(int), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) {
    cudaStreamSynchronize(s);
    return fail(h_err, err_len, ISX_ERR_CUDA, std::string("stream: ") + cudaGetErrorString(e));
  }
  uint64_t size = 0;
  int status = 0;
  std::memcpy(&size, res + 8, 8);
  std::memcpy(&status, res + 16, sizeof(int));
  *h_size = (size_t)size;
  if (status == kStCapacity)
    return fail(h_err, err_len, ISX_ERR_CAPACITY,
                "output buffer too small: the stream needs " + std::to_string(size) + " bytes of capacity");
  if (status == kStRange)
    return fail(h_err, err_len, ISX_ERR_ARG, "a sample exceeds the tile's bit depth (values must be below 2^bits)");
  if (status != 0)
    return fail(h_err, err_len, ISX_ERR_INTERNAL,
                "internal consistency check failed on the device (code " + std::to_string(status) + ")");
  return ISX_OK;
}
