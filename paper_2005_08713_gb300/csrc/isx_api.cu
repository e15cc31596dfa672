// isx_api.cu — the C ABI of include/isx.h: context, scratch arena,
// argument checks, tile planning and the kernel sequences of encode and
// decode.
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>
#include <algorithm>

#include "../../include/isx.h"
#include "isx_internal.cuh"
#include "isx_kernels.h"

namespace isx {
void encode_set_attributes();
void decode_set_attributes();
}  // namespace isx

using namespace isx;

// Optional per-stage timing: events recorded between the kernel groups of
// a call, folded into running totals by isx_stage_times().
struct StageTimer : StageMarks {
  bool on = false;
  std::vector<cudaEvent_t> pool;
  std::vector<std::pair<std::string, std::pair<cudaEvent_t, cudaEvent_t>>> pending;
  std::vector<std::pair<std::string, std::pair<double, int64_t>>> totals;   // name -> (ms, count)
  size_t next = 0;
  cudaEvent_t cur = nullptr;
  std::string cur_name;
  cudaEvent_t get() {
    if (next == pool.size()) {
      cudaEvent_t e;
      cudaEventCreate(&e);
      pool.push_back(e);
    }
    return pool[next++];
  }
  void mark(const char* name, cudaStream_t s) override {
    if (!on) return;
    cudaEvent_t e = get();
    cudaEventRecord(e, s);
    if (cur) pending.push_back({cur_name, {cur, e}});
    cur = name ? e : nullptr;
    cur_name = name ? name : "";
  }
  void collect() {
    for (auto& p : pending) {
      float ms = 0.f;
      if (cudaEventSynchronize(p.second.second) != cudaSuccess) continue;
      cudaEventElapsedTime(&ms, p.second.first, p.second.second);
      bool found = false;
      for (auto& t : totals)
        if (t.first == p.first) { t.second.first += ms; t.second.second += 1; found = true; break; }
      if (!found) totals.push_back({p.first, {(double)ms, 1}});
    }
    pending.clear();
    next = 0;
    cur = nullptr;
  }
};

struct isx_ctx {
  StageTimer timer;
  int device = 0;
  size_t budget = 0;
  uint8_t* arena = nullptr;
  size_t arena_size = 0;
  TileDev* h_tiles = nullptr;      // pinned staging for descriptors
  size_t h_tiles_cap = 0;
  int64_t* h_index = nullptr;      // pinned staging for decode tile indices
  size_t h_index_cap = 0;
  int32_t* h_task = nullptr;       // pinned staging: tiles taking the fused shared-memory path
  size_t h_task_cap = 0;
  cudaEvent_t staging_free = nullptr;
  int* d_status = nullptr;
  uint8_t* d_io = nullptr;         // device staging of the host-buffer calls
  size_t d_io_cap = 0;
  std::string err;
  int launches = 0;
};

namespace {

isx_status fail(isx_ctx* c, isx_status st, const std::string& msg) {
  if (c) c->err = msg;
  return st;
}

isx_status cuda_fail(isx_ctx* c, cudaError_t e, const char* where) {
  return fail(c, ISX_ERR_CUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

#define ISX_CUDA(call)                                     \
  do {                                                     \
    cudaError_t e_ = (call);                               \
    if (e_ != cudaSuccess) return cuda_fail(ctx, e_, #call); \
  } while (0)

// Bump allocator over the context's arena; sizes are aligned to 256 bytes.
struct Carve {
  size_t used = 0;
  size_t take(size_t bytes) {
    size_t off = used;
    used += (bytes + 255) & ~(size_t)255;
    return off;
  }
};

isx_status ensure_arena(isx_ctx* ctx, size_t need) {
  if (need <= ctx->arena_size) return ISX_OK;
  if (ctx->budget && need > ctx->budget)
    return fail(ctx, ISX_ERR_OOM, "scratch of " + std::to_string(need) + " bytes exceeds the HBM budget");
  ISX_CUDA(cudaDeviceSynchronize());
  if (ctx->arena) cudaFree(ctx->arena);
  ctx->arena = nullptr;
  ctx->arena_size = 0;
  size_t sz = need + need / 8;
  if (ctx->budget && sz > ctx->budget) sz = need;
  cudaError_t e = cudaMalloc(&ctx->arena, sz);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return fail(ctx, ISX_ERR_OOM, std::string("cudaMalloc of scratch failed: ") + cudaGetErrorString(e));
  }
  ctx->arena_size = sz;
  return ISX_OK;
}

isx_status ensure_staging(isx_ctx* ctx, size_t n_tiles) {
  ISX_CUDA(cudaEventSynchronize(ctx->staging_free));
  if (n_tiles > ctx->h_tiles_cap) {
    if (ctx->h_tiles) cudaFreeHost(ctx->h_tiles);
    ctx->h_tiles = nullptr;
    size_t cap = std::max<size_t>(n_tiles, 1024);
    ISX_CUDA(cudaMallocHost(&ctx->h_tiles, cap * sizeof(TileDev)));
    ctx->h_tiles_cap = cap;
  }
  if (n_tiles > ctx->h_task_cap) {
    if (ctx->h_task) cudaFreeHost(ctx->h_task);
    ctx->h_task = nullptr;
    size_t cap = std::max<size_t>(n_tiles, 1024);
    ISX_CUDA(cudaMallocHost(&ctx->h_task, cap * sizeof(int32_t)));
    ctx->h_task_cap = cap;
  }
  if (n_tiles > ctx->h_index_cap) {
    if (ctx->h_index) cudaFreeHost(ctx->h_index);
    ctx->h_index = nullptr;
    size_t cap = std::max<size_t>(n_tiles, 1024);
    ISX_CUDA(cudaMallocHost(&ctx->h_index, cap * sizeof(int64_t)));
    ctx->h_index_cap = cap;
  }
  return ISX_OK;
}

bool tile_ok(const isx_tile_desc& t, std::string* why) {
  if (t.width < 1 || t.width > 65535 || t.height < 1 || t.height > 65535) { *why = "width/height out of 1..65535"; return false; }
  if (t.channels != 1 && t.channels != 3) { *why = "channels must be 1 or 3"; return false; }
  if (t.bits < 1 || t.bits > 16) { *why = "bits out of 1..16"; return false; }
  if (t.levels < 0 || t.levels > kMaxLevels) { *why = "levels out of 0..15"; return false; }
  if (t.x0 < 0 || t.y0 < 0) { *why = "negative tile origin"; return false; }
  for (int l = 0; l <= t.levels; ++l)
    if (t.qstep_log2[l] > 15) { *why = "qstep_log2 out of 0..15"; return false; }
  return true;
}

// blocks of a tile (all levels, or LL + levels > zmin) and padded coefficients
void tile_counts(const isx_tile_desc& t, int zmin, int64_t* nb, int64_t* ncoef) {
  int64_t b = 0, c = 0;
  int lw = level_dim(t.width, t.levels), lh = level_dim(t.height, t.levels);
  b += (int64_t)ceil_div(lw, kCell) * ceil_div(lh, kCell);
  c += (int64_t)pad4(lw) * pad4(lh);
  for (int l = t.levels; l >= 1 && l > zmin; --l) {
    int gw = level_dim(t.width, l), gh = level_dim(t.height, l);
    b += (int64_t)ceil_div(gw, kCell) * ceil_div(gh, kCell);
    c += 3LL * pad4(gw) * pad4(gh);
  }
  *nb = b * t.channels;
  *ncoef = c * t.channels;
}

void fill_tiledev(TileDev& d, const isx_tile_desc& t) {
  d.pixels = (const uint8_t*)t.pixels;
  d.pitch = t.row_pitch_bytes;
  d.w = t.width; d.h = t.height; d.C = t.channels; d.bits = t.bits; d.L = t.levels;
  d.x0 = t.x0; d.y0 = t.y0;
  for (int k = 0; k < 16; ++k) d.q[k] = k <= t.levels ? t.qstep_log2[k] : 0;
}

struct EncodePlan {
  int64_t n_blocks = 0, coef_bytes = 0, plane_total = 0, header_total = 0, sym_bytes = 0;
  int max_levels = 0, max_dim = 1;
  int n_fused = 0, max_plane_bytes = 0;
};

isx_status plan_encode(isx_ctx* ctx, const isx_tile_desc* tiles, int32_t n, bool need_pixels, bool allow_fused, EncodePlan& P) {
  isx_status st = ensure_staging(ctx, (size_t)n);
  if (st != ISX_OK) return st;
  for (int32_t i = 0; i < n; ++i) {
    const isx_tile_desc& t = tiles[i];
    std::string why;
    if (!tile_ok(t, &why)) return fail(ctx, ISX_ERR_ARG, "tile " + std::to_string(i) + ": " + why);
    if (need_pixels && (!t.pixels || t.row_pitch_bytes < (int64_t)t.width * t.channels * (t.bits <= 8 ? 1 : 2)))
      return fail(ctx, ISX_ERR_ARG, "tile " + std::to_string(i) + ": missing pixels or row pitch too small");
    int64_t nb, nc;
    tile_counts(t, 0, &nb, &nc);
    TileDev& d = ctx->h_tiles[i];
    fill_tiledev(d, t);
    d.nb = (int32_t)nb;
    d.block_base = P.n_blocks;
    d.coef_base = P.coef_bytes;
    d.fused = allow_fused && fused_tile(t.width, t.height, t.bits) ? 1 : 0;
    d.plane_base = d.fused ? 0 : P.plane_total;
    if (d.fused) {
      ctx->h_task[P.n_fused++] = i;
      P.max_plane_bytes = std::max(P.max_plane_bytes, fused_plane_bytes(t.width, t.height));
    } else {
      P.plane_total += (int64_t)t.channels * t.width * t.height;
    }
    d.sym_base = P.sym_bytes;
    P.n_blocks += nb;
    P.coef_bytes += nc * (t.bits <= 12 ? 2 : 4);
    // symbol regions: dmax planes of p*w*h/8 bytes per block, each rounded up to 16
    P.sym_bytes += ((int64_t)dmax_of_bits(t.bits) * (nc / 8 + 16 * nb) + 15) & ~15LL;   // 16-byte aligned regions
    P.header_total += 32 + 4 * nb;
    P.max_levels = std::max(P.max_levels, t.levels);
    P.max_dim = std::max(P.max_dim, std::max(t.width, t.height));
  }
  return ISX_OK;
}

}  // namespace

extern "C" {

isx_status isx_create(isx_ctx** out, int device, size_t hbm_budget_bytes) {
  if (!out) return ISX_ERR_ARG;
  *out = nullptr;
  isx_ctx* ctx = new isx_ctx();
  ctx->device = device;
  ctx->budget = hbm_budget_bytes;
  cudaError_t e = cudaSetDevice(device);
  if (e == cudaSuccess) e = cudaMalloc(&ctx->d_status, sizeof(int));
  if (e == cudaSuccess) e = cudaMemset(ctx->d_status, 0, sizeof(int));
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ctx->staging_free, cudaEventDisableTiming);
  if (e != cudaSuccess) {
    cudaGetLastError();
    delete ctx;
    return ISX_ERR_CUDA;
  }
  encode_set_attributes();
  decode_set_attributes();
  transform_set_attributes();
  *out = ctx;
  return ISX_OK;
}

void isx_destroy(isx_ctx* ctx) {
  if (!ctx) return;
  cudaSetDevice(ctx->device);
  cudaDeviceSynchronize();
  if (ctx->arena) cudaFree(ctx->arena);
  if (ctx->d_io) cudaFree(ctx->d_io);
  if (ctx->d_status) cudaFree(ctx->d_status);
  if (ctx->h_tiles) cudaFreeHost(ctx->h_tiles);
  if (ctx->h_index) cudaFreeHost(ctx->h_index);
  if (ctx->h_task) cudaFreeHost(ctx->h_task);
  if (ctx->staging_free) cudaEventDestroy(ctx->staging_free);
  for (cudaEvent_t e : ctx->timer.pool) cudaEventDestroy(e);
  delete ctx;
}

isx_status isx_set_timing(isx_ctx* ctx, int32_t enable) {
  if (!ctx) return ISX_ERR_ARG;
  ctx->timer.collect();
  ctx->timer.on = enable != 0;
  ctx->timer.totals.clear();
  return ISX_OK;
}

int32_t isx_stage_times(isx_ctx* ctx, char* names, int64_t names_len, double* ms, int64_t* counts, int32_t cap) {
  if (!ctx) return -1;
  ctx->timer.collect();
  int32_t n = 0;
  std::string all;
  for (auto& t : ctx->timer.totals) {
    if (n >= cap) break;
    if (ms) ms[n] = t.second.first;
    if (counts) counts[n] = t.second.second;
    all += t.first;
    all += '\n';
    ++n;
  }
  if (names && names_len > 0) {
    size_t k = std::min<size_t>(all.size(), (size_t)names_len - 1);
    std::memcpy(names, all.data(), k);
    names[k] = 0;
  }
  return n;
}

const char* isx_last_error(isx_ctx* ctx) { return ctx ? ctx->err.c_str() : "null context"; }

int32_t isx_last_launch_count(isx_ctx* ctx) { return ctx ? ctx->launches : 0; }

isx_status isx_sync_status(isx_ctx* ctx, void* stream) {
  if (!ctx) return ISX_ERR_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  ISX_CUDA(cudaStreamSynchronize(s));
  int st = 0;
  ISX_CUDA(cudaMemcpy(&st, ctx->d_status, sizeof(int), cudaMemcpyDeviceToHost));
  ISX_CUDA(cudaMemset(ctx->d_status, 0, sizeof(int)));
  switch (st) {
    case 0: return ISX_OK;
    case kStCapacity: return fail(ctx, ISX_ERR_CAPACITY, "output buffer too small; required size in tile_offsets[n_tiles]");
    case kStCorrupt: return fail(ctx, ISX_ERR_CORRUPT, "malformed compressed stream");
    case kStTimeout: return fail(ctx, ISX_ERR_TIMEOUT, "device wait gave up");
    case kStRange: return fail(ctx, ISX_ERR_ARG, "a sample exceeds its tile's bit depth (values must be below 2^bits)");
    default: return fail(ctx, ISX_ERR_CUDA, "internal consistency check failed on the device (code " + std::to_string(st) + ")");
  }
}

isx_status isx_forward_coefficients(isx_ctx* ctx, const isx_tile_desc* tiles, int32_t n_tiles, int32_t* d_coef, void* stream) {
  if (!ctx || !tiles || n_tiles < 1 || !d_coef) return fail(ctx, ISX_ERR_ARG, "bad arguments");
  cudaStream_t s = (cudaStream_t)stream;
  ISX_CUDA(cudaSetDevice(ctx->device));
  EncodePlan P;
  isx_status st = plan_encode(ctx, tiles, n_tiles, true, false, P);
  if (st != ISX_OK) return st;
  Carve cv;
  size_t o_tiles = cv.take(sizeof(TileDev) * n_tiles);
  size_t o_A = cv.take(4 * (size_t)P.plane_total);
  size_t o_B = cv.take(4 * (size_t)P.plane_total);
  st = ensure_arena(ctx, cv.used);
  if (st != ISX_OK) return st;
  TileDev* d_tiles = (TileDev*)(ctx->arena + o_tiles);
  int32_t* A = (int32_t*)(ctx->arena + o_A);
  int32_t* B = (int32_t*)(ctx->arena + o_B);
  ISX_CUDA(cudaMemcpyAsync(d_tiles, ctx->h_tiles, sizeof(TileDev) * n_tiles, cudaMemcpyHostToDevice, s));
  ISX_CUDA(cudaEventRecord(ctx->staging_free, s));
  int L = launch_forward_transform(d_tiles, n_tiles, P.max_levels, P.max_dim, A, B, ctx->d_status, s);
  L += launch_quantise_planes(d_tiles, n_tiles, A, d_coef, s);
  ctx->launches = L;
  ISX_CUDA(cudaGetLastError());
  return ISX_OK;
}

isx_status isx_encode_tiles(isx_ctx* ctx, const isx_tile_desc* tiles, int32_t n_tiles, void* d_out, size_t out_capacity,
                            uint64_t* d_tile_offsets, void* stream) {
  if (!ctx) return ISX_ERR_ARG;
  if (!tiles || n_tiles < 1 || !d_tile_offsets || (!d_out && out_capacity))
    return fail(ctx, ISX_ERR_ARG, "bad arguments");
  if (reinterpret_cast<uintptr_t>(d_out) & 3) return fail(ctx, ISX_ERR_ARG, "d_out must be 4-byte aligned");
  cudaStream_t s = (cudaStream_t)stream;
  ISX_CUDA(cudaSetDevice(ctx->device));
  EncodePlan P;
  isx_status st = plan_encode(ctx, tiles, n_tiles, true, true, P);
  if (st != ISX_OK) return st;
  const int64_t NB = P.n_blocks;
  const int64_t n_part = NB / 2048 + 2;
  Carve cv;
  size_t o_tiles = cv.take(sizeof(TileDev) * n_tiles);
  size_t o_task = cv.take(sizeof(int32_t) * (size_t)std::max(P.n_fused, 1));
  size_t o_blocks = cv.take(sizeof(BlockDev) * NB);
  size_t o_A = cv.take(4 * (size_t)P.plane_total);
  size_t o_B = cv.take(4 * (size_t)P.plane_total);
  size_t o_coef = cv.take((size_t)P.coef_bytes);
  size_t o_sym = cv.take((size_t)P.sym_bytes);
  size_t o_stats = cv.take(sizeof(BlockStats) * NB);
  size_t o_codes = cv.take(sizeof(BlockCode) * NB);
  size_t o_hdrs = cv.take(enc_hdr_bytes() * NB);
  size_t o_is = cv.take(8 * NB), o_fp = cv.take(8 * NB), o_perm = cv.take(8 * NB), o_bucket = cv.take(8 * 64);
  size_t o_part = cv.take(8 * n_part), o_tot = cv.take(64);
  st = ensure_arena(ctx, cv.used);
  if (st != ISX_OK) return st;
  uint8_t* ar = ctx->arena;
  TileDev* d_tiles = (TileDev*)(ar + o_tiles);
  int32_t* d_task = (int32_t*)(ar + o_task);
  ISX_CUDA(cudaMemcpyAsync(d_tiles, ctx->h_tiles, sizeof(TileDev) * n_tiles, cudaMemcpyHostToDevice, s));
  if (P.n_fused) ISX_CUDA(cudaMemcpyAsync(d_task, ctx->h_task, sizeof(int32_t) * P.n_fused, cudaMemcpyHostToDevice, s));
  ISX_CUDA(cudaEventRecord(ctx->staging_free, s));
  BlockDev* d_blocks = (BlockDev*)(ar + o_blocks);
  int32_t* A = (int32_t*)(ar + o_A);
  int32_t* B = (int32_t*)(ar + o_B);
  uint8_t* coef = ar + o_coef;
  StageTimer& T = ctx->timer;
  if (T.on && !T.pending.empty()) T.collect();
  T.mark("encode.plan", s);
  int L = launch_plan_blocks(d_tiles, n_tiles, 0, d_blocks, s);
  T.mark("encode.transform", s);
  L += launch_fused_forward(d_tiles, d_task, P.n_fused, P.max_plane_bytes, d_blocks, coef, ctx->d_status, s);
  if (P.n_fused < n_tiles) {
    T.mark("encode.transform_global", s);
    L += launch_forward_transform(d_tiles, n_tiles, P.max_levels, P.max_dim, A, B, ctx->d_status, s);
    T.mark("encode.pack", s);
    L += launch_pack_blocks(d_tiles, d_blocks, NB, A, coef, s);
  }
  EncodeBuffers eb;
  eb.tiles = d_tiles; eb.n_tiles = n_tiles; eb.blocks = d_blocks; eb.n_blocks = NB; eb.coef = coef;
  eb.sym = ar + o_sym;
  eb.stats = (BlockStats*)(ar + o_stats);
  eb.codes = (BlockCode*)(ar + o_codes);
  eb.hdrs = ar + o_hdrs;
  eb.item_size = (int64_t*)(ar + o_is); eb.final_pos = (int64_t*)(ar + o_fp);
  eb.scan_part = (int64_t*)(ar + o_part); eb.totals = (int64_t*)(ar + o_tot);
  eb.bucket = (int64_t*)(ar + o_bucket); eb.perm = (int64_t*)(ar + o_perm);
  eb.out = (uint8_t*)d_out; eb.out_capacity = (int64_t)out_capacity;
  eb.tile_offsets = d_tile_offsets; eb.status = ctx->d_status;
  L += launch_encode_coding(eb, s, &T);
  T.mark(nullptr, s);
  ctx->launches = L;
  ISX_CUDA(cudaGetLastError());
  return ISX_OK;
}

isx_status isx_decode_region(isx_ctx* ctx, const void* d_stream, const uint64_t* d_tile_offsets, const isx_tile_desc* tiles,
                             int32_t n_tiles, int32_t level, int32_t rx, int32_t ry, int32_t rw, int32_t rh, int32_t drop_lsb_planes,
                             void* d_out, int64_t out_pitch_bytes, void* stream) {
  if (!ctx) return ISX_ERR_ARG;
  if (!d_stream || !d_tile_offsets || !tiles || n_tiles < 1 || !d_out || rw < 1 || rh < 1 || level < 0 || level > kMaxLevels ||
      drop_lsb_planes < 0 || drop_lsb_planes > kMaxD)
    return fail(ctx, ISX_ERR_ARG, "bad arguments");
  cudaStream_t s = (cudaStream_t)stream;
  ISX_CUDA(cudaSetDevice(ctx->device));
  isx_status st = ensure_staging(ctx, (size_t)n_tiles);
  if (st != ISX_OK) return st;
  const int z = level;
  int C = -1, bits = -1;
  int32_t nsel = 0;
  int64_t n_blocks = 0, plane_total = 0, sym_cap = 0, max_items = 0;
  int max_levels = 0, max_dim = 1, n_fused = 0, max_plane_bytes = 0;
  // fused tiles write their pixels themselves; three-channel ones pass int16 planes between their CTAs
  const bool fstore = true;
  int64_t fplane_total = 0;
  for (int32_t i = 0; i < n_tiles; ++i) {
    const isx_tile_desc& t = tiles[i];
    std::string why;
    if (!tile_ok(t, &why)) return fail(ctx, ISX_ERR_ARG, "tile " + std::to_string(i) + ": " + why);
    const int zw = level_dim(t.width, z), zh = level_dim(t.height, z);
    const int tx = t.x0 >> z, ty = t.y0 >> z;
    if (tx >= rx + rw || ty >= ry + rh || tx + zw <= rx || ty + zh <= ry) continue;
    if (z > t.levels) return fail(ctx, ISX_ERR_ARG, "level exceeds the levels of tile " + std::to_string(i));
    if (C < 0) { C = t.channels; bits = t.bits; }
    if (t.channels != C || (t.bits <= 8) != (bits <= 8))
      return fail(ctx, ISX_ERR_ARG, "tiles of one region must share channels and sample size");
    int64_t nb, nc;
    tile_counts(t, z, &nb, &nc);
    // symbols of every kept plane: at most (1 + magnitude bits) planes of p*w*h/8 bytes each, plus padding
    sym_cap += (int64_t)(t.bits <= 12 ? 16 : kMaxD) * (nc / 8) + 16 * kMaxD * nb;
    max_items += (int64_t)(t.bits <= 12 ? 16 : kMaxD) * nb;
    TileDev& d = ctx->h_tiles[nsel];
    fill_tiledev(d, t);
    d.nb = (int32_t)nb;
    d.block_base = n_blocks;
    d.coef_base = 0;
    d.fused = fused_tile(zw, zh, t.bits) ? 1 : 0;
    d.plane_base = d.fused && fstore ? fplane_total : plane_total;
    if (d.fused) {
      ctx->h_task[n_fused++] = nsel;
      max_plane_bytes = std::max(max_plane_bytes, fused_plane_bytes(zw, zh));
    }
    ctx->h_index[nsel] = i;
    ++nsel;
    n_blocks += nb;
    if (d.fused && fstore) fplane_total += t.channels == 3 ? (3LL * zw * zh + 7) & ~7LL : 0;   // 16-byte aligned planes
    else plane_total += (int64_t)t.channels * zw * zh;
    max_levels = std::max(max_levels, t.levels);
    max_dim = std::max(max_dim, std::max(t.width, t.height));
  }
  if (out_pitch_bytes < (int64_t)rw * std::max(C, 1) * (bits > 8 ? 2 : 1)) return fail(ctx, ISX_ERR_ARG, "output pitch too small");
  ctx->launches = 0;
  if (nsel == 0) return ISX_OK;
  Carve cv;
  size_t o_tiles = cv.take(sizeof(TileDev) * nsel);
  size_t o_idx = cv.take(8 * (size_t)nsel);
  size_t o_task = cv.take(4 * (size_t)std::max(n_fused, 1));
  size_t o_blocks = cv.take(sizeof(BlockDev) * n_blocks);
  size_t o_bb = cv.take(8 * n_blocks), o_bl = cv.take(4 * n_blocks);
  size_t o_info = cv.take(sizeof(DecInfo) * n_blocks), o_sb = cv.take(8 * n_blocks), o_so = cv.take(8 * n_blocks);
  size_t o_part = cv.take(8 * (n_blocks / 2048 + 2)), o_tot = cv.take(64);
  size_t o_tab = cv.take(dec_table_bytes() * n_blocks), o_bucket = cv.take(8 * 2 * 512), o_items = cv.take(8 * (size_t)max_items);
  size_t o_sym = cv.take((size_t)sym_cap + 64);
  size_t o_A = cv.take(4 * (size_t)plane_total), o_B = cv.take(4 * (size_t)plane_total);
  size_t o_fp = cv.take(2 * (size_t)fplane_total), o_tk = cv.take(4 * (size_t)std::max(n_fused, 1));
  st = ensure_arena(ctx, cv.used);
  if (st != ISX_OK) return st;
  uint8_t* ar = ctx->arena;
  TileDev* d_tiles = (TileDev*)(ar + o_tiles);
  int64_t* d_idx = (int64_t*)(ar + o_idx);
  ISX_CUDA(cudaMemcpyAsync(d_tiles, ctx->h_tiles, sizeof(TileDev) * nsel, cudaMemcpyHostToDevice, s));
  ISX_CUDA(cudaMemcpyAsync(d_idx, ctx->h_index, 8 * (size_t)nsel, cudaMemcpyHostToDevice, s));
  int32_t* d_task = (int32_t*)(ar + o_task);
  if (n_fused) ISX_CUDA(cudaMemcpyAsync(d_task, ctx->h_task, 4 * (size_t)n_fused, cudaMemcpyHostToDevice, s));
  ISX_CUDA(cudaEventRecord(ctx->staging_free, s));
  DecodeBuffers db;
  db.tiles = d_tiles; db.n_tiles = nsel; db.tile_index = d_idx;
  db.stream = (const uint8_t*)d_stream; db.stream_offsets = d_tile_offsets;
  db.blocks = (BlockDev*)(ar + o_blocks); db.block_byte = (int64_t*)(ar + o_bb); db.block_len = (int32_t*)(ar + o_bl);
  db.n_blocks = n_blocks; db.z = z; db.drop = drop_lsb_planes;
  db.planes = (int32_t*)(ar + o_A); db.status = ctx->d_status;
  db.info = (DecInfo*)(ar + o_info); db.sym_bytes = (int64_t*)(ar + o_sb); db.sym_off = (int64_t*)(ar + o_so);
  db.scan_part = (int64_t*)(ar + o_part); db.totals = (int64_t*)(ar + o_tot);
  db.sym = ar + o_sym; db.sym_cap = sym_cap;
  db.tables = ar + o_tab; db.bucket = (int64_t*)(ar + o_bucket); db.items = (int64_t*)(ar + o_items); db.max_items = max_items;
  StageTimer& T = ctx->timer;
  if (T.on && !T.pending.empty()) T.collect();
  int L = launch_decode_blocks(db, s, &T);
  T.mark("decode.inverse_transform", s);
  FusedStore fs{d_out, out_pitch_bytes, rx, ry, rw, rh, (int16_t*)(ar + o_fp), (uint32_t*)(ar + o_tk)};
  L += launch_fused_inverse(d_tiles, d_task, n_fused, max_plane_bytes, db, fstore ? &fs : nullptr, s);
  if (n_fused < nsel) {
    T.mark("decode.inverse_global", s);
    L += launch_inverse_transform(d_tiles, nsel, max_levels, z, max_dim, (int32_t*)(ar + o_A), (int32_t*)(ar + o_B), s);
  }
  if (!fstore || n_fused < nsel) {
    T.mark("decode.store", s);
    L += launch_store_region(d_tiles, nsel, z, (int32_t*)(ar + o_A), d_out, out_pitch_bytes, rx, ry, rw, rh, fstore, s);
  }
  T.mark(nullptr, s);
  ctx->launches = L;
  ISX_CUDA(cudaGetLastError());
  return ISX_OK;
}

isx_status isx_encode_tiles_host(isx_ctx* ctx, const isx_tile_desc* tiles, int32_t n_tiles, void* h_out, size_t out_capacity,
                                 uint64_t* h_tile_offsets, void* stream) {
  if (!ctx) return ISX_ERR_ARG;
  if (!tiles || n_tiles < 1 || !h_tile_offsets || (!h_out && out_capacity)) return fail(ctx, ISX_ERR_ARG, "bad arguments");
  cudaStream_t s = (cudaStream_t)stream;
  ISX_CUDA(cudaSetDevice(ctx->device));
  // Group tiles whose host pixels lie in one contiguous span (e.g. tiles of
  // one image) so that each span is copied once.
  struct Span { const uint8_t* lo; const uint8_t* hi; size_t dev; };
  std::vector<int32_t> order(n_tiles);
  for (int32_t i = 0; i < n_tiles; ++i) order[i] = i;
  auto extent = [&](int32_t i, const uint8_t** lo, const uint8_t** hi) {
    const isx_tile_desc& t = tiles[i];
    int bpp = t.channels * (t.bits <= 8 ? 1 : 2);
    *lo = (const uint8_t*)t.pixels;
    *hi = *lo + (int64_t)(t.height - 1) * t.row_pitch_bytes + (int64_t)t.width * bpp;
  };
  for (int32_t i = 0; i < n_tiles; ++i) {
    std::string why;
    if (!tile_ok(tiles[i], &why)) return fail(ctx, ISX_ERR_ARG, "tile " + std::to_string(i) + ": " + why);
    if (!tiles[i].pixels || tiles[i].row_pitch_bytes < (int64_t)tiles[i].width * tiles[i].channels * (tiles[i].bits <= 8 ? 1 : 2))
      return fail(ctx, ISX_ERR_ARG, "tile " + std::to_string(i) + ": missing pixels or row pitch too small");
  }
  std::sort(order.begin(), order.end(), [&](int32_t a, int32_t b) { return tiles[a].pixels < tiles[b].pixels; });
  std::vector<Span> spans;
  std::vector<int32_t> span_of(n_tiles);
  size_t dev_total = 0;
  for (int32_t k = 0; k < n_tiles; ++k) {
    const uint8_t *lo, *hi;
    extent(order[k], &lo, &hi);
    if (!spans.empty() && lo <= spans.back().hi) {
      spans.back().hi = std::max(spans.back().hi, hi);
    } else {
      spans.push_back({lo, hi, 0});
    }
    span_of[order[k]] = (int32_t)spans.size() - 1;
  }
  for (auto& sp : spans) {
    sp.dev = dev_total;
    dev_total += ((size_t)(sp.hi - sp.lo) + 255) & ~(size_t)255;
  }
  const size_t out_dev = (dev_total + 255) & ~(size_t)255;
  const size_t off_dev = out_dev + ((out_capacity + 255) & ~(size_t)255);
  const size_t io_need = off_dev + 8 * (size_t)(n_tiles + 1) + 256;
  if (io_need > ctx->d_io_cap) {
    ISX_CUDA(cudaDeviceSynchronize());
    if (ctx->d_io) cudaFree(ctx->d_io);
    ctx->d_io = nullptr;
    ctx->d_io_cap = 0;
    cudaError_t e = cudaMalloc(&ctx->d_io, io_need);
    if (e != cudaSuccess) { cudaGetLastError(); return fail(ctx, ISX_ERR_OOM, "cudaMalloc of I/O staging failed"); }
    ctx->d_io_cap = io_need;
  }
  for (const auto& sp : spans)
    ISX_CUDA(cudaMemcpyAsync(ctx->d_io + sp.dev, sp.lo, (size_t)(sp.hi - sp.lo), cudaMemcpyHostToDevice, s));
  std::vector<isx_tile_desc> dt(tiles, tiles + n_tiles);
  for (int32_t i = 0; i < n_tiles; ++i) {
    const Span& sp = spans[span_of[i]];
    dt[i].pixels = ctx->d_io + sp.dev + ((const uint8_t*)tiles[i].pixels - sp.lo);
  }
  uint64_t* d_off = (uint64_t*)(ctx->d_io + off_dev);
  isx_status st = isx_encode_tiles(ctx, dt.data(), n_tiles, ctx->d_io + out_dev, out_capacity, d_off, stream);
  if (st != ISX_OK) return st;
  int L = ctx->launches;
  ISX_CUDA(cudaMemcpyAsync(h_tile_offsets, d_off, 8 * (size_t)(n_tiles + 1), cudaMemcpyDeviceToHost, s));
  st = isx_sync_status(ctx, stream);
  ctx->launches = L;
  if (st != ISX_OK) return st;
  uint64_t total = h_tile_offsets[n_tiles];
  if (total) ISX_CUDA(cudaMemcpyAsync(h_out, ctx->d_io + out_dev, (size_t)total, cudaMemcpyDeviceToHost, s));
  ISX_CUDA(cudaStreamSynchronize(s));
  return ISX_OK;
}

isx_status isx_decode_region_host(isx_ctx* ctx, const void* h_stream, const uint64_t* h_tile_offsets, const isx_tile_desc* tiles,
                                  int32_t n_tiles, int32_t level, int32_t rx, int32_t ry, int32_t rw, int32_t rh, int32_t drop_lsb_planes,
                                  void* h_out, int64_t out_pitch_bytes, void* stream) {
  if (!ctx) return ISX_ERR_ARG;
  if (!h_stream || !h_tile_offsets || !tiles || n_tiles < 1 || !h_out || rw < 1 || rh < 1) return fail(ctx, ISX_ERR_ARG, "bad arguments");
  cudaStream_t s = (cudaStream_t)stream;
  ISX_CUDA(cudaSetDevice(ctx->device));
  int C = tiles[0].channels, bpp = C * (tiles[0].bits <= 8 ? 1 : 2);
  const size_t total = (size_t)h_tile_offsets[n_tiles];
  const size_t row_bytes = (size_t)rw * bpp;
  const size_t off_dev = (total + 255) & ~(size_t)255;
  const size_t out_dev = off_dev + ((8 * (size_t)(n_tiles + 1) + 255) & ~(size_t)255);
  const size_t io_need = out_dev + row_bytes * rh + 256;
  if (io_need > ctx->d_io_cap) {
    ISX_CUDA(cudaDeviceSynchronize());
    if (ctx->d_io) cudaFree(ctx->d_io);
    ctx->d_io = nullptr;
    ctx->d_io_cap = 0;
    cudaError_t e = cudaMalloc(&ctx->d_io, io_need);
    if (e != cudaSuccess) { cudaGetLastError(); return fail(ctx, ISX_ERR_OOM, "cudaMalloc of I/O staging failed"); }
    ctx->d_io_cap = io_need;
  }
  ISX_CUDA(cudaMemcpyAsync(ctx->d_io, h_stream, total, cudaMemcpyHostToDevice, s));
  ISX_CUDA(cudaMemcpyAsync(ctx->d_io + off_dev, h_tile_offsets, 8 * (size_t)(n_tiles + 1), cudaMemcpyHostToDevice, s));
  // the rectangle is decoded into a dense, zeroed device buffer, then copied out row by row
  ISX_CUDA(cudaMemsetAsync(ctx->d_io + out_dev, 0, row_bytes * rh, s));
  isx_status st = isx_decode_region(ctx, ctx->d_io, (const uint64_t*)(ctx->d_io + off_dev), tiles, n_tiles, level, rx, ry, rw, rh,
                                    drop_lsb_planes, ctx->d_io + out_dev, (int64_t)row_bytes, stream);
  if (st != ISX_OK) return st;
  ISX_CUDA(cudaMemcpy2DAsync(h_out, (size_t)out_pitch_bytes, ctx->d_io + out_dev, row_bytes, row_bytes, (size_t)rh,
                             cudaMemcpyDeviceToHost, s));
  int L = ctx->launches;
  st = isx_sync_status(ctx, stream);
  ctx->launches = L;
  return st;
}

}  // extern "C"
