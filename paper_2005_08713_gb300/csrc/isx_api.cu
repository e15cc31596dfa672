// isx_api.cu — the C ABI of include/isx.h: context, scratch arena,
// argument checks, tile planning and the kernel sequences of encode and
// decode.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>
#include <algorithm>

#include "../../include/isx.h"
#include "isx_internal.cuh"
#include "isx_kernels.h"
#include "isx_host_plan.h"

namespace isx {
cudaError_t decode_set_attributes();
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

// Threads per CTA of the fused transforms for each tile size class (bytes
// of the tile's int16 channel plane); set by isx_set_schedule or tuned by
// isx_autotune.
struct Schedule {
  int fwd[ISX_SIZE_CLASSES];
  int inv[ISX_SIZE_CLASSES];
};

// One set of pinned staging buffers for a call's descriptors.  A context
// rotates through kStagingSets of them, so that a call waits only for the
// host-to-device copies of the call kStagingSets calls back (queued work of
// the calls in between does not hold the host).
struct Staging {
  TileDev* h_tiles = nullptr;      // descriptors
  size_t h_tiles_cap = 0;
  int64_t* h_index = nullptr;      // decode tile indices
  size_t h_index_cap = 0;
  int32_t* h_task = nullptr;       // tiles taking the fused shared-memory path
  size_t h_task_cap = 0;
  cudaEvent_t free = nullptr;      // recorded after the copies out of this set
};
constexpr int kStagingSets = 8;

// Host-buffer decodes of at least kIoMinBytes of pixels (and kIoMinTiles
// tiles) overlap the copy of their pixels back with the inverse transform,
// in up to kIoChunks chunks.
constexpr int kIoChunks = 8, kIoMinTiles = 32;
constexpr size_t kIoMinBytes = (size_t)64 << 20;

struct isx_ctx {
  StageTimer timer;
  int device = 0;
  size_t budget = 0;
  uint8_t* arena = nullptr;
  size_t arena_size = 0;
  Staging stage[kStagingSets];
  int stage_next = 0;
  int* d_status = nullptr;
  uint8_t* d_io = nullptr;         // device staging of the host-buffer calls
  size_t d_io_cap = 0;
  Schedule sched;
  std::string err;
  int launches = 0;
  uint64_t* stamps = nullptr;      // per-tile timestamps (isx_set_tile_stamps), 4 x stamp_n
  int32_t stamp_n = 0;
  isx_rect_copy* h_copy = nullptr; // pinned staging of isx_copy_rects
  isx_rect_copy* d_copy = nullptr;
  size_t copy_cap = 0;
  cudaEvent_t copy_free = nullptr;
  // overlapped host-buffer decodes (created on first use): the stream of
  // the copies back to the host, and an event per chunk
  cudaStream_t io_out = nullptr;
  cudaEvent_t io_ev[kIoChunks] = {};
};

namespace {

// upper bounds (plane bytes) of the fused size classes
constexpr int kClassBytes[ISX_SIZE_CLASSES] = {4096, 16384, 49152, 98304, kSmemPlaneBytes};

int class_of(int plane_bytes) {
  for (int k = 0; k < ISX_SIZE_CLASSES; ++k)
    if (plane_bytes <= kClassBytes[k]) return k;
  return ISX_SIZE_CLASSES - 1;
}

Schedule default_schedule() {
  Schedule S;
  const int t[ISX_SIZE_CLASSES] = {256, 256, 512, 1024, 1024};
  for (int k = 0; k < ISX_SIZE_CLASSES; ++k) S.fwd[k] = S.inv[k] = t[k];
  return S;
}

bool valid_threads(int t) { return t == 256 || t == 512 || t == 1024; }

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

// Bump allocator over a device region; sizes are aligned to 256 bytes.
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

// The next staging set, its previous copies complete, with room for n entries.
isx_status ensure_staging(isx_ctx* ctx, size_t n, Staging** out) {
  Staging& g = ctx->stage[ctx->stage_next];
  ctx->stage_next = (ctx->stage_next + 1) % kStagingSets;
  ISX_CUDA(cudaEventSynchronize(g.free));
  if (n > g.h_tiles_cap || n > g.h_task_cap || n > g.h_index_cap) {
    // Freeing pinned memory synchronises the device: every set grows now,
    // so that later calls (whose copies and kernels may be in flight on
    // other streams) find theirs large enough.
    const size_t cap = std::max<size_t>(n, 1024);
    for (Staging& h : ctx->stage) {
      if (h.h_tiles_cap >= n && h.h_task_cap >= n && h.h_index_cap >= n) continue;
      ISX_CUDA(cudaEventSynchronize(h.free));
      if (h.h_tiles_cap < n) {
        if (h.h_tiles) cudaFreeHost(h.h_tiles);
        h.h_tiles = nullptr;
        h.h_tiles_cap = 0;
        ISX_CUDA(cudaMallocHost(&h.h_tiles, cap * sizeof(TileDev)));
        h.h_tiles_cap = cap;
      }
      if (h.h_task_cap < n) {
        if (h.h_task) cudaFreeHost(h.h_task);
        h.h_task = nullptr;
        h.h_task_cap = 0;
        ISX_CUDA(cudaMallocHost(&h.h_task, cap * sizeof(int32_t)));
        h.h_task_cap = cap;
      }
      if (h.h_index_cap < n) {
        if (h.h_index) cudaFreeHost(h.h_index);
        h.h_index = nullptr;
        h.h_index_cap = 0;
        ISX_CUDA(cudaMallocHost(&h.h_index, cap * sizeof(int64_t)));
        h.h_index_cap = cap;
      }
    }
  }
  *out = &g;
  return ISX_OK;
}

bool fused_inverse_fits_int16(const isx_tile_desc& t, int z, int drop) { return inverse_state_bound(t, z, drop) <= 32767.0; }

// Tiles of the fused path grouped by size class: task[] lists them class by
// class; each class launches with its own plane size and thread count.
struct FusedClass {
  int begin = 0, count = 0, smem = 0, threads = 256, slots = 1;   // slots: CTAs per tile, the class's most channels
};

struct FusedTask {
  int32_t task;
  int plane_bytes, channels;
};

// Chunks of a host-buffer decode whose copies back overlap its inverse
// transform: chunk k holds the call's tiles cut[k] .. cut[k+1]-1 (tile
// indices; cut[0] = 0); the fused inverse of chunk k records ev[k] once its
// pixels are stored.
struct IoGate {
  int n = 0;
  int32_t cut[kIoChunks + 1] = {};
  cudaEvent_t ev[kIoChunks] = {};
};

// The sub-range [*pos, e) of a class's tasks whose tile (tile_of(task))
// lies below `end`; advances *pos to e.
template <class F>
int gate_range(const int32_t* task, int count, int* pos, int32_t end, F tile_of) {
  int e = *pos;
  while (e < count && tile_of(task[e]) < end) ++e;
  const int b = *pos;
  *pos = e;
  return b;
}

void group_fused(const std::vector<FusedTask>& fused, const int* threads, int32_t* task, FusedClass* cls) {
  int pos = 0;
  for (int k = 0; k < ISX_SIZE_CLASSES; ++k) {
    cls[k] = FusedClass();
    cls[k].begin = pos;
    cls[k].threads = threads[k];
    for (const auto& f : fused) {
      if (class_of(f.plane_bytes) != k) continue;
      task[pos++] = f.task;
      cls[k].smem = std::max(cls[k].smem, f.plane_bytes);
      cls[k].slots = std::max(cls[k].slots, f.channels);
    }
    cls[k].count = pos - cls[k].begin;
  }
}

// ------------------------------------------------------------ encode
struct EncodeLayout {
  int32_t n_tiles = 0;
  int64_t n_blocks = 0, coef_bytes = 0, plane_total = 0, sym_bytes = 0, pst_slots = 0;
  int max_levels = 0, max_dim = 1, max_c = 1, n_fused = 0;
  FusedClass cls[ISX_SIZE_CLASSES];
  int64_t level_blocks[16] = {};
  int level_quads[16] = {};
  uint64_t* stamps = nullptr;
  int32_t stamp_n = 0;
  size_t o_tiles = 0, o_task = 0, o_blocks = 0, o_A = 0, o_B = 0, o_coef = 0, o_sym = 0, o_stats = 0, o_pst = 0, o_codes = 0, o_hdrs = 0;
  size_t o_is = 0, o_fp = 0, o_perm = 0, o_bucket = 0, o_part = 0, o_tot = 0, total = 0;
};

// Host planning of an encode: descriptors into h_tiles[n], fused tasks into
// h_task[n], sizes and the device layout into E.
isx_status plan_encode(const isx_tile_desc* tiles, int32_t n, bool allow_fused, const Schedule& S, TileDev* h_tiles, int32_t* h_task,
                       EncodeLayout& E, std::string* err, uint64_t* stamps = nullptr, int32_t stamp_n = 0) {
  E = EncodeLayout();
  E.n_tiles = n;
  if (stamps && stamp_n < n) {
    *err = "the tile stamp array holds fewer entries than the call's tiles";
    return ISX_ERR_ARG;
  }
  E.stamps = stamps;
  E.stamp_n = stamp_n;
  std::vector<FusedTask> fused;
  for (int32_t i = 0; i < n; ++i) {
    const isx_tile_desc& t = tiles[i];
    std::string why;
    if (!tile_ok(t, &why)) { *err = "tile " + std::to_string(i) + ": " + why; return ISX_ERR_ARG; }
    if (!t.pixels || t.row_pitch_bytes < (int64_t)t.width * t.channels * (t.bits <= 8 ? 1 : 2)) {
      *err = "tile " + std::to_string(i) + ": missing pixels or row pitch too small";
      return ISX_ERR_ARG;
    }
    int64_t nb, nc;
    tile_counts(t, 0, &nb, &nc);
    level_blocks(t, E.level_blocks, E.level_quads);
    TileDev& d = h_tiles[i];
    fill_tiledev(d, t);
    d.stamps = stamps;
    d.stamp_n = stamp_n;
    d.stamp_i = i;
    d.nb = (int32_t)nb;
    d.block_base = E.n_blocks;
    d.coef_base = E.coef_bytes;
    // the fused kernels hold the plane in int16: only when every state of the forward transform fits
    d.fused = allow_fused && fused_tile(t.width, t.height) && d.coef16 ? 1 : 0;
    d.plane_base = d.fused ? 0 : E.plane_total;
    if (d.fused) fused.push_back({i, fused_plane_bytes(t.width, t.height), t.channels});
    else E.plane_total += (int64_t)t.channels * t.width * t.height;
    d.sym_base = E.sym_bytes;
    d.pst_base = E.pst_slots;
    E.pst_slots += nb * dmax_of_bits(t.bits);
    E.n_blocks += nb;
    E.coef_bytes += nc * (d.coef16 ? 2 : 4);
    E.max_c = std::max(E.max_c, t.channels);
    // symbol regions: dmax planes of p*w*h/8 bytes per block, each rounded up to 16
    E.sym_bytes += ((int64_t)dmax_of_bits(t.bits) * (nc / 8 + 16 * nb) + 15) & ~15LL;
    E.max_levels = std::max(E.max_levels, t.levels);
    E.max_dim = std::max(E.max_dim, std::max(t.width, t.height));
  }
  E.n_fused = (int)fused.size();
  group_fused(fused, S.fwd, h_task, E.cls);
  const int64_t NB = E.n_blocks;
  Carve cv;
  E.o_tiles = cv.take(sizeof(TileDev) * n);
  E.o_task = cv.take(sizeof(int32_t) * (size_t)std::max(E.n_fused, 1));
  E.o_blocks = cv.take(sizeof(BlockDev) * NB);
  E.o_A = cv.take(4 * (size_t)E.plane_total);
  E.o_B = cv.take(4 * (size_t)E.plane_total);
  E.o_coef = cv.take((size_t)E.coef_bytes);
  E.o_sym = cv.take((size_t)E.sym_bytes);
  E.o_stats = cv.take(sizeof(BlockStats) * NB);
  E.o_pst = cv.take(sizeof(PlaneStats) * (size_t)E.pst_slots);
  E.o_codes = cv.take(sizeof(BlockCode) * NB);
  E.o_hdrs = cv.take(enc_hdr_bytes() * NB);
  E.o_is = cv.take(8 * NB);
  E.o_fp = cv.take(8 * NB);
  E.o_perm = cv.take(8 * NB);
  E.o_bucket = cv.take(8 * 64);
  E.o_part = cv.take(8 * (NB / 2048 + 2));
  E.o_tot = cv.take(64);
  E.total = cv.used;
  return ISX_OK;
}

// The kernels of an encode, on descriptors already in the region at `base`.
// Enqueues kernels (and nothing else) on s.
int launch_encode(const EncodeLayout& E, uint8_t* base, void* d_out, size_t out_capacity, uint64_t* d_tile_offsets, int* d_status,
                  StageMarks* T, cudaStream_t s) {
  TileDev* d_tiles = (TileDev*)(base + E.o_tiles);
  int32_t* d_task = (int32_t*)(base + E.o_task);
  BlockDev* d_blocks = (BlockDev*)(base + E.o_blocks);
  int32_t* A = (int32_t*)(base + E.o_A);
  int32_t* B = (int32_t*)(base + E.o_B);
  uint8_t* coef = base + E.o_coef;
  T->mark("encode.plan", s);
  if (E.stamps) {   // start: the earliest kernel of a tile (a minimum), end: its tile header (a maximum)
    cudaMemsetAsync(E.stamps, 0xff, 8 * (size_t)E.stamp_n, s);
    cudaMemsetAsync(E.stamps + E.stamp_n, 0, 8 * (size_t)E.stamp_n, s);
  }
  int L = launch_plan_blocks(d_tiles, E.n_tiles, 0, d_blocks, s);
  T->mark("encode.transform", s);
  for (const FusedClass& c : E.cls)
    L += launch_fused_forward(d_tiles, d_task + c.begin, c.count, c.slots, c.smem, c.threads, d_blocks, coef, d_status, s);  if (E.n_fused < E.n_tiles) {
    T->mark("encode.transform_global", s);
    L += launch_forward_transform(d_tiles, E.n_tiles, E.max_levels, E.max_dim, E.max_c, A, B, d_status, s);
    T->mark("encode.pack", s);
    L += launch_pack_blocks(d_tiles, d_blocks, E.n_blocks, A, coef, s);
  }
  EncodeBuffers eb;
  eb.tiles = d_tiles; eb.n_tiles = E.n_tiles; eb.blocks = d_blocks; eb.n_blocks = E.n_blocks; eb.coef = coef;
  eb.sym = base + E.o_sym;
  eb.stats = (BlockStats*)(base + E.o_stats);
  eb.pst = (PlaneStats*)(base + E.o_pst);
  eb.codes = (BlockCode*)(base + E.o_codes);
  eb.hdrs = base + E.o_hdrs;
  eb.item_size = (int64_t*)(base + E.o_is); eb.final_pos = (int64_t*)(base + E.o_fp);
  eb.scan_part = (int64_t*)(base + E.o_part); eb.totals = (int64_t*)(base + E.o_tot);
  eb.bucket = (int64_t*)(base + E.o_bucket); eb.perm = (int64_t*)(base + E.o_perm);
  eb.out = (uint8_t*)d_out; eb.out_capacity = (int64_t)out_capacity;
  eb.tile_offsets = d_tile_offsets; eb.status = d_status;
  for (int l = 0; l < 16; ++l) {
    eb.level_blocks[l] = E.level_blocks[l];
    eb.level_quads[l] = E.level_quads[l];
  }
  L += launch_encode_coding(eb, s, T);
  T->mark(nullptr, s);
  return L;
}

// ------------------------------------------------------------ decode
// One decode job: the part of tile `tile` inside (rx, ry, rw, rh) (level-z
// pixels) into out, whose first byte is pixel (rx, ry).
struct Job {
  int32_t tile, rx, ry, rw, rh;
  void* out;
  int64_t pitch;
};

struct DecodeLayout {
  int32_t nsel = 0;
  int z = 0, drop = 0;
  int64_t n_blocks = 0, plane_total = 0, fplane_total = 0, sym_cap = 0, max_items = 0;
  int max_levels = 0, max_dim = 1, max_c = 1, n_fused = 0, n_win = 0, max_win = 1;
  FusedClass cls[ISX_SIZE_CLASSES];
  uint64_t* stamps = nullptr;
  int32_t stamp_n = 0;
  size_t o_win = 0;
  size_t o_tiles = 0, o_idx = 0, o_task = 0, o_blocks = 0, o_bb = 0, o_bl = 0, o_info = 0, o_sb = 0, o_so = 0, o_part = 0, o_tot = 0;
  size_t o_tab = 0, o_bucket = 0, o_items = 0, o_sym = 0, o_A = 0, o_B = 0, o_fp = 0, o_tk = 0, total = 0;
  size_t o_perm = 0, o_icnt = 0, o_ibase = 0, o_big = 0;
};

// Host planning of a decode: one descriptor per job whose tile meets its
// rectangle (h_tiles, h_index, h_task hold n_jobs entries).
isx_status plan_decode(const isx_tile_desc* tiles, int32_t n_tiles, const Job* jobs, int32_t n_jobs, int z, int drop, const Schedule& S,
                       TileDev* h_tiles, int64_t* h_index, int32_t* h_task, DecodeLayout& D, std::string* err,
                       uint64_t* stamps = nullptr, int32_t stamp_n = 0, std::vector<WinDev>* wins = nullptr) {
  D = DecodeLayout();
  if (wins) wins->clear();
  D.z = z;
  D.drop = drop;
  if (stamps && stamp_n < n_tiles) {
    *err = "the tile stamp array holds fewer entries than the stream's tiles";
    return ISX_ERR_ARG;
  }
  D.stamps = stamps;
  D.stamp_n = stamp_n;
  std::vector<FusedTask> fused;
  for (int32_t j = 0; j < n_jobs; ++j) {
    const Job& jb = jobs[j];
    if (jb.tile < 0 || jb.tile >= n_tiles) { *err = "job " + std::to_string(j) + ": tile index out of range"; return ISX_ERR_ARG; }
    if (!jb.out || jb.rw < 1 || jb.rh < 1) { *err = "job " + std::to_string(j) + ": bad output rectangle"; return ISX_ERR_ARG; }
    const isx_tile_desc& t = tiles[jb.tile];
    std::string why;
    if (!tile_ok(t, &why)) { *err = "tile " + std::to_string(jb.tile) + ": " + why; return ISX_ERR_ARG; }
    const int zw = level_dim(t.width, z), zh = level_dim(t.height, z);
    const int tx = t.x0 >> z, ty = t.y0 >> z;
    if (tx >= jb.rx + jb.rw || ty >= jb.ry + jb.rh || tx + zw <= jb.rx || ty + zh <= jb.ry) continue;
    if (z > t.levels) { *err = "level exceeds the levels of tile " + std::to_string(jb.tile); return ISX_ERR_ARG; }
    if (jb.pitch < (int64_t)jb.rw * t.channels * (t.bits <= 8 ? 1 : 2)) {
      *err = "job " + std::to_string(j) + ": output pitch too small";
      return ISX_ERR_ARG;
    }
    // A tile too large for the fused inverse whose level-z extent the rectangle covers only in part
    // is decoded through a window: only the blocks and samples the rectangle depends on.
    const int ax = std::max(jb.rx - tx, 0), bx = std::min(jb.rx + jb.rw - tx, zw);
    const int ay = std::max(jb.ry - ty, 0), by = std::min(jb.ry + jb.rh - ty, zh);
    const bool fusable = fused_tile(zw, zh) && fused_inverse_fits_int16(t, z, drop);
    const bool windowed = wins && !fusable && (bx - ax < zw || by - ay < zh);
    WinDev W;
    int64_t nb, nc, win_elems = 0;
    if (windowed) {
      win_elems = plan_window(t, z, ax, bx, ay, by, W);
      window_counts(t, W, &nb, &nc);
    } else {
      tile_counts(t, z, &nb, &nc);
    }
    // symbols of every kept plane: at most 1 + bitlen(F) planes (sign and magnitude; F bounds every
    // coefficient the encoder writes) of p*w*h/8 bytes each, plus padding
    const double F = forward_state_bound(t);
    int64_t planes = 1;
    while (planes < kMaxD && std::ldexp(1.0, (int)planes - 1) <= F) ++planes;
    D.sym_cap += planes * (nc / 8) + 16 * kMaxD * nb;
    D.max_items += planes * nb;
    TileDev& d = h_tiles[D.nsel];
    fill_tiledev(d, t);
    d.stamps = stamps;
    d.stamp_n = stamp_n;
    d.stamp_i = jb.tile;
    d.nb = (int32_t)nb;
    d.block_base = D.n_blocks;
    d.coef_base = 0;
    d.fused = fusable ? 1 : 0;
    d.win = -1;
    d.dst = (uint8_t*)jb.out;
    d.dpitch = jb.pitch;
    d.rx = jb.rx; d.ry = jb.ry; d.rw = jb.rw; d.rh = jb.rh;
    if (d.fused) {
      // tiles with a colour transform hand the int16 planes of channels 0..2 between CTAs: 16-byte aligned
      d.plane_base = D.fplane_total;
      if (d.ct) D.fplane_total += (3LL * zw * zh + 7) & ~7LL;
      fused.push_back({D.nsel, fused_plane_bytes(zw, zh), t.channels});
    } else if (windowed) {
      d.plane_base = D.plane_total;
      D.plane_total += (win_elems + 3) & ~3LL;
      d.win = (int32_t)wins->size();
      wins->push_back(W);
      D.max_win = std::max({D.max_win, bx - ax, by - ay});
      if (z < t.levels) {
        const WinLevel& v = W.lev[z + 1];
        D.max_win = std::max({D.max_win, (v.lx1 - v.lx0) + (v.hx1 - v.hx0), (v.ly1 - v.ly0) + (v.hy1 - v.hy0)});
      }
    } else {
      d.plane_base = D.plane_total;
      D.plane_total += (int64_t)t.channels * zw * zh;
    }
    h_index[D.nsel] = jb.tile;
    ++D.nsel;
    D.n_blocks += nb;
    D.max_levels = std::max(D.max_levels, t.levels);
    if (!windowed) D.max_dim = std::max(D.max_dim, std::max(t.width, t.height));   // grids of the whole-tile passes
    D.max_c = std::max(D.max_c, t.channels);
  }
  D.n_fused = (int)fused.size();
  D.n_win = wins ? (int)wins->size() : 0;
  group_fused(fused, S.inv, h_task, D.cls);
  const int64_t nb = D.n_blocks;
  Carve cv;
  D.o_tiles = cv.take(sizeof(TileDev) * (size_t)std::max(D.nsel, 1));
  D.o_idx = cv.take(8 * (size_t)std::max(D.nsel, 1));
  D.o_task = cv.take(4 * (size_t)std::max(D.n_fused, 1));
  D.o_blocks = cv.take(sizeof(BlockDev) * nb);
  D.o_bb = cv.take(8 * nb);
  D.o_bl = cv.take(4 * nb);
  D.o_info = cv.take(sizeof(DecInfo) * nb);
  D.o_sb = cv.take(8 * nb);
  D.o_so = cv.take(8 * nb);
  D.o_part = cv.take(8 * (nb / 2048 + 2));
  D.o_tot = cv.take(64);
  D.o_tab = cv.take(dec_table_bytes() * nb);
  D.o_bucket = cv.take(8 * 2 * 512);
  D.o_items = cv.take(8 * (size_t)D.max_items);
  D.o_perm = cv.take(8 * nb);
  D.o_icnt = cv.take(8 * nb);
  D.o_ibase = cv.take(8 * nb);
  D.o_big = cv.take(8 * (size_t)D.max_items);
  D.o_win = cv.take(sizeof(WinDev) * (size_t)std::max(D.n_win, 1));
  D.o_sym = cv.take((size_t)D.sym_cap + 64);
  D.o_A = cv.take(4 * (size_t)D.plane_total);
  D.o_B = cv.take(4 * (size_t)D.plane_total);
  D.o_fp = cv.take(2 * (size_t)D.fplane_total);
  D.o_tk = cv.take(4 * (size_t)std::max(D.n_fused, 1));
  D.total = cv.used;
  return ISX_OK;
}

// Decodes of at most this many blocks (about 300 tiles of 256 x 256) run in
// latency mode (DecodeBuffers::latency_mode).
constexpr int64_t kLatencyBlocks = 8192;

// The kernels (and ticket clears) of a decode on descriptors already at base.
int launch_decode(const DecodeLayout& D, uint8_t* base, const void* d_stream, const uint64_t* d_tile_offsets, int* d_status,
                  StageMarks* T, cudaStream_t s, const IoGate* gate = nullptr, const int32_t* h_task = nullptr,
                  const int64_t* h_index = nullptr) {
  if (D.nsel == 0) return 0;
  TileDev* d_tiles = (TileDev*)(base + D.o_tiles);
  int32_t* d_task = (int32_t*)(base + D.o_task);
  DecodeBuffers db;
  db.tiles = d_tiles; db.n_tiles = D.nsel; db.tile_index = (int64_t*)(base + D.o_idx);
  db.stream = (const uint8_t*)d_stream; db.stream_offsets = d_tile_offsets;
  db.blocks = (BlockDev*)(base + D.o_blocks); db.block_byte = (int64_t*)(base + D.o_bb); db.block_len = (int32_t*)(base + D.o_bl);
  db.n_blocks = D.n_blocks; db.z = D.z; db.drop = D.drop;
  db.planes = (int32_t*)(base + D.o_A); db.status = d_status;
  db.info = (DecInfo*)(base + D.o_info); db.sym_bytes = (int64_t*)(base + D.o_sb); db.sym_off = (int64_t*)(base + D.o_so);
  db.scan_part = (int64_t*)(base + D.o_part); db.totals = (int64_t*)(base + D.o_tot);
  db.sym = base + D.o_sym; db.sym_cap = D.sym_cap;
  db.tables = base + D.o_tab; db.bucket = (int64_t*)(base + D.o_bucket); db.items = (int64_t*)(base + D.o_items);
  db.max_items = D.max_items;
  db.perm = (int64_t*)(base + D.o_perm); db.item_cnt = (int64_t*)(base + D.o_icnt); db.item_base = (int64_t*)(base + D.o_ibase);
  db.big = (int64_t*)(base + D.o_big);
  db.wins = (const WinDev*)(base + D.o_win);
  // a decode of few blocks leaves most of the GPU idle: its long segments are decoded one warp each
  db.latency_mode = D.n_blocks <= kLatencyBlocks;
  db.global_rebuild = D.n_fused < D.nsel;
  if (D.stamps) {   // start: its stream header parsed (a minimum), end: its pixels stored (a maximum)
    cudaMemsetAsync(D.stamps + 2 * (size_t)D.stamp_n, 0xff, 8 * (size_t)D.stamp_n, s);
    cudaMemsetAsync(D.stamps + 3 * (size_t)D.stamp_n, 0, 8 * (size_t)D.stamp_n, s);
  }
  int L = launch_decode_blocks(db, s, T);
  T->mark("decode.inverse_transform", s);
  uint32_t* tickets = (uint32_t*)(base + D.o_tk);
  if (D.n_fused) cudaMemsetAsync(tickets, 0, 4 * (size_t)D.n_fused, s);
  // chunk by chunk when every tile takes the fused inverse (tasks are
  // selections, h_index their tiles): chunk k's pixels are then stored when
  // its event fires
  const bool gated = gate && h_task && h_index && D.n_fused == D.nsel && D.n_win == 0;
  if (gated) {
    int pos[ISX_SIZE_CLASSES] = {};
    for (int k = 0; k < gate->n; ++k) {
      for (int ci = 0; ci < ISX_SIZE_CLASSES; ++ci) {
        const FusedClass& c = D.cls[ci];
        const int b = gate_range(h_task + c.begin, c.count, &pos[ci], gate->cut[k + 1],
                                 [h_index](int32_t sel) { return (int32_t)h_index[sel]; });
        if (pos[ci] > b)
          L += launch_fused_inverse(d_tiles, d_task + c.begin + b, pos[ci] - b, c.slots, c.smem, c.threads, db,
                                    (int16_t*)(base + D.o_fp), tickets + c.begin + b, s);
      }
      cudaEventRecord(gate->ev[k], s);
    }
    // The chunks assume each class's tasks in tile order (the jobs of a
    // region decode are); any task left over runs now, and every chunk
    // counts as stored only after it.
    bool rest = false;
    for (int ci = 0; ci < ISX_SIZE_CLASSES; ++ci) {
      const FusedClass& c = D.cls[ci];
      if (pos[ci] < c.count) {
        L += launch_fused_inverse(d_tiles, d_task + c.begin + pos[ci], c.count - pos[ci], c.slots, c.smem, c.threads, db,
                                  (int16_t*)(base + D.o_fp), tickets + c.begin + pos[ci], s);
        rest = true;
      }
    }
    if (rest)
      for (int k = 0; k < gate->n; ++k) cudaEventRecord(gate->ev[k], s);
  } else {
    for (const FusedClass& c : D.cls)
      L += launch_fused_inverse(d_tiles, d_task + c.begin, c.count, c.slots, c.smem, c.threads, db, (int16_t*)(base + D.o_fp),
                                tickets + c.begin, s);
  }
  if (D.n_fused < D.nsel) {
    T->mark("decode.inverse_global", s);
    L += launch_inverse_transform(d_tiles, D.nsel, D.max_levels, D.z, D.max_dim, D.max_c, (int32_t*)(base + D.o_A),
                                  (int32_t*)(base + D.o_B), s);
    T->mark("decode.store", s);
    L += launch_store_region(d_tiles, D.nsel, D.z, (int32_t*)(base + D.o_A), s);
  }
  if (D.n_win) {
    T->mark("decode.inverse_window", s);
    L += launch_window_inverse(d_tiles, D.nsel, D.max_levels, D.z, D.max_c, db.wins, (int32_t*)(base + D.o_A), D.max_win, s);
  }
  if (gate && !gated)   // some tiles took another path: every chunk is complete only now
    for (int k = 0; k < gate->n; ++k) cudaEventRecord(gate->ev[k], s);
  T->mark(nullptr, s);
  return L;
}

struct NoMarks : StageMarks {
  void mark(const char*, cudaStream_t) override {}
};

// Decode of jobs through the context: plan, arena, descriptor upload, kernels.
isx_status decode_jobs_ctx(isx_ctx* ctx, const void* d_stream, const uint64_t* d_tile_offsets, const isx_tile_desc* tiles,
                           int32_t n_tiles, const Job* jobs, int32_t n_jobs, int z, int drop, cudaStream_t s,
                           const IoGate* gate = nullptr) {
  ISX_CUDA(cudaSetDevice(ctx->device));
  Staging* g = nullptr;
  isx_status st = ensure_staging(ctx, (size_t)std::max(n_jobs, 1), &g);
  if (st != ISX_OK) return st;
  DecodeLayout D;
  std::string err;
  std::vector<WinDev> wins;
  st = plan_decode(tiles, n_tiles, jobs, n_jobs, z, drop, ctx->sched, g->h_tiles, g->h_index, g->h_task, D, &err, ctx->stamps,
                   ctx->stamp_n, &wins);
  if (st != ISX_OK) return fail(ctx, st, err);
  ctx->launches = 0;
  if (D.nsel == 0) {
    if (gate)
      for (int k = 0; k < gate->n; ++k) ISX_CUDA(cudaEventRecord(gate->ev[k], s));
    return ISX_OK;
  }
  st = ensure_arena(ctx, D.total);
  if (st != ISX_OK) return st;
  uint8_t* ar = ctx->arena;
  ISX_CUDA(cudaMemcpyAsync(ar + D.o_tiles, g->h_tiles, sizeof(TileDev) * D.nsel, cudaMemcpyHostToDevice, s));
  ISX_CUDA(cudaMemcpyAsync(ar + D.o_idx, g->h_index, 8 * (size_t)D.nsel, cudaMemcpyHostToDevice, s));
  if (D.n_fused) ISX_CUDA(cudaMemcpyAsync(ar + D.o_task, g->h_task, 4 * (size_t)D.n_fused, cudaMemcpyHostToDevice, s));
  // windows from pageable memory: the copy is complete when the call returns
  if (D.n_win) ISX_CUDA(cudaMemcpyAsync(ar + D.o_win, wins.data(), sizeof(WinDev) * (size_t)D.n_win, cudaMemcpyHostToDevice, s));
  ISX_CUDA(cudaEventRecord(g->free, s));
  StageTimer& T = ctx->timer;
  if (T.on && !T.pending.empty()) T.collect();
  ctx->launches = launch_decode(D, ar, d_stream, d_tile_offsets, ctx->d_status, &T, s, gate, g->h_task, g->h_index);
  ISX_CUDA(cudaGetLastError());
  return ISX_OK;
}

}  // namespace

// A prepared encode or decode with its own device memory: launching it only
// enqueues kernels (and ticket clears), so it can be captured in a CUDA graph.
struct isx_plan {
  int kind = 0;   // 1 encode, 2 decode
  int device = 0;
  EncodeLayout E;
  DecodeLayout D;
  uint8_t* mem = nullptr;
  size_t mem_bytes = 0;
  int* d_status = nullptr;
  int launches = 0;
  std::string err;
};

extern "C" {

isx_status isx_create(isx_ctx** out, int device, size_t hbm_budget_bytes) {
  if (!out) return ISX_ERR_ARG;
  *out = nullptr;
  isx_ctx* ctx = new isx_ctx();
  ctx->device = device;
  ctx->budget = hbm_budget_bytes;
  ctx->sched = default_schedule();
  cudaError_t e = cudaSetDevice(device);
  if (e == cudaSuccess) e = cudaMalloc(&ctx->d_status, sizeof(int));
  if (e == cudaSuccess) e = cudaMemset(ctx->d_status, 0, sizeof(int));
  for (int k = 0; k < kStagingSets && e == cudaSuccess; ++k) e = cudaEventCreateWithFlags(&ctx->stage[k].free, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ctx->copy_free, cudaEventDisableTiming);
  if (e != cudaSuccess) {
    cudaGetLastError();
    isx_destroy(ctx);
    return ISX_ERR_CUDA;
  }
  if (e == cudaSuccess) e = encode_set_attributes();
  if (e == cudaSuccess) e = decode_set_attributes();
  if (e == cudaSuccess) e = transform_set_attributes();
  if (e != cudaSuccess) {
    cudaGetLastError();
    isx_destroy(ctx);
    return ISX_ERR_CUDA;
  }
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
  for (Staging& g : ctx->stage) {
    if (g.h_tiles) cudaFreeHost(g.h_tiles);
    if (g.h_index) cudaFreeHost(g.h_index);
    if (g.h_task) cudaFreeHost(g.h_task);
    if (g.free) cudaEventDestroy(g.free);
  }
  if (ctx->copy_free) cudaEventDestroy(ctx->copy_free);
  if (ctx->io_out) cudaStreamDestroy(ctx->io_out);
  for (cudaEvent_t e : ctx->io_ev)
    if (e) cudaEventDestroy(e);
  if (ctx->h_copy) cudaFreeHost(ctx->h_copy);
  if (ctx->d_copy) cudaFree(ctx->d_copy);
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

isx_status isx_copy_rects(isx_ctx* ctx, const isx_rect_copy* copies, int32_t n, void* stream) {
  if (!ctx) return ISX_ERR_ARG;
  if (n < 0 || (n > 0 && !copies)) return fail(ctx, ISX_ERR_ARG, "bad arguments");
  for (int32_t i = 0; i < n; ++i)
    if (copies[i].row_bytes < 0 || copies[i].rows < 0 || ((copies[i].row_bytes > 0 && copies[i].rows > 0) && (!copies[i].src || !copies[i].dst)))
      return fail(ctx, ISX_ERR_ARG, "copy " + std::to_string(i) + ": bad rectangle");
  ctx->launches = 0;
  // each rectangle runs as pieces of at most kCopyPieceRows rows, one CTA a piece
  int64_t pieces = 0;
  for (int32_t i = 0; i < n; ++i)
    if (copies[i].row_bytes > 0 && copies[i].rows > 0) pieces += (copies[i].rows + kCopyPieceRows - 1) / kCopyPieceRows;
  if (pieces == 0) return ISX_OK;
  if (pieces > INT32_MAX) return fail(ctx, ISX_ERR_ARG, "too many rectangle pieces for one launch");
  ISX_CUDA(cudaSetDevice(ctx->device));
  cudaStream_t s = (cudaStream_t)stream;
  ISX_CUDA(cudaEventSynchronize(ctx->copy_free));   // the previous call's descriptors have been copied
  if ((size_t)pieces > ctx->copy_cap) {
    ISX_CUDA(cudaDeviceSynchronize());
    if (ctx->h_copy) cudaFreeHost(ctx->h_copy);
    if (ctx->d_copy) cudaFree(ctx->d_copy);
    ctx->h_copy = nullptr;
    ctx->d_copy = nullptr;
    ctx->copy_cap = 0;
    const size_t cap = std::max<size_t>((size_t)pieces, 65536);
    ISX_CUDA(cudaMallocHost(&ctx->h_copy, cap * sizeof(isx_rect_copy)));
    ISX_CUDA(cudaMalloc(&ctx->d_copy, cap * sizeof(isx_rect_copy)));
    ctx->copy_cap = cap;
  }
  int64_t k = 0;
  for (int32_t i = 0; i < n; ++i) {
    const isx_rect_copy& c = copies[i];
    if (c.row_bytes <= 0 || c.rows <= 0) continue;
    for (int32_t r = 0; r < c.rows; r += kCopyPieceRows) {
      isx_rect_copy& p = ctx->h_copy[k++];
      p = c;
      p.src = static_cast<const uint8_t*>(c.src) + (int64_t)r * c.src_pitch;
      p.dst = static_cast<uint8_t*>(c.dst) + (int64_t)r * c.dst_pitch;
      p.rows = std::min(kCopyPieceRows, c.rows - r);
    }
  }
  const int n_pieces = (int)pieces;
  ISX_CUDA(cudaMemcpyAsync(ctx->d_copy, ctx->h_copy, (size_t)n_pieces * sizeof(isx_rect_copy), cudaMemcpyHostToDevice, s));
  ISX_CUDA(cudaEventRecord(ctx->copy_free, s));
  ctx->launches = launch_copy_rects(ctx->d_copy, n_pieces, s);
  ISX_CUDA(cudaGetLastError());
  return ISX_OK;
}

isx_status isx_set_tile_stamps(isx_ctx* ctx, uint64_t* d_stamps, int32_t n_tiles) {
  if (!ctx) return ISX_ERR_ARG;
  if (d_stamps && n_tiles < 1) return fail(ctx, ISX_ERR_ARG, "stamps need n_tiles >= 1");
  ctx->stamps = d_stamps;
  ctx->stamp_n = d_stamps ? n_tiles : 0;
  return ISX_OK;
}

int32_t isx_decode_path(const isx_tile_desc* tile, int32_t level, int32_t drop_lsb_planes, double* h_bound) {
  std::string why;
  if (!tile || !tile_ok(*tile, &why) || level < 0 || level > tile->levels || drop_lsb_planes < 0) return -1;
  const double b = inverse_state_bound(*tile, level, drop_lsb_planes);
  if (h_bound) *h_bound = b;
  const int zw = level_dim(tile->width, level), zh = level_dim(tile->height, level);
  return fused_tile(zw, zh) && b <= 32767.0 ? 1 : 0;
}

int32_t isx_last_launch_count(isx_ctx* ctx) { return ctx ? ctx->launches : 0; }

}  // extern "C"

namespace {
isx_status status_of(isx_ctx* ctx, std::string* err, int st) {
  switch (st) {
    case 0: return ISX_OK;
    case kStCapacity: *err = "output buffer too small; required size in tile_offsets[n_tiles]"; return ISX_ERR_CAPACITY;
    case kStCorrupt: *err = "malformed compressed stream"; return ISX_ERR_CORRUPT;
    case kStTimeout: *err = "device wait gave up"; return ISX_ERR_TIMEOUT;
    case kStRange: *err = "a sample exceeds its tile's bit depth (values must be below 2^bits)"; return ISX_ERR_ARG;
    case kStInternal:
      *err = "internal consistency check failed on the device (the encoder's segment sizes disagree with its symbols)";
      return ISX_ERR_INTERNAL;
    default: *err = "unknown device status " + std::to_string(st); return ISX_ERR_INTERNAL;
  }
  (void)ctx;
}
}  // namespace

extern "C" {

isx_status isx_sync_status(isx_ctx* ctx, void* stream) {
  if (!ctx) return ISX_ERR_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  ISX_CUDA(cudaStreamSynchronize(s));
  int st = 0;
  ISX_CUDA(cudaMemcpy(&st, ctx->d_status, sizeof(int), cudaMemcpyDeviceToHost));
  ISX_CUDA(cudaMemset(ctx->d_status, 0, sizeof(int)));
  std::string msg;
  isx_status r = status_of(ctx, &msg, st);
  if (r != ISX_OK) ctx->err = msg;
  return r;
}

isx_status isx_forward_coefficients(isx_ctx* ctx, const isx_tile_desc* tiles, int32_t n_tiles, int32_t* d_coef, void* stream) {
  if (!ctx || !tiles || n_tiles < 1 || !d_coef) return fail(ctx, ISX_ERR_ARG, "bad arguments");
  cudaStream_t s = (cudaStream_t)stream;
  ISX_CUDA(cudaSetDevice(ctx->device));
  Staging* g = nullptr;
  isx_status st = ensure_staging(ctx, (size_t)n_tiles, &g);
  if (st != ISX_OK) return st;
  EncodeLayout E;
  std::string err;
  st = plan_encode(tiles, n_tiles, false, ctx->sched, g->h_tiles, g->h_task, E, &err);
  if (st != ISX_OK) return fail(ctx, st, err);
  Carve cv;
  size_t o_tiles = cv.take(sizeof(TileDev) * n_tiles);
  size_t o_A = cv.take(4 * (size_t)E.plane_total);
  size_t o_B = cv.take(4 * (size_t)E.plane_total);
  st = ensure_arena(ctx, cv.used);
  if (st != ISX_OK) return st;
  TileDev* d_tiles = (TileDev*)(ctx->arena + o_tiles);
  int32_t* A = (int32_t*)(ctx->arena + o_A);
  int32_t* B = (int32_t*)(ctx->arena + o_B);
  ISX_CUDA(cudaMemcpyAsync(d_tiles, g->h_tiles, sizeof(TileDev) * n_tiles, cudaMemcpyHostToDevice, s));
  ISX_CUDA(cudaEventRecord(g->free, s));
  int L = launch_forward_transform(d_tiles, n_tiles, E.max_levels, E.max_dim, E.max_c, A, B, ctx->d_status, s);
  L += launch_quantise_planes(d_tiles, n_tiles, A, d_coef, s);
  ctx->launches = L;
  ISX_CUDA(cudaGetLastError());
  return ISX_OK;
}

}  // extern "C"

namespace {
isx_status decode_region_impl(isx_ctx* ctx, const void* d_stream, const uint64_t* d_tile_offsets, const isx_tile_desc* tiles,
                              int32_t n_tiles, int32_t level, int32_t rx, int32_t ry, int32_t rw, int32_t rh, int32_t drop_lsb_planes,
                              void* d_out, int64_t out_pitch_bytes, void* stream, const IoGate* gate);

// The copy stream and events of the overlapped host-buffer decodes, created on first use.
isx_status ensure_io(isx_ctx* ctx) {
  if (!ctx->io_out) ISX_CUDA(cudaStreamCreateWithFlags(&ctx->io_out, cudaStreamNonBlocking));
  for (cudaEvent_t& e : ctx->io_ev)
    if (!e) ISX_CUDA(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
  return ISX_OK;
}
}  // namespace

extern "C" {

isx_status isx_decode_region(isx_ctx* ctx, const void* d_stream, const uint64_t* d_tile_offsets, const isx_tile_desc* tiles,
                             int32_t n_tiles, int32_t level, int32_t rx, int32_t ry, int32_t rw, int32_t rh, int32_t drop_lsb_planes,
                             void* d_out, int64_t out_pitch_bytes, void* stream) {
  return decode_region_impl(ctx, d_stream, d_tile_offsets, tiles, n_tiles, level, rx, ry, rw, rh, drop_lsb_planes, d_out,
                            out_pitch_bytes, stream, nullptr);
}

}  // extern "C"

extern "C" {

isx_status isx_encode_tiles(isx_ctx* ctx, const isx_tile_desc* tiles, int32_t n_tiles, void* d_out, size_t out_capacity,
                            uint64_t* d_tile_offsets, void* stream) {
  if (!ctx) return ISX_ERR_ARG;
  if (!tiles || n_tiles < 1 || !d_tile_offsets || (!d_out && out_capacity))
    return fail(ctx, ISX_ERR_ARG, "bad arguments");
  if (reinterpret_cast<uintptr_t>(d_out) & 3) return fail(ctx, ISX_ERR_ARG, "d_out must be 4-byte aligned");
  cudaStream_t s = (cudaStream_t)stream;
  ISX_CUDA(cudaSetDevice(ctx->device));
  Staging* g = nullptr;
  isx_status st = ensure_staging(ctx, (size_t)n_tiles, &g);
  if (st != ISX_OK) return st;
  EncodeLayout E;
  std::string err;
  st = plan_encode(tiles, n_tiles, true, ctx->sched, g->h_tiles, g->h_task, E, &err, ctx->stamps, ctx->stamp_n);
  if (st != ISX_OK) return fail(ctx, st, err);
  st = ensure_arena(ctx, E.total);
  if (st != ISX_OK) return st;
  uint8_t* ar = ctx->arena;
  ISX_CUDA(cudaMemcpyAsync(ar + E.o_tiles, g->h_tiles, sizeof(TileDev) * n_tiles, cudaMemcpyHostToDevice, s));
  if (E.n_fused) ISX_CUDA(cudaMemcpyAsync(ar + E.o_task, g->h_task, sizeof(int32_t) * E.n_fused, cudaMemcpyHostToDevice, s));
  ISX_CUDA(cudaEventRecord(g->free, s));
  StageTimer& T = ctx->timer;
  if (T.on && !T.pending.empty()) T.collect();
  ctx->launches = launch_encode(E, ar, d_out, out_capacity, d_tile_offsets, ctx->d_status, &T, s);
  ISX_CUDA(cudaGetLastError());
  return ISX_OK;
}

}  // extern "C"

namespace {
isx_status decode_region_impl(isx_ctx* ctx, const void* d_stream, const uint64_t* d_tile_offsets, const isx_tile_desc* tiles,
                              int32_t n_tiles, int32_t level, int32_t rx, int32_t ry, int32_t rw, int32_t rh, int32_t drop_lsb_planes,
                              void* d_out, int64_t out_pitch_bytes, void* stream, const IoGate* gate) {
  if (!ctx) return ISX_ERR_ARG;
  if (!d_stream || !d_tile_offsets || !tiles || n_tiles < 1 || !d_out || rw < 1 || rh < 1 || level < 0 || level > kMaxLevels ||
      drop_lsb_planes < 0 || drop_lsb_planes > kMaxD)
    return fail(ctx, ISX_ERR_ARG, "bad arguments");
  // one job per tile meeting the rectangle; all write into the one output
  std::vector<Job> jobs;
  int C = -1, bits = -1;
  for (int32_t i = 0; i < n_tiles; ++i) {
    const isx_tile_desc& t = tiles[i];
    // tiles outside the rectangle are not read: only the ones it meets are checked
    if (t.width < 1 || t.height < 1 || t.x0 < 0 || t.y0 < 0) return fail(ctx, ISX_ERR_ARG, "tile " + std::to_string(i) + ": bad geometry");
    const int zw = level_dim(t.width, level), zh = level_dim(t.height, level);
    const int tx = t.x0 >> level, ty = t.y0 >> level;
    if (tx >= rx + rw || ty >= ry + rh || tx + zw <= rx || ty + zh <= ry) continue;
    std::string why;
    if (!tile_ok(t, &why)) return fail(ctx, ISX_ERR_ARG, "tile " + std::to_string(i) + ": " + why);
    if (C < 0) { C = t.channels; bits = t.bits; }
    if (t.channels != C || (t.bits <= 8) != (bits <= 8))
      return fail(ctx, ISX_ERR_ARG, "tiles of one region must share channels and sample size");
    jobs.push_back(Job{i, rx, ry, rw, rh, d_out, out_pitch_bytes});
  }
  if (out_pitch_bytes < (int64_t)rw * std::max(C, 1) * (bits > 8 ? 2 : 1)) return fail(ctx, ISX_ERR_ARG, "output pitch too small");
  ctx->launches = 0;
  if (jobs.empty()) {
    if (gate)
      for (int k = 0; k < gate->n; ++k) ISX_CUDA(cudaEventRecord(gate->ev[k], (cudaStream_t)stream));
    return ISX_OK;
  }
  return decode_jobs_ctx(ctx, d_stream, d_tile_offsets, tiles, n_tiles, jobs.data(), (int32_t)jobs.size(), level, drop_lsb_planes,
                         (cudaStream_t)stream, gate);
}
}  // namespace

extern "C" {

isx_status isx_decode_jobs(isx_ctx* ctx, const void* d_stream, const uint64_t* d_tile_offsets, const isx_tile_desc* tiles,
                           int32_t n_tiles, const isx_decode_job* jobs, int32_t n_jobs, int32_t level, int32_t drop_lsb_planes,
                           void* stream) {
  if (!ctx) return ISX_ERR_ARG;
  if (!d_stream || !d_tile_offsets || !tiles || n_tiles < 1 || !jobs || n_jobs < 0 || level < 0 || level > kMaxLevels ||
      drop_lsb_planes < 0 || drop_lsb_planes > kMaxD)
    return fail(ctx, ISX_ERR_ARG, "bad arguments");
  std::vector<Job> J((size_t)n_jobs);
  for (int32_t j = 0; j < n_jobs; ++j)
    J[j] = Job{jobs[j].tile, jobs[j].rx, jobs[j].ry, jobs[j].rw, jobs[j].rh, jobs[j].d_out, jobs[j].out_pitch_bytes};
  ctx->launches = 0;
  if (n_jobs == 0) return ISX_OK;
  return decode_jobs_ctx(ctx, d_stream, d_tile_offsets, tiles, n_tiles, J.data(), n_jobs, level, drop_lsb_planes, (cudaStream_t)stream);
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
  if (n_tiles >= kIoMinTiles && row_bytes * (size_t)rh >= kIoMinBytes) {
    // Large calls: the inverse transform runs chunk by chunk (consecutive
    // tiles, cut where a new row of tiles starts when one is near), and each
    // chunk's rows go back on io_out while the next chunk is inverted.  A row
    // is copied back last by the last chunk with a tile on it, after every
    // tile on it is stored, so overlapping chunks leave the right pixels.
    isx_status se = ensure_io(ctx);
    if (se != ISX_OK) return se;
    IoGate gate;
    const int K = std::min(kIoChunks, n_tiles / 4);
    const int32_t step = (n_tiles + K - 1) / K;
    int n = 0;
    gate.cut[0] = 0;
    while (gate.cut[n] < n_tiles) {
      int32_t i = std::min(n_tiles, gate.cut[n] + step), j = i;
      while (j < n_tiles && j < i + step / 2 && tiles[j].y0 == tiles[j - 1].y0) ++j;
      if (j < n_tiles && j < i + step / 2) i = j;
      if (n + 1 == K) i = n_tiles;
      gate.cut[++n] = i;
    }
    gate.n = n;
    for (int k = 0; k < n; ++k) gate.ev[k] = ctx->io_ev[k];
    isx_status st = decode_region_impl(ctx, ctx->d_io, (const uint64_t*)(ctx->d_io + off_dev), tiles, n_tiles, level, rx, ry, rw, rh,
                                       drop_lsb_planes, ctx->d_io + out_dev, (int64_t)row_bytes, stream, &gate);
    if (st != ISX_OK) return st;
    int L = ctx->launches;
    const uint8_t* d_rows = ctx->d_io + out_dev;
    std::vector<char> covered((size_t)rh, 0);
    for (int k = 0; k < n; ++k) {
      int ya = ry + rh, yb = ry;   // the rows of the rectangle that chunk k's tiles cover at this level
      for (int32_t i = gate.cut[k]; i < gate.cut[k + 1]; ++i) {
        const int t0 = tiles[i].y0 >> level, t1 = t0 + level_dim(tiles[i].height, level);
        const int u0 = tiles[i].x0 >> level, u1 = u0 + level_dim(tiles[i].width, level);
        if (std::max(t0, ry) < std::min(t1, ry + rh) && std::max(u0, rx) < std::min(u1, rx + rw)) {
          ya = std::min(ya, std::max(t0, ry));
          yb = std::max(yb, std::min(t1, ry + rh));
        }
      }
      if (ya >= yb) continue;
      ISX_CUDA(cudaStreamWaitEvent(ctx->io_out, gate.ev[k], 0));
      ISX_CUDA(cudaMemcpy2DAsync((uint8_t*)h_out + (size_t)(ya - ry) * (size_t)out_pitch_bytes, (size_t)out_pitch_bytes,
                                 d_rows + (size_t)(ya - ry) * row_bytes, row_bytes, row_bytes, (size_t)(yb - ya), cudaMemcpyDeviceToHost,
                                 ctx->io_out));
      for (int y = ya; y < yb; ++y) covered[(size_t)(y - ry)] = 1;
    }
    // rows no tile covers: zeros (the clear ran before the last chunk's inverse)
    ISX_CUDA(cudaStreamWaitEvent(ctx->io_out, gate.ev[n - 1], 0));
    for (int y = 0; y < rh;) {
      if (covered[(size_t)y]) { ++y; continue; }
      int e = y;
      while (e < rh && !covered[(size_t)e]) ++e;
      ISX_CUDA(cudaMemcpy2DAsync((uint8_t*)h_out + (size_t)y * (size_t)out_pitch_bytes, (size_t)out_pitch_bytes, d_rows + (size_t)y * row_bytes,
                                 row_bytes, row_bytes, (size_t)(e - y), cudaMemcpyDeviceToHost, ctx->io_out));
      y = e;
    }
    ISX_CUDA(cudaStreamSynchronize(ctx->io_out));
    st = isx_sync_status(ctx, stream);
    ctx->launches = L;
    return st;
  }
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


isx_status isx_decode_jobs_scratch(isx_ctx* ctx, const isx_tile_desc* tiles, int32_t n_tiles, const isx_decode_job* jobs,
                                   int32_t n_jobs, int32_t level, int32_t drop_lsb_planes, size_t* bytes) {
  if (!ctx) return ISX_ERR_ARG;
  if (!tiles || n_tiles < 1 || !jobs || n_jobs < 0 || !bytes || level < 0 || level > kMaxLevels) return fail(ctx, ISX_ERR_ARG, "bad arguments");
  std::vector<Job> J((size_t)n_jobs);
  for (int32_t j = 0; j < n_jobs; ++j)
    J[j] = Job{jobs[j].tile, jobs[j].rx, jobs[j].ry, jobs[j].rw, jobs[j].rh, jobs[j].d_out, jobs[j].out_pitch_bytes};
  std::vector<TileDev> ht((size_t)std::max(n_jobs, 1));
  std::vector<int64_t> hidx((size_t)std::max(n_jobs, 1));
  std::vector<int32_t> htask((size_t)std::max(n_jobs, 1));
  DecodeLayout D;
  std::string err;
  std::vector<WinDev> wins;   // the same windows as isx_decode_jobs
  isx_status st = plan_decode(tiles, n_tiles, J.data(), n_jobs, level, drop_lsb_planes, ctx->sched, ht.data(), hidx.data(), htask.data(),
                              D, &err, nullptr, 0, &wins);
  if (st != ISX_OK) return fail(ctx, st, err);
  *bytes = D.nsel ? D.total : 0;
  return ISX_OK;
}

isx_status isx_reserve_scratch(isx_ctx* ctx, size_t bytes) {
  if (!ctx) return ISX_ERR_ARG;
  ISX_CUDA(cudaSetDevice(ctx->device));
  return ensure_arena(ctx, bytes);
}

size_t isx_scratch_bytes(isx_ctx* ctx) { return ctx ? ctx->arena_size : 0; }

// ---------------------------------------------------------------- schedule
isx_status isx_get_schedule(isx_ctx* ctx, isx_schedule* out) {
  if (!ctx || !out) return ISX_ERR_ARG;
  for (int k = 0; k < ISX_SIZE_CLASSES; ++k) {
    out->forward_threads[k] = ctx->sched.fwd[k];
    out->inverse_threads[k] = ctx->sched.inv[k];
  }
  return ISX_OK;
}

isx_status isx_set_schedule(isx_ctx* ctx, const isx_schedule* sch) {
  if (!ctx || !sch) return ISX_ERR_ARG;
  for (int k = 0; k < ISX_SIZE_CLASSES; ++k)
    if (!valid_threads(sch->forward_threads[k]) || !valid_threads(sch->inverse_threads[k]))
      return fail(ctx, ISX_ERR_ARG, "threads per CTA must be 256, 512 or 1024");
  for (int k = 0; k < ISX_SIZE_CLASSES; ++k) {
    ctx->sched.fwd[k] = sch->forward_threads[k];
    ctx->sched.inv[k] = sch->inverse_threads[k];
  }
  return ISX_OK;
}

isx_status isx_autotune(isx_ctx* ctx, const isx_tile_desc* tiles, int32_t n_tiles, int32_t reps, void* stream) {
  if (!ctx) return ISX_ERR_ARG;
  if (!tiles || n_tiles < 1 || reps < 1) return fail(ctx, ISX_ERR_ARG, "bad arguments");
  cudaStream_t s = (cudaStream_t)stream;
  ISX_CUDA(cudaSetDevice(ctx->device));
  static const int kCand[3] = {256, 512, 1024};
  // encode once into a scratch stream, growing it if the estimate is short
  std::vector<TileDev> ht(n_tiles);
  std::vector<int32_t> htask(n_tiles);
  EncodeLayout E;
  std::string err;
  isx_status st = plan_encode(tiles, n_tiles, true, ctx->sched, ht.data(), htask.data(), E, &err);
  if (st != ISX_OK) return fail(ctx, st, err);
  size_t cap = 4096;
  for (int32_t i = 0; i < n_tiles; ++i)
    cap += (size_t)tiles[i].width * tiles[i].height * tiles[i].channels * 4 + 4096;
  uint8_t* d_mem = nullptr;
  const size_t stream_off = (E.total + 255) & ~(size_t)255;
  const size_t offs_off = stream_off + ((cap + 255) & ~(size_t)255);
  ISX_CUDA(cudaMalloc(&d_mem, offs_off + 8 * (size_t)(n_tiles + 1)));
  struct Free { uint8_t* p; ~Free() { if (p) cudaFree(p); } } guard{d_mem};
  ISX_CUDA(cudaMemcpy(d_mem + E.o_tiles, ht.data(), sizeof(TileDev) * n_tiles, cudaMemcpyHostToDevice));
  if (E.n_fused) ISX_CUDA(cudaMemcpy(d_mem + E.o_task, htask.data(), 4 * (size_t)E.n_fused, cudaMemcpyHostToDevice));
  NoMarks nm;
  uint64_t* d_offs = (uint64_t*)(d_mem + offs_off);
  launch_encode(E, d_mem, d_mem + stream_off, cap, d_offs, ctx->d_status, &nm, s);
  st = isx_sync_status(ctx, stream);
  if (st != ISX_OK) return st;
  cudaEvent_t e0, e1;
  ISX_CUDA(cudaEventCreate(&e0));
  ISX_CUDA(cudaEventCreate(&e1));
  auto time_ms = [&](auto&& launch) {
    cudaEventRecord(e0, s);
    for (int r = 0; r < reps; ++r) launch();
    cudaEventRecord(e1, s);
    cudaEventSynchronize(e1);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    return ms;
  };
  Schedule best = ctx->sched;
  for (int k = 0; k < ISX_SIZE_CLASSES; ++k) {
    const FusedClass& c = E.cls[k];
    if (!c.count) continue;
    float best_ms = 1e30f;
    for (int t : kCand) {
      const float ms = time_ms([&] {
        launch_fused_forward((TileDev*)(d_mem + E.o_tiles), (int32_t*)(d_mem + E.o_task) + c.begin, c.count, c.slots, c.smem, t,
                             (BlockDev*)(d_mem + E.o_blocks), d_mem + E.o_coef, ctx->d_status, s);
      });
      if (ms < best_ms) { best_ms = ms; best.fwd[k] = t; }
    }
  }
  // decode every tile whole into its own output
  std::vector<Job> jobs(n_tiles);
  size_t out_bytes = 0;
  for (int32_t i = 0; i < n_tiles; ++i) {
    const isx_tile_desc& t = tiles[i];
    const int64_t pitch = (int64_t)t.width * t.channels * (t.bits <= 8 ? 1 : 2);
    jobs[i] = Job{i, t.x0, t.y0, t.width, t.height, (void*)(uintptr_t)out_bytes, pitch};
    out_bytes += ((size_t)pitch * t.height + 15) & ~(size_t)15;
  }
  std::vector<TileDev> dt(n_tiles);
  std::vector<int64_t> didx(n_tiles);
  std::vector<int32_t> dtask(n_tiles);
  DecodeLayout D;
  uint8_t* d_dec = nullptr;
  ISX_CUDA(cudaMalloc(&d_dec, out_bytes));
  struct Free2 { uint8_t* p; ~Free2() { if (p) cudaFree(p); } } guard2{d_dec};
  for (auto& j : jobs) j.out = d_dec + (uintptr_t)j.out;
  st = plan_decode(tiles, n_tiles, jobs.data(), n_tiles, 0, 0, ctx->sched, dt.data(), didx.data(), dtask.data(), D, &err);
  if (st != ISX_OK) return fail(ctx, st, err);
  st = ensure_arena(ctx, D.total);
  if (st != ISX_OK) return st;
  uint8_t* ar = ctx->arena;
  ISX_CUDA(cudaMemcpy(ar + D.o_tiles, dt.data(), sizeof(TileDev) * D.nsel, cudaMemcpyHostToDevice));
  ISX_CUDA(cudaMemcpy(ar + D.o_idx, didx.data(), 8 * (size_t)D.nsel, cudaMemcpyHostToDevice));
  if (D.n_fused) ISX_CUDA(cudaMemcpy(ar + D.o_task, dtask.data(), 4 * (size_t)D.n_fused, cudaMemcpyHostToDevice));
  launch_decode(D, ar, d_mem + stream_off, d_offs, ctx->d_status, &nm, s);
  st = isx_sync_status(ctx, stream);
  if (st != ISX_OK) return st;
  DecodeBuffers db;   // the fused inverse reads only these fields
  db.blocks = (BlockDev*)(ar + D.o_blocks); db.info = (DecInfo*)(ar + D.o_info); db.sym_off = (int64_t*)(ar + D.o_so);
  db.sym = ar + D.o_sym; db.totals = (int64_t*)(ar + D.o_tot); db.sym_cap = D.sym_cap; db.z = 0;
  uint32_t* tickets = (uint32_t*)(ar + D.o_tk);
  for (int k = 0; k < ISX_SIZE_CLASSES; ++k) {
    const FusedClass& c = D.cls[k];
    if (!c.count) continue;
    float best_ms = 1e30f;
    for (int t : kCand) {
      const float ms = time_ms([&] {
        cudaMemsetAsync(tickets + c.begin, 0, 4 * (size_t)c.count, s);
        launch_fused_inverse((TileDev*)(ar + D.o_tiles), (int32_t*)(ar + D.o_task) + c.begin, c.count, c.slots, c.smem, t, db,
                             (int16_t*)(ar + D.o_fp), tickets + c.begin, s);
      });
      if (ms < best_ms) { best_ms = ms; best.inv[k] = t; }
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  ISX_CUDA(cudaGetLastError());
  st = isx_sync_status(ctx, stream);
  if (st != ISX_OK) return st;
  ctx->sched = best;
  return ISX_OK;
}

// ---------------------------------------------------------------- plans
isx_status isx_plan_encode(isx_ctx* ctx, const isx_tile_desc* tiles, int32_t n_tiles, isx_plan** out) {
  if (!ctx) return ISX_ERR_ARG;
  if (!out || !tiles || n_tiles < 1) return fail(ctx, ISX_ERR_ARG, "bad arguments");
  *out = nullptr;
  ISX_CUDA(cudaSetDevice(ctx->device));
  isx_plan* P = new isx_plan();
  P->kind = 1;
  P->device = ctx->device;
  std::vector<TileDev> ht(n_tiles);
  std::vector<int32_t> htask(n_tiles);
  std::string err;
  isx_status st = plan_encode(tiles, n_tiles, true, ctx->sched, ht.data(), htask.data(), P->E, &err, ctx->stamps, ctx->stamp_n);
  cudaError_t e = cudaSuccess;
  if (st == ISX_OK) {
    P->mem_bytes = P->E.total;
    e = cudaMalloc(&P->mem, P->mem_bytes);
    if (e == cudaSuccess) e = cudaMalloc(&P->d_status, sizeof(int));
    if (e == cudaSuccess) e = cudaMemset(P->d_status, 0, sizeof(int));
    if (e == cudaSuccess) e = cudaMemcpy(P->mem + P->E.o_tiles, ht.data(), sizeof(TileDev) * n_tiles, cudaMemcpyHostToDevice);
    if (e == cudaSuccess && P->E.n_fused)
      e = cudaMemcpy(P->mem + P->E.o_task, htask.data(), 4 * (size_t)P->E.n_fused, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) { cudaGetLastError(); st = ISX_ERR_OOM; err = std::string("plan memory: ") + cudaGetErrorString(e); }
  }
  if (st != ISX_OK) {
    isx_plan_destroy(P);
    return fail(ctx, st, err);
  }
  *out = P;
  return ISX_OK;
}

isx_status isx_plan_decode(isx_ctx* ctx, const isx_tile_desc* tiles, int32_t n_tiles, const isx_decode_job* jobs, int32_t n_jobs,
                           int32_t level, int32_t drop_lsb_planes, isx_plan** out) {
  if (!ctx) return ISX_ERR_ARG;
  if (!out || !tiles || n_tiles < 1 || !jobs || n_jobs < 1 || level < 0 || level > kMaxLevels || drop_lsb_planes < 0 ||
      drop_lsb_planes > kMaxD)
    return fail(ctx, ISX_ERR_ARG, "bad arguments");
  *out = nullptr;
  ISX_CUDA(cudaSetDevice(ctx->device));
  isx_plan* P = new isx_plan();
  P->kind = 2;
  P->device = ctx->device;
  std::vector<Job> J((size_t)n_jobs);
  for (int32_t j = 0; j < n_jobs; ++j)
    J[j] = Job{jobs[j].tile, jobs[j].rx, jobs[j].ry, jobs[j].rw, jobs[j].rh, jobs[j].d_out, jobs[j].out_pitch_bytes};
  std::vector<TileDev> ht(n_jobs);
  std::vector<int64_t> hidx(n_jobs);
  std::vector<int32_t> htask(n_jobs);
  std::string err;
  std::vector<WinDev> wins;
  isx_status st = plan_decode(tiles, n_tiles, J.data(), n_jobs, level, drop_lsb_planes, ctx->sched, ht.data(), hidx.data(), htask.data(),
                              P->D, &err, ctx->stamps, ctx->stamp_n, &wins);
  cudaError_t e = cudaSuccess;
  if (st == ISX_OK) {
    P->mem_bytes = P->D.total;
    e = cudaMalloc(&P->mem, P->mem_bytes);
    if (e == cudaSuccess) e = cudaMalloc(&P->d_status, sizeof(int));
    if (e == cudaSuccess) e = cudaMemset(P->d_status, 0, sizeof(int));
    if (e == cudaSuccess && P->D.nsel) {
      e = cudaMemcpy(P->mem + P->D.o_tiles, ht.data(), sizeof(TileDev) * P->D.nsel, cudaMemcpyHostToDevice);
      if (e == cudaSuccess) e = cudaMemcpy(P->mem + P->D.o_idx, hidx.data(), 8 * (size_t)P->D.nsel, cudaMemcpyHostToDevice);
      if (e == cudaSuccess && P->D.n_fused)
        e = cudaMemcpy(P->mem + P->D.o_task, htask.data(), 4 * (size_t)P->D.n_fused, cudaMemcpyHostToDevice);
      if (e == cudaSuccess && P->D.n_win)
        e = cudaMemcpy(P->mem + P->D.o_win, wins.data(), sizeof(WinDev) * (size_t)P->D.n_win, cudaMemcpyHostToDevice);
    }
    if (e != cudaSuccess) { cudaGetLastError(); st = ISX_ERR_OOM; err = std::string("plan memory: ") + cudaGetErrorString(e); }
  }
  if (st != ISX_OK) {
    isx_plan_destroy(P);
    return fail(ctx, st, err);
  }
  *out = P;
  return ISX_OK;
}

isx_status isx_plan_launch_encode(isx_plan* plan, void* d_out, size_t out_capacity, uint64_t* d_tile_offsets, void* stream) {
  if (!plan || plan->kind != 1) return ISX_ERR_ARG;
  if (!d_tile_offsets || (!d_out && out_capacity) || (reinterpret_cast<uintptr_t>(d_out) & 3)) {
    plan->err = "bad arguments (d_out must be 4-byte aligned)";
    return ISX_ERR_ARG;
  }
  NoMarks nm;
  plan->launches = launch_encode(plan->E, plan->mem, d_out, out_capacity, d_tile_offsets, plan->d_status, &nm, (cudaStream_t)stream);
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) { plan->err = cudaGetErrorString(e); return ISX_ERR_CUDA; }
  return ISX_OK;
}

isx_status isx_plan_launch_decode(isx_plan* plan, const void* d_stream, const uint64_t* d_tile_offsets, void* stream) {
  if (!plan || plan->kind != 2) return ISX_ERR_ARG;
  if (!d_stream || !d_tile_offsets) { plan->err = "bad arguments"; return ISX_ERR_ARG; }
  NoMarks nm;
  plan->launches = launch_decode(plan->D, plan->mem, d_stream, d_tile_offsets, plan->d_status, &nm, (cudaStream_t)stream);
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) { plan->err = cudaGetErrorString(e); return ISX_ERR_CUDA; }
  return ISX_OK;
}

isx_status isx_plan_sync_status(isx_plan* plan, void* stream) {
  if (!plan) return ISX_ERR_ARG;
  cudaError_t e = cudaStreamSynchronize((cudaStream_t)stream);
  int st = 0;
  if (e == cudaSuccess) e = cudaMemcpy(&st, plan->d_status, sizeof(int), cudaMemcpyDeviceToHost);
  if (e == cudaSuccess) e = cudaMemset(plan->d_status, 0, sizeof(int));
  if (e != cudaSuccess) { plan->err = cudaGetErrorString(e); return ISX_ERR_CUDA; }
  return status_of(nullptr, &plan->err, st);
}

size_t isx_plan_device_bytes(const isx_plan* plan) { return plan ? plan->mem_bytes + sizeof(int) : 0; }

int32_t isx_plan_launch_count(const isx_plan* plan) { return plan ? plan->launches : 0; }

const char* isx_plan_last_error(const isx_plan* plan) { return plan ? plan->err.c_str() : "null plan"; }

void isx_plan_destroy(isx_plan* plan) {
  if (!plan) return;
  cudaSetDevice(plan->device);
  if (plan->mem || plan->d_status) cudaDeviceSynchronize();
  if (plan->mem) cudaFree(plan->mem);
  if (plan->d_status) cudaFree(plan->d_status);
  delete plan;
}

}  // extern "C"
