// C ABI of libgsr (declared in include/gsr.h): scene arena, workspace
// management, launch sequence of one render / pose-gradient / batch call,
// CUDA-graph capture of batches, and the parity exports.
//
// Host arithmetic that feeds the binary32 projection (pose rounding, the
// field-of-view guard) is compiled without floating-point contraction so that
// it is the same IEEE sequence on every host.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <functional>
#include <map>
#include <string>
#include <vector>

#include "gsr.h"
#include "gsr_internal.h"

using namespace gsr;

namespace {

thread_local std::string g_err;

gs_status fail(gs_status st, const std::string& msg) {
  g_err = msg;
  return st;
}

#define GS_CUDA(x)                                                                              \
  do {                                                                                          \
    const cudaError_t e_ = (x);                                                                 \
    if (e_ != cudaSuccess) return fail(GS_ERR_CUDA, std::string(#x) + ": " + cudaGetErrorString(e_)); \
  } while (0)

#define GS_TRY(x)                     \
  do {                                \
    const gs_status s_ = (x);         \
    if (s_ != GS_OK) return s_;       \
  } while (0)

struct DevBuf {
  void* p = nullptr;
  size_t bytes = 0;
};

// Bumped by every device (re)allocation of a workspace buffer and by every
// change of a launch configuration: a captured graph holds the buffers'
// addresses and the launch shapes, and is replayed only while this is
// unchanged since its capture.
std::atomic<uint64_t> g_alloc_gen{0};

gs_status ensure(DevBuf& b, size_t bytes) {
  if (b.bytes >= bytes && b.p) return GS_OK;
  g_alloc_gen.fetch_add(1);
  if (b.p) cudaFree(b.p);
  b.p = nullptr;
  b.bytes = 0;
  const size_t alloc = std::max<size_t>(bytes, 256);
  const cudaError_t e = cudaMalloc(&b.p, alloc);
  if (e != cudaSuccess) {
    cudaGetLastError();
    b.p = nullptr;
    return fail(e == cudaErrorMemoryAllocation ? GS_ERR_OOM : GS_ERR_CUDA,
                std::string("cudaMalloc(") + std::to_string(alloc) + "): " + cudaGetErrorString(e));
  }
  b.bytes = alloc;
  return GS_OK;
}

void release(DevBuf& b) {
  if (b.p) cudaFree(b.p);
  b.p = nullptr;
  b.bytes = 0;
}

template <typename T>
T* dp(const DevBuf& b) {
  return reinterpret_cast<T*>(b.p);
}

// Loss inputs of a pose-gradient call, one entry per view (host arrays of
// device pointers).
struct GradIn {
  const float* const* target_rgb;
  const float* const* target_depth;
  const float* const* pixel_weight;  // NULL, or per-view entries that may be NULL
  float depth_weight;
  double* result;  // device destination, kResultStride doubles per view, or NULL (scene buffer)
};

constexpr int kResultStride = 8;  // (loss, grad rho, grad phi, pad) per view
constexpr int kUploadBands = 4;   // tile-row bands of a host-target pose-gradient call

// Loss targets uploaded in bands of tile rows (single-view host-target calls):
// band b covers tile rows [tile_row[b], tile_row[b + 1]) and its rows are on
// the device once ready[b] has completed; its tangent pass waits for nothing else.
struct Bands {
  int n = 0;
  uint32_t tile_row[kMaxBands + 1] = {};
  cudaEvent_t ready[kMaxBands] = {};
};

// Outputs of a visibility-check call (device pointers; uv is never NULL: the
// caller's array or the scene's scratch).
struct VisOut {
  uint8_t* mask;
  float2* uv;
  float* grad;
  int32_t* vis_gid;
  float2* vis_uv;
};

// A captured batch: replayed while everything but the poses is unchanged.
struct GraphCache {
  bool valid = false;
  cudaGraphExec_t exec = nullptr;
  std::vector<char> key;       // cameras, outputs, loss inputs of the capture
  char* host_table = nullptr;  // pinned call table (ranges + views), read by the graph's upload node
  cudaEvent_t done = nullptr;
  cudaStream_t capture = nullptr;
  int n_views = 0;
  uint64_t gen = 0;  // g_alloc_gen at capture
};

}  // namespace

namespace gsr {
// lets other translation units (the no-allocation entry point) set the message
void set_last_error(const std::string& msg) { g_err = msg; }
}  // namespace gsr

// A partition of the scene (a VastGaussian-style cell, Sec. 3.1): index range,
// bounding box of its means, largest scale, and whether it is on the device.
constexpr int kPartBoxes = 6;  // boxes of mean +- k s for k = 1, 2, 4, ..., 32
struct Part {
  int64_t begin = 0, end = 0;
  double lo[3] = {0, 0, 0}, hi[3] = {0, 0, 0};  // box of the means
  double klo[kPartBoxes][3], khi[kPartBoxes][3];  // box of mean_i +- 2^j s_i (s_i: largest scale)
  double smax = 0.0;
  bool resident = false;
};

struct gs_scene {
  int device = 0;
  int sm_count = 1;
  std::string device_name;
  // launch configurations by call shape (the views' sizes), set by the
  // autotuner, gs_scene_set_launch or gs_tune_load; absent shapes use the defaults
  std::map<std::string, LaunchCfg> launch;
  int64_t n = 0;
  int sh_degree = 0, feat_dim = 0, nsh4 = 1;
  DevBuf pos, cov, sh, feat;
  std::vector<int64_t> part_off;
  std::vector<Part> parts;
  bool streaming = false;  // partitions are uploaded from the pinned copy on first use
  float4* h_pos = nullptr;  // pinned packed copy (streaming only), same layout as the device arena
  float4* h_cov = nullptr;
  float4* h_sh = nullptr;
  uint4* h_feat = nullptr;
  int64_t h2d_bytes = 0;
  int last_active = 0;
  // workspace
  DevBuf rec_a, rec_b, rec_c, rec_m, rec_j;
  uint32_t rec_cap = 0, jac_cap = 0;
  DevBuf tile_count, tile_offset, tile_cursor, partials, chunks;
  uint32_t tile_cap = 0;
  DevBuf pairs, pairs_tmp;
  uint32_t pair_cap = 0;
  DevBuf ctr, result, views;
  Counters* ctr_host = nullptr;
  double* result_host = nullptr;
  // loss targets uploaded from host memory (gs_render_pose_grad_host) on a side
  // stream that overlaps the projection and binning kernels
  DevBuf targets;
  // visibility check: final transmittance and last index of its forward
  // render, per-record accumulators, (U, V) scratch, compaction counters
  DevBuf vis_T, vis_last, vis_acc, vis_uv, vis_blk;
  cudaStream_t copy_st = nullptr;
  cudaEvent_t ev_call = nullptr, ev_targets = nullptr;
  // pinned copy of the call table for synchronous calls: its upload must not
  // queue behind large host-to-device copies (a pageable source is staged and
  // copied in order with them)
  char* table_host = nullptr;
  size_t table_host_bytes = 0;
  // banded tangent pass: two streams that take the bands in turn, and the
  // events between the binning, the band uploads and the band launches
  cudaStream_t band_st[2] = {nullptr, nullptr};
  // the shading pass runs on side_st beside the binning (fork after the
  // projection, join before the compositing)
  cudaStream_t side_st = nullptr;
  cudaEvent_t ev_proj = nullptr, ev_shade = nullptr;
  cudaEvent_t ev_binned = nullptr;
  cudaEvent_t ev_band[kMaxBands] = {};
  cudaEvent_t ev_band_done[kMaxBands] = {};
  // kernel timing: one set of GS_KERNEL_COUNT + 1 events per timed call
  bool timing = false;
  struct TimedCall {
    std::vector<cudaEvent_t> ev;  // GS_KERNEL_COUNT + 1 events
    int n_kernels;                // kernels bracketed by ev[0..n_kernels]
  };
  std::vector<TimedCall> ev_pending;
  std::vector<std::vector<cudaEvent_t>> ev_free;
  double kt_ms[GS_KERNEL_COUNT] = {};
  int64_t kt_n[GS_KERNEL_COUNT] = {};
  // last call
  std::vector<View> last_views;
  uint32_t last_tiles = 0;
  GraphCache graph;       // forward batches
  GraphCache graph_grad;  // pose-gradient batches
  GraphCache graph_sync;  // synchronous single-view pose gradients
};

namespace {

// Call-shape key of a launch configuration: the views' sizes as a sorted
// multiset, "WxH*count" joined by commas.
std::string shape_key(const std::vector<std::pair<int, int>>& sizes) {
  std::map<std::pair<int, int>, int> m;
  for (const auto& wh : sizes) ++m[wh];
  std::string k;
  for (const auto& e : m) {
    if (!k.empty()) k += ',';
    k += std::to_string(e.first.first) + "x" + std::to_string(e.first.second) + "*" + std::to_string(e.second);
  }
  return k;
}

std::string shape_key(const std::vector<View>& hv) {
  std::vector<std::pair<int, int>> sz;
  for (const View& V : hv) sz.emplace_back(V.width, V.height);
  return shape_key(sz);
}

LaunchCfg launch_cfg(const gs_scene* s, const std::vector<View>& hv) {
  if (s->launch.empty()) return LaunchCfg{};
  const auto it = s->launch.find(shape_key(hv));
  return it == s->launch.end() ? LaunchCfg{} : it->second;
}

SceneDev scene_dev(const gs_scene* s) {
  SceneDev d;
  d.pos = dp<float4>(s->pos);
  d.cov = dp<float4>(s->cov);
  d.sh = dp<float4>(s->sh);
  d.feat = s->feat_dim ? dp<uint4>(s->feat) : nullptr;
  d.n = (int)s->n;
  d.sh_degree = s->sh_degree;
  d.nsh4 = s->nsh4;
  d.feat_dim = s->feat_dim;
  return d;
}

Work work_of(gs_scene* s, uint32_t n_tiles) {
  Work w;
  w.rec_a = dp<float4>(s->rec_a);
  w.rec_b = dp<float4>(s->rec_b);
  w.rec_c = dp<float4>(s->rec_c);
  w.rec_m = dp<uint4>(s->rec_m);
  w.rec_j = dp<float>(s->rec_j);
  w.rec_cap = s->rec_cap;
  w.rec_seg = s->rec_cap / kRecRegions;
  w.tile_count = dp<uint32_t>(s->tile_count);
  w.tile_offset = dp<uint32_t>(s->tile_offset);
  w.tile_cursor = dp<uint32_t>(s->tile_cursor);
  w.n_tiles = n_tiles;
  w.pairs = dp<uint2>(s->pairs);
  w.pairs_tmp = dp<uint2>(s->pairs_tmp);
  w.pair_cap = s->pair_cap;
  w.ctr = dp<Counters>(s->ctr);
  w.partials = dp<double>(s->partials);
  // chunk sums, then the view counters; one view has at least one tile, so
  // tile_cap bounds both the chunk and the view count
  w.chunk_part = dp<double>(s->chunks);
  w.view_ctr = reinterpret_cast<uint32_t*>(w.chunk_part + (size_t)s->tile_cap * kPartialStride);
  w.n_chunks = 0;
  w.n_views = 0;
  w.result = dp<double>(s->result);
  return w;
}

gs_status grow_records(gs_scene* s, uint64_t rec_cap, bool grad) {
  rec_cap = std::min<uint64_t>(rec_cap, 0x7fffffffull);
  rec_cap = (rec_cap + kRecRegions - 1) / kRecRegions * kRecRegions;  // equal segments
  if (rec_cap > s->rec_cap) {
    GS_TRY(ensure(s->rec_a, rec_cap * sizeof(float4)));
    GS_TRY(ensure(s->rec_b, rec_cap * sizeof(float4)));
    GS_TRY(ensure(s->rec_c, rec_cap * sizeof(float4)));
    GS_TRY(ensure(s->rec_m, rec_cap * sizeof(uint4)));
    s->rec_cap = (uint32_t)rec_cap;
  }
  if (grad && s->jac_cap < s->rec_cap) {
    GS_TRY(ensure(s->rec_j, (size_t)s->rec_cap * kJacStride * sizeof(float)));
    s->jac_cap = s->rec_cap;
  }
  return GS_OK;
}

gs_status grow_pairs(gs_scene* s, uint64_t pair_cap) {
  pair_cap = std::min<uint64_t>(pair_cap, 0xffffffffull);
  if (pair_cap > s->pair_cap) {
    GS_TRY(ensure(s->pairs, pair_cap * sizeof(uint2)));
    GS_TRY(ensure(s->pairs_tmp, pair_cap * sizeof(uint2)));
    s->pair_cap = (uint32_t)pair_cap;
  }
  return GS_OK;
}

gs_status grow_tiles(gs_scene* s, uint64_t n_tiles) {
  if (n_tiles + 1 > s->tile_cap) {
    const uint64_t cap = n_tiles + 1;
    GS_TRY(ensure(s->tile_count, cap * sizeof(uint32_t)));
    GS_TRY(ensure(s->tile_offset, cap * sizeof(uint32_t)));
    GS_TRY(ensure(s->tile_cursor, cap * sizeof(uint32_t)));
    GS_TRY(ensure(s->partials, cap * kPartialStride * sizeof(double)));
    GS_TRY(ensure(s->chunks, cap * (kPartialStride * sizeof(double) + sizeof(uint32_t))));
    s->tile_cap = (uint32_t)cap;
  }
  return GS_OK;
}

bool finite_pos(float x) { return std::isfinite(x) && x > 0.0f; }

gs_status check_cam(const gs_camera& c) {
  if (c.width < 1 || c.height < 1 || c.width > 65535 * kTile || c.height > 65535 * kTile)
    return fail(GS_ERR_INVALID_ARG, "camera size out of range");
  if (!finite_pos(c.fx) || !finite_pos(c.fy) || !std::isfinite(c.cx) || !std::isfinite(c.cy))
    return fail(GS_ERR_INVALID_ARG, "camera intrinsics must be finite with fx, fy > 0");
  return GS_OK;
}

gs_status check_pose(const gs_pose& p) {
  for (int k = 0; k < 16; ++k)
    if (!std::isfinite(p.T_cw[k])) return fail(GS_ERR_INVALID_ARG, "pose has a non-finite entry");
  return GS_OK;
}

// Build the per-view device parameters (outputs the caller did not ask for
// are not written; the pose gradient needs none of them).
gs_status build_views(gs_scene* s, int nv, const gs_camera* cams, const gs_pose* poses, const gs_outputs* outs,
                      const GradIn* g, std::vector<View>& hv, uint64_t& n_tiles) {
  hv.assign(nv, View{});
  n_tiles = 0;
  uint32_t n_chunks = 0;
  for (int v = 0; v < nv; ++v) {
    GS_TRY(check_cam(cams[v]));
    GS_TRY(check_pose(poses[v]));
  }
  for (int v = 0; v < nv; ++v) {
    const gs_camera& c = cams[v];
    const double* T = poses[v].T_cw;
    View& V = hv[v];
    for (int a = 0; a < 3; ++a) {
      for (int b = 0; b < 3; ++b) {
        V.R[3 * a + b] = (float)T[4 * a + b];
        V.Rl[3 * a + b] = (float)(T[4 * a + b] - (double)V.R[3 * a + b]);
      }
      V.t[a] = (float)T[4 * a + 3];
      V.tl[a] = (float)(T[4 * a + 3] - (double)V.t[a]);
    }
    for (int a = 0; a < 3; ++a)
      V.cw[a] = (float)(-(T[a] * T[3] + T[4 + a] * T[7] + T[8 + a] * T[11]));
    V.fx = c.fx;
    V.fy = c.fy;
    V.cx = c.cx;
    V.cy = c.cy;
    const float hw = 0.5f * (float)c.width, hh = 0.5f * (float)c.height;
    const float qx = hw / c.fx, qy = hh / c.fy;
    V.limx = 1.3f * qx;
    V.limy = 1.3f * qy;
    V.jb2 = c.fx * c.fx * (1.0f + V.limx * V.limx) + c.fy * c.fy * (1.0f + V.limy * V.limy);
    V.width = c.width;
    V.height = c.height;
    V.tiles_x = (c.width + kTile - 1) / kTile;
    V.tiles_y = (c.height + kTile - 1) / kTile;
    V.tile_base = (uint32_t)n_tiles;
    V.chunk_base = n_chunks;
    n_tiles += (uint64_t)V.tiles_x * V.tiles_y;
    n_chunks += (uint32_t)(((uint64_t)V.tiles_x * V.tiles_y + kChunkTiles - 1) / kChunkTiles);
    const gs_outputs o = outs ? outs[v] : gs_outputs{};
    const uint64_t P = (uint64_t)c.width * c.height;
    V.rgb = o.rgb;
    V.depth = o.depth;
    V.alpha = o.alpha;
    V.final_T = o.final_T;
    V.feats = s->feat_dim ? o.feats : nullptr;
    V.last_idx = o.last_idx;
    if (g) {
      V.target_rgb = g->target_rgb[v];
      V.target_depth = g->target_depth[v];
      V.pixel_weight = g->pixel_weight ? g->pixel_weight[v] : nullptr;
      V.depth_weight = g->depth_weight;
      V.inv_3p = (float)(1.0 / (3.0 * (double)P));
      V.inv_p = (float)(1.0 / (double)P);
    }
  }
  if (n_tiles >= 0x7fffffffull) return fail(GS_ERR_INVALID_ARG, "too many tiles in one call");
  return GS_OK;
}

// Enqueue one call. When `upload_src` is given the view table is copied from
// it (pinned memory, for graph capture); otherwise from hv (pageable: the copy
// is staged before cudaMemcpyAsync returns).
// Device call table: ranges (1 + partitions entries) followed by the views.
size_t table_ranges_bytes(const gs_scene* s) { return (1 + s->parts.size()) * sizeof(int4); }
size_t table_bytes(const gs_scene* s, int nv) { return table_ranges_bytes(s) + (size_t)nv * sizeof(View); }

void fill_table(const gs_scene* s, const std::vector<View>& hv, const std::vector<int4>& ranges, char* dst) {
  std::memset(dst, 0, table_ranges_bytes(s));
  std::memcpy(dst, ranges.data(), ranges.size() * sizeof(int4));
  std::memcpy(dst + table_ranges_bytes(s), hv.data(), hv.size() * sizeof(View));
}

// `graph`: the call is being captured (no timing events). `after_table`, if
// given, is called once the table upload is on the stream (the host-target
// path issues its target copies there, so that the table goes first).
gs_status enqueue(gs_scene* s, const std::vector<View>& hv, const std::vector<int4>& ranges, uint64_t n_tiles,
                  const GradIn* g, cudaStream_t st, const char* upload_src, cudaEvent_t targets_ready = nullptr,
                  const VisOut* vis = nullptr, const Bands* bands = nullptr, bool graph = false,
                  const std::function<gs_status()>* after_table = nullptr, bool keep_table = false) {
  const int nv = (int)hv.size();
  const bool jac = g != nullptr || vis != nullptr;  // per-record pose Jacobian
  GS_TRY(grow_tiles(s, n_tiles));
  GS_TRY(ensure(s->views, table_bytes(s, nv)));
  if (g && !g->result) GS_TRY(ensure(s->result, (size_t)nv * kResultStride * sizeof(double)));
  if (s->rec_cap == 0) {
    const uint64_t guess = std::max<uint64_t>(1u << 16, (uint64_t)s->n * nv / 4);
    GS_TRY(grow_records(s, guess, jac));
    GS_TRY(grow_pairs(s, guess * 8));
  } else {
    GS_TRY(grow_records(s, s->rec_cap, jac));
  }
  if (s->pair_cap == 0) GS_TRY(grow_pairs(s, (uint64_t)s->rec_cap * 8));
  if (vis) {
    GS_TRY(ensure(s->vis_acc, (size_t)s->rec_cap * kVisAcc * sizeof(float)));
    GS_TRY(ensure(s->vis_blk, ((size_t)s->n / kVisBlock + 1) * sizeof(uint32_t)));
  }
  View* dviews = reinterpret_cast<View*>(static_cast<char*>(s->views.p) + table_ranges_bytes(s));
  if (keep_table) {
    // the device table is current (a device-side pose update rewrote it)
  } else if (upload_src) {
    GS_CUDA(cudaMemcpyAsync(s->views.p, upload_src, table_bytes(s, nv), cudaMemcpyHostToDevice, st));
  } else {
    std::vector<char> tab(table_bytes(s, nv));
    fill_table(s, hv, ranges, tab.data());
    GS_CUDA(cudaMemcpyAsync(s->views.p, tab.data(), tab.size(), cudaMemcpyHostToDevice, st));
  }
  if (after_table) GS_TRY((*after_table)());
  Work w = work_of(s, (uint32_t)n_tiles);
  w.ranges = dp<int4>(s->views);
  if (g) {
    const View& L = hv.back();
    w.n_chunks = L.chunk_base + (uint32_t)(((uint64_t)L.tiles_x * L.tiles_y + kChunkTiles - 1) / kChunkTiles);
    w.n_views = (uint32_t)nv;
  }
  GS_CUDA(cudaMemsetAsync(w.tile_count, 0, (n_tiles + 1) * sizeof(uint32_t), st));
  GS_CUDA(cudaMemsetAsync(w.ctr, 0, sizeof(Counters), st));
  const SceneDev sc = scene_dev(s);
  std::vector<cudaEvent_t> ev;
  const bool timed = s->timing && !graph;  // no events inside captured graphs
  if (timed) {
    if (!s->ev_free.empty()) {
      ev = std::move(s->ev_free.back());
      s->ev_free.pop_back();
    } else {
      ev.resize(GS_KERNEL_COUNT + 1);
      for (auto& e : ev) GS_CUDA(cudaEventCreate(&e));
    }
  }
  auto mark = [&](int k) -> cudaError_t { return timed ? cudaEventRecord(ev[k], st) : cudaSuccess; };
  bool feats = false;
  for (const View& V : hv) feats = feats || V.feats != nullptr;
  const LaunchCfg cfg = launch_cfg(s, hv);
  const int mode = g ? kModeTan : (feats && s->feat_dim) ? kModeFwdFeat : kModeFwd;
  const int grid = s->sm_count * std::max(1, cfg.grid_mult[mode]);  // projection, shading, scatter, sort
  GS_CUDA(mark(0));
  GS_CUDA(launch_project(sc, dviews, nv, w, grid, st));
  GS_CUDA(mark(1));
  // The shading pass reads only what the projection wrote, and the binning
  // (scan, scatter, sort) reads nothing the shading writes (the sort's tie key,
  // the Gaussian index in rec_b.w, is written by the projection alone), so the
  // two run side by side and join before the compositing. Kernel timing keeps
  // them in order.
  const bool fork = !timed && s->side_st != nullptr;
  if (fork) {
    GS_CUDA(cudaEventRecord(s->ev_proj, st));
    GS_CUDA(cudaStreamWaitEvent(s->side_st, s->ev_proj, 0));
    GS_CUDA(launch_shade(sc, dviews, w, jac, grid, s->side_st));
    if (vis) {  // Algorithm 1's in-image test and the reverse pass's zeroed accumulator need no binning
      GS_CUDA(cudaMemsetAsync(dp<float>(s->vis_acc), 0, (size_t)s->rec_cap * kVisAcc * sizeof(float), s->side_st));
      GS_CUDA(launch_vis_inimage(sc, dviews, vis->mask, vis->uv, vis->grad, s->sm_count * 8, s->side_st));
    }
    GS_CUDA(cudaEventRecord(s->ev_shade, s->side_st));
  } else {
    GS_CUDA(launch_shade(sc, dviews, w, jac, grid, st));
  }
  GS_CUDA(mark(2));
  GS_CUDA(launch_scan_tiles(w, st));
  GS_CUDA(mark(3));
  GS_CUDA(launch_scatter(dviews, w, grid, st));
  GS_CUDA(mark(4));
  GS_CUDA(launch_sort_tiles(w, grid, st));
  if (fork) GS_CUDA(cudaStreamWaitEvent(st, s->ev_shade, 0));
  GS_CUDA(mark(5));
  if (!g || feats) GS_CUDA(launch_composite(sc, dviews, nv, w, feats, cfg, s->sm_count, st));
  if (g) {
    // the tangent pass re-renders the same values (without features) and adds
    // the loss and its pose gradient
    double* res = g->result ? g->result : w.result;
    if (bands && bands->n > 0 && nv == 1) {
      // band b of the tangent pass starts when the binning is done and its
      // target rows are on the device; consecutive bands run on two streams so
      // that one band's last tiles overlap the next band's first ones
      GS_CUDA(cudaEventRecord(s->ev_binned, st));
      const View& V = hv[0];
      for (int b = 0; b < bands->n; ++b) {
        const cudaStream_t bs = s->band_st[b & 1];
        GS_CUDA(cudaStreamWaitEvent(bs, s->ev_binned, 0));
        GS_CUDA(cudaStreamWaitEvent(bs, bands->ready[b], 0));
        const uint32_t t0 = V.tile_base + bands->tile_row[b] * (uint32_t)V.tiles_x;
        const uint32_t t1 = V.tile_base + bands->tile_row[b + 1] * (uint32_t)V.tiles_x;
        GS_CUDA(launch_composite_tangent_range(sc, dviews, nv, w, res, cfg, s->sm_count, bs, t0, t1,
                                               &w.ctr->band_queue[b]));
        GS_CUDA(cudaEventRecord(s->ev_band_done[b], bs));
      }
      for (int b = 0; b < bands->n; ++b) GS_CUDA(cudaStreamWaitEvent(st, s->ev_band_done[b], 0));
    } else {
      if (targets_ready) GS_CUDA(cudaStreamWaitEvent(st, targets_ready, 0));  // only this pass reads the targets
      GS_CUDA(launch_composite_tangent(sc, dviews, nv, w, res, cfg, s->sm_count, st));
    }
    GS_CUDA(launch_reduce_tangent(dviews, nv, w, res, st));
  }
  GS_CUDA(mark(6));
  if (vis) {
    // Algorithm 1: reverse pass of sum RGB, then the per-Gaussian tests
    float* acc = dp<float>(s->vis_acc);
    if (!fork) GS_CUDA(cudaMemsetAsync(acc, 0, (size_t)s->rec_cap * kVisAcc * sizeof(float), st));
    GS_CUDA(launch_vis_backward(dviews, nv, w, acc, s->sm_count, st));
    GS_CUDA(mark(7));
    if (!fork) GS_CUDA(launch_vis_inimage(sc, dviews, vis->mask, vis->uv, vis->grad, s->sm_count * 8, st));
    GS_CUDA(launch_vis_chain(dviews, w, acc, vis->mask, vis->grad, s->sm_count * 8, st));
    GS_CUDA(launch_vis_compact(vis->mask, vis->uv, (int)s->n, dp<uint32_t>(s->vis_blk), vis->vis_gid, vis->vis_uv,
                               st));
    GS_CUDA(mark(8));
  }
  if (timed) s->ev_pending.push_back({std::move(ev), vis ? 8 : 6});
  s->last_views = hv;
  s->last_tiles = (uint32_t)n_tiles;
  return GS_OK;
}

// Binary32 covariance of one Gaussian in the fixed operation order of the
// scene-packing kernel (host copy used when partitions are streamed).
void host_cov3d(const float* sc, const float* q, float S[6]) {
  const float qw = q[0], qx = q[1], qy = q[2], qz = q[3];
  const float n2 = qw * qw + qx * qx + qy * qy + qz * qz;
  float w = 1.0f, x = 0.0f, y = 0.0f, z = 0.0f;
  if (n2 > 0.0f) {
    const float nr = std::sqrt(n2);
    w = qw / nr;
    x = qx / nr;
    y = qy / nr;
    z = qz / nr;
  }
  const float xx = x * x, yy = y * y, zz = z * z, xy = x * y, xz = x * z, yz = y * z;
  const float wx = w * x, wy = w * y, wz = w * z;
  const float r[3][3] = {{1.0f - 2.0f * (yy + zz), 2.0f * (xy - wz), 2.0f * (xz + wy)},
                         {2.0f * (xy + wz), 1.0f - 2.0f * (xx + zz), 2.0f * (yz - wx)},
                         {2.0f * (xz - wy), 2.0f * (yz + wx), 1.0f - 2.0f * (xx + yy)}};
  float m[3][3];
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b) m[a][b] = r[a][b] * sc[b];
  const int ia[6] = {0, 0, 0, 1, 1, 2}, ib[6] = {0, 1, 2, 1, 2, 2};
  for (int k = 0; k < 6; ++k) {
    const float* u = m[ia[k]];
    const float* v = m[ib[k]];
    S[k] = u[0] * v[0] + u[1] * v[1] + u[2] * v[2];
  }
}

// Conservative test whether any Gaussian of the partition can reach the view's
// tiles. A Gaussian of largest scale s at depth z has a pixel radius of at most
// 3 s |J|_F + 3.5 px with |J|_F <= jb / z (guard clamp included), i.e. a world
// footprint of at most k s with k = 3.3 jb / f; the partition's box of
// mean_i +- k' s_i (k' = the next precomputed power of two >= k) therefore
// holds every Gaussian's footprint, and the image is widened by 32 px for the
// constant part and tile rounding. If all corners of that box lie outside one
// frustum plane (or in front of the near plane), no Gaussian of the partition
// has a non-empty tile rectangle, so skipping the partition changes nothing.
bool part_in_view(const Part& P, const View& V) {
  double R[9], t[3];
  for (int k = 0; k < 9; ++k) R[k] = (double)V.R[k] + (double)V.Rl[k];
  for (int k = 0; k < 3; ++k) t[k] = (double)V.t[k] + (double)V.tl[k];
  const double fx = V.fx, fy = V.fy;
  const double lx = 1.3 * 0.5 * V.width / fx, ly = 1.3 * 0.5 * V.height / fy;
  const double jb = std::sqrt(fx * fx * (1.0 + lx * lx) + fy * fy * (1.0 + ly * ly));
  const double k = 3.3 * jb / std::min(fx, fy);
  double blo[3], bhi[3];
  int j = 0;
  while (j < kPartBoxes && (double)(1 << j) < k) ++j;
  for (int a = 0; a < 3; ++a) {
    if (j < kPartBoxes) {
      blo[a] = P.klo[j][a];
      bhi[a] = P.khi[j][a];
    } else {  // very wide field of view: pad the means' box by k s_max
      blo[a] = P.lo[a] - k * P.smax;
      bhi[a] = P.hi[a] + k * P.smax;
    }
  }
  const double M = 32.0;
  const double a0 = (-M - V.cx) / fx, a1 = (16.0 * V.tiles_x + M - V.cx) / fx;
  const double b0 = (-M - V.cy) / fy, b1 = (16.0 * V.tiles_y + M - V.cy) / fy;
  bool out_near = true, out_l = true, out_r = true, out_t = true, out_b = true;
  for (int c = 0; c < 8; ++c) {
    const double X[3] = {(c & 1) ? bhi[0] : blo[0], (c & 2) ? bhi[1] : blo[1], (c & 4) ? bhi[2] : blo[2]};
    double q[3];
    for (int a = 0; a < 3; ++a) q[a] = R[3 * a] * X[0] + R[3 * a + 1] * X[1] + R[3 * a + 2] * X[2] + t[a];
    out_near = out_near && q[2] < 0.2;
    out_l = out_l && (q[0] - a0 * q[2]) < 0.0;
    out_r = out_r && (a1 * q[2] - q[0]) < 0.0;
    out_t = out_t && (q[1] - b0 * q[2]) < 0.0;
    out_b = out_b && (b1 * q[2] - q[1]) < 0.0;
  }
  return !(out_near || out_l || out_r || out_t || out_b);
}

// Upload a streamed partition that is not on the device yet (no-op otherwise).
gs_status make_resident(gs_scene* s, Part& P, cudaStream_t st) {
  if (!s->streaming || P.resident || P.end <= P.begin) return GS_OK;
  const size_t b = (size_t)P.begin, c = (size_t)(P.end - P.begin);
  GS_CUDA(cudaMemcpyAsync(dp<float4>(s->pos) + b, s->h_pos + b, c * sizeof(float4), cudaMemcpyHostToDevice, st));
  GS_CUDA(cudaMemcpyAsync(dp<float4>(s->cov) + 2 * b, s->h_cov + 2 * b, 2 * c * sizeof(float4),
                          cudaMemcpyHostToDevice, st));
  GS_CUDA(cudaMemcpyAsync(dp<float4>(s->sh) + b * s->nsh4, s->h_sh + b * s->nsh4, c * s->nsh4 * sizeof(float4),
                          cudaMemcpyHostToDevice, st));
  s->h2d_bytes += (int64_t)(c * (3 + s->nsh4) * sizeof(float4));
  if (s->feat_dim) {
    GS_CUDA(cudaMemcpyAsync(dp<uint4>(s->feat) + 4 * b, s->h_feat + 4 * b, 4 * c * sizeof(uint4),
                            cudaMemcpyHostToDevice, st));
    s->h2d_bytes += (int64_t)(4 * c * sizeof(uint4));
  }
  P.resident = true;
  return GS_OK;
}

// Partitions in view of any view of the call: uploads the non-resident ones
// (streaming scenes) on the stream and returns the index ranges the
// projection walks, in ascending order (header entry first).
gs_status prepare_call(gs_scene* s, const std::vector<View>& hv, cudaStream_t st, std::vector<int4>& ranges) {
  ranges.assign(1, make_int4(0, 0, 0, 0));
  int total = 0, active = 0;
  for (Part& P : s->parts) {
    if (P.end <= P.begin) continue;
    bool need = false;
    for (const View& V : hv) need = need || part_in_view(P, V);
    if (!need) continue;
    ++active;
    GS_TRY(make_resident(s, P, st));
    if (ranges.size() > 1 && ranges.back().y == (int)P.begin) {
      ranges.back().y = (int)P.end;  // merge adjacent partitions
    } else {
      ranges.push_back(make_int4((int)P.begin, (int)P.end, total, 0));
    }
    total += (int)(P.end - P.begin);
  }
  ranges[0] = make_int4((int)ranges.size() - 1, total, 0, 0);
  s->last_active = active;
  return GS_OK;
}

// Record capacity the last call needed: every segment must hold its count.
uint64_t records_capacity_needed(const Counters& c) {
  uint64_t mx = 0;
  for (int k = 0; k < kRecRegions; ++k) mx = std::max<uint64_t>(mx, c.rec_region[k]);
  return mx * kRecRegions;
}

// Indices of the filled record slots (segment k holds min(count_k, seg) records).
std::vector<uint32_t> filled_records(const Counters& c, uint32_t rec_cap) {
  std::vector<uint32_t> idx;
  const uint32_t seg = rec_cap / kRecRegions;
  for (int k = 0; k < kRecRegions; ++k)
    for (uint32_t j = 0; j < std::min(c.rec_region[k], seg); ++j) idx.push_back(k * seg + j);
  return idx;
}

gs_status read_counters(gs_scene* s, cudaStream_t st, Counters& c) {
  GS_CUDA(cudaMemcpyAsync(s->ctr_host, s->ctr.p, sizeof(Counters), cudaMemcpyDeviceToHost, st));
  GS_CUDA(cudaStreamSynchronize(st));
  c = *s->ctr_host;
  return GS_OK;
}

// Synchronous call with the regrow rule: render, check the counters, and if the
// workspace was too small grow it and render again.
// With a pose gradient the (loss, gradient) of the first view are copied to
// s->result_host in the same round trip as the counters.
gs_status run_sync(gs_scene* s, const std::vector<View>& hv, uint64_t n_tiles, const GradIn* g, cudaStream_t st,
                   cudaEvent_t targets_ready = nullptr, const VisOut* vis = nullptr, const Bands* bands = nullptr,
                   const std::function<gs_status()>* after_table = nullptr) {
  std::vector<int4> ranges;
  GS_TRY(prepare_call(s, hv, st, ranges));
  // the table from pinned memory: a synchronous call's previous upload is done
  const size_t tb = table_bytes(s, (int)hv.size());
  if (s->table_host_bytes < tb) {
    if (s->table_host) cudaFreeHost(s->table_host);
    s->table_host = nullptr;
    s->table_host_bytes = 0;
    GS_CUDA(cudaMallocHost(&s->table_host, tb));
    s->table_host_bytes = tb;
  }
  fill_table(s, hv, ranges, s->table_host);
  for (int attempt = 0; attempt < 4; ++attempt) {
    GS_TRY(enqueue(s, hv, ranges, n_tiles, g, st, s->table_host, targets_ready, vis, bands, false,
                   attempt == 0 ? after_table : nullptr));
    GS_CUDA(cudaMemcpyAsync(s->ctr_host, s->ctr.p, sizeof(Counters), cudaMemcpyDeviceToHost, st));
    if (g && !g->result)
      GS_CUDA(cudaMemcpyAsync(s->result_host, s->result.p, 7 * sizeof(double), cudaMemcpyDeviceToHost, st));
    GS_CUDA(cudaStreamSynchronize(st));
    const Counters c = *s->ctr_host;
    if (c.error) return fail(GS_ERR_INTERNAL, "device consistency check failed: the binning handed out a pair slot past the scanned tile counts");
    if (!c.overflow) return GS_OK;
    if (c.overflow & 4u) return fail(GS_ERR_CAPACITY, "more than 2^32 (tile, Gaussian) pairs in one call");
    const uint64_t need = records_capacity_needed(c);
    uint64_t need_rec = std::max<uint64_t>(s->rec_cap, need + need / 4 + 1024);
    uint64_t need_pair = std::max<uint64_t>(s->pair_cap, (uint64_t)c.pair_total + c.pair_total / 4 + 4096);
    if (c.overflow & 1u)  // pair count is incomplete when records overflowed
      need_pair = std::max<uint64_t>(need_pair, (uint64_t)s->pair_cap * (need_rec / std::max<uint32_t>(1, s->rec_cap) + 1));
    GS_CUDA(cudaStreamSynchronize(st));
    GS_TRY(grow_records(s, need_rec, g != nullptr || vis != nullptr));
    GS_TRY(grow_pairs(s, need_pair));
  }
  return fail(GS_ERR_CAPACITY, "workspace did not converge");
}

// IEEE half bit pattern -> float (host side, for the parity export)
float half_bits_to_float(uint16_t h) {
  const uint32_t sign = (uint32_t)(h >> 15) << 31;
  const uint32_t e = (h >> 10) & 0x1f, m = h & 0x3ff;
  float v;
  if (e == 0) {
    v = std::ldexp((float)m, -24);
  } else if (e == 31) {
    v = m ? NAN : INFINITY;
  } else {
    v = std::ldexp((float)(m | 0x400), (int)e - 25);
  }
  uint32_t bits;
  std::memcpy(&bits, &v, 4);
  bits |= sign;
  std::memcpy(&v, &bits, 4);
  return v;
}

gs_status check_scene(const gs_scene* s) {
  if (!s) return fail(GS_ERR_INVALID_ARG, "scene is NULL");
  return GS_OK;
}

gs_status set_device(const gs_scene* s) {
  GS_CUDA(cudaSetDevice(s->device));
  return GS_OK;
}

gs_status check_grad_args(const float* target_rgb, const float* target_depth, float depth_weight) {
  if (!target_rgb || !target_depth) return fail(GS_ERR_INVALID_ARG, "target_rgb and target_depth are required");
  if (!std::isfinite(depth_weight) || depth_weight < 0.0f)
    return fail(GS_ERR_INVALID_ARG, "depth_weight must be finite and >= 0");
  return GS_OK;
}

}  // namespace

namespace {

// Replay the cached graph if the batch layout (key) is unchanged, else capture
// a new one. Everything the capture needs is allocated before capturing.
gs_status run_graph(gs_scene* s, GraphCache& G, const std::vector<char>& key, const std::vector<View>& hv,
                    uint64_t n_tiles, const GradIn* g, cudaStream_t st, bool copy_back = false) {
  const int n_views = (int)hv.size();
  std::vector<int4> ranges;
  const bool ready = G.valid && G.key == key && G.gen == g_alloc_gen.load();
  if (ready) GS_CUDA(cudaEventSynchronize(G.done));  // previous replay read the table
  GS_TRY(prepare_call(s, hv, st, ranges));  // uploads partitions on st before the graph runs
  if (!ready) {
    if (G.exec) cudaGraphExecDestroy(G.exec);
    G.exec = nullptr;
    G.valid = false;
    if (G.host_table) cudaFreeHost(G.host_table);
    G.host_table = nullptr;
    if (!G.done) GS_CUDA(cudaEventCreateWithFlags(&G.done, cudaEventDisableTiming));
    GS_CUDA(cudaMallocHost(&G.host_table, table_bytes(s, n_views)));
    fill_table(s, hv, ranges, G.host_table);
    GS_TRY(grow_tiles(s, n_tiles));
    GS_TRY(ensure(s->views, table_bytes(s, n_views)));
    if (g && !g->result) GS_TRY(ensure(s->result, (size_t)n_views * kResultStride * sizeof(double)));
    const uint64_t guess = std::max<uint64_t>(1u << 16, (uint64_t)s->n * n_views / 4);
    GS_TRY(grow_records(s, s->rec_cap ? s->rec_cap : guess, g != nullptr));
    GS_TRY(grow_pairs(s, s->pair_cap ? s->pair_cap : guess * 8));
    // capture on a private stream (the legacy default stream cannot be captured);
    // the graph is then launched on the caller's stream
    if (!G.capture) GS_CUDA(cudaStreamCreateWithFlags(&G.capture, cudaStreamNonBlocking));
    GS_CUDA(cudaStreamSynchronize(st));
    cudaGraph_t graph = nullptr;
    GS_CUDA(cudaStreamBeginCapture(G.capture, cudaStreamCaptureModeThreadLocal));
    gs_status est = enqueue(s, hv, ranges, n_tiles, g, G.capture, G.host_table, nullptr, nullptr, nullptr, true);
    if (est == GS_OK && copy_back) {  // the counters and the (loss, gradient) to the pinned host copies
      if (cudaMemcpyAsync(s->ctr_host, s->ctr.p, sizeof(Counters), cudaMemcpyDeviceToHost, G.capture) != cudaSuccess ||
          cudaMemcpyAsync(s->result_host, s->result.p, 7 * sizeof(double), cudaMemcpyDeviceToHost, G.capture) !=
              cudaSuccess)
        est = fail(GS_ERR_CUDA, "cudaMemcpyAsync in the captured call failed");
    }
    const cudaError_t ce = cudaStreamEndCapture(G.capture, &graph);
    if (est != GS_OK) {
      if (graph) cudaGraphDestroy(graph);
      return est;
    }
    if (ce != cudaSuccess) return fail(GS_ERR_CUDA, std::string("cudaStreamEndCapture: ") + cudaGetErrorString(ce));
    const cudaError_t ie = cudaGraphInstantiate(&G.exec, graph, 0);
    cudaGraphDestroy(graph);
    if (ie != cudaSuccess) return fail(GS_ERR_CUDA, std::string("cudaGraphInstantiate: ") + cudaGetErrorString(ie));
    G.key = key;
    G.n_views = n_views;
    G.gen = g_alloc_gen.load();
    G.valid = true;
  } else {
    fill_table(s, hv, ranges, G.host_table);
    s->last_views = hv;
    s->last_tiles = (uint32_t)n_tiles;
  }
  GS_CUDA(cudaGraphLaunch(G.exec, st));
  GS_CUDA(cudaEventRecord(G.done, st));
  return GS_OK;
}

template <typename T>
void append_bytes(std::vector<char>& key, const T* p, size_t n) {
  const char* b = reinterpret_cast<const char*>(p);
  key.insert(key.end(), b, b + n * sizeof(T));
}

// A synchronous single-view pose gradient replayed from a CUDA graph: one
// launch instead of the call's memsets, table upload and six kernel launches.
// The graph is keyed on everything but the pose (the view with its pose fields
// cleared); a call that overflows the workspace is redone by the regrow path
// and the next call captures again. With kernel timing on, the ordinary path
// runs (graphs carry no timing events).
gs_status run_sync_graphed(gs_scene* s, const std::vector<View>& hv, uint64_t n_tiles, const GradIn* g,
                           cudaStream_t st) {
  if (s->timing || hv.size() != 1 || g->result) return run_sync(s, hv, n_tiles, g, st);
  View k = hv[0];
  std::memset(k.R, 0, sizeof(k.R));
  std::memset(k.t, 0, sizeof(k.t));
  std::memset(k.Rl, 0, sizeof(k.Rl));
  std::memset(k.tl, 0, sizeof(k.tl));
  std::memset(k.cw, 0, sizeof(k.cw));
  std::vector<char> key;
  append_bytes(key, &k, 1);
  append_bytes(key, &n_tiles, 1);
  GS_TRY(run_graph(s, s->graph_sync, key, hv, n_tiles, g, st, true));  // the graph copies the results back
  GS_CUDA(cudaStreamSynchronize(st));
  const Counters& c = *s->ctr_host;
  if (c.error) return fail(GS_ERR_INTERNAL, "device consistency check failed: the binning handed out a pair slot past the scanned tile counts");
  if (c.overflow) {
    s->graph_sync.valid = false;
    return run_sync(s, hv, n_tiles, g, st);
  }
  return GS_OK;
}

}  // namespace

extern "C" {

const char* gs_last_error(void) { return g_err.c_str(); }

const char* gs_version(void) { return "gsr 0.1 (sm_103a)"; }

gs_status gs_create_scene(const gs_scene_desc* d, gs_scene** out) {
  g_err.clear();
  if (!d || !out) return fail(GS_ERR_INVALID_ARG, "desc and out are required");
  *out = nullptr;
  if (d->n < 0 || d->n >= 0x7fffffffLL) return fail(GS_ERR_INVALID_ARG, "n out of range");
  if (d->sh_degree < 0 || d->sh_degree > 3) return fail(GS_ERR_INVALID_ARG, "sh_degree must be 0..3");
  if (d->feat_dim != 0 && d->feat_dim != 32) return fail(GS_ERR_INVALID_ARG, "feat_dim must be 0 or 32");
  if (d->n > 0 && (!d->means || !d->scales || !d->quats || !d->opacities || !d->sh))
    return fail(GS_ERR_INVALID_ARG, "scene arrays are required when n > 0");
  if (d->n > 0 && d->feat_dim && !d->feats_bf16) return fail(GS_ERR_INVALID_ARG, "feats_bf16 required");
  if (d->n_partitions < 0) return fail(GS_ERR_INVALID_ARG, "n_partitions < 0");
  std::vector<int64_t> parts;
  if (d->n_partitions > 0) {
    if (!d->partition_offsets) return fail(GS_ERR_INVALID_ARG, "partition_offsets required");
    parts.assign(d->partition_offsets, d->partition_offsets + d->n_partitions + 1);
    if (parts.front() != 0 || parts.back() != d->n) return fail(GS_ERR_INVALID_ARG, "partition table must span [0, n]");
    for (int k = 0; k < d->n_partitions; ++k)
      if (parts[k + 1] < parts[k]) return fail(GS_ERR_INVALID_ARG, "partition offsets must ascend");
  } else {
    parts = {0, d->n};
  }
  gs_scene* s = new gs_scene();
  s->n = d->n;
  s->sh_degree = d->sh_degree;
  s->feat_dim = d->feat_dim;
  s->part_off = parts;
  const int K3 = 3 * (d->sh_degree + 1) * (d->sh_degree + 1);
  s->nsh4 = (K3 + 3) / 4;
  auto cleanup = [&](gs_status st) {
    gs_destroy_scene(s);
    return st;
  };
  cudaError_t e = cudaGetDevice(&s->device);
  if (e != cudaSuccess) return cleanup(fail(GS_ERR_CUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e)));
  cudaDeviceProp prop;
  e = cudaGetDeviceProperties(&prop, s->device);
  if (e != cudaSuccess) return cleanup(fail(GS_ERR_CUDA, std::string("cudaGetDeviceProperties: ") + cudaGetErrorString(e)));
  s->sm_count = prop.multiProcessorCount;
  s->device_name = prop.name;
  e = cudaStreamCreateWithFlags(&s->side_st, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&s->ev_proj, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&s->ev_shade, cudaEventDisableTiming);
  if (e != cudaSuccess) return cleanup(fail(GS_ERR_CUDA, std::string("stream / event creation: ") + cudaGetErrorString(e)));
  const size_t n = (size_t)d->n;
  gs_status st;
  if ((st = ensure(s->pos, n * sizeof(float4))) != GS_OK) return cleanup(st);
  if ((st = ensure(s->cov, 2 * n * sizeof(float4))) != GS_OK) return cleanup(st);
  if ((st = ensure(s->sh, n * s->nsh4 * sizeof(float4))) != GS_OK) return cleanup(st);
  if (s->feat_dim && (st = ensure(s->feat, n * 4 * sizeof(uint4))) != GS_OK) return cleanup(st);
  if ((st = ensure(s->ctr, sizeof(Counters))) != GS_OK) return cleanup(st);
  if ((st = ensure(s->result, 8 * sizeof(double))) != GS_OK) return cleanup(st);
  if (cudaMallocHost(&s->ctr_host, sizeof(Counters)) != cudaSuccess ||
      cudaMallocHost(&s->result_host, 8 * sizeof(double)) != cudaSuccess) {
    cudaGetLastError();
    return cleanup(fail(GS_ERR_OOM, "pinned host allocation failed"));
  }
  // partitions: index ranges, bounding boxes of the means, largest scale
  {
    std::vector<float> hm, hs;
    const float *m = d->means, *sc = d->scales;
    if (n > 0 && d->device_resident) {
      hm.resize(3 * n);
      hs.resize(3 * n);
      e = cudaMemcpy(hm.data(), d->means, 3 * n * sizeof(float), cudaMemcpyDeviceToHost);
      if (e == cudaSuccess) e = cudaMemcpy(hs.data(), d->scales, 3 * n * sizeof(float), cudaMemcpyDeviceToHost);
      if (e != cudaSuccess) return cleanup(fail(GS_ERR_CUDA, std::string("cudaMemcpy: ") + cudaGetErrorString(e)));
      m = hm.data();
      sc = hs.data();
    }
    for (size_t k = 0; k + 1 < parts.size(); ++k) {
      Part P;
      P.begin = parts[k];
      P.end = parts[k + 1];
      for (int a = 0; a < 3; ++a) {
        P.lo[a] = 1e300;
        P.hi[a] = -1e300;
        for (int j = 0; j < kPartBoxes; ++j) {
          P.klo[j][a] = 1e300;
          P.khi[j][a] = -1e300;
        }
      }
      for (int64_t i = P.begin; i < P.end; ++i) {
        const double si = std::max(std::fabs((double)sc[3 * i]),
                                   std::max(std::fabs((double)sc[3 * i + 1]), std::fabs((double)sc[3 * i + 2])));
        P.smax = std::max(P.smax, si);
        for (int a = 0; a < 3; ++a) {
          const double x = m[3 * i + a];
          P.lo[a] = std::min(P.lo[a], x);
          P.hi[a] = std::max(P.hi[a], x);
          for (int j = 0; j < kPartBoxes; ++j) {
            P.klo[j][a] = std::min(P.klo[j][a], x - (double)(1 << j) * si);
            P.khi[j][a] = std::max(P.khi[j][a], x + (double)(1 << j) * si);
          }
        }
      }
      s->parts.push_back(P);
    }
  }
  s->streaming = !d->device_resident && d->n_partitions > 0 && n > 0;
  if (s->streaming) {
    // pack on the host into pinned memory in the device layout; partitions are
    // uploaded on first use by a call whose views they can reach
    if (cudaMallocHost(&s->h_pos, n * sizeof(float4)) != cudaSuccess ||
        cudaMallocHost(&s->h_cov, 2 * n * sizeof(float4)) != cudaSuccess ||
        cudaMallocHost(&s->h_sh, n * s->nsh4 * sizeof(float4)) != cudaSuccess ||
        (s->feat_dim && cudaMallocHost(&s->h_feat, n * 4 * sizeof(uint4)) != cudaSuccess)) {
      cudaGetLastError();
      return cleanup(fail(GS_ERR_OOM, "pinned host allocation for the streamed scene failed"));
    }
    for (size_t i = 0; i < n; ++i) {
      float S[6];
      host_cov3d(d->scales + 3 * i, d->quats + 4 * i, S);
      const float* sc = d->scales + 3 * i;
      const float smax = std::max(sc[0], std::max(sc[1], sc[2]));
      s->h_pos[i] = make_float4(d->means[3 * i], d->means[3 * i + 1], d->means[3 * i + 2], smax);
      s->h_cov[2 * i] = make_float4(S[0], S[1], S[2], S[3]);
      s->h_cov[2 * i + 1] = make_float4(S[4], S[5], d->opacities[i], 0.0f);
      float* so = reinterpret_cast<float*>(s->h_sh + i * s->nsh4);
      for (int k = 0; k < 4 * s->nsh4; ++k) so[k] = (k < K3) ? d->sh[i * K3 + k] : 0.0f;
      if (s->feat_dim) std::memcpy(s->h_feat + 4 * i, d->feats_bf16 + 32 * i, 64);
    }
  } else {
    for (Part& P : s->parts) P.resident = true;
  }
  if (n > 0 && !s->streaming) {
    const float *m = d->means, *sc = d->scales, *q = d->quats, *o = d->opacities, *sh = d->sh;
    const uint16_t* f = d->feats_bf16;
    DevBuf staging;
    if (!d->device_resident) {
      const size_t fb = s->feat_dim ? n * 32 * sizeof(uint16_t) : 0;
      const size_t bytes = n * (3 + 3 + 4 + 1 + K3) * sizeof(float) + fb;
      if ((st = ensure(staging, bytes)) != GS_OK) return cleanup(st);
      char* p = static_cast<char*>(staging.p);
      auto put = [&](const void* src, size_t b) {
        void* dst = p;
        p += b;
        return std::make_pair(dst, cudaMemcpy(dst, src, b, cudaMemcpyHostToDevice));
      };
      auto r1 = put(m, n * 3 * 4), r2 = put(sc, n * 3 * 4), r3 = put(q, n * 4 * 4), r4 = put(o, n * 4),
           r5 = put(sh, n * K3 * 4);
      std::pair<void*, cudaError_t> r6{nullptr, cudaSuccess};
      if (fb) r6 = put(f, fb);
      for (auto* r : {&r1, &r2, &r3, &r4, &r5, &r6})
        if (r->second != cudaSuccess) {
          release(staging);
          return cleanup(fail(GS_ERR_CUDA, std::string("cudaMemcpy: ") + cudaGetErrorString(r->second)));
        }
      m = (const float*)r1.first;
      sc = (const float*)r2.first;
      q = (const float*)r3.first;
      o = (const float*)r4.first;
      sh = (const float*)r5.first;
      f = (const uint16_t*)r6.first;
    }
    e = launch_pack_scene(m, sc, q, o, sh, K3, f, s->feat_dim, (int)n, s->nsh4, dp<float4>(s->pos), dp<float4>(s->cov),
                          dp<float4>(s->sh), s->feat_dim ? dp<uint4>(s->feat) : nullptr, 0);
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    release(staging);
    if (e != cudaSuccess) return cleanup(fail(GS_ERR_CUDA, std::string("pack: ") + cudaGetErrorString(e)));
  }
  // occupancy queries of every compositor variant outside any stream capture
  for (int m = 0; m < kModeCount; ++m)
    for (int v = 0; v < kCompVariants; ++v) composite_variant_info(m, v);
  *out = s;
  return GS_OK;
}

void gs_destroy_scene(gs_scene* s) {
  if (!s) return;
  cudaSetDevice(s->device);
  cudaDeviceSynchronize();
  for (GraphCache* G : {&s->graph, &s->graph_grad, &s->graph_sync}) {
    if (G->exec) cudaGraphExecDestroy(G->exec);
    if (G->host_table) cudaFreeHost(G->host_table);
    if (G->done) cudaEventDestroy(G->done);
    if (G->capture) cudaStreamDestroy(G->capture);
  }
  for (auto& tc : s->ev_pending)
    for (cudaEvent_t e : tc.ev) cudaEventDestroy(e);
  for (auto& ev : s->ev_free)
    for (cudaEvent_t e : ev) cudaEventDestroy(e);
  for (DevBuf* b : {&s->pos, &s->cov, &s->sh, &s->feat, &s->rec_a, &s->rec_b, &s->rec_c, &s->rec_m, &s->rec_j,
                    &s->tile_count, &s->tile_offset, &s->tile_cursor, &s->partials, &s->chunks, &s->pairs, &s->pairs_tmp,
                    &s->ctr, &s->result, &s->views, &s->vis_T, &s->vis_last, &s->vis_acc, &s->vis_uv, &s->vis_blk})
    release(*b);
  for (void* h : {(void*)s->h_pos, (void*)s->h_cov, (void*)s->h_sh, (void*)s->h_feat})
    if (h) cudaFreeHost(h);
  if (s->ctr_host) cudaFreeHost(s->ctr_host);
  if (s->table_host) cudaFreeHost(s->table_host);
  if (s->result_host) cudaFreeHost(s->result_host);
  release(s->targets);
  if (s->copy_st) cudaStreamDestroy(s->copy_st);
  for (cudaStream_t b : s->band_st)
    if (b) cudaStreamDestroy(b);
  if (s->side_st) cudaStreamDestroy(s->side_st);
  if (s->ev_proj) cudaEventDestroy(s->ev_proj);
  if (s->ev_shade) cudaEventDestroy(s->ev_shade);
  if (s->ev_binned) cudaEventDestroy(s->ev_binned);
  for (int b = 0; b < kMaxBands; ++b) {
    if (s->ev_band[b]) cudaEventDestroy(s->ev_band[b]);
    if (s->ev_band_done[b]) cudaEventDestroy(s->ev_band_done[b]);
  }
  if (s->ev_call) cudaEventDestroy(s->ev_call);
  if (s->ev_targets) cudaEventDestroy(s->ev_targets);
  delete s;
}

gs_status gs_scene_reserve(gs_scene* s, int64_t max_records, int64_t max_pairs) {
  g_err.clear();
  GS_TRY(check_scene(s));
  if (max_records < 0 || max_pairs < 0) return fail(GS_ERR_INVALID_ARG, "negative reservation");
  GS_TRY(set_device(s));
  GS_CUDA(cudaDeviceSynchronize());
  GS_TRY(grow_records(s, (uint64_t)max_records, true));
  GS_TRY(grow_pairs(s, (uint64_t)max_pairs));
  return GS_OK;
}

gs_status gs_render(gs_scene* s, const gs_camera* cam, const gs_pose* pose, const gs_outputs* out, void* stream) {
  g_err.clear();
  GS_TRY(check_scene(s));
  if (!cam || !pose) return fail(GS_ERR_INVALID_ARG, "cam and pose are required");
  GS_TRY(set_device(s));
  std::vector<View> hv;
  uint64_t n_tiles;
  GS_TRY(build_views(s, 1, cam, pose, out, nullptr, hv, n_tiles));
  return run_sync(s, hv, n_tiles, nullptr, (cudaStream_t)stream);
}

gs_status gs_render_async(gs_scene* s, const gs_camera* cam, const gs_pose* pose, const gs_outputs* out,
                          void* stream) {
  g_err.clear();
  GS_TRY(check_scene(s));
  if (!cam || !pose) return fail(GS_ERR_INVALID_ARG, "cam and pose are required");
  GS_TRY(set_device(s));
  std::vector<View> hv;
  uint64_t n_tiles;
  GS_TRY(build_views(s, 1, cam, pose, out, nullptr, hv, n_tiles));
  std::vector<int4> ranges;
  GS_TRY(prepare_call(s, hv, (cudaStream_t)stream, ranges));
  return enqueue(s, hv, ranges, n_tiles, nullptr, (cudaStream_t)stream, nullptr);
}

gs_status gs_render_pose_grad(gs_scene* s, const gs_camera* cam, const gs_pose* pose, const float* target_rgb,
                              const float* target_depth, const float* pixel_weight, float depth_weight,
                              const gs_outputs* out, double* loss_out, double* grad_xi_out, void* stream) {
  g_err.clear();
  GS_TRY(check_scene(s));
  if (!cam || !pose) return fail(GS_ERR_INVALID_ARG, "cam and pose are required");
  GS_TRY(check_grad_args(target_rgb, target_depth, depth_weight));
  GS_TRY(set_device(s));
  GradIn g{&target_rgb, &target_depth, &pixel_weight, depth_weight, nullptr};
  std::vector<View> hv;
  uint64_t n_tiles;
  GS_TRY(build_views(s, 1, cam, pose, out, &g, hv, n_tiles));
  const cudaStream_t st = (cudaStream_t)stream;
  GS_TRY(run_sync_graphed(s, hv, n_tiles, &g, st));
  if (loss_out) *loss_out = s->result_host[0];
  if (grad_xi_out)
    for (int k = 0; k < 6; ++k) grad_xi_out[k] = s->result_host[1 + k];
  return GS_OK;
}

gs_status gs_render_pose_grad_host(gs_scene* s, const gs_camera* cam, const gs_pose* pose,
                                   const float* target_rgb, const float* target_depth, const float* pixel_weight,
                                   float depth_weight, const gs_outputs* out, double* loss_out, double* grad_xi_out,
                                   void* stream) {
  g_err.clear();
  GS_TRY(check_scene(s));
  if (!cam || !pose) return fail(GS_ERR_INVALID_ARG, "cam and pose are required");
  GS_TRY(check_grad_args(target_rgb, target_depth, depth_weight));
  GS_TRY(set_device(s));
  GS_TRY(check_cam(*cam));
  const cudaStream_t st = (cudaStream_t)stream;
  const size_t P = (size_t)cam->width * cam->height;
  // Pinned (page-locked, device-mapped) host targets are read in place by the
  // tangent pass over the CPU-GPU link: each pixel's targets once, at the end
  // of its tile, spread over the whole pass. A bulk copy instead slows the
  // memory-bound projection and binning kernels it overlaps by about a quarter.
  {
    const void* dev[3] = {nullptr, nullptr, nullptr};
    const void* hp[3] = {target_rgb, target_depth, pixel_weight};
    bool mapped = true;
    for (int k = 0; k < 3 && mapped; ++k) {
      if (!hp[k]) continue;
      cudaPointerAttributes a;
      if (cudaPointerGetAttributes(&a, hp[k]) != cudaSuccess) {
        cudaGetLastError();
        mapped = false;
      } else {
        mapped = a.type == cudaMemoryTypeHost && a.devicePointer != nullptr;
        dev[k] = a.devicePointer;
      }
    }
    if (mapped) {
      const float* tr = static_cast<const float*>(dev[0]);
      const float* td = static_cast<const float*>(dev[1]);
      const float* tw = static_cast<const float*>(dev[2]);
      GradIn g{&tr, &td, &tw, depth_weight, nullptr};
      std::vector<View> hv;
      uint64_t n_tiles;
      GS_TRY(build_views(s, 1, cam, pose, out, &g, hv, n_tiles));
      GS_TRY(run_sync_graphed(s, hv, n_tiles, &g, st));
      if (loss_out) *loss_out = s->result_host[0];
      if (grad_xi_out)
        for (int k = 0; k < 6; ++k) grad_xi_out[k] = s->result_host[1 + k];
      return GS_OK;
    }
  }
  // pageable targets: uploaded by the copy engine, in bands
  GS_TRY(ensure(s->targets, (pixel_weight ? 5 : 4) * P * sizeof(float)));
  if (!s->copy_st) GS_CUDA(cudaStreamCreateWithFlags(&s->copy_st, cudaStreamNonBlocking));
  if (!s->ev_call) GS_CUDA(cudaEventCreateWithFlags(&s->ev_call, cudaEventDisableTiming));
  if (!s->ev_targets) GS_CUDA(cudaEventCreateWithFlags(&s->ev_targets, cudaEventDisableTiming));
  if (!s->ev_binned) {
    GS_CUDA(cudaEventCreateWithFlags(&s->ev_binned, cudaEventDisableTiming));
    for (int b = 0; b < kMaxBands; ++b) {
      GS_CUDA(cudaEventCreateWithFlags(&s->ev_band[b], cudaEventDisableTiming));
      GS_CUDA(cudaEventCreateWithFlags(&s->ev_band_done[b], cudaEventDisableTiming));
    }
    for (cudaStream_t& b : s->band_st) GS_CUDA(cudaStreamCreateWithFlags(&b, cudaStreamNonBlocking));
  }
  float* d_rgb = dp<float>(s->targets);
  float* d_dep = d_rgb + 3 * P;
  float* d_w = pixel_weight ? d_rgb + 4 * P : nullptr;
  // The uploads (16 or 20 B per pixel at the host link's ~200 GB/s) start after
  // the work already on the caller's stream, which may still read the buffers,
  // and after the call table, which the first kernel needs (queued behind tens
  // of MB of targets it would hold everything back). They go in bands of tile
  // rows: band b's tangent pass needs only its rows, so the later bands upload
  // while the projection, the binning and the earlier bands run.
  const int W = cam->width, H = cam->height;
  const int tiles_y = (H + kTile - 1) / kTile;
  Bands bands;
  bands.n = std::min(kUploadBands, tiles_y);
  for (int b = 0; b <= bands.n; ++b) bands.tile_row[b] = (uint32_t)((int64_t)tiles_y * b / bands.n);
  for (int b = 0; b < bands.n; ++b) bands.ready[b] = s->ev_band[b];
  // issued once the call table is on the stream (see enqueue)
  const std::function<gs_status()> upload = [&]() -> gs_status {
    GS_CUDA(cudaEventRecord(s->ev_call, st));
    GS_CUDA(cudaStreamWaitEvent(s->copy_st, s->ev_call, 0));
    for (int b = 0; b < bands.n; ++b) {
      const size_t y0 = (size_t)bands.tile_row[b] * kTile;
      const size_t y1 = std::min((size_t)bands.tile_row[b + 1] * kTile, (size_t)H);
      const size_t off = y0 * W, bytes = (y1 - y0) * W * sizeof(float);
      // the three colour planes of the band in one strided copy
      GS_CUDA(cudaMemcpy2DAsync(d_rgb + off, P * sizeof(float), target_rgb + off, P * sizeof(float), bytes, 3,
                                cudaMemcpyHostToDevice, s->copy_st));
      GS_CUDA(cudaMemcpyAsync(d_dep + off, target_depth + off, bytes, cudaMemcpyHostToDevice, s->copy_st));
      if (d_w) GS_CUDA(cudaMemcpyAsync(d_w + off, pixel_weight + off, bytes, cudaMemcpyHostToDevice, s->copy_st));
      GS_CUDA(cudaEventRecord(s->ev_band[b], s->copy_st));
    }
    return GS_OK;
  };
  const float* tr = d_rgb;
  const float* td = d_dep;
  const float* tw = d_w;
  GradIn g{&tr, &td, &tw, depth_weight, nullptr};
  std::vector<View> hv;
  uint64_t n_tiles;
  GS_TRY(build_views(s, 1, cam, pose, out, &g, hv, n_tiles));
  GS_TRY(run_sync(s, hv, n_tiles, &g, st, nullptr, nullptr, &bands, &upload));
  if (loss_out) *loss_out = s->result_host[0];
  if (grad_xi_out)
    for (int k = 0; k < 6; ++k) grad_xi_out[k] = s->result_host[1 + k];
  return GS_OK;
}

gs_status gs_render_pose_grad_async(gs_scene* s, const gs_camera* cam, const gs_pose* pose, const float* target_rgb,
                                    const float* target_depth, const float* pixel_weight, float depth_weight,
                                    const gs_outputs* out, double* result_dev, void* stream) {
  g_err.clear();
  GS_TRY(check_scene(s));
  if (!cam || !pose || !result_dev) return fail(GS_ERR_INVALID_ARG, "cam, pose and result_dev are required");
  GS_TRY(check_grad_args(target_rgb, target_depth, depth_weight));
  GS_TRY(set_device(s));
  GradIn g{&target_rgb, &target_depth, &pixel_weight, depth_weight, result_dev};
  std::vector<View> hv;
  uint64_t n_tiles;
  GS_TRY(build_views(s, 1, cam, pose, out, &g, hv, n_tiles));
  std::vector<int4> ranges;
  GS_TRY(prepare_call(s, hv, (cudaStream_t)stream, ranges));
  return enqueue(s, hv, ranges, n_tiles, &g, (cudaStream_t)stream, nullptr);
}

gs_status gs_render_batch(gs_scene* s, int n_views, const gs_camera* cams, const gs_pose* poses,
                          const gs_outputs* outs, unsigned flags, void* stream) {
  g_err.clear();
  GS_TRY(check_scene(s));
  if (n_views < 1 || !cams || !poses || !outs) return fail(GS_ERR_INVALID_ARG, "n_views >= 1, cams, poses, outs required");
  if (flags & ~GS_BATCH_GRAPH) return fail(GS_ERR_INVALID_ARG, "unknown flag");
  GS_TRY(set_device(s));
  const cudaStream_t st = (cudaStream_t)stream;
  std::vector<View> hv;
  uint64_t n_tiles;
  GS_TRY(build_views(s, n_views, cams, poses, outs, nullptr, hv, n_tiles));
  if (!(flags & GS_BATCH_GRAPH)) return run_sync(s, hv, n_tiles, nullptr, st);
  std::vector<char> key;
  append_bytes(key, cams, n_views);
  append_bytes(key, outs, n_views);
  return run_graph(s, s->graph, key, hv, n_tiles, nullptr, st);
}

gs_status gs_render_pose_grad_batch(gs_scene* s, int n_views, const gs_camera* cams, const gs_pose* poses,
                                    const float* const* target_rgb, const float* const* target_depth,
                                    const float* const* pixel_weight, float depth_weight, const gs_outputs* outs,
                                    double* loss_out, double* grad_out, double* results_dev, unsigned flags,
                                    void* stream) {
  g_err.clear();
  GS_TRY(check_scene(s));
  if (n_views < 1 || !cams || !poses || !target_rgb || !target_depth)
    return fail(GS_ERR_INVALID_ARG, "n_views >= 1, cams, poses, target_rgb, target_depth required");
  if (flags & ~GS_BATCH_GRAPH) return fail(GS_ERR_INVALID_ARG, "unknown flag");
  for (int v = 0; v < n_views; ++v) GS_TRY(check_grad_args(target_rgb[v], target_depth[v], depth_weight));
  if ((flags & GS_BATCH_GRAPH) && !results_dev) return fail(GS_ERR_INVALID_ARG, "graph mode needs results_dev");
  GS_TRY(set_device(s));
  const cudaStream_t st = (cudaStream_t)stream;
  GradIn g{target_rgb, target_depth, pixel_weight, depth_weight, results_dev};
  std::vector<View> hv;
  uint64_t n_tiles;
  GS_TRY(build_views(s, n_views, cams, poses, outs, &g, hv, n_tiles));
  if (flags & GS_BATCH_GRAPH) {
    std::vector<char> key;
    append_bytes(key, cams, n_views);
    if (outs) append_bytes(key, outs, n_views);
    append_bytes(key, target_rgb, n_views);
    append_bytes(key, target_depth, n_views);
    if (pixel_weight) append_bytes(key, pixel_weight, n_views);
    append_bytes(key, &depth_weight, 1);
    append_bytes(key, &results_dev, 1);
    return run_graph(s, s->graph_grad, key, hv, n_tiles, &g, st);
  }
  GS_TRY(run_sync(s, hv, n_tiles, &g, st));
  double* res = results_dev ? results_dev : dp<double>(s->result);
  std::vector<double> host((size_t)n_views * kResultStride);
  GS_CUDA(cudaMemcpyAsync(host.data(), res, host.size() * sizeof(double), cudaMemcpyDeviceToHost, st));
  GS_CUDA(cudaStreamSynchronize(st));
  for (int v = 0; v < n_views; ++v) {
    if (loss_out) loss_out[v] = host[(size_t)v * kResultStride];
    if (grad_out)
      for (int k = 0; k < 6; ++k) grad_out[6 * v + k] = host[(size_t)v * kResultStride + 1 + k];
  }
  return GS_OK;
}

gs_status gs_scene_stream_stats(gs_scene* s, int64_t* h2d_bytes, int* resident_partitions,
                                int* active_partitions) {
  g_err.clear();
  GS_TRY(check_scene(s));
  int res = 0;
  for (const Part& P : s->parts) res += P.resident ? 1 : 0;
  if (h2d_bytes) *h2d_bytes = s->h2d_bytes;
  if (resident_partitions) *resident_partitions = res;
  if (active_partitions) *active_partitions = s->last_active;
  return GS_OK;
}

gs_status gs_scene_shape(const gs_scene* s, int64_t* n, int* sh_degree, int* feat_dim) {
  g_err.clear();
  GS_TRY(check_scene(s));
  if (n) *n = s->n;
  if (sh_degree) *sh_degree = s->sh_degree;
  if (feat_dim) *feat_dim = s->feat_dim;
  return GS_OK;
}

gs_status gs_scene_evict(gs_scene* s) {
  g_err.clear();
  GS_TRY(check_scene(s));
  if (!s->streaming) return GS_OK;
  GS_TRY(set_device(s));
  GS_CUDA(cudaDeviceSynchronize());
  for (Part& P : s->parts) P.resident = false;
  return GS_OK;
}

gs_status gs_scene_set_timing(gs_scene* s, int enable) {
  g_err.clear();
  GS_TRY(check_scene(s));
  s->timing = enable != 0;
  return GS_OK;
}

gs_status gs_scene_kernel_times(gs_scene* s, double* total_ms, int64_t* launches) {
  g_err.clear();
  GS_TRY(check_scene(s));
  if (!total_ms) return fail(GS_ERR_INVALID_ARG, "total_ms is required");
  GS_TRY(set_device(s));
  for (auto& tc : s->ev_pending) {
    GS_CUDA(cudaEventSynchronize(tc.ev[tc.n_kernels]));
    for (int k = 0; k < tc.n_kernels; ++k) {
      float ms = 0.f;
      GS_CUDA(cudaEventElapsedTime(&ms, tc.ev[k], tc.ev[k + 1]));
      s->kt_ms[k] += ms;
      s->kt_n[k] += 1;
    }
    s->ev_free.push_back(std::move(tc.ev));
  }
  s->ev_pending.clear();
  for (int k = 0; k < GS_KERNEL_COUNT; ++k) {
    total_ms[k] = s->kt_ms[k];
    if (launches) launches[k] = s->kt_n[k];
    s->kt_ms[k] = 0.0;
    s->kt_n[k] = 0;
  }
  return GS_OK;
}

gs_status gs_visibility(gs_scene* s, const gs_camera* cam, const gs_pose* pose, uint8_t* mask, float* uv,
                        float* grad_mean, int32_t* visible_ids, float* visible_uv, int64_t* n_visible,
                        void* stream) {
  g_err.clear();
  GS_TRY(check_scene(s));
  if (!cam || !pose || !mask) return fail(GS_ERR_INVALID_ARG, "cam, pose and mask are required");
  for (const void* q : {(const void*)uv, (const void*)visible_uv})
    if (reinterpret_cast<uintptr_t>(q) % 8) return fail(GS_ERR_INVALID_ARG, "uv arrays must be 8-byte aligned");
  if (reinterpret_cast<uintptr_t>(grad_mean) % 4 || reinterpret_cast<uintptr_t>(visible_ids) % 4)
    return fail(GS_ERR_INVALID_ARG, "grad_mean and visible_ids must be 4-byte aligned");
  GS_TRY(set_device(s));
  GS_TRY(check_cam(*cam));
  const cudaStream_t st = (cudaStream_t)stream;
  const size_t P = (size_t)cam->width * cam->height;
  GS_TRY(ensure(s->vis_T, P * sizeof(float)));
  GS_TRY(ensure(s->vis_last, P * sizeof(uint32_t)));
  if (!uv) GS_TRY(ensure(s->vis_uv, (size_t)std::max<int64_t>(s->n, 1) * sizeof(float2)));
  // the in-image test covers every Gaussian: a streamed scene becomes resident
  for (Part& Pt : s->parts) GS_TRY(make_resident(s, Pt, st));
  gs_outputs o{};
  o.final_T = dp<float>(s->vis_T);
  o.last_idx = dp<uint32_t>(s->vis_last);
  std::vector<View> hv;
  uint64_t n_tiles;
  GS_TRY(build_views(s, 1, cam, pose, &o, nullptr, hv, n_tiles));
  const VisOut vo{mask, uv ? reinterpret_cast<float2*>(uv) : dp<float2>(s->vis_uv), grad_mean, visible_ids,
                  reinterpret_cast<float2*>(visible_uv)};
  GS_TRY(run_sync(s, hv, n_tiles, nullptr, st, nullptr, &vo));
  if (n_visible) *n_visible = (int64_t)s->ctr_host->vis_count;
  return GS_OK;
}

gs_status gs_scene_blend_count(gs_scene* s, void* stream, int64_t* blended) {
  g_err.clear();
  GS_TRY(check_scene(s));
  if (!blended) return fail(GS_ERR_INVALID_ARG, "blended is required");
  GS_TRY(set_device(s));
  Counters c;
  GS_TRY(read_counters(s, (cudaStream_t)stream, c));
  *blended = (int64_t)c.blends;
  return GS_OK;
}

gs_status gs_scene_work_counts(gs_scene* s, void* stream, int64_t* blended, int64_t* evaluated) {
  g_err.clear();
  GS_TRY(check_scene(s));
  GS_TRY(set_device(s));
  Counters c;
  GS_TRY(read_counters(s, (cudaStream_t)stream, c));
  if (blended) *blended = (int64_t)c.blends;
  if (evaluated) *evaluated = (int64_t)c.evals;
  return GS_OK;
}

// ---- launch configurations and the autotuner ------------------------------

}  // extern "C"

namespace {

gs_status check_mode_cams(int mode, int n_views, const gs_camera* cams) {
  if (mode < 0 || mode >= kModeCount) return fail(GS_ERR_INVALID_ARG, "mode must be GS_MODE_FORWARD, _FEATURES or _POSE_GRAD");
  if (n_views < 1 || !cams) return fail(GS_ERR_INVALID_ARG, "n_views >= 1 and cams are required");
  for (int v = 0; v < n_views; ++v) GS_TRY(check_cam(cams[v]));
  return GS_OK;
}

std::string cams_key(int n_views, const gs_camera* cams) {
  std::vector<std::pair<int, int>> sz;
  for (int v = 0; v < n_views; ++v) sz.emplace_back(cams[v].width, cams[v].height);
  return shape_key(sz);
}

void fill_launch(const LaunchCfg& c, int mode, gs_launch* out) {
  const CompVariantInfo vi = composite_variant_info(mode, c.variant[mode]);
  out->variant = c.variant[mode];
  out->ctas_per_sm = c.per_sm[mode] > 0 && c.per_sm[mode] < vi.occupancy ? c.per_sm[mode] : vi.occupancy;
  out->grid_mult = c.grid_mult[mode];
  out->batch = vi.batch;
  out->min_blocks = vi.min_blocks;
  out->occupancy = vi.occupancy;
}

gs_status set_cfg(gs_scene* s, int mode, const std::string& key, int variant, int per_sm, int grid_mult) {
  if (variant < 0 || variant >= kCompVariants) return fail(GS_ERR_INVALID_ARG, "variant out of range");
  if (per_sm < 0 || per_sm > 64) return fail(GS_ERR_INVALID_ARG, "ctas_per_sm must be 0..64");
  if (grid_mult < 1 || grid_mult > 64) return fail(GS_ERR_INVALID_ARG, "grid_mult must be 1..64");
  LaunchCfg& c = s->launch[key];
  c.variant[mode] = variant;
  c.per_sm[mode] = per_sm;
  c.grid_mult[mode] = grid_mult;
  g_alloc_gen.fetch_add(1);  // captured graphs hold the old launch shapes
  return GS_OK;
}

}  // namespace

extern "C" {

gs_status gs_scene_set_launch(gs_scene* s, int mode, int n_views, const gs_camera* cams, const gs_launch* cfg) {
  g_err.clear();
  GS_TRY(check_scene(s));
  GS_TRY(check_mode_cams(mode, n_views, cams));
  if (!cfg) return fail(GS_ERR_INVALID_ARG, "cfg is required");
  return set_cfg(s, mode, cams_key(n_views, cams), cfg->variant, cfg->ctas_per_sm, cfg->grid_mult);
}

gs_status gs_scene_get_launch(gs_scene* s, int mode, int n_views, const gs_camera* cams, gs_launch* cfg) {
  g_err.clear();
  GS_TRY(check_scene(s));
  GS_TRY(check_mode_cams(mode, n_views, cams));
  if (!cfg) return fail(GS_ERR_INVALID_ARG, "cfg is required");
  GS_TRY(set_device(s));
  const auto it = s->launch.find(cams_key(n_views, cams));
  fill_launch(it == s->launch.end() ? LaunchCfg{} : it->second, mode, cfg);
  return GS_OK;
}

gs_status gs_autotune(gs_scene* s, int mode, int n_views, const gs_camera* cams, const gs_pose* poses, int reps,
                      gs_tune_result* result, void* stream) {
  g_err.clear();
  GS_TRY(check_scene(s));
  GS_TRY(check_mode_cams(mode, n_views, cams));
  if (!poses) return fail(GS_ERR_INVALID_ARG, "poses are required");
  for (int v = 0; v < n_views; ++v) GS_TRY(check_pose(poses[v]));
  if (mode == kModeFwdFeat && !s->feat_dim) return fail(GS_ERR_INVALID_ARG, "GS_MODE_FEATURES needs a scene with features");
  if (reps < 1) reps = 5;
  GS_TRY(set_device(s));
  const cudaStream_t st = (cudaStream_t)stream;
  const std::string key = cams_key(n_views, cams);
  // output buffers of every view (the tuner's own); the pose-gradient mode uses
  // the forward renders at the same poses as its targets
  std::vector<DevBuf> bufs((size_t)n_views);
  auto free_all = [&]() {
    cudaStreamSynchronize(st);
    for (DevBuf& b : bufs) release(b);
  };
  std::vector<gs_outputs> outs((size_t)n_views);
  for (int v = 0; v < n_views; ++v) {
    const size_t P = (size_t)cams[v].width * cams[v].height;
    const size_t nf = mode == kModeFwdFeat ? 32 : 0;
    const gs_status e = ensure(bufs[v], (6 + nf) * P * sizeof(float));
    if (e != GS_OK) {
      free_all();
      return e;
    }
    float* b = static_cast<float*>(bufs[v].p);
    outs[v] = gs_outputs{b, b + 3 * P, b + 4 * P, b + 5 * P, nf ? b + 6 * P : nullptr, nullptr};
  }
  std::vector<const float*> trgb((size_t)n_views), tdep((size_t)n_views);
  for (int v = 0; v < n_views; ++v) {
    trgb[v] = outs[v].rgb;
    tdep[v] = outs[v].depth;
  }
  GradIn g{trgb.data(), tdep.data(), nullptr, 0.1f, nullptr};
  std::vector<View> hv;
  uint64_t n_tiles = 0;
  gs_status stt = build_views(s, n_views, cams, poses, outs.data(), mode == kModeTan ? &g : nullptr, hv, n_tiles);
  if (stt != GS_OK) {
    free_all();
    return stt;
  }
  if (mode == kModeTan) {  // the targets, and a first synchronous call that sizes the workspace
    std::vector<View> hf;
    uint64_t nt = 0;
    stt = build_views(s, n_views, cams, poses, outs.data(), nullptr, hf, nt);
    if (stt == GS_OK) stt = run_sync(s, hf, nt, nullptr, st);
  }
  if (stt == GS_OK) stt = run_sync(s, hv, n_tiles, mode == kModeTan ? &g : nullptr, st);
  if (stt != GS_OK) {
    free_all();
    return stt;
  }
  const LaunchCfg saved = s->launch.count(key) ? s->launch[key] : LaunchCfg{};
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  GS_CUDA(cudaEventCreate(&e0));
  GS_CUDA(cudaEventCreate(&e1));
  std::vector<int4> ranges;
  // median device time of `reps` asynchronous calls under configuration c
  auto time_cfg = [&](const LaunchCfg& c, double& ms) -> gs_status {
    s->launch[key] = c;
    GS_TRY(prepare_call(s, hv, st, ranges));
    GS_TRY(enqueue(s, hv, ranges, n_tiles, mode == kModeTan ? &g : nullptr, st, nullptr));  // warm
    std::vector<double> t;
    for (int r = 0; r < reps; ++r) {
      GS_CUDA(cudaEventRecord(e0, st));
      GS_TRY(enqueue(s, hv, ranges, n_tiles, mode == kModeTan ? &g : nullptr, st, nullptr));
      GS_CUDA(cudaEventRecord(e1, st));
      GS_CUDA(cudaEventSynchronize(e1));
      float f = 0.f;
      GS_CUDA(cudaEventElapsedTime(&f, e0, e1));
      t.push_back(f);
    }
    Counters c2;
    GS_TRY(read_counters(s, st, c2));
    if (c2.overflow) return fail(GS_ERR_CAPACITY, "workspace overflow while tuning");
    std::sort(t.begin(), t.end());
    ms = t[t.size() / 2];
    return GS_OK;
  };
  LaunchCfg best = saved, cur = saved;
  best.variant[mode] = 0;
  best.per_sm[mode] = 0;
  best.grid_mult[mode] = 8;
  double ms_default = 0.0, ms_best = 0.0;
  int tried = 0;
  gs_status err = time_cfg(best, ms_default);
  ms_best = ms_default;
  ++tried;
  // compositor variant x persistent CTAs per SM, at the default grid multiple
  for (int v = 0; v < kCompVariants && err == GS_OK; ++v) {
    const int occ = composite_variant_info(mode, v).occupancy;
    for (int p = occ; p >= std::max(1, occ - 2) && err == GS_OK; --p) {
      if (v == 0 && p == occ) continue;  // the default, timed above
      cur = best;
      cur.variant[mode] = v;
      cur.per_sm[mode] = p == occ ? 0 : p;
      double ms = 0.0;
      err = time_cfg(cur, ms);
      ++tried;
      if (err == GS_OK && ms < ms_best) {
        ms_best = ms;
        best = cur;
      }
    }
  }
  // then the CTAs per SM of the projection, shading, scatter and sort
  for (int gm : {2, 4, 16, 32}) {
    if (err != GS_OK) break;
    cur = best;
    cur.grid_mult[mode] = gm;
    double ms = 0.0;
    err = time_cfg(cur, ms);
    ++tried;
    if (err == GS_OK && ms < ms_best) {
      ms_best = ms;
      best = cur;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  free_all();
  if (err != GS_OK) {
    s->launch[key] = saved;
    g_alloc_gen.fetch_add(1);
    return err;
  }
  s->launch[key] = best;
  g_alloc_gen.fetch_add(1);  // captured graphs hold the old launch shapes
  if (result) {
    fill_launch(best, mode, &result->best);
    result->ms_default = ms_default;
    result->ms_best = ms_best;
    result->candidates = tried;
  }
  return GS_OK;
}

gs_status gs_tune_save(const gs_scene* s, const char* path) {
  g_err.clear();
  GS_TRY(check_scene(s));
  if (!path) return fail(GS_ERR_INVALID_ARG, "path is required");
  // keep the lines of other devices and shapes, replace this device's entries for this scene's shapes
  std::vector<std::string> keep;
  if (FILE* f = std::fopen(path, "r")) {
    char line[1024];
    while (std::fgets(line, sizeof line, f)) {
      std::string l(line);
      while (!l.empty() && (l.back() == '\n' || l.back() == '\r')) l.pop_back();
      if (l.empty() || l.rfind("#", 0) == 0) continue;
      const size_t a = l.find('|'), b = l.find('|', a + 1), c = l.find('|', b + 1);
      if (a == std::string::npos || b == std::string::npos || c == std::string::npos) continue;
      const std::string dev = l.substr(0, a), key = l.substr(b + 1, c - b - 1);
      if (dev == s->device_name + "/" + std::to_string(s->sm_count) && s->launch.count(key)) continue;
      keep.push_back(l);
    }
    std::fclose(f);
  }
  FILE* f = std::fopen(path, "w");
  if (!f) return fail(GS_ERR_INVALID_ARG, std::string("cannot write ") + path);
  std::fprintf(f, "# libgsr launch configurations: device/SMs|mode|shape|variant ctas_per_sm grid_mult\n");
  for (const std::string& l : keep) std::fprintf(f, "%s\n", l.c_str());
  for (const auto& e : s->launch)
    for (int m = 0; m < kModeCount; ++m)
      std::fprintf(f, "%s/%d|%d|%s|%d %d %d\n", s->device_name.c_str(), s->sm_count, m, e.first.c_str(),
                   e.second.variant[m], e.second.per_sm[m], e.second.grid_mult[m]);
  const bool ok = std::fclose(f) == 0;
  return ok ? GS_OK : fail(GS_ERR_INVALID_ARG, std::string("cannot write ") + path);
}

gs_status gs_tune_load(gs_scene* s, const char* path, int* loaded) {
  g_err.clear();
  GS_TRY(check_scene(s));
  if (!path) return fail(GS_ERR_INVALID_ARG, "path is required");
  FILE* f = std::fopen(path, "r");
  if (!f) return fail(GS_ERR_INVALID_ARG, std::string("cannot read ") + path);
  const std::string dev = s->device_name + "/" + std::to_string(s->sm_count);
  int n = 0;
  char line[1024];
  gs_status st = GS_OK;
  while (st == GS_OK && std::fgets(line, sizeof line, f)) {
    std::string l(line);
    while (!l.empty() && (l.back() == '\n' || l.back() == '\r')) l.pop_back();
    if (l.empty() || l.rfind("#", 0) == 0) continue;
    const size_t a = l.find('|'), b = l.find('|', a + 1), c = l.find('|', b + 1);
    if (a == std::string::npos || b == std::string::npos || c == std::string::npos || l.substr(0, a) != dev) continue;
    int mode = -1, v = 0, p = 0, gm = 0;
    if (std::sscanf(l.c_str() + a + 1, "%d", &mode) != 1 || std::sscanf(l.c_str() + c + 1, "%d %d %d", &v, &p, &gm) != 3 ||
        mode < 0 || mode >= kModeCount) {
      st = fail(GS_ERR_INVALID_ARG, "malformed line in " + std::string(path) + ": " + l);
      break;
    }
    st = set_cfg(s, mode, l.substr(b + 1, c - b - 1), v, p, gm);
    n += st == GS_OK;
  }
  std::fclose(f);
  if (loaded) *loaded = n;
  return st;
}

gs_status gs_scene_status(gs_scene* s, void* stream, int64_t* needed_records, int64_t* needed_pairs) {
  g_err.clear();
  GS_TRY(check_scene(s));
  GS_TRY(set_device(s));
  Counters c;
  GS_TRY(read_counters(s, (cudaStream_t)stream, c));
  if (needed_records) *needed_records = (int64_t)records_capacity_needed(c);
  if (needed_pairs) *needed_pairs = c.pair_total;
  if (c.error) return fail(GS_ERR_INTERNAL, "device consistency check failed: the binning handed out a pair slot past the scanned tile counts");
  if (c.overflow) return fail(GS_ERR_CAPACITY, "workspace too small for the last asynchronous call");
  return GS_OK;
}

gs_status gs_get_tile_lists(gs_scene* s, int view, uint64_t* keys, uint32_t* gids, int64_t* tile_start,
                            int64_t capacity, int64_t* n_pairs, void* stream) {
  g_err.clear();
  GS_TRY(check_scene(s));
  if (view < 0 || view >= (int)s->last_views.size()) return fail(GS_ERR_INVALID_ARG, "no such view in the last call");
  if (!keys || !gids || !tile_start || !n_pairs) return fail(GS_ERR_INVALID_ARG, "output pointers required");
  GS_TRY(set_device(s));
  const cudaStream_t st = (cudaStream_t)stream;
  Counters c;
  GS_TRY(read_counters(s, st, c));
  if (c.overflow) return fail(GS_ERR_CAPACITY, "last call overflowed its workspace");
  const View& V = s->last_views[view];
  const uint32_t nt = (uint32_t)(V.tiles_x * V.tiles_y);
  std::vector<uint32_t> off(nt + 1);
  GS_CUDA(cudaMemcpy(off.data(), dp<uint32_t>(s->tile_offset) + V.tile_base, (nt + 1) * sizeof(uint32_t),
                     cudaMemcpyDeviceToHost));
  const int64_t np = (int64_t)off[nt] - off[0];
  *n_pairs = np;
  for (uint32_t t = 0; t <= nt; ++t) tile_start[t] = (int64_t)off[t] - off[0];
  if (np > capacity) return fail(GS_ERR_INVALID_ARG, "capacity too small");
  std::vector<uint2> pr((size_t)np);
  if (np) GS_CUDA(cudaMemcpy(pr.data(), dp<uint2>(s->pairs) + off[0], np * sizeof(uint2), cudaMemcpyDeviceToHost));
  const uint32_t nrec = s->rec_cap;
  std::vector<float4> rb(nrec);
  if (nrec) GS_CUDA(cudaMemcpy(rb.data(), s->rec_b.p, nrec * sizeof(float4), cudaMemcpyDeviceToHost));
  for (uint32_t t = 0; t < nt; ++t)
    for (uint32_t j = off[t] - off[0]; j < off[t + 1] - off[0]; ++j) {
      keys[j] = ((uint64_t)t << 32) | pr[j].x;
      float gf = rb[pr[j].y].w;
      int32_t gi;
      std::memcpy(&gi, &gf, 4);
      gids[j] = (uint32_t)gi;
    }
  return GS_OK;
}

gs_status gs_get_records(gs_scene* s, int view, int32_t* rec, int64_t capacity, int64_t* n_records, void* stream) {
  g_err.clear();
  GS_TRY(check_scene(s));
  if (view < 0 || view >= (int)s->last_views.size()) return fail(GS_ERR_INVALID_ARG, "no such view in the last call");
  if (!rec || !n_records) return fail(GS_ERR_INVALID_ARG, "output pointers required");
  GS_TRY(set_device(s));
  Counters c;
  GS_TRY(read_counters(s, (cudaStream_t)stream, c));
  if (c.overflow) return fail(GS_ERR_CAPACITY, "last call overflowed its workspace");
  const uint32_t nrec = s->rec_cap;
  std::vector<float4> ra(nrec), rb(nrec), rc(nrec);
  std::vector<uint4> rm(nrec);
  if (nrec) {
    GS_CUDA(cudaMemcpy(rc.data(), s->rec_c.p, nrec * sizeof(float4), cudaMemcpyDeviceToHost));
    GS_CUDA(cudaMemcpy(ra.data(), s->rec_a.p, nrec * sizeof(float4), cudaMemcpyDeviceToHost));
    GS_CUDA(cudaMemcpy(rb.data(), s->rec_b.p, nrec * sizeof(float4), cudaMemcpyDeviceToHost));
    GS_CUDA(cudaMemcpy(rm.data(), s->rec_m.p, nrec * sizeof(uint4), cudaMemcpyDeviceToHost));
  }
  int64_t k = 0;
  for (const uint32_t r : filled_records(c, s->rec_cap)) {
    if ((int)rm[r].z != view) continue;
    if (k < capacity) {
      int32_t* o = rec + 10 * k;
      std::memcpy(&o[0], &rb[r].w, 4);
      o[1] = (int32_t)(rm[r].x & 0xffff);
      o[2] = (int32_t)(rm[r].x >> 16);
      o[3] = (int32_t)(rm[r].y & 0xffff);
      o[4] = (int32_t)(rm[r].y >> 16);
      o[5] = (int32_t)rm[r].w;
      uint32_t lo2;
      std::memcpy(&lo2, &rc[r].w, 4);
      const float ulo = half_bits_to_float((uint16_t)(lo2 & 0xffff)), vlo = half_bits_to_float((uint16_t)(lo2 >> 16));
      std::memcpy(&o[6], &ra[r].x, 4);
      std::memcpy(&o[7], &ulo, 4);
      std::memcpy(&o[8], &ra[r].y, 4);
      std::memcpy(&o[9], &vlo, 4);
    }
    ++k;
  }
  *n_records = k;
  if (k > capacity) return fail(GS_ERR_INVALID_ARG, "capacity too small");
  return GS_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Pose refinement with the Adam step on the device. After a first synchronous
// iteration (which sizes the workspace), every iteration is the pose-gradient
// launch sequence followed by one small kernel that takes the Adam step from
// the gradient in the result buffer, applies T <- Exp(-step) T in fp64 and
// rewrites the view's pose fields in the device call table. One iteration is
// captured as a CUDA graph and replayed, so the host enqueues all iterations
// without waiting for any of them.
// ---------------------------------------------------------------------------
namespace {

struct RefineState {
  double T[16];
  double m[6], v[6];
  double b1t, b2t;  // beta1^t, beta2^t after t iterations
  int it;           // iterations taken
  int pad;
};

// One warp per view: lanes 0-5 take the Adam step of one tangent coordinate,
// lanes 0-11 one entry of the updated 3x4 pose and of the view's pose fields.
// sticky: bits 0-2 the overflow bits of a call, bit 8 a device consistency failure.
__global__ void __launch_bounds__(128) k_refine_update(View* __restrict__ views, int nv,
                                                       const double* __restrict__ result,
                                                       RefineState* __restrict__ rs, gs_refine_opts o, int iters,
                                                       double* __restrict__ hist,
                                                       const Counters* __restrict__ ctr,
                                                       unsigned int* __restrict__ sticky) {
  const int v = blockIdx.x * 4 + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (v >= nv) return;
  const unsigned int bad = ctr->overflow | (ctr->error ? 0x100u : 0u);
  if (bad) {  // this iteration's render is incomplete: stop updating
    if (lane == 0) atomicOr(sticky, bad);
    return;
  }
  if (*sticky) return;
  RefineState& S = rs[v];
  const int it = S.it;
  if (it >= iters) return;
  const double* r = result + (size_t)v * kResultStride;
  if (hist && lane == 0) hist[(size_t)v * iters + it] = r[0];
  const double b1t = S.b1t * o.beta1, b2t = S.b2t * o.beta2;
  double xi = 0.0;  // this lane's coordinate of -step
  if (lane < 6) {
    const double g = r[1 + lane];
    const double m = o.beta1 * S.m[lane] + (1.0 - o.beta1) * g;
    const double vv = o.beta2 * S.v[lane] + (1.0 - o.beta2) * g * g;
    S.m[lane] = m;
    S.v[lane] = vv;
    const double lr = lane < 3 ? o.lr_trans : o.lr_rot;
    xi = -(lr * (m / (1.0 - b1t)) / (sqrt(vv / (1.0 - b2t)) + o.eps));
  }
  double x[6];
  for (int k = 0; k < 6; ++k) x[k] = __shfl_sync(0xffffffffu, xi, k);
  // Exp of the twist (rho, phi) = x: R = I + a K + b K^2, V = I + b K + c K^2
  const double* w = x + 3;
  const double t2 = w[0] * w[0] + w[1] * w[1] + w[2] * w[2];
  const double t = sqrt(t2);
  double a, b, c;
  if (t < 1e-6) {  // series of sin t / t, (1 - cos t) / t^2, (t - sin t) / t^3
    a = 1.0 - t2 / 6.0;
    b = 0.5 - t2 / 24.0;
    c = 1.0 / 6.0 - t2 / 120.0;
  } else {
    double sn, cs;
    sincos(t, &sn, &cs);
    const double it2 = 1.0 / t2;
    a = sn / t;
    b = (1.0 - cs) * it2;
    c = (t - sn) * it2 / t;
  }
  double out = 0.0;
  const int i = lane >> 2, j = lane & 3;  // lanes 0-11: entry (i, j) of the new 3x4 pose
  if (lane < 12) {
    // row i of K = [phi]x and of K^2 = phi phi^T - |phi|^2 I
    const double kr[3] = {i == 0 ? 0.0 : (i == 1 ? w[2] : -w[1]), i == 0 ? -w[2] : (i == 1 ? 0.0 : w[0]),
                          i == 0 ? w[1] : (i == 1 ? -w[0] : 0.0)};
    const double wi = i == 0 ? w[0] : (i == 1 ? w[1] : w[2]);
    double e[4];  // row i of Exp
    double tv = 0.0;
    for (int q = 0; q < 3; ++q) {
      const double id = (i == q) ? 1.0 : 0.0;
      const double k2 = wi * w[q] - id * t2;
      e[q] = id + a * kr[q] + b * k2;
      tv += (id + b * kr[q] + c * k2) * x[q];
    }
    e[3] = tv;
    out = e[0] * S.T[j] + e[1] * S.T[4 + j] + e[2] * S.T[8 + j] + e[3] * S.T[12 + j];
  }
  __syncwarp();
  if (lane < 12) S.T[4 * i + j] = out;
  if (lane == 0) {
    S.b1t = b1t;
    S.b2t = b2t;
    S.it = it + 1;
  }
  // the view's pose fields, split as the host splits them (rounded products and sums)
  View& V = views[v];
  if (lane < 12) {
    const float hi = (float)out, lo = (float)(out - (double)hi);
    if (j < 3) {
      V.R[3 * i + j] = hi;
      V.Rl[3 * i + j] = lo;
    } else {
      V.t[i] = hi;
      V.tl[i] = lo;
    }
  }
  const int l3 = lane < 3 ? lane : 0;  // column l3 of R against the translation
  const double r0 = __shfl_sync(0xffffffffu, out, l3), r1 = __shfl_sync(0xffffffffu, out, 4 + l3);
  const double r2 = __shfl_sync(0xffffffffu, out, 8 + l3);
  const double t0 = __shfl_sync(0xffffffffu, out, 3), t1 = __shfl_sync(0xffffffffu, out, 7);
  const double tz = __shfl_sync(0xffffffffu, out, 11);
  if (lane < 3) V.cw[lane] = (float)(-__dadd_rn(__dadd_rn(__dmul_rn(r0, t0), __dmul_rn(r1, t1)), __dmul_rn(r2, tz)));
}

}  // namespace

namespace gsr {

gs_status refine_on_device(gs_scene* s, int nv, const gs_camera* cams, gs_pose* poses,
                           const float* const* target_rgb, const float* const* target_depth,
                           const float* const* pixel_weight, const gs_refine_opts* o, double* loss_history,
                           cudaStream_t st, bool* used) {
  *used = false;
  if (s->streaming || s->parts.size() != 1) return GS_OK;  // partitions culled per pose: the host loop
  *used = true;
  if (o->iterations == 0) return GS_OK;
  GS_TRY(set_device(s));
  for (int v = 0; v < nv; ++v) GS_TRY(check_grad_args(target_rgb[v], target_depth[v], o->depth_weight));
  GradIn g{target_rgb, target_depth, pixel_weight, o->depth_weight, nullptr};
  const int iters = o->iterations;
  std::vector<RefineState> h0(nv);
  for (int v = 0; v < nv; ++v) {
    std::memcpy(h0[v].T, poses[v].T_cw, sizeof(h0[v].T));
    std::fill(h0[v].m, h0[v].m + 6, 0.0);
    std::fill(h0[v].v, h0[v].v + 6, 0.0);
    h0[v].b1t = 1.0;
    h0[v].b2t = 1.0;
    h0[v].it = 0;
    h0[v].pad = 0;
  }
  RefineState* drs = nullptr;
  double* dhist = nullptr;
  unsigned int* dsticky = nullptr;
  cudaStream_t cap = nullptr;
  cudaGraphExec_t exec = nullptr;
  auto cleanup = [&]() {
    if (exec) cudaGraphExecDestroy(exec);
    if (cap) cudaStreamDestroy(cap);
    if (drs) cudaFree(drs);
    if (dhist) cudaFree(dhist);
    if (dsticky) cudaFree(dsticky);
  };
  if (cudaMalloc(&drs, nv * sizeof(RefineState)) != cudaSuccess ||
      (loss_history && cudaMalloc(&dhist, (size_t)nv * iters * sizeof(double)) != cudaSuccess) ||
      cudaMalloc(&dsticky, sizeof(unsigned int)) != cudaSuccess) {
    cudaGetLastError();
    cleanup();
    return fail(GS_ERR_OOM, "refinement state allocation failed");
  }
  const int blocks = (nv + 3) / 4;
  gs_status status = GS_OK;
  auto launch_update = [&](cudaStream_t on) -> gs_status {
    View* dviews = reinterpret_cast<View*>(static_cast<char*>(s->views.p) + table_ranges_bytes(s));
    k_refine_update<<<blocks, 128, 0, on>>>(dviews, nv, dp<double>(s->result), drs, *o, iters, dhist,
                                            dp<Counters>(s->ctr), dsticky);
    GS_CUDA(cudaGetLastError());
    return GS_OK;
  };
  for (int attempt = 0;; ++attempt) {
    if (exec) cudaGraphExecDestroy(exec);
    exec = nullptr;
    std::vector<View> hv;
    uint64_t n_tiles;
    status = build_views(s, nv, cams, poses, nullptr, &g, hv, n_tiles);
    if (status != GS_OK) break;
    // iteration 0 synchronously: sizes the workspace and fills the device call table
    status = run_sync(s, hv, n_tiles, &g, st);
    if (status != GS_OK) break;
    {  // headroom for the records and pairs of the poses to come
      const Counters c = *s->ctr_host;
      const uint64_t need = records_capacity_needed(c);
      status = grow_records(s, need + need / 2 + 1024, true);
      if (status == GS_OK) status = grow_pairs(s, (uint64_t)c.pair_total + c.pair_total / 2 + 4096);
      if (status != GS_OK) break;
    }
    std::vector<int4> ranges;
    status = prepare_call(s, hv, st, ranges);
    if (status != GS_OK) break;
    if (cudaMemcpyAsync(drs, h0.data(), nv * sizeof(RefineState), cudaMemcpyHostToDevice, st) != cudaSuccess ||
        cudaMemsetAsync(dsticky, 0, sizeof(unsigned int), st) != cudaSuccess) {
      status = fail(GS_ERR_CUDA, "refinement state upload failed");
      break;
    }
    status = launch_update(st);
    if (status != GS_OK) break;
    if (iters > 1 && !s->timing) {
      // one iteration as a graph (kernel timing needs the eager path's events)
      if (!cap && cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking) != cudaSuccess) {
        status = fail(GS_ERR_CUDA, "capture stream creation failed");
        break;
      }
      cudaGraph_t graph = nullptr;
      if (cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
        status = fail(GS_ERR_CUDA, "cudaStreamBeginCapture failed");
        break;
      }
      gs_status est = enqueue(s, hv, ranges, n_tiles, &g, cap, nullptr, nullptr, nullptr, nullptr, true, nullptr,
                              true);
      if (est == GS_OK) est = launch_update(cap);
      const cudaError_t ce = cudaStreamEndCapture(cap, &graph);
      if (est == GS_OK && ce != cudaSuccess)
        est = fail(GS_ERR_CUDA, std::string("cudaStreamEndCapture: ") + cudaGetErrorString(ce));
      if (est == GS_OK) {
        const cudaError_t ie = cudaGraphInstantiate(&exec, graph, 0);
        if (ie != cudaSuccess) est = fail(GS_ERR_CUDA, std::string("cudaGraphInstantiate: ") + cudaGetErrorString(ie));
      }
      if (graph) cudaGraphDestroy(graph);
      status = est;
      for (int it = 1; it < iters && status == GS_OK; ++it) {
        const cudaError_t le = cudaGraphLaunch(exec, st);
        if (le != cudaSuccess) status = fail(GS_ERR_CUDA, std::string("cudaGraphLaunch: ") + cudaGetErrorString(le));
      }
    } else {
      for (int it = 1; it < iters && status == GS_OK; ++it) {
        status = enqueue(s, hv, ranges, n_tiles, &g, st, nullptr, nullptr, nullptr, nullptr, false, nullptr, true);
        if (status == GS_OK) status = launch_update(st);
      }
    }
    if (status != GS_OK) break;
    unsigned int sticky = 0;
    std::vector<RefineState> h1(nv);
    if (cudaMemcpyAsync(&sticky, dsticky, sizeof(sticky), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaMemcpyAsync(h1.data(), drs, nv * sizeof(RefineState), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        (loss_history && cudaMemcpyAsync(loss_history, dhist, (size_t)nv * iters * sizeof(double),
                                         cudaMemcpyDeviceToHost, st) != cudaSuccess) ||
        cudaStreamSynchronize(st) != cudaSuccess) {
      status = fail(GS_ERR_CUDA, "refinement read-back failed");
      break;
    }
    if (sticky & 0x100u) {
      status = fail(GS_ERR_INTERNAL, "device consistency check failed: the binning handed out a pair slot past the scanned tile counts");
      break;
    }
    if (sticky & 4u) {
      status = fail(GS_ERR_CAPACITY, "more than 2^32 (tile, Gaussian) pairs in one call");
      break;
    }
    if (sticky) {  // a later pose outgrew the workspace: double it and start again
      if (attempt == 3) {
        status = fail(GS_ERR_CAPACITY, "refinement workspace did not converge");
        break;
      }
      status = grow_records(s, (uint64_t)s->rec_cap * 2, true);
      if (status == GS_OK) status = grow_pairs(s, (uint64_t)s->pair_cap * 2);
      if (status != GS_OK) break;
      continue;
    }
    for (int v = 0; v < nv; ++v) std::memcpy(poses[v].T_cw, h1[v].T, sizeof(poses[v].T_cw));
    break;
  }
  if (status != GS_OK) cudaStreamSynchronize(st);  // nothing of this call may still use its state
  cleanup();
  return status;
}

}  // namespace gsr
