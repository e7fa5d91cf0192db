// gs_render_noalloc: the forward render of gs_render with every piece of
// working memory taken from one fixed, file-scope device array instead of
// cudaMalloc. The paper has no counterpart; it exists for callers that must
// not allocate device memory at call time (see include/gsr.h).
//
// The array below is reserved in every GPU's memory as soon as the library is
// loaded there, and stays reserved until the process exits. Its host-side
// name is only a stand-in: host code obtains the device address with
// cudaGetSymbolAddress, once per device, the first time the entry point runs
// on that device.
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>
#include <mutex>
#include <string>

#include "gsr.h"
#include "gsr_internal.h"

static __device__ __align__(256) unsigned char gs_noalloc_scratch[GS_NOALLOC_SCRATCH_BYTES];

namespace gsr {
void set_last_error(const std::string& msg);
}

namespace {

using namespace gsr;

constexpr size_t kMaxDevices = 64;
std::mutex g_setup_mu;
unsigned char* g_scratch_addr[kMaxDevices] = {};

constexpr size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

// projection blocks of 256 Gaussians: one per block at the Gaussian limit
constexpr int kProjBlocks = GS_NOALLOC_MAX_GAUSSIANS / 256;
static_assert(GS_NOALLOC_MAX_GAUSSIANS % (256 * kRecRegions) == 0, "two projection blocks per record segment");

// Byte offsets of each buffer inside the scratch array, for the stated limits.
struct Layout {
  static constexpr size_t G = GS_NOALLOC_MAX_GAUSSIANS;
  static constexpr size_t P = GS_NOALLOC_MAX_PAIRS;
  static constexpr size_t TL = GS_NOALLOC_MAX_TILES + 1;
  static constexpr size_t pos = 0;
  static constexpr size_t cov = align256(pos + G * sizeof(float4));
  static constexpr size_t sh = align256(cov + 2 * G * sizeof(float4));
  static constexpr size_t feat = align256(sh + 12 * G * sizeof(float4));
  static constexpr size_t rec_a = align256(feat + 4 * G * sizeof(uint4));
  static constexpr size_t rec_b = align256(rec_a + G * sizeof(float4));
  static constexpr size_t rec_c = align256(rec_b + G * sizeof(float4));
  static constexpr size_t rec_m = align256(rec_c + G * sizeof(float4));
  static constexpr size_t tcount = align256(rec_m + G * sizeof(uint4));
  static constexpr size_t toffset = align256(tcount + TL * sizeof(uint32_t));
  static constexpr size_t tcursor = align256(toffset + TL * sizeof(uint32_t));
  static constexpr size_t pairs = align256(tcursor + TL * sizeof(uint32_t));
  static constexpr size_t pairs_tmp = align256(pairs + P * sizeof(uint2));
  static constexpr size_t ctr = align256(pairs_tmp + P * sizeof(uint2));
  static constexpr size_t view = align256(ctr + sizeof(Counters));
  static constexpr size_t ranges = align256(view + sizeof(View));
  static constexpr size_t end = align256(ranges + 2 * sizeof(int4));
};
static_assert(Layout::end <= GS_NOALLOC_SCRATCH_BYTES, "no-alloc limits do not fit the scratch array");

gs_status nfail(gs_status st, const std::string& msg) {
  set_last_error(msg);
  return st;
}

#define NA_CUDA(x)                                                                                   \
  do {                                                                                               \
    const cudaError_t e_ = (x);                                                                      \
    if (e_ != cudaSuccess) return nfail(GS_ERR_CUDA, std::string(#x) + ": " + cudaGetErrorString(e_)); \
  } while (0)

// Device address of the scratch array on the current device (set up once).
gs_status scratch_on_device(int dev, unsigned char** out) {
  if (dev < 0 || (size_t)dev >= kMaxDevices) return nfail(GS_ERR_INVALID_ARG, "device ordinal out of range");
  std::lock_guard<std::mutex> lk(g_setup_mu);
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, gs_noalloc_scratch);
    if (e != cudaSuccess || !p)
      return nfail(GS_ERR_CUDA, std::string("cudaGetSymbolAddress(scratch): ") + cudaGetErrorString(e));
    g_scratch_addr[dev] = static_cast<unsigned char*>(p);
  }
  *out = g_scratch_addr[dev];
  return GS_OK;
}

}  // namespace

extern "C" gs_status gs_render_noalloc(const gs_scene_desc* d, const gs_camera* cam, const gs_pose* pose,
                                       const gs_outputs* out, void* stream) {
  set_last_error("");
  if (!d || !cam || !pose) return nfail(GS_ERR_INVALID_ARG, "desc, cam and pose are required");
  if (!d->device_resident) return nfail(GS_ERR_INVALID_ARG, "gs_render_noalloc needs device-resident scene arrays");
  if (d->n < 0 || d->n > GS_NOALLOC_MAX_GAUSSIANS)
    return nfail(GS_ERR_INVALID_ARG, "n = " + std::to_string(d->n) + " exceeds the no-alloc limit of " +
                                         std::to_string(GS_NOALLOC_MAX_GAUSSIANS) + " Gaussians");
  if (d->sh_degree < 0 || d->sh_degree > 3) return nfail(GS_ERR_INVALID_ARG, "sh_degree must be 0..3");
  if (d->feat_dim != 0 && d->feat_dim != 32) return nfail(GS_ERR_INVALID_ARG, "feat_dim must be 0 or 32");
  if (d->n > 0 && (!d->means || !d->scales || !d->quats || !d->opacities || !d->sh || (d->feat_dim && !d->feats_bf16)))
    return nfail(GS_ERR_INVALID_ARG, "scene arrays are required when n > 0");
  if (cam->width < 1 || cam->height < 1 || !(std::isfinite(cam->fx) && cam->fx > 0.f) ||
      !(std::isfinite(cam->fy) && cam->fy > 0.f) || !std::isfinite(cam->cx) || !std::isfinite(cam->cy))
    return nfail(GS_ERR_INVALID_ARG, "camera size or intrinsics out of range");
  for (int k = 0; k < 16; ++k)
    if (!std::isfinite(pose->T_cw[k])) return nfail(GS_ERR_INVALID_ARG, "pose has a non-finite entry");
  const int tiles_x = (cam->width + kTile - 1) / kTile, tiles_y = (cam->height + kTile - 1) / kTile;
  const long long n_tiles = (long long)tiles_x * tiles_y;
  if (n_tiles > GS_NOALLOC_MAX_TILES)
    return nfail(GS_ERR_INVALID_ARG, "image needs " + std::to_string(n_tiles) + " tiles; the no-alloc limit is " +
                                         std::to_string(GS_NOALLOC_MAX_TILES));
  int dev = 0;
  NA_CUDA(cudaGetDevice(&dev));
  unsigned char* base = nullptr;
  const gs_status ss = scratch_on_device(dev, &base);
  if (ss != GS_OK) return ss;
  int sm_count = 1;
  NA_CUDA(cudaDeviceGetAttribute(&sm_count, cudaDevAttrMultiProcessorCount, dev));
  const cudaStream_t st = (cudaStream_t)stream;
  const int n = (int)d->n;
  const int K3 = 3 * (d->sh_degree + 1) * (d->sh_degree + 1);
  const int nsh4 = (K3 + 3) / 4;

  // per-view parameters, built exactly as for gs_render
  View V;
  std::memset(&V, 0, sizeof(V));
  const double* T = pose->T_cw;
  for (int a = 0; a < 3; ++a) {
    for (int b = 0; b < 3; ++b) {
      V.R[3 * a + b] = (float)T[4 * a + b];
      V.Rl[3 * a + b] = (float)(T[4 * a + b] - (double)V.R[3 * a + b]);
    }
    V.t[a] = (float)T[4 * a + 3];
    V.tl[a] = (float)(T[4 * a + 3] - (double)V.t[a]);
    V.cw[a] = (float)(-(T[a] * T[3] + T[4 + a] * T[7] + T[8 + a] * T[11]));
  }
  V.fx = cam->fx;
  V.fy = cam->fy;
  V.cx = cam->cx;
  V.cy = cam->cy;
  const float hw = 0.5f * (float)cam->width, hh = 0.5f * (float)cam->height;
  const float qx = hw / cam->fx, qy = hh / cam->fy;
  V.limx = 1.3f * qx;
  V.limy = 1.3f * qy;
  V.jb2 = cam->fx * cam->fx * (1.0f + V.limx * V.limx) + cam->fy * cam->fy * (1.0f + V.limy * V.limy);
  V.width = cam->width;
  V.height = cam->height;
  V.tiles_x = tiles_x;
  V.tiles_y = tiles_y;
  V.tile_base = 0;
  if (out) {
    V.rgb = out->rgb;
    V.depth = out->depth;
    V.alpha = out->alpha;
    V.final_T = out->final_T;
    V.feats = d->feat_dim ? out->feats : nullptr;
    V.last_idx = out->last_idx;
  }

  float4* pos = reinterpret_cast<float4*>(base + Layout::pos);
  float4* cov = reinterpret_cast<float4*>(base + Layout::cov);
  float4* sh = reinterpret_cast<float4*>(base + Layout::sh);
  uint4* feat = reinterpret_cast<uint4*>(base + Layout::feat);
  View* dview = reinterpret_cast<View*>(base + Layout::view);
  Work w{};  // zero, except the members with defaults (the whole tile space)
  w.rec_a = reinterpret_cast<float4*>(base + Layout::rec_a);
  w.rec_b = reinterpret_cast<float4*>(base + Layout::rec_b);
  w.rec_c = reinterpret_cast<float4*>(base + Layout::rec_c);
  w.rec_m = reinterpret_cast<uint4*>(base + Layout::rec_m);
  w.rec_j = nullptr;
  w.rec_cap = GS_NOALLOC_MAX_GAUSSIANS;
  // Segment b % 64 receives the records of projection block b. The projection
  // below always runs kProjBlocks = 32768 / 256 = 128 blocks, one per 256
  // Gaussians whatever the SM count, so a segment takes the records of two
  // blocks, at most 2 x 256 = 512 = rec_cap / 64, and cannot overflow.
  w.rec_seg = GS_NOALLOC_MAX_GAUSSIANS / kRecRegions;
  w.tile_count = reinterpret_cast<uint32_t*>(base + Layout::tcount);
  w.tile_offset = reinterpret_cast<uint32_t*>(base + Layout::toffset);
  w.tile_cursor = reinterpret_cast<uint32_t*>(base + Layout::tcursor);
  w.n_tiles = (uint32_t)n_tiles;
  w.pairs = reinterpret_cast<uint2*>(base + Layout::pairs);
  w.pairs_tmp = reinterpret_cast<uint2*>(base + Layout::pairs_tmp);
  w.pair_cap = GS_NOALLOC_MAX_PAIRS;
  w.ctr = reinterpret_cast<Counters*>(base + Layout::ctr);
  int4* dranges = reinterpret_cast<int4*>(base + Layout::ranges);
  w.ranges = dranges;
  const int4 hranges[2] = {make_int4(1, n, 0, 0), make_int4(0, n, 0, 0)};  // one range: every Gaussian

  SceneDev sc;
  sc.pos = pos;
  sc.cov = cov;
  sc.sh = sh;
  sc.feat = d->feat_dim ? feat : nullptr;
  sc.n = n;
  sc.sh_degree = d->sh_degree;
  sc.nsh4 = nsh4;
  sc.feat_dim = d->feat_dim;

  // the scratch keeps the previous call's contents: reset what must start at zero
  NA_CUDA(cudaMemsetAsync(w.tile_count, 0, (n_tiles + 1) * sizeof(uint32_t), st));
  NA_CUDA(cudaMemsetAsync(w.ctr, 0, sizeof(Counters), st));
  NA_CUDA(cudaMemcpyAsync(dview, &V, sizeof(View), cudaMemcpyHostToDevice, st));
  NA_CUDA(cudaMemcpyAsync(dranges, hranges, sizeof(hranges), cudaMemcpyHostToDevice, st));
  NA_CUDA(launch_pack_scene(d->means, d->scales, d->quats, d->opacities, d->sh, K3, d->feats_bf16, d->feat_dim, n,
                            nsh4, pos, cov, sh, d->feat_dim ? feat : nullptr, st));
  NA_CUDA(launch_project(sc, dview, 1, w, kProjBlocks, st));
  NA_CUDA(launch_shade(sc, dview, w, false, sm_count * 8, st));
  NA_CUDA(launch_scan_tiles(w, st));
  NA_CUDA(launch_scatter(dview, w, sm_count * 8, st));
  NA_CUDA(launch_sort_tiles(w, sm_count * 8, st));
  const bool feats = d->feat_dim && out && out->feats;
  NA_CUDA(launch_composite(sc, dview, 1, w, feats, LaunchCfg{}, sm_count, st));
  Counters c;
  NA_CUDA(cudaMemcpyAsync(&c, w.ctr, sizeof(Counters), cudaMemcpyDeviceToHost, st));
  NA_CUDA(cudaStreamSynchronize(st));
  if (c.overflow & 1u)  // cannot happen with the fixed projection grid; reported apart from the pairs
    return nfail(GS_ERR_INTERNAL, "a record segment overflowed in the no-alloc render");
  if (c.overflow)
    return nfail(GS_ERR_CAPACITY, "the view needs " + std::to_string(c.pair_total) +
                                      " (tile, Gaussian) pairs; the no-alloc limit is " +
                                      std::to_string(GS_NOALLOC_MAX_PAIRS));
  return GS_OK;
}
