// Internal declarations of libgsr: device layout, per-view parameters and the
// kernel launchers shared by the translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "gsr.h"

namespace gsr {

constexpr int kTile = 16;          // tile edge in pixels
constexpr int kTileThreads = 256;  // one thread per pixel of a tile
constexpr int kSortCap = 2048;     // (tile, Gaussian) pairs a tile sorts in shared memory
constexpr int kJacStride = 48;     // floats per record of the pose Jacobian (45 used)
constexpr int kPartialStride = 8;  // doubles per tile partial (loss + 6 grad + pad)
constexpr int kChunkTiles = 64;    // tiles per first-level chunk of the fp64 pose reduction
constexpr int kWarpSortMax = 256;  // longest tile list sorted by one warp (registers)
constexpr int kVisAcc = 8;         // floats per record of the visibility check's accumulator
constexpr int kVisBlock = 2048;    // Gaussians per block of the visibility compaction
constexpr int kRecRegions = 64;    // record-allocation counters (block index mod 64)
constexpr int kMaxBands = 8;       // tile-row bands of a tangent pass that overlaps its target upload

// Per-view parameters (device copy built on the host for every call).
struct View {
  float R[9];           // world-to-camera rotation (binary32, row-major)
  float t[3];           // world-to-camera translation
  float Rl[9];          // R - double(R): low parts for the float-float centre
  float tl[3];          // t - double(t)
  float fx, fy, cx, cy;
  float limx, limy;     // 1.3 x half field of view, in normalised coordinates
  float cw[3];          // camera centre in world coordinates
  float jb2;            // fx^2 (1 + limx^2) + fy^2 (1 + limy^2): bound on z^2 |J|_F^2
  int width, height, tiles_x, tiles_y;
  uint32_t tile_base;   // first global tile index of this view
  uint32_t chunk_base;  // first reduction chunk (kChunkTiles tiles) of this view
  float* rgb;           // outputs (device; NULL = not written)
  float* depth;
  float* alpha;
  float* final_T;
  float* feats;
  uint32_t* last_idx;
  const float* target_rgb;   // loss inputs (pose gradient only)
  const float* target_depth;
  const float* pixel_weight;
  float depth_weight;
  float inv_3p;         // 1 / (3 W H)
  float inv_p;          // 1 / (W H)
  float pad1;
};

// Device counters and status of one call (zeroed at its start).
// Records live in kRecRegions equal segments of the record arrays; block b of
// the projection appends to segment b % kRecRegions, so no single counter
// serialises the whole grid. rec_region[k] may exceed the segment size (then
// the overflow bit is set and the count tells the host how much to grow).
struct Counters {
  unsigned int rec_region[kRecRegions];  // records requested per segment
  unsigned int pair_total;  // pairs requested by the binning
  unsigned int overflow;    // bit 0: records, bit 1: pairs, bit 2: pair count >= 2^32
  unsigned int fwd_queue;   // persistent tile queue of the forward render
  unsigned int tan_queue;   // persistent tile queue of the tangent (pose-gradient) render
  unsigned int error;       // device-side consistency failure
  unsigned int vis_count;   // Gaussians the visibility check keeps (M = M^r and M^i)
  unsigned long long blends;  // (pixel, Gaussian) pairs blended by the tangent or visibility reverse pass
  unsigned long long evals;   // list entries the tangent pass's pixels examined before their stop, or
                              // (pixel, Gaussian) pairs the visibility reverse pass evaluated
  unsigned int band_queue[kMaxBands];  // tile queues of a tangent pass launched in bands of tile rows
};

// Scene arena (device pointers).
struct SceneDev {
  const float4* pos;   // n: (x, y, z, max scale)
  const float4* cov;   // 2n: (S00, S01, S02, S11), (S12, S22, opacity, 0)
  const float4* sh;    // n * nsh4: SH coefficients, coefficient-major, padded to float4
  const uint4* feat;   // n * 4: 32 bfloat16 features, or NULL
  int n;
  int sh_degree;
  int nsh4;
  int feat_dim;
};

// Per-call workspace (device pointers and capacities).
struct Work {
  float4* rec_a;       // (u, v high parts, conic A, conic B)
  float4* rec_b;       // (conic C, opacity, depth z, Gaussian index bits)
  float4* rec_c;       // (r, g, b, half2 low parts of u and v)
  uint4* rec_m;        // (x0 | x1 << 16, y0 | y1 << 16, view, depth bits)
  float* rec_j;        // kJacStride floats per record (pose gradient only)
  uint32_t rec_cap;    // multiple of kRecRegions
  uint32_t rec_seg;    // rec_cap / kRecRegions
  uint32_t* tile_count;   // n_tiles + 1
  uint32_t* tile_offset;  // n_tiles + 1 (exclusive scan)
  uint32_t* tile_cursor;  // n_tiles
  uint32_t n_tiles;
  uint2* pairs;        // (depth bits, record index), sorted per tile by the compositor
  uint2* pairs_tmp;    // scratch for tiles longer than kSortCap
  uint32_t pair_cap;
  Counters* ctr;
  double* partials;    // n_tiles * kPartialStride
  double* chunk_part;  // n_chunks * kPartialStride: fp64 sums of kChunkTiles tile partials
  uint32_t* view_ctr;  // n_views: chunks of the view summed (zeroed by the scan)
  uint32_t n_chunks;
  uint32_t n_views;
  double* result;      // 7 doubles (loss, grad)
  // Gaussian index ranges the projection walks (partitions in view):
  // ranges[0] = (count, total length, 0, 0), ranges[1 + k] = (begin, end, prefix, 0)
  const int4* ranges;
  // tiles [tile_begin, tile_end) of the tangent pass taken from *queue (NULL:
  // the whole tile space from the counters' own queue)
  uint32_t tile_begin = 0;
  uint32_t tile_end = 0xffffffffu;
  unsigned int* queue = nullptr;
};

// Compositor modes and their variants (staging batch x resident-CTA bound);
// variant 0 of each mode is the default, the autotuner may pick another.
enum { kModeFwd = 0, kModeFwdFeat = 1, kModeTan = 2, kModeCount = 3 };
constexpr int kCompVariants = 4;
struct CompVariantInfo {
  int batch;       // Gaussians staged per batch
  int min_blocks;  // resident CTAs per SM its registers allow for
  int occupancy;   // resident CTAs per SM on this device (registers and shared memory)
};
CompVariantInfo composite_variant_info(int mode, int variant);

// Launch configuration of one call shape: per compositor mode, the variant,
// the persistent CTAs per SM (0: the variant's occupancy) and the CTAs per SM
// of the projection, shading, scatter and sort kernels.
struct LaunchCfg {
  int variant[kModeCount] = {0, 0, 0};
  int per_sm[kModeCount] = {0, 0, 0};
  int grid_mult[kModeCount] = {8, 8, 8};
};

// launchers (return the CUDA error of the launch)
cudaError_t launch_pack_scene(const float* means, const float* scales, const float* quats,
                              const float* opacities, const float* sh, int sh_k3, const uint16_t* feats,
                              int feat_dim, int n, int nsh4, float4* pos, float4* cov, float4* sh_out,
                              uint4* feat_out, cudaStream_t st);
cudaError_t launch_project(const SceneDev& sc, const View* views, int n_views, const Work& w, int grid,
                           cudaStream_t st);
cudaError_t launch_shade(const SceneDev& sc, const View* views, const Work& w, bool grad, int grid,
                         cudaStream_t st);
cudaError_t launch_scan_tiles(const Work& w, cudaStream_t st);
cudaError_t launch_sort_tiles(const Work& w, int grid, cudaStream_t st);
cudaError_t launch_scatter(const View* views, const Work& w, int grid, cudaStream_t st);
// feats: some view writes the feature map (else the feature-free kernel runs);
// persistent grid from cfg and the SM count
cudaError_t launch_composite(const SceneDev& sc, const View* views, int n_views, const Work& w, bool feats,
                             const LaunchCfg& cfg, int sm_count, cudaStream_t st);
// forward render plus the pose gradient (tangent mode): per-tile fp32 partials
// of (loss, dL/drho, dL/dphi) in w.partials; launch_reduce_tangent then sums
// them in fixed order into result (kPartialStride doubles per view)
cudaError_t launch_composite_tangent(const SceneDev& sc, const View* views, int n_views, const Work& w,
                                     double* result, const LaunchCfg& cfg, int sm_count, cudaStream_t st);
// the same pass over tiles [tile_begin, tile_end) with its own queue counter
cudaError_t launch_composite_tangent_range(const SceneDev& sc, const View* views, int n_views, const Work& w,
                                           double* result, const LaunchCfg& cfg, int sm_count, cudaStream_t st,
                                           uint32_t tile_begin, uint32_t tile_end, unsigned int* queue);
// the fp64 chunk and view sums of the tangent pass's tile partials, once every
// tile of the call is done
cudaError_t launch_reduce_tangent(const View* views, int n_views, const Work& w, double* result, cudaStream_t st);

// Algorithm 1 visibility check, after a forward render of one view that wrote
// final_T and last_idx and a shading pass that wrote the pose Jacobian:
// reverse pass into acc (kVisAcc floats per record, zeroed by the caller);
// persistent grid of the resident blocks on sm_count SMs
cudaError_t launch_vis_backward(const View* views, int n_views, const Work& w, float* acc, int sm_count,
                                cudaStream_t st);
// every Gaussian: projected centre (U, V) and M^i (mask bit 2); zeroes grad
cudaError_t launch_vis_inimage(const SceneDev& sc, const View* views, uint8_t* mask, float2* uv, float* grad,
                               int grid, cudaStream_t st);
// every record: mean gradient of sum RGB, M^r (bit 1), M (bit 0), count
cudaError_t launch_vis_chain(const View* views, const Work& w, const float* acc, uint8_t* mask, float* grad,
                             int grid, cudaStream_t st);
// kept Gaussians in ascending order: ids and (U, V); blk holds n / kVisBlock + 1 counters
cudaError_t launch_vis_compact(const uint8_t* mask, const float2* uv, int n, uint32_t* blk, int32_t* vis_gid,
                               float2* vis_uv, cudaStream_t st);

// Adam pose refinement with the update on the device (single-partition,
// non-streamed scenes; *used = false otherwise, and nothing is done). n views
// refined together; loss_history: host, n x iterations or NULL.
gs_status refine_on_device(gs_scene* s, int n_views, const gs_camera* cams, gs_pose* poses,
                           const float* const* target_rgb, const float* const* target_depth,
                           const float* const* pixel_weight, const gs_refine_opts* opts, double* loss_history,
                           cudaStream_t st, bool* used);


}  // namespace gsr
