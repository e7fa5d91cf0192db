// Probabilistic mutual matching (PMM) of a query and a rendered feature map,
// coarse to fine: Hi^2-GSLoc Sec. 3.4, Eq. 11.
//
// Coarse level. Each 8 x 8 block of the fine maps becomes one coarse cell: its
// mean, L2-normalised in binary32 (k_pmm_codes) and split into two bfloat16
// vectors, hi = bf16(u) and lo = bf16(u - hi), which carry u to about 2^-17.
// The cosine matrix M of all query cells against all rendered cells is the
// 32-deep contraction hi_q . hi_r + lo_q . hi_r + hi_q . lo_r (the lo . lo term
// is below 2^-17), computed tile by tile on the 5th generation tensor cores
// (tcgen05.mma, bf16 operands in shared memory, fp32 accumulator in tensor
// memory) and never stored: M is the fp32-accurate cosine of the unrounded
// cell means, not that of bf16-rounded ones (which would move the dual-softmax
// decisions whose margins are below about 1e-2). Two passes over the tiles:
//   1. row and column sums of exp((M - 1) / tau), hence the row and column
//      log-sum-exps r_i, c_j of M / tau (|M| <= 1 makes 1 / tau a fixed
//      shift, so one exponential serves the row and the column);
//   2. per row i the first argmax over j of log P_M + r_i = 2 M / tau - c_j,
//      per column j the first argmax over i of 2 M / tau - r_i.
// Partial results per tile row / column are reduced in a fixed order, and a
// query cell i matches rendered cell j when each is the other's argmax (MNN).
//
// Fine level. For every coarse match the 64 fine query vectors of cell i and
// the 64 rendered vectors of cell j (normalised in fp32) give a 64 x 64 cosine
// matrix; the same dual softmax and MNN inside the window pair give the fine
// matches (one CTA per coarse match).
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <cstring>
#include <string>

#include "gsr_pmm.h"

namespace gsr {
void set_last_error(const std::string& msg);
}

namespace {

constexpr int kC = 32;         // channels
constexpr int kRatio = 8;      // H_f / H_c
constexpr int kTile = 128;     // cells per tile side (MMA M = N = 128)
constexpr uint32_t kTmemCols = 128;
constexpr int kWaitLimit = GS_PMM_DEFAULT_WAIT_POLLS;  // polls of an mbarrier before giving up (far beyond a 2-MMA tile)
constexpr int kMaxCells = 1 << 18;
constexpr int kScanThreads = 1024;
constexpr int kWin = kRatio * kRatio;  // fine vectors per window
constexpr int kCode = 2 * kC;          // bf16 per coarse code: hi[32], then lo[32]
static_assert(kWin == 64, "k_pmm_fine splits the 64 window rows into two halves of 32 columns");

// Tensor-core operand layout of a block of kTile codes (no swizzle, K-major):
// the byte offset of the 16-byte chunk (row r, k-chunk c) is that of core
// matrix (r / 8, c), 128 bytes each, with the 8 k-chunks of a row group (hi
// 0..3, lo 0..3) adjacent, so row groups are kChunks x 128 = 1024 bytes apart.
// The codes kernel also writes every block of kTile cells in this layout, so
// that a tile's operand is one contiguous kTileBytes bulk copy.
constexpr int kChunks = kCode * 2 / 16;         // 16-byte k-chunks per code
constexpr int kTileBytes = kTile * kCode * 2;   // one operand block (16 KB)
__host__ __device__ __forceinline__ int core_off(int r, int c) {
  return ((r >> 3) * kChunks + c) * 128 + (r & 7) * 16;
}

// ---------------------------------------------------------------------------
// coarse codes: a CTA takes 32 horizontally adjacent cells; warp c sums channel c
// of each cell (lane = cell: the 32 lanes read one contiguous row of 256
// pixels), warp 0 forms the norms, and the codes leave as one contiguous block
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(1024) k_pmm_codes(const float* __restrict__ F, int H, int W, int Wc, int n_cells,
                                                    unsigned short* __restrict__ codes,
                                                    unsigned char* __restrict__ tiled) {
  __shared__ float m_s[kC][32];
  __shared__ float inv_s[32];
  __shared__ unsigned short u_s[32][kCode + 2];  // padded rows: the per-channel stores hit distinct banks
  const int c = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int cy = blockIdx.y, cx = blockIdx.x * 32 + lane;
  const bool ok = cx < Wc;
  float m = 0.0f;
  if (ok) {
    const float* base = F + (size_t)c * H * W + (size_t)(cy * kRatio) * W + cx * kRatio;
    float s = 0.0f;  // block sum in row-major order
#pragma unroll
    for (int dy = 0; dy < kRatio; ++dy) {
      const float4 a = *reinterpret_cast<const float4*>(base + (size_t)dy * W);
      const float4 b = *reinterpret_cast<const float4*>(base + (size_t)dy * W + 4);
      s = __fadd_rn(s, a.x);
      s = __fadd_rn(s, a.y);
      s = __fadd_rn(s, a.z);
      s = __fadd_rn(s, a.w);
      s = __fadd_rn(s, b.x);
      s = __fadd_rn(s, b.y);
      s = __fadd_rn(s, b.z);
      s = __fadd_rn(s, b.w);
    }
    m = __fmul_rn(s, 1.0f / (kRatio * kRatio));  // exact scaling
  }
  m_s[c][lane] = m;
  __syncthreads();
  if (c == 0) {  // squares summed over channels in channel order
    float ss = 0.0f;
#pragma unroll
    for (int k = 0; k < kC; ++k) ss = __fadd_rn(ss, __fmul_rn(m_s[k][lane], m_s[k][lane]));
    inv_s[lane] = __fsqrt_rn(ss);
  }
  __syncthreads();
  const float n = inv_s[lane];
  const float u = n > 0.0f ? __fdiv_rn(m, n) : 0.0f;
  const __nv_bfloat16 hi = __float2bfloat16_rn(u);
  const __nv_bfloat16 lo = __float2bfloat16_rn(__fsub_rn(u, __bfloat162float(hi)));  // exact difference
  u_s[lane][c] = __bfloat16_as_ushort(hi);
  u_s[lane][kC + c] = __bfloat16_as_ushort(lo);
  __syncthreads();
  const int cell0 = cy * Wc + blockIdx.x * 32;
  const int ncell = min(32, Wc - blockIdx.x * 32);
  // 32 cells x 64 bf16, contiguous in the output: two 16-bit values per thread
  const int t = threadIdx.x;
  if (t < ncell * kC) {
    const int e = 2 * t;
    const uint32_t v = (uint32_t)u_s[e / kCode][e % kCode] | ((uint32_t)u_s[e / kCode][e % kCode + 1] << 16);
    reinterpret_cast<uint32_t*>(codes + (size_t)cell0 * kCode)[t] = v;
    const int cell = cell0 + e / kCode, el = e % kCode;  // the same two values in the tiled copy
    const size_t off = (size_t)(cell / kTile) * kTileBytes + core_off(cell % kTile, el / 8) + (el % 8) * 2;
    *reinterpret_cast<uint32_t*>(tiled + off) = v;
  }
}

// ---------------------------------------------------------------------------
// tcgen05 helpers (inline PTX)
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// Shared-memory matrix descriptor: K-major, no swizzle. The operand is stored
// as 8 x 16-byte core matrices; adjacent core matrices along K are `lbo` bytes
// apart and adjacent 8-row groups `sbo` bytes apart.
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);
  d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
  d |= (uint64_t)1 << 46;  // descriptor version field (0b001)
  return d;                 // base offset 0, relative LBO, no swizzle
}

// Instruction descriptor of tcgen05.mma kind::f16: fp32 accumulator, bf16 A and
// B, both K-major, N = M = 128.
constexpr uint32_t kIdesc = (1u << 4)                         // D format: f32
                            | (1u << 7)                       // A format: bf16
                            | (1u << 10)                      // B format: bf16
                            | ((uint32_t)(kTile >> 3) << 17)  // N >> 3
                            | ((uint32_t)(kTile >> 4) << 24);  // M >> 4

__device__ __forceinline__ void mma_bf16(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}"
      ::"r"(tmem_d), "l"(adesc), "l"(bdesc), "r"(kIdesc), "r"(accumulate)
      : "memory");
}

__device__ __forceinline__ void mma_commit(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}

// bounded wait for the phase `parity` of an mbarrier: at most `limit` polls,
// false when they run out (limit 0 gives up at once)
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, int limit) {
  for (int it = 0; it < limit; ++it) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(bar), "r"(parity)
        : "memory");
    if (done) return true;
  }
  return false;
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// 16 consecutive fp32 accumulator columns of this thread's lane
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16]) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
      "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr)
      : "memory");
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int k = 0; k < 16; ++k) v[k] = __uint_as_float(r[k]);
}

// ---------------------------------------------------------------------------
// similarity tiles
// ---------------------------------------------------------------------------
constexpr int kTileThreads = 256;  // warp w: tensor-memory lanes 32 (w % 4) .. +31, columns 64 (w / 4) .. +63

struct TileSmem {
  uint4 a[kTile * kCode * 2 / 16];  // A codes (rows of M), hi then lo, core-matrix layout (16 KB)
  uint4 b[kTile * kCode * 2 / 16];  // B codes (columns of M) (16 KB)
  float colv[4][kTile];          // pass 1: column partials per row quarter
  float rowv[2][kTile];          // row partials per column half
  int rowi[2][kTile];            // pass 2: their column index
  float lse_c[kTile];            // pass 2: log-sum-exp of the tile's columns
  unsigned long long bar;       // MMA completion
  unsigned long long load_bar;  // operand bulk copies
  uint32_t tmem;
};
// one CTA uses 128 of the 512 tensor-memory columns of an SM; the dynamic
// shared-memory request keeps at most 4 CTAs on an SM so allocation never waits
constexpr size_t kTileSmemBytes = 48 * 1024;
static_assert(sizeof(TileSmem) <= kTileSmemBytes, "tile shared memory");


// lane l ends with the sum over the warp's lanes of v[l & 15] (the 16 columns of
// a chunk, each summed over the warp's 32 rows)
__device__ __forceinline__ float reduce_scatter16(float (&v)[16], int lane) {
#pragma unroll
  for (int s = 8; s >= 1; s >>= 1) {
    const bool up = (lane & s) != 0;
#pragma unroll
    for (int i = 0; i < s; ++i) {
      const float send = up ? v[i] : v[i + s];
      const float keep = up ? v[i + s] : v[i];
      v[i] = keep + __shfl_xor_sync(0xffffffffu, send, s);
    }
  }
  return v[0] + __shfl_xor_sync(0xffffffffu, v[0], 16);
}

// 2^x for x in [-120, 1]: the results stay normal binary32 numbers, so the
// flush-to-zero form of the hardware approximation is exact enough here
__device__ __forceinline__ float ex2_ftz(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// argmax order: larger value wins, equal values go to the smaller index
__device__ __forceinline__ bool better(float v, int i, float bv, int bi) { return v > bv || (v == bv && i < bi); }

// Tiles of M = A B^T (A, B: n x 32 bf16 codes), 128 x 128 each, persistent.
// PASS 1: prow_v[cb n + i] = sum over the tile's columns j of exp((M_ij - 1) / tau)
//         and pcol_v[rb n + j] = the same over the tile's rows (row block rb,
//         column block cb).
// PASS 2: prow_v / prow_i = the best 2 M_ij / tau - lse_c[j] of row i within the
//         tile and its column (the first on ties). With A = query, B = rendered
//         and lse_c = column log-sum-exps this is the row argmax of log P_M; with
//         the operands swapped and the row log-sum-exps, its column argmax.
template <int PASS>
__global__ void __launch_bounds__(kTileThreads, 4) k_pmm_tiles(const unsigned char* __restrict__ ca,
                                                               const unsigned char* __restrict__ cb,
                                                            int n, int nb, float s_exp, float s_two,
                                                            const float* __restrict__ lse_c,
                                                            float* __restrict__ prow_v, int* __restrict__ prow_i,
                                                            float* __restrict__ pcol_v, int* __restrict__ err,
                                                            int wait_limit) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  TileSmem& S = *reinterpret_cast<TileSmem*>(smem_raw);
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int quarter = warp & 3, half = warp >> 2;
  const int lrow = quarter * 32 + lane;  // this thread's row of the tile
  const uint32_t bar = smem_u32(&S.bar);
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&S.tmem)),
                 "r"(kTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  const uint32_t load_bar = smem_u32(&S.load_bar);
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar) : "memory");
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(load_bar) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = S.tmem;
  const uint32_t tbase = tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(half * 64);
  const uint32_t sa = smem_u32(S.a), sb = smem_u32(S.b);
  // Operand staging: each tile's two operand blocks (A = codes of its row
  // block, B = of its column block) are contiguous kTileBytes blocks of the
  // tiled codes, already in the MMA layout, so one thread moves them with two
  // bulk copies that complete on load_bar (no load/store instructions, no
  // register staging). The next tile's copies start as soon as this tile's
  // MMAs have read the operands, and overlap the epilogue.
  auto stage_ops = [&](int t) {  // thread 0 only
    const int rb_ = t / nb, cb_ = t - rb_ * nb;
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(load_bar), "r"(2 * kTileBytes)
                 : "memory");
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                 ::"r"(sa), "l"(ca + (size_t)rb_ * kTileBytes), "r"(kTileBytes), "r"(load_bar)
                 : "memory");
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                 ::"r"(sb), "l"(cb + (size_t)cb_ * kTileBytes), "r"(kTileBytes), "r"(load_bar)
                 : "memory");
  };
  uint32_t phase = 0, load_phase = 0;
  const int n_tiles = nb * nb;
  if (tid == 0 && (int)blockIdx.x < n_tiles) stage_ops(blockIdx.x);
  for (int t = blockIdx.x; t < n_tiles; t += gridDim.x) {  // block-uniform
    const int rb_ = t / nb, cb_ = t - rb_ * nb;
    const int grow = rb_ * kTile + lrow;  // global row (A index) of this thread
    if (PASS == 2 && tid < kTile) S.lse_c[tid] = cb_ * kTile + tid < n ? lse_c[cb_ * kTile + tid] : 0.0f;
    tc_fence_before();  // the previous tile's accumulator reads are done
    __syncthreads();
    // Thread 0 waits for the operands, issues the MMAs and polls their
    // completion; the other warps wait at the barrier (their polls would crowd
    // the MIO queue the other CTAs' epilogues use), which then orders every
    // thread's tensor-memory reads after the completion.
    bool done = true;
    if (tid == 0 && !mbar_wait(load_bar, load_phase, kWaitLimit)) {  // operands never arrived
      atomicExch(err, 1);
      done = false;
      mbar_wait(load_bar, load_phase, kWaitLimit);  // drain before the shared memory is released
    } else if (tid == 0) {
      tc_fence_after();
      // hi . hi, lo . hi, hi . lo, each K = 32 as two K = 16 steps (k-chunks
      // (0, 1) then (2, 3) at +256 bytes); the lo half starts 512 bytes in
      constexpr uint32_t kSbo = kChunks * 128;
      mma_bf16(tmem, smem_desc(sa, 128, kSbo), smem_desc(sb, 128, kSbo), 0u);
      mma_bf16(tmem, smem_desc(sa + 256, 128, kSbo), smem_desc(sb + 256, 128, kSbo), 1u);
      mma_bf16(tmem, smem_desc(sa + 512, 128, kSbo), smem_desc(sb, 128, kSbo), 1u);
      mma_bf16(tmem, smem_desc(sa + 768, 128, kSbo), smem_desc(sb + 256, 128, kSbo), 1u);
      mma_bf16(tmem, smem_desc(sa, 128, kSbo), smem_desc(sb + 512, 128, kSbo), 1u);
      mma_bf16(tmem, smem_desc(sa + 256, 128, kSbo), smem_desc(sb + 768, 128, kSbo), 1u);
      mma_commit(bar);
      done = mbar_wait(bar, phase, wait_limit);
      if (!done) {
        atomicExch(err, 1);
        mbar_wait(bar, phase, kWaitLimit);  // the MMA in flight completes before tensor memory is freed
      } else if (t + (int)gridDim.x < n_tiles) {
        stage_ops(t + gridDim.x);  // the MMAs have read the operands: copy the next tile's
      }
    }
    phase ^= 1u;
    load_phase ^= 1u;
    if (__syncthreads_or(!done)) break;  // the accumulator did not arrive in time: reported, drained
    tc_fence_after();
    const bool row_ok = grow < n;
    // interior tiles (every row and column below n) take the unmasked path
    const bool interior = (rb_ + 1) * kTile <= n && (cb_ + 1) * kTile <= n;
    if (PASS == 1) {
      float rsum = 0.0f;
#pragma unroll 2
      for (int ch = 0; ch < 4; ++ch) {
        float v[16];
        tmem_ld16(tbase + (uint32_t)(ch * 16), v);
        if (interior) {
#pragma unroll
          for (int k = 0; k < 16; ++k) {
            v[k] = ex2_ftz(fmaf(v[k], s_exp, -s_exp));  // exp((M - 1) / tau)
            rsum += v[k];
          }
        } else {
          const int col0 = cb_ * kTile + half * 64 + ch * 16;
#pragma unroll
          for (int k = 0; k < 16; ++k) {
            const float e = ex2_ftz(fmaf(v[k], s_exp, -s_exp));
            v[k] = (row_ok && col0 + k < n) ? e : 0.0f;
            rsum += v[k];
          }
        }
        const float cs = reduce_scatter16(v, lane);
        if (lane < 16) S.colv[quarter][half * 64 + ch * 16 + lane] = cs;
      }
      S.rowv[half][lrow] = rsum;
    } else {
      float best = -INFINITY;
      int bidx = 0x7fffffff;
#pragma unroll 2
      for (int ch = 0; ch < 4; ++ch) {
        float v[16];
        tmem_ld16(tbase + (uint32_t)(ch * 16), v);
        const int l0 = half * 64 + ch * 16;
        const float4* lc4 = reinterpret_cast<const float4*>(S.lse_c + l0);
        float lc[16];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const float4 x = lc4[q];
          lc[4 * q] = x.x;
          lc[4 * q + 1] = x.y;
          lc[4 * q + 2] = x.z;
          lc[4 * q + 3] = x.w;
        }
        const int col0 = cb_ * kTile + l0;
        if (interior) {
#pragma unroll
          for (int k = 0; k < 16; ++k) {
            const float rv = fmaf(v[k], s_two, -lc[k]);
            if (rv > best) {  // ascending columns: the first maximum stays
              best = rv;
              bidx = col0 + k;
            }
          }
        } else {
          const int lim = row_ok ? min(16, n - col0) : 0;
#pragma unroll
          for (int k = 0; k < 16; ++k) {
            const float rv = fmaf(v[k], s_two, -lc[k]);
            if (k < lim && rv > best) {
              best = rv;
              bidx = col0 + k;
            }
          }
        }
      }
      S.rowv[half][lrow] = best;
      S.rowi[half][lrow] = bidx;
    }
    tc_fence_before();
    __syncthreads();
    if (tid < kTile) {  // rows: the two column halves in order
      const int r = rb_ * kTile + tid;
      if (r < n) {
        if (PASS == 1) {
          prow_v[(size_t)cb_ * n + r] = S.rowv[0][tid] + S.rowv[1][tid];
        } else {
          const bool h1 = better(S.rowv[1][tid], S.rowi[1][tid], S.rowv[0][tid], S.rowi[0][tid]);
          prow_v[(size_t)cb_ * n + r] = h1 ? S.rowv[1][tid] : S.rowv[0][tid];
          prow_i[(size_t)cb_ * n + r] = h1 ? S.rowi[1][tid] : S.rowi[0][tid];
        }
      }
    } else if (PASS == 1) {  // columns: the four row quarters in order
      const int l = tid - kTile, col = cb_ * kTile + l;
      if (col < n) pcol_v[(size_t)rb_ * n + col] = ((S.colv[0][l] + S.colv[1][l]) + S.colv[2][l]) + S.colv[3][l];
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols) : "memory");
  }
}

// Fixed-order reductions of the per-tile partials: a CTA takes 32 rows (or
// columns), warp g of its 8 the partials g, g + 8, ... in ascending order
// (coalesced over the 32 rows), then the 8 warp results are combined in order.
constexpr int kRedRows = 32;
constexpr int kRedWarps = 8;

__global__ void __launch_bounds__(kRedRows * kRedWarps) k_pmm_lse(const float* __restrict__ part, int nb, int n,
                                                                  float inv_tau, float* __restrict__ lse) {
  __shared__ float sp[kRedWarps][kRedRows];
  const int lane = threadIdx.x & 31, g = threadIdx.x >> 5;
  const int i = blockIdx.x * kRedRows + lane;
  float s = 0.0f;
  if (i < n) {
#pragma unroll 4
    for (int b = g; b < nb; b += kRedWarps) s += part[(size_t)b * n + i];
  }
  sp[g][lane] = s;
  __syncthreads();
  if (g == 0 && i < n) {
    float t = sp[0][lane];
#pragma unroll
    for (int k = 1; k < kRedWarps; ++k) t += sp[k][lane];
    lse[i] = inv_tau + logf(t);  // log sum exp(M / tau) = 1 / tau + log sum exp((M - 1) / tau)
  }
}

__global__ void __launch_bounds__(kRedRows * kRedWarps) k_pmm_best(const float* __restrict__ pv,
                                                                   const int* __restrict__ pi, int nb, int n,
                                                                   int* __restrict__ best) {
  __shared__ float sv[kRedWarps][kRedRows];
  __shared__ int si[kRedWarps][kRedRows];
  const int lane = threadIdx.x & 31, g = threadIdx.x >> 5;
  const int i = blockIdx.x * kRedRows + lane;
  float bv = -INFINITY;
  int bi = 0x7fffffff;
  if (i < n) {
#pragma unroll 4
    for (int b = g; b < nb; b += kRedWarps) {
      const float v = pv[(size_t)b * n + i];
      const int x = pi[(size_t)b * n + i];
      if (better(v, x, bv, bi)) {
        bv = v;
        bi = x;
      }
    }
  }
  sv[g][lane] = bv;
  si[g][lane] = bi;
  __syncthreads();
  if (g == 0 && i < n) {
#pragma unroll
    for (int k = 1; k < kRedWarps; ++k)
      if (better(sv[k][lane], si[k][lane], bv, bi)) {
        bv = sv[k][lane];
        bi = si[k][lane];
      }
    best[i] = bi;
  }
}

// the coarse similarity of two split codes, with the three products of the tiles
__device__ __forceinline__ float dot_codes(const __nv_bfloat16* a, const __nv_bfloat16* b) {
  float s = 0.0f;
#pragma unroll
  for (int k = 0; k < kC; ++k) {
    const float ah = __bfloat162float(a[k]), al = __bfloat162float(a[kC + k]);
    const float bh = __bfloat162float(b[k]), bl = __bfloat162float(b[kC + k]);
    s = fmaf(ah, bh, fmaf(al, bh, fmaf(ah, bl, s)));
  }
  return s;
}


// mutual nearest neighbours: flag[i] = 1 when query cell i and rendered cell
// row_best[i] are each other's argmax, with P_M of the pair (an argmax left at
// its sentinel by non-finite features matches nothing). After a timed-out
// tile pass (*err set) nothing matches, so the fine level has no work.
__global__ void k_pmm_mnn(int n, const int* __restrict__ row_best, const int* __restrict__ col_best,
                          const __nv_bfloat16* __restrict__ cq, const __nv_bfloat16* __restrict__ cr,
                          const float* __restrict__ lse_row, const float* __restrict__ lse_col, float s_two,
                          int* __restrict__ flag, float* __restrict__ prob, const int* __restrict__ err) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  if (*err) {
    flag[i] = 0;
    return;
  }
  const int j = row_best[i];
  const bool mutual = j >= 0 && j < n && col_best[j] == i;
  flag[i] = mutual ? 1 : 0;
  if (mutual) prob[i] = expf(dot_codes(cq + (size_t)i * kCode, cr + (size_t)j * kCode) * s_two - lse_row[i] - lse_col[j]);
}

// the matches at their scanned positions, in ascending query order
__global__ void k_pmm_mnn_scatter(int n, const int* __restrict__ row_best, const int* __restrict__ flag,
                                  const int* __restrict__ off, const float* __restrict__ prob_in,
                                  int* __restrict__ coarse, float* __restrict__ prob) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n || !flag[i]) return;
  const int pos = off[i];
  coarse[2 * pos] = i;
  coarse[2 * pos + 1] = row_best[i];
  prob[pos] = prob_in[i];
}

// ---------------------------------------------------------------------------
// fine level: one CTA of 64 threads per coarse match
// ---------------------------------------------------------------------------
constexpr int kQs = kC + 1;  // row stride of the staged query vectors (conflict-free reads by row)

__global__ void __launch_bounds__(kWin, 8) k_pmm_fine(const float* __restrict__ Fq, const float* __restrict__ Fr,
                                                      int H, int W, int Wc, const int* __restrict__ coarse,
                                                      float inv_tau, float s_exp, float s_two,
                                                      int* __restrict__ slot_r, float* __restrict__ slot_p,
                                                      int* __restrict__ win_count, const int* __restrict__ n_coarse) {
  __shared__ __align__(16) float ur[kWin][kC];  // rendered unit vectors (read as float4 broadcasts)
  __shared__ float Mf[kWin][kWin + 1];          // similarities; first the query unit vectors (row stride kQs)
  __shared__ float lr[kWin], lc[kWin];
  __shared__ float rsh[2][kWin];                // row exp sums of the two column halves
  __shared__ int rbest[kWin], cbest[kWin];
  static_assert(kWin * kQs <= kWin * (kWin + 1), "the staged query vectors fit in the similarity buffer");
  const int k = blockIdx.x, a = threadIdx.x;
  if (k >= *n_coarse) return;  // launched for every cell; the coarse count is known on the device only
  const int ci = coarse[2 * k], cj = coarse[2 * k + 1];
  const size_t HW = (size_t)H * W;
  const int qy = (ci / Wc) * kRatio + a / kRatio, qx = (ci % Wc) * kRatio + a % kRatio;
  const int ry = (cj / Wc) * kRatio + a / kRatio, rx = (cj % Wc) * kRatio + a % kRatio;
  float* uqs = &Mf[0][0];
  {  // thread a normalises query vector a and rendered vector a (fp32, channel order)
    float vq[kC], vr[kC];
    float sq = 0.0f, sr = 0.0f;
#pragma unroll
    for (int c = 0; c < kC; ++c) {
      vq[c] = Fq[c * HW + (size_t)qy * W + qx];
      vr[c] = Fr[c * HW + (size_t)ry * W + rx];
      sq = fmaf(vq[c], vq[c], sq);
      sr = fmaf(vr[c], vr[c], sr);
    }
    const float iq = sq > 0.0f ? 1.0f / sqrtf(sq) : 0.0f, ir = sr > 0.0f ? 1.0f / sqrtf(sr) : 0.0f;
#pragma unroll
    for (int c = 0; c < kC; ++c) {
      uqs[a * kQs + c] = vq[c] * iq;
      ur[a][c] = vr[c] * ir;
    }
  }
  __syncthreads();
  // thread a: query rows r0 and r0 + 32 against the 32 columns of half h, so
  // that every broadcast of a rendered vector feeds both rows
  const int r0 = a & 31, h = a >> 5;
  float q0[kC], q1[kC];
#pragma unroll
  for (int c = 0; c < kC; ++c) {
    q0[c] = uqs[r0 * kQs + c];
    q1[c] = uqs[(r0 + 32) * kQs + c];
  }
  __syncthreads();  // the query vectors are in registers before the similarities overwrite them
  float rs0 = 0.0f, rs1 = 0.0f;  // exp sums of rows r0 and r0 + 32 over this half
  for (int b = 32 * h; b < 32 * h + 32; b += 4) {
    float m0[4] = {0.0f, 0.0f, 0.0f, 0.0f}, m1[4] = {0.0f, 0.0f, 0.0f, 0.0f};
#pragma unroll
    for (int q = 0; q < kC / 4; ++q) {
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const float4 x = reinterpret_cast<const float4*>(ur[b + u])[q];
        m0[u] = fmaf(q0[4 * q], x.x, m0[u]);
        m0[u] = fmaf(q0[4 * q + 1], x.y, m0[u]);
        m0[u] = fmaf(q0[4 * q + 2], x.z, m0[u]);
        m0[u] = fmaf(q0[4 * q + 3], x.w, m0[u]);
        m1[u] = fmaf(q1[4 * q], x.x, m1[u]);
        m1[u] = fmaf(q1[4 * q + 1], x.y, m1[u]);
        m1[u] = fmaf(q1[4 * q + 2], x.z, m1[u]);
        m1[u] = fmaf(q1[4 * q + 3], x.w, m1[u]);
      }
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      Mf[r0][b + u] = m0[u];
      Mf[r0 + 32][b + u] = m1[u];
      rs0 += exp2f((m0[u] - 1.0f) * s_exp);
      rs1 += exp2f((m1[u] - 1.0f) * s_exp);
    }
  }
  rsh[h][r0] = rs0;
  rsh[h][r0 + 32] = rs1;
  __syncthreads();
  lr[a] = inv_tau + logf(rsh[0][a] + rsh[1][a]);
  __syncthreads();
  float cs = 0.0f;  // column a
  for (int i = 0; i < kWin; ++i) cs += exp2f((Mf[i][a] - 1.0f) * s_exp);
  lc[a] = inv_tau + logf(cs);
  __syncthreads();
  {
    float bv = -INFINITY;
    int bi = 0;
    for (int b = 0; b < kWin; ++b) {
      const float v = Mf[a][b] * s_two - lc[b];
      if (v > bv) {
        bv = v;
        bi = b;
      }
    }
    rbest[a] = bi;
    bv = -INFINITY;
    bi = 0;
    for (int i = 0; i < kWin; ++i) {
      const float v = Mf[i][a] * s_two - lr[i];
      if (v > bv) {
        bv = v;
        bi = i;
      }
    }
    cbest[a] = bi;
  }
  __syncthreads();
  const int b = rbest[a];
  const bool mutual = cbest[b] == a;
  const int by = (cj / Wc) * kRatio + b / kRatio, bx = (cj % Wc) * kRatio + b % kRatio;
  slot_r[(size_t)k * kWin + a] = mutual ? by * W + bx : -1;
  slot_p[(size_t)k * kWin + a] = mutual ? expf(Mf[a][b] * s_two - lr[a] - lc[b]) : 0.0f;
  const unsigned bal = __ballot_sync(0xffffffffu, mutual);
  if ((a & 31) == 0) rbest[a] = __popc(bal);  // rows are no longer read: reuse for the two warp counts
  __syncthreads();
  if (a == 0) win_count[k] = rbest[0] + rbest[32];
}

// exclusive scan of n_win counts (one CTA): offsets and the total
__global__ void __launch_bounds__(kScanThreads) k_pmm_scan(int n_win, const int* __restrict__ cnt,
                                                           int* __restrict__ off, int* __restrict__ total,
                                                           const int* __restrict__ n_dev) {
  __shared__ uint32_t wsum[32];
  if (n_dev) n_win = *n_dev;  // a count produced on the device (the coarse matches)
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int per = (n_win + 31) / 32;  // a contiguous chunk per warp, read in coalesced steps of 32
  const int b = w * per, e = min(n_win, b + per);
  uint32_t s = 0;
  for (int k = b + lane; k < e; k += 32) s += (uint32_t)cnt[k];
  s = __reduce_add_sync(0xffffffffu, s);
  if (lane == 0) wsum[w] = s;
  __syncthreads();
  if (w == 0) {
    const uint32_t x = wsum[lane];
    uint32_t y = x;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t t = __shfl_up_sync(0xffffffffu, y, o);
      if (lane >= o) y += t;
    }
    wsum[lane] = y - x;
    if (lane == 31) *total = (int)y;
  }
  __syncthreads();
  uint32_t run = wsum[w];
  for (int k0 = b; k0 < e; k0 += 32) {
    const int k = k0 + lane;
    const uint32_t c = k < e ? (uint32_t)cnt[k] : 0u;
    uint32_t incl = c;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t t = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += t;
    }
    if (k < e) off[k] = (int)(run + incl - c);
    run += __shfl_sync(0xffffffffu, incl, 31);
  }
}

// fine matches of window k at its offset, in query-pixel order (64 threads)
__global__ void __launch_bounds__(kWin) k_pmm_fine_scatter(int W, int Wc, const int* __restrict__ coarse,
                                                           const int* __restrict__ slot_r,
                                                           const float* __restrict__ slot_p,
                                                           const int* __restrict__ off, int* __restrict__ fine,
                                                           float* __restrict__ prob, const int* __restrict__ n_coarse) {
  __shared__ int w0;
  const int k = blockIdx.x, a = threadIdx.x;
  if (k >= *n_coarse) return;
  const int r = slot_r[(size_t)k * kWin + a];
  const unsigned bal = __ballot_sync(0xffffffffu, r >= 0);
  if (a == 0) w0 = __popc(bal);
  __syncthreads();
  if (r < 0) return;
  const int pos = off[k] + (a >= 32 ? w0 : 0) + __popc(bal & ((1u << (a & 31)) - 1u));
  const int ci = coarse[2 * k];
  const int qy = (ci / Wc) * kRatio + a / kRatio, qx = (ci % Wc) * kRatio + a % kRatio;
  fine[3 * pos] = k;
  fine[3 * pos + 1] = qy * W + qx;
  fine[3 * pos + 2] = r;
  prob[pos] = slot_p[(size_t)k * kWin + a];
}

}  // namespace

// ---------------------------------------------------------------------------
// C ABI
// ---------------------------------------------------------------------------
struct gs_pmm {
  int device = 0, sm_count = 1;
  int C = 0, H = 0, W = 0, Hc = 0, Wc = 0, n = 0, nb = 0;
  void* arena = nullptr;
  __nv_bfloat16 *codes_q = nullptr, *codes_r = nullptr;
  unsigned char *tiled_q = nullptr, *tiled_r = nullptr;  // the codes in the tensor-core operand layout
  float *prow_v = nullptr, *pcol_v = nullptr, *lse_row = nullptr, *lse_col = nullptr;
  int *prow_i = nullptr, *pcol_i = nullptr, *row_best = nullptr, *col_best = nullptr;
  int *coarse = nullptr, *fine = nullptr, *slot_r = nullptr, *counters = nullptr, *win_cnt = nullptr,
      *win_off = nullptr;
  float *coarse_p = nullptr, *fine_p = nullptr, *slot_p = nullptr;
  int* host = nullptr;  // pinned: counts and error flag
  int wait_limit = kWaitLimit;  // polls of a tensor-core completion wait
};

namespace {

gs_status pmm_fail(gs_status st, const std::string& msg) {
  gsr::set_last_error(msg);
  return st;
}

#define PMM_CUDA(x)                                                                    \
  do {                                                                                 \
    const cudaError_t e_ = (x);                                                        \
    if (e_ != cudaSuccess) return pmm_fail(GS_ERR_CUDA, std::string(#x) + ": " + cudaGetErrorString(e_)); \
  } while (0)

size_t align_up(size_t x) { return (x + 255) & ~(size_t)255; }

}  // namespace

extern "C" {

gs_status gs_pmm_create(int channels, int height, int width, gs_pmm** out) {
  if (!out) return pmm_fail(GS_ERR_INVALID_ARG, "out is required");
  *out = nullptr;
  if (channels != kC) return pmm_fail(GS_ERR_INVALID_ARG, "PMM needs 32 feature channels");
  if (height < kRatio || width < kRatio || height % kRatio || width % kRatio || height > 8192 || width > 8192)
    return pmm_fail(GS_ERR_INVALID_ARG, "feature maps must be 8..8192 pixels, multiples of 8");
  const int Hc = height / kRatio, Wc = width / kRatio, n = Hc * Wc;
  if (n > kMaxCells) return pmm_fail(GS_ERR_INVALID_ARG, "more than 2^18 coarse cells");
  gs_pmm* m = new gs_pmm();
  m->C = channels;
  m->H = height;
  m->W = width;
  m->Hc = Hc;
  m->Wc = Wc;
  m->n = n;
  m->nb = (n + kTile - 1) / kTile;
  cudaError_t e = cudaGetDevice(&m->device);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&m->sm_count, cudaDevAttrMultiProcessorCount, m->device);
  const size_t nn = (size_t)n, part = (size_t)m->nb * nn;
  size_t off = 0;
  auto take = [&](size_t bytes) {
    const size_t o = off;
    off = align_up(off + bytes);
    return o;
  };
  const size_t o_cq = take(nn * kCode * 2), o_cr = take(nn * kCode * 2);
  const size_t tiled_bytes = (size_t)m->nb * kTileBytes;  // whole blocks: rows past n stay zero
  const size_t o_tq = take(tiled_bytes), o_tr = take(tiled_bytes);
  const size_t o_prv = take(part * 4), o_pri = take(part * 4), o_pcv = take(part * 4), o_pci = take(part * 4);
  const size_t o_lr = take(nn * 4), o_lc = take(nn * 4), o_rb = take(nn * 4), o_cb = take(nn * 4);
  const size_t o_co = take(nn * 8), o_cp = take(nn * 4);
  const size_t o_sr = take(nn * kWin * 4), o_sp = take(nn * kWin * 4);
  const size_t o_fi = take(nn * kWin * 12), o_fp = take(nn * kWin * 4);
  const size_t o_wc = take(nn * 4), o_wo = take(nn * 4);
  const size_t o_ct = take(4 * 4);
  if (e == cudaSuccess) e = cudaMalloc(&m->arena, off);
  // rows of the tiled codes past n are never written: zero operands of the ragged last block
  if (e == cudaSuccess) e = cudaMemset(static_cast<char*>(m->arena) + o_tq, 0, o_tr + tiled_bytes - o_tq);
  if (e == cudaSuccess) e = cudaMallocHost(reinterpret_cast<void**>(&m->host), 4 * sizeof(int));
  if (e != cudaSuccess) {
    gs_pmm_destroy(m);
    return pmm_fail(e == cudaErrorMemoryAllocation ? GS_ERR_OOM : GS_ERR_CUDA,
                    std::string("gs_pmm_create: ") + cudaGetErrorString(e));
  }
  char* base = static_cast<char*>(m->arena);
  m->codes_q = reinterpret_cast<__nv_bfloat16*>(base + o_cq);
  m->codes_r = reinterpret_cast<__nv_bfloat16*>(base + o_cr);
  m->tiled_q = reinterpret_cast<unsigned char*>(base + o_tq);
  m->tiled_r = reinterpret_cast<unsigned char*>(base + o_tr);
  m->prow_v = reinterpret_cast<float*>(base + o_prv);
  m->prow_i = reinterpret_cast<int*>(base + o_pri);
  m->pcol_v = reinterpret_cast<float*>(base + o_pcv);
  m->pcol_i = reinterpret_cast<int*>(base + o_pci);
  m->lse_row = reinterpret_cast<float*>(base + o_lr);
  m->lse_col = reinterpret_cast<float*>(base + o_lc);
  m->row_best = reinterpret_cast<int*>(base + o_rb);
  m->col_best = reinterpret_cast<int*>(base + o_cb);
  m->coarse = reinterpret_cast<int*>(base + o_co);
  m->coarse_p = reinterpret_cast<float*>(base + o_cp);
  m->slot_r = reinterpret_cast<int*>(base + o_sr);
  m->slot_p = reinterpret_cast<float*>(base + o_sp);
  m->fine = reinterpret_cast<int*>(base + o_fi);
  m->fine_p = reinterpret_cast<float*>(base + o_fp);
  m->win_cnt = reinterpret_cast<int*>(base + o_wc);
  m->win_off = reinterpret_cast<int*>(base + o_wo);
  m->counters = reinterpret_cast<int*>(base + o_ct);
  *out = m;
  return GS_OK;
}

gs_status gs_pmm_set_wait_limit(gs_pmm* m, int polls) {
  if (!m) return pmm_fail(GS_ERR_INVALID_ARG, "matcher is NULL");
  if (polls < 0) return pmm_fail(GS_ERR_INVALID_ARG, "polls must be >= 0");
  m->wait_limit = polls;
  return GS_OK;
}

gs_status gs_pmm_shape(const gs_pmm* m, int* channels, int* height, int* width) {
  if (!m) return pmm_fail(GS_ERR_INVALID_ARG, "matcher is NULL");
  if (channels) *channels = m->C;
  if (height) *height = m->H;
  if (width) *width = m->W;
  return GS_OK;
}

void gs_pmm_destroy(gs_pmm* m) {
  if (!m) return;
  cudaSetDevice(m->device);
  if (m->arena) {
    cudaDeviceSynchronize();
    cudaFree(m->arena);
  }
  if (m->host) cudaFreeHost(m->host);
  delete m;
}

gs_status gs_pmm_match(gs_pmm* m, const float* feat_query, const float* feat_render, float tau,
                       gs_pmm_result* out, void* stream) {
  gsr::set_last_error("");
  if (!m || !feat_query || !feat_render || !out) return pmm_fail(GS_ERR_INVALID_ARG, "matcher, maps and out are required");
  if (((uintptr_t)feat_query | (uintptr_t)feat_render) & 15u)
    return pmm_fail(GS_ERR_INVALID_ARG, "feature maps must be 16-byte aligned");
  if (!(tau >= 0.025f) || !std::isfinite(tau)) return pmm_fail(GS_ERR_INVALID_ARG, "tau must be finite and >= 0.025");
  PMM_CUDA(cudaSetDevice(m->device));
  const cudaStream_t st = (cudaStream_t)stream;
  const int n = m->n, nb = m->nb;
  const float inv_tau = 1.0f / tau;
  const float s_exp = 1.4426950408889634f * inv_tau;  // exp(x / tau) = exp2(x log2(e) / tau)
  const float s_two = 2.0f * inv_tau;
  PMM_CUDA(cudaMemsetAsync(m->counters, 0, 4 * sizeof(int), st));
  const dim3 cgrid((unsigned)((m->Wc + 31) / 32), (unsigned)m->Hc);
  unsigned short* cq16 = reinterpret_cast<unsigned short*>(m->codes_q);
  unsigned short* cr16 = reinterpret_cast<unsigned short*>(m->codes_r);
  k_pmm_codes<<<cgrid, 1024, 0, st>>>(feat_query, m->H, m->W, m->Wc, n, cq16, m->tiled_q);
  k_pmm_codes<<<cgrid, 1024, 0, st>>>(feat_render, m->H, m->W, m->Wc, n, cr16, m->tiled_r);
  PMM_CUDA(cudaGetLastError());
  static bool attr = false;
  if (!attr) {
    PMM_CUDA(cudaFuncSetAttribute(k_pmm_tiles<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kTileSmemBytes));
    PMM_CUDA(cudaFuncSetAttribute(k_pmm_tiles<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kTileSmemBytes));
    attr = true;
  }
  const int tiles = nb * nb;
  const int grid = tiles < 4 * m->sm_count ? tiles : 4 * m->sm_count;
  const unsigned char* cq = m->tiled_q;
  const unsigned char* cr = m->tiled_r;
  int* err = m->counters + 3;
  const int rg = (n + 255) / 256;
  // pass 1: row and column exp sums, then the log-sum-exps
  k_pmm_tiles<1><<<grid, kTileThreads, kTileSmemBytes, st>>>(cq, cr, n, nb, s_exp, s_two, nullptr, m->prow_v,
                                                             nullptr, m->pcol_v, err, m->wait_limit);
  PMM_CUDA(cudaGetLastError());
  const int rd = (n + kRedRows - 1) / kRedRows;
  k_pmm_lse<<<rd, kRedRows * kRedWarps, 0, st>>>(m->prow_v, nb, n, inv_tau, m->lse_row);
  k_pmm_lse<<<rd, kRedRows * kRedWarps, 0, st>>>(m->pcol_v, nb, n, inv_tau, m->lse_col);
  // pass 2: row argmax of log P_M, then (operands swapped) its column argmax
  k_pmm_tiles<2><<<grid, kTileThreads, kTileSmemBytes, st>>>(cq, cr, n, nb, s_exp, s_two, m->lse_col, m->prow_v,
                                                             m->prow_i, nullptr, err, m->wait_limit);
  k_pmm_best<<<rd, kRedRows * kRedWarps, 0, st>>>(m->prow_v, m->prow_i, nb, n, m->row_best);
  k_pmm_tiles<2><<<grid, kTileThreads, kTileSmemBytes, st>>>(cr, cq, n, nb, s_exp, s_two, m->lse_row, m->prow_v,
                                                             m->prow_i, nullptr, err, m->wait_limit);
  k_pmm_best<<<rd, kRedRows * kRedWarps, 0, st>>>(m->prow_v, m->prow_i, nb, n, m->col_best);
  PMM_CUDA(cudaGetLastError());
  // mutual nearest neighbours in ascending query order
  k_pmm_mnn<<<rg, 256, 0, st>>>(n, m->row_best, m->col_best, m->codes_q, m->codes_r, m->lse_row, m->lse_col, s_two,
                                m->win_cnt, m->slot_p, err);
  k_pmm_scan<<<1, kScanThreads, 0, st>>>(n, m->win_cnt, m->win_off, m->counters, nullptr);
  k_pmm_mnn_scatter<<<rg, 256, 0, st>>>(n, m->row_best, m->win_cnt, m->win_off, m->slot_p, m->coarse, m->coarse_p);
  PMM_CUDA(cudaGetLastError());
  // fine level without a round trip: one CTA per cell (the most coarse matches
  // there can be); those past the device-side coarse count return at once
  k_pmm_fine<<<n, kWin, 0, st>>>(feat_query, feat_render, m->H, m->W, m->Wc, m->coarse, inv_tau, s_exp, s_two,
                                 m->slot_r, m->slot_p, m->win_cnt, m->counters);
  k_pmm_scan<<<1, kScanThreads, 0, st>>>(0, m->win_cnt, m->win_off, m->counters + 1, m->counters);
  k_pmm_fine_scatter<<<n, kWin, 0, st>>>(m->W, m->Wc, m->coarse, m->slot_r, m->slot_p, m->win_off, m->fine,
                                         m->fine_p, m->counters);
  PMM_CUDA(cudaGetLastError());
  PMM_CUDA(cudaMemcpyAsync(m->host, m->counters, 4 * sizeof(int), cudaMemcpyDeviceToHost, st));
  PMM_CUDA(cudaStreamSynchronize(st));
  if (m->host[3])
    return pmm_fail(GS_ERR_TIMEOUT, "a tensor-core completion wait ran out of polls (limit " +
                                        std::to_string(m->wait_limit) + "); the matcher stays usable");
  const int n_coarse = m->host[0];
  out->n_cells = n;
  out->codes_q = reinterpret_cast<const uint16_t*>(m->codes_q);
  out->codes_r = reinterpret_cast<const uint16_t*>(m->codes_r);
  out->lse_row = m->lse_row;
  out->lse_col = m->lse_col;
  out->row_best = m->row_best;
  out->col_best = m->col_best;
  out->n_coarse = n_coarse;
  out->coarse = m->coarse;
  out->coarse_prob = m->coarse_p;
  out->n_fine = m->host[1];
  out->fine = m->fine;
  out->fine_prob = m->fine_p;
  return GS_OK;
}

}  // extern "C"
