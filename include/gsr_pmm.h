/* gsr_pmm.h -- probabilistic mutual matching (PMM) of rendered and query
 * feature maps on GB300 (sm_103a): the coarse-to-fine dense matching of the
 * dense refinement stage of Hi^2-GSLoc (arXiv 2507.15683, Sec. 3.4, Eq. 11).
 *
 * Sec. 3.4: at the coarse level (H_f / H_c = 8) the cosine similarity M of
 * every query position with every rendered position, the dual softmax
 *   P_M = softmax_j(M / tau) (.) softmax_i(M / tau)                 (Eq. 11)
 * and mutual nearest neighbours on P_M give the coarse correspondences; the
 * same operations inside the w x w windows (w = 8) of fine pixels at each
 * coarse correspondence give the fine correspondences.
 *
 * Readings (the paper is silent): the coarse maps are the 8 x 8 block means of
 * the fine maps; vectors are L2-normalised (zero stays zero); tau = 0.1; ties
 * in an argmax go to the lower index; the fine window of a coarse position is
 * its 8 x 8 block. The coarse similarities are fp32-accurate cosines of the
 * unrounded cell means: each binary32 unit mean u is split into bfloat16
 * hi = bf16(u) and lo = bf16(u - hi) for the tensor cores, and M = hi.hi +
 * lo.hi + hi.lo with fp32 accumulation (error about 2^-17).
 *
 * All pointers named feat_* and every pointer in gs_pmm_result are device
 * memory. Thread safety: one matcher per stream at a time.
 */
#ifndef GSR_PMM_H
#define GSR_PMM_H

#include "gsr.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct gs_pmm gs_pmm;

/* A matcher for feature maps of `channels` (32) channels and height x width
 * pixels, both multiples of 8. It owns its device workspace (about
 * 4 (H W / 64)^2 / 32 bytes of partial sums plus the match lists). Errors:
 * INVALID_ARG (channels != 32, sizes not multiples of 8 or above 8192), OOM,
 * CUDA. */
gs_status gs_pmm_create(int channels, int height, int width, gs_pmm** out);
void gs_pmm_destroy(gs_pmm* matcher);

/* The feature-map shape the matcher was created for (host pointers, each may
 * be NULL). Errors: INVALID_ARG (NULL matcher). */
gs_status gs_pmm_shape(const gs_pmm* matcher, int* channels, int* height, int* width);

/* Results of the last gs_pmm_match; the device arrays belong to the matcher
 * and stay valid until its next call or destruction. A cell is a coarse
 * position, index cy * (W / 8) + cx; a pixel is y * W + x. */
typedef struct {
  int32_t n_cells;           /* (H / 8) * (W / 8) */
  const uint16_t* codes_q;   /* n_cells x 64 bfloat16: unit coarse query vectors u as hi[32], lo[32] (u = hi + lo) */
  const uint16_t* codes_r;   /* n_cells x 64: rendered */
  const float* lse_row;      /* n_cells: log sum_j exp(M_ij / tau), query cell i */
  const float* lse_col;      /* n_cells: log sum_i exp(M_ij / tau), rendered cell j */
  const int32_t* row_best;   /* n_cells: argmax_j P_M[i, j] */
  const int32_t* col_best;   /* n_cells: argmax_i P_M[i, j] */
  int64_t n_coarse;          /* coarse correspondences (mutual nearest neighbours) */
  const int32_t* coarse;     /* n_coarse x 2: (query cell, rendered cell), ascending query cell */
  const float* coarse_prob;  /* n_coarse: P_M of the pair */
  int64_t n_fine;            /* fine correspondences */
  const int32_t* fine;       /* n_fine x 3: (coarse index, query pixel, rendered pixel), in coarse then query order */
  const float* fine_prob;    /* n_fine: window P_M of the pair */
} gs_pmm_result;

/* Match feat_query against feat_render, both channels x height x width fp32
 * planar (the layout of gs_outputs.feats), with temperature tau (>= 0.025, so
 * that exp(-2 / tau) stays a normal binary32 number; 0.1 in the paper's
 * setting). Synchronous on `stream`: the counts in *out are valid on return.
 * Errors: INVALID_ARG, CUDA, TIMEOUT (a tensor-core completion wait ran out
 * of polls: the tile kernel drains the MMA in flight, frees its tensor
 * memory and stops, the later kernels find no match, and the matcher stays
 * usable for the next call). */
gs_status gs_pmm_match(gs_pmm* matcher, const float* feat_query, const float* feat_render, float tau,
                       gs_pmm_result* out, void* stream);

/* The bound on every tensor-core completion wait of the matcher's tile
 * kernels, in mbarrier polls (default GS_PMM_DEFAULT_WAIT_POLLS, far beyond
 * the two MMAs of a tile). A wait that runs out sets a device error flag and
 * gs_pmm_match returns GS_ERR_TIMEOUT instead of spinning on. polls = 0 makes
 * every first wait give up at once: the host-visible way to exercise that
 * path without a fault (the drain that follows keeps the default bound).
 * Errors: INVALID_ARG (NULL matcher, polls < 0). */
#define GS_PMM_DEFAULT_WAIT_POLLS (1 << 22)
gs_status gs_pmm_set_wait_limit(gs_pmm* matcher, int polls);

#ifdef __cplusplus
}
#endif

#endif /* GSR_PMM_H */
