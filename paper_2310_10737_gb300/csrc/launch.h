// launch.h -- host-side launchers of the device kernels (library internal).
#pragma once
#include <cuda_runtime.h>

#include <cstdint>

#include "sg_common.h"

namespace sg {

// Component-word SISO decoding (sogrand_decode).  Pointers are device
// memory; every output may be null.
struct DecodeArgs {
  int64_t n_words;
  const float *llr_ch;   // [W][n]
  const float *llr_a;    // [W][n] or null
  uint8_t *hard;         // [W][n]
  float *llr_app;        // [W][n]
  float *llr_ext;        // [W][n]
  float *p_miss;         // [W]
  int64_t *queries;      // [W]
  uint64_t *list_words;  // [W][L][nm]
  float *list_app;       // [W][L]
  int32_t *list_count;   // [W]
  int32_t *xf_count;     // [1] words that needed the extended-range remainder (diagnostic)
  unsigned long long *wsum;  // [1] += summed pattern weights of all queries (may be null)
};

// Block-turbo decoding of product codes (plain form: one launch per half).
struct ProductArgs {
  int64_t n_frames;
  int32_t nr, nc;        // frame: nc rows of nr bits (nr = row code's n, nc = column code's n)
  int32_t hbw;           // words of hard decisions kept per frame: max(nr, nc)
  int32_t diag;          // 1: QC-GLDPC, the second set of words are the wrapped diagonals of the n x n frame
                         // (bit i of word w is bit ((w + i) mod n, i)) instead of its columns
  const float *llr_ch;   // [F][nc][nr] row-major
  float alpha;
  int32_t max_half;      // 2 * max iterations
  float *le;             // [F][n][n] extrinsic state (scratch)
  uint64_t *hb;          // [F][n][nm] hard decisions of the last half, rows or columns (scratch)
  int32_t *fstate;       // [F] 0 running, 1 decoded, 2 max iterations, 3 invalid input (scratch)
  int32_t *hmax;         // [F] max queries of the current half (scratch)
  uint8_t *bits;         // [F][n*n/8] out, row-major, LSB first
  int32_t *half_iters;   // [F] out
  uint8_t *status;       // [F] out: 0 decoded, 1 max iterations, 2 invalid input
  int64_t *queries;      // [F] out (total)
  int64_t *par_queries;  // [F] out ("parallelized": sum over halves of the per-half max)
  int32_t *active;       // [1] frames still running after the last check (scratch, may be null)
  int32_t *xf_count;
  unsigned long long *wsum;  // [1] += summed pattern weights of all queries (may be null)
  // persistent form only (scratch)
  int32_t *queue;             // [F * max_half] frame-halves: frame + 1 once a slot is filled, else 0
  int32_t *half_cur;          // [F] current half iteration of each frame
  int32_t *done_words;        // [F] words of the current half completed
  int32_t *bad;               // [F] a non-finite input was seen
  int32_t *ctrl;              // [8] slots reserved, word tickets, finished frames, error, active warps
  int32_t max_spin;           // microseconds of accumulated back-off without work before giving up
  int32_t *half_stop;         // [F] or null: park the frame after this half (serving epochs)
  // serving: the launch decodes the frames named by a list (buffer indices;
  // an entry -(f + 1) marks frame f as newly admitted: its counters are
  // cleared and its status set to 255, "in progress"), each for at most
  // epoch_halves halves; n_frames is then the list's length
  int32_t *frame_list;        // [n_frames] or null: frames 0 .. n_frames-1, all new
  int32_t epoch_halves;       // > 0 with frame_list and half_stop
  int32_t grid_cap;           // > 0: at most this many blocks
  // plain form only: query count of every word of the current half, [F][hbw] (or null)
  int32_t *wq;
  // persistent form: the blocks' remaining-mass areas in global memory (block
  // b uses dp_area + b * dp_stride), for at most dp_blocks blocks; null: in
  // shared memory
  unsigned char *dp_area;
  int32_t dp_stride, dp_blocks;
};

template <int NPL, class SYN>
cudaError_t launch_decode(const DevCode &code, const SisoParams &P, const DecodeArgs &a, cudaStream_t s);

template <int NPL, class SYN>
cudaError_t launch_trace(const DevCode &code, const float *lam, int max_q, uint64_t *out, int32_t *count,
                         int32_t *c_out, cudaStream_t s);

template <int NPL, class SYN>
cudaError_t launch_product_init(const DevCode &code, const ProductArgs &a, cudaStream_t s);

// Product launchers take the row code (words of a row half) and the column
// code (words of a column half); a square product code passes one code twice.
// GEN = false is the square product code of one code (rowc == colc,
// nr == nc == n, no diagonals); GEN = true any other geometry.
template <int NPL, class SYN, bool GEN>
cudaError_t launch_product_half(const DevCode &rowc, const DevCode &colc, const SisoParams &P, const ProductArgs &a,
                                int half, cudaStream_t s);

template <int NPL, class SYN>
cudaError_t launch_product_check(const DevCode &rowc, const DevCode &colc, const ProductArgs &a, int half,
                                 cudaStream_t s);

// The batched form's two launches: the list set-up (k_persistent_init) and
// the decoder.  `part` selects them: PERSISTENT_ALL both, PERSISTENT_INIT the
// set-up only, PERSISTENT_DECODE the decoder only, PERSISTENT_DECODE_PDL the
// decoder as a programmatic dependent launch: it may start once every block
// of the previous kernel on the stream has begun to leave (the decoder's
// warps signal that when they drain), so a chain of decoders overlaps only
// at the tails.  The decoder reads nothing the previous kernel writes.
enum PersistentPart { PERSISTENT_ALL = 0, PERSISTENT_INIT = 1, PERSISTENT_DECODE = 2, PERSISTENT_DECODE_PDL = 3 };
template <int NPL, class SYN, bool GEN>
cudaError_t launch_product_persistent(const DevCode &rowc, const DevCode &colc, const SisoParams &P,
                                      const ProductArgs &a, cudaStream_t s, int part = PERSISTENT_ALL);

// shared-memory layout sizes of a code: per warp, and the block's remaining-mass area
int dp_area_bytes(int npl, int syn_bytes, int jmax);
// bytes of one block's slice of a global remaining-mass region
int dp_slice_bytes(int npl, int syn_bytes, int jmax);

}  // namespace sg
