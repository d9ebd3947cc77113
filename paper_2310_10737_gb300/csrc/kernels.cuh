// kernels.cuh -- __global__ kernels and their launchers (instantiated per lane
// width in inst_npl*.cu).
//
//   k_decode        sogrand_decode: warp-per-word SISO over many independent
//                   component words (Sec. V-B, Fig. siso);
//   k_trace         test hook: the canonical query order of one word;
//   k_product_half  one half iteration of block turbo decoding (Sec. VI,
//                   steps 1/2): every row (odd half) or column (even half) of
//                   every running frame is decoded with lambda = L_Ch +
//                   alpha L_E(previous half) and its L_E and hard decision are
//                   stored;
//   k_product_check hard decision of the whole frame: every row and every
//                   column must satisfy H x = 0 (Sec. VI), else continue.
#pragma once
#include <algorithm>

#include "launch.h"
#include "siso_warp.cuh"

namespace sg {

constexpr int TPB = 32 * WARPS_PER_BLOCK;

// dynamic shared memory of one block of a single-code kernel
template <int NPL, class SYN>
__host__ __device__ inline int block_scratch_bytes(int jmax) {
  return Layout<NPL, SYN>::block_bytes(jmax);
}

// The block's tail (lock word of its remaining-mass area and the warps'
// tally slots) in shared memory after the warps' areas (`wstride` bytes
// each); the remaining-mass area after the tail, or the block's own slice of
// a global region when the launch passes one.  The area serves about 1% of
// component decodings or fewer; in global memory it leaves the SM's on-chip
// memory to L1, which holds the hot query-order entries (a block of a long
// code kept 14 KB of shared memory for it).
__device__ __forceinline__ unsigned char *block_tail(unsigned char *smem, int wstride) {
  return smem + WARPS_PER_BLOCK * wstride;
}
__device__ __forceinline__ unsigned char *block_dp_area(unsigned char *smem, int wstride, unsigned char *dp_global,
                                                        int dp_stride) {
  return dp_global ? dp_global + (size_t)blockIdx.x * dp_stride : block_tail(smem, wstride) + TAIL_BYTES;
}

// Bind warp `warp`'s view: its area in shared memory (`wstride` bytes a warp),
// the block's remaining-mass area `dpb` and tail `tl`.
template <int NPL, class SYN>
__device__ __forceinline__ void bind_scratch(Scratch<NPL, SYN> &sc, unsigned char *smem, int warp, int wstride,
                                             unsigned char *dpb, unsigned char *tl) {
  sc.bind(smem + warp * wstride, dpb, tl);
}

// Clear the block's remaining-mass lock and store its poll limit (every
// thread of the block calls this).  P.lock_preheld starts the block with the
// lock taken, as if a warp held it and never released it.
__device__ __forceinline__ void init_block_lock(unsigned char *tl, const SisoParams &P) {
  if (threadIdx.x == 0) {
    int *lock = reinterpret_cast<int *>(tl);
    lock[0] = P.lock_preheld ? 1 : 0;
    lock[1] = P.lock_polls;
  }
  __syncthreads();
}

// ---------------------------------------------------------------------------
// LANES: the query order is enumerated by the lanes (DevCode::ord_lanes)
// instead of read from the order table; a kernel of its own, so that the
// table path's code and register allocation stay as they are.
template <int NPL, class SYN, int MINB, bool LANES>
__global__ void __launch_bounds__(TPB, MINB) k_decode(const DevCode code, const SisoParams P, const DecodeArgs a) {
  extern __shared__ __align__(16) unsigned char smem[];
  using LY = Layout<NPL, SYN>;
  constexpr int NM = (32 * NPL + 63) / 64;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  unsigned char *tl = block_tail(smem, LY::warp_bytes);
  init_block_lock(tl, P);
  Scratch<NPL, SYN> sc;
  bind_scratch(sc, smem, warp, LY::warp_bytes, tl + TAIL_BYTES, tl);
  const int n = code.n;
  const int64_t nwarps = (int64_t)gridDim.x * WARPS_PER_BLOCK;
  for (int64_t w = (int64_t)blockIdx.x * WARPS_PER_BLOCK + warp; w < a.n_words; w += nwarps) {
    const size_t base = (size_t)w * n;
    float lam[NPL];
#pragma unroll
    for (int k = 0; k < NPL; k++) {
      const int i = lane + 32 * k;
      float x = 0.f;
      if (i < n) {
        x = __ldg(a.llr_ch + base + i);
        if (a.llr_a) x = __fadd_rn(x, __ldg(a.llr_a + base + i));
      }
      lam[k] = x;
    }
    float lapp[NPL];
    WordResult res;
    int used_xf = 0;
    siso_word<NPL, SYN, LANES>(code, P, sc, lam, lane, lapp, res, &used_xf);
    const bool empty = res.nhit == 0;
#pragma unroll
    for (int k = 0; k < NPL; k++) {
      const int i = lane + 32 * k;
      if (i < n) {
        if (a.llr_app) a.llr_app[base + i] = lapp[k];
        if (a.llr_ext) a.llr_ext[base + i] = empty ? 0.f : __fsub_rn(lapp[k], sc.lam_at(i));
        if (a.hard) a.hard[base + i] = lapp[k] < 0.f ? 1 : 0;
      }
    }
    if (lane == 0) {
      if (a.p_miss) a.p_miss[w] = res.pmiss;
      if (a.queries) a.queries[w] = res.queries;
      if (a.list_count) a.list_count[w] = res.nhit;
      if ((used_xf & 1) && a.xf_count) atomicAdd(a.xf_count, 1);
      if (a.wsum) atomicAdd(a.wsum, (unsigned long long)res.wsum);
    }
    if (a.list_words || a.list_app) {
      for (int l = lane; l < P.L; l += 32) {
        if (a.list_words)
#pragma unroll
          for (int wd = 0; wd < NM; wd++)
            a.list_words[((size_t)w * P.L + l) * NM + wd] = l < res.nhit ? sc.cw()[l * NM + wd] : 0ull;
        if (a.list_app) a.list_app[(size_t)w * P.L + l] = l < res.nhit ? sc.wl()[l] : 0.f;
      }
    }
    __syncwarp();
  }
}

template <int NPL, class SYN>
__global__ void k_trace(const DevCode code, const float *lam_in, int max_q, uint64_t *out, int32_t *count,
                        int32_t *c_out) {
  extern __shared__ __align__(16) unsigned char smem[];
  using LY = Layout<NPL, SYN>;
  const int lane = threadIdx.x & 31;
  unsigned char *tl = block_tail(smem, LY::warp_bytes);
  init_block_lock(tl, SisoParams{1, 1, 0.f});
  Scratch<NPL, SYN> sc;
  bind_scratch(sc, smem, 0, LY::warp_bytes, tl + TAIL_BYTES, tl);
  float lam[NPL];
#pragma unroll
  for (int k = 0; k < NPL; k++) {
    const int i = lane + 32 * k;
    lam[k] = i < code.n ? lam_in[i] : 0.f;
  }
  const int q = trace_word<NPL, SYN>(code, sc, lam, lane, max_q, out, c_out);
  if (lane == 0) *count = q;
}

// ---------------------------------------------------------------------------
// product codes
// ---------------------------------------------------------------------------
enum : int32_t { F_RUN = 0, F_DECODED = 1, F_MAXIT = 2, F_BAD_PENDING = 3, F_BAD = 4 };

// Loads that must see writes made by other SMs during the same kernel (the
// persistent form) bypass L1.
template <bool COHERENT>
__device__ __forceinline__ float ld_state(const float *p) {
  if constexpr (COHERENT) return __ldcg(p);
  return *p;
}
template <bool COHERENT>
__device__ __forceinline__ uint64_t ld_state(const uint64_t *p) {
  if constexpr (COHERENT) return __ldcg(reinterpret_cast<const unsigned long long *>(p));
  return *p;
}

// Per-warp tallies live in the warp's shared slot (not in registers, which
// the search needs) and reach the global counters once, when the warp exits.
__device__ __forceinline__ void tally_clear(unsigned long long *slot, int lane) {
  if (lane == 0) slot[0] = slot[1] = 0ull;
  __syncwarp();
}
__device__ __forceinline__ void tally_flush(const unsigned long long *slot, unsigned long long *wsum, int32_t *xf_count,
                                            int lane) {
  __syncwarp();
  if (lane != 0) return;
  if (wsum && slot[0]) atomicAdd(wsum, slot[0]);
  if (xf_count && slot[1]) atomicAdd(xf_count, (int32_t)slot[1]);
}

// A word's context (frame, word, half, list index) is kept at the start of
// the frame-check area sc.W(), which nothing else uses during a word (the
// word's lambda follows it), and read back after the search: the registers
// that held it are free while the search runs.
struct WordCtx {
  int64_t f, li;
  int32_t wd, half;
};
static_assert(sizeof(WordCtx) <= 32, "the word's lambda follows the context in the frame-check area");

// One component word of frame f in half `half` (rows when odd): lambda =
// L_Ch + fl32(alpha L_E) (L_A = 0 in the first half), SOGRAND, then L_E and
// the hard decision of L_APP are stored and the query counters updated.
// `code` is the code of this half's words (the row code in a row half, the
// column code in a column half).  GEN: the frame is a.nc rows of a.nr bits
// and the second set of words may be wrapped diagonals (a.diag); otherwise
// it is a square code.n x code.n frame with columns as the second set.
// Returns the word's query count (-1: non-finite input).
template <int NPL, class SYN, bool COHERENT, bool GEN, bool LANES = false>
__device__ __forceinline__ int product_word(const DevCode &code, const SisoParams &P, const ProductArgs &a,
                                            const Scratch<NPL, SYN> &sc, int64_t f, int wd, int half, int lane) {
  constexpr int NM = (32 * NPL + 63) / 64;
#ifdef SG_PHASE_PROFILE
  const long long t0 = clock64();
#endif
  const int n = code.n, nr = GEN ? a.nr : n;
  const bool rows = (half & 1) != 0, diag = GEN && a.diag;
  const size_t fb = (size_t)f * nr * (GEN ? a.nc : n);
  float lam[NPL];
#pragma unroll
  for (int k = 0; k < NPL; k++) {
    const int i = lane + 32 * k;
    float x = 0.f;
    if (i < n) {
      const size_t pos = fb + (rows ? (size_t)wd * nr + i
                                    : (diag ? (size_t)((wd + i) % nr) * nr + i : (size_t)i * nr + wd));
      x = __ldg(a.llr_ch + pos);
      if (half > 1) x = __fadd_rn(x, __fmul_rn(a.alpha, ld_state<COHERENT>(a.le + pos)));  // L_A = alpha L_E
    }
    lam[k] = x;
  }
  float lapp[NPL];
  WordResult res;
  int used_xf = 0;
  WordCtx *ctx = reinterpret_cast<WordCtx *>(sc.W());
  if (lane == 0) {
    ctx->f = f;
    ctx->wd = wd;
    ctx->half = half;
  }
  __syncwarp();
  siso_word<NPL, SYN, LANES>(code, P, sc, lam, lane, lapp, res, &used_xf);
  bool rows2;
  {
    const volatile WordCtx *vc = ctx;
    f = vc->f;
    wd = vc->wd;
    rows2 = (vc->half & 1) != 0;
  }
  const size_t fb2 = (size_t)f * nr * (GEN ? a.nc : n);
  const bool empty = res.nhit == 0;
  unsigned hb[NPL];
#pragma unroll
  for (int k = 0; k < NPL; k++) {
    const int i = lane + 32 * k;
    if (i < n) {
      const size_t pos = fb2 + (rows2 ? (size_t)wd * nr + i
                                     : (diag ? (size_t)((wd + i) % nr) * nr + i : (size_t)i * nr + wd));
      a.le[pos] = (empty || res.queries < 0) ? 0.f : __fsub_rn(lapp[k], sc.lam_at(i));
    }
    hb[k] = __ballot_sync(FULL, i < n && lapp[k] < 0.f);
  }
  if (lane == 0) {
    uint64_t *dst = a.hb + ((size_t)f * (GEN ? a.hbw : n) + wd) * NM;
#pragma unroll
    for (int wd2 = 0; wd2 < NM; wd2++) {
      uint64_t v = hb[2 * wd2];
      if (2 * wd2 + 1 < NPL) v |= (uint64_t)hb[2 * wd2 + 1] << 32;
      dst[wd2] = v;
    }
    if (a.wq) a.wq[(size_t)f * (GEN ? a.hbw : n) + wd] = res.queries;
    if (res.queries >= 0) {
      atomicAdd(reinterpret_cast<unsigned long long *>(a.queries + f), (unsigned long long)res.queries);
      atomicMax(a.hmax + f, res.queries);
      sc.tally()[0] += (unsigned long long)res.wsum;
    }
    sc.tally()[1] += used_xf & 1;
    if ((used_xf & 2) && a.ctrl) atomicExch(a.ctrl + 3, 2);  // stops a persistent launch: reported as a timeout
  }
  __syncwarp();
#ifdef SG_PHASE_PROFILE
  if (lane == 0) {
    SG_PROF(10, clock64() - t0);
    SG_PROF(11, 1);
  }
#endif
  return res.queries;
}

// Hard decision of frame f after a half: W holds its words (rows after an
// odd half, columns after an even one): xc.n words of wc.n bits, wc the code
// of these words and xc the code across them.  Every word is a codeword of wc
// iff parity(word & H_wc row t) = 0 for all t; every word of the other
// orientation is a codeword of xc iff, for every t, the XOR of the words
// selected by H_xc row t is zero (bit-sliced, no transpose).  Warp-uniform.
template <int NPL>
__device__ __forceinline__ bool frame_valid(const DevCode &wc, const DevCode &xc, const uint64_t *W, int lane) {
  constexpr int NM = (32 * NPL + 63) / 64;
  const int nw = xc.n;  // words in W
  bool ok = true;
#pragma unroll
  for (int k = 0; k < NPL; k++) {
    const int wd = lane + 32 * k;
    if (wd < nw) {
      for (int t = 0; t < wc.m && ok; t++) {
        int p = 0;
#pragma unroll
        for (int x = 0; x < NM; x++) p ^= __popcll(W[wd * NM + x] & __ldg(wc.hrow + t * NM + x));
        if (p & 1) ok = false;
      }
    }
  }
  ok = __all_sync(FULL, ok);
  for (int t = 0; t < xc.m && ok; t++) {
    uint64_t acc[NM];
#pragma unroll
    for (int x = 0; x < NM; x++) acc[x] = 0;
#pragma unroll
    for (int k = 0; k < NPL; k++) {
      const int wd = lane + 32 * k;
      if (wd < nw && ((__ldg(xc.hrow + t * NM + (wd >> 6)) >> (wd & 63)) & 1ull))
#pragma unroll
        for (int x = 0; x < NM; x++) acc[x] ^= W[wd * NM + x];
    }
    bool zero = true;
#pragma unroll
    for (int x = 0; x < NM; x++) {
      const unsigned lo_ = __reduce_xor_sync(FULL, (unsigned)acc[x]);
      const unsigned hi_ = __reduce_xor_sync(FULL, (unsigned)(acc[x] >> 32));
      zero = zero && lo_ == 0 && hi_ == 0;
    }
    ok = ok && zero;
  }
  return ok;
}

// QC-GLDPC frame check: W holds the n words of the last half (rows, or the
// wrapped diagonals after a diagonal half).  Each must be a codeword, and so
// must each word of the other set, whose syndrome is gathered bit by bit:
// after a row half diagonal x has bit j = bit j of row (x + j) mod n; after a
// diagonal half row x has bit j = bit j of diagonal (x - j) mod n.
template <int NPL>
__device__ __forceinline__ bool frame_valid_diag(const DevCode &code, const uint64_t *W, bool rows, int lane) {
  constexpr int NM = (32 * NPL + 63) / 64;
  const int n = code.n;
  bool ok = true;
#pragma unroll
  for (int k = 0; k < NPL; k++) {
    const int x = lane + 32 * k;
    if (x < n) {
      for (int t = 0; t < code.m && ok; t++) {
        int p = 0;
#pragma unroll
        for (int y = 0; y < NM; y++) p ^= __popcll(W[x * NM + y] & __ldg(code.hrow + t * NM + y));
        if (p & 1) ok = false;
      }
      uint64_t syn = 0;
      for (int j = 0; j < n; j++) {
        const int w = rows ? (x + j) % n : (x - j + n) % n;
        if ((W[w * NM + (j >> 6)] >> (j & 63)) & 1ull) syn ^= __ldg(code.hcol + j);
      }
      if (syn) ok = false;
    }
  }
  return __all_sync(FULL, ok);
}

// Write the frame's decision as row-major bits and its status.  W holds the
// words of the last half: rows (bit j of word i is bit (i, j)), columns
// (bit i of word j is bit (i, j)) or, for a QC-GLDPC, wrapped diagonals (bit j
// of word (i - j) mod n is bit (i, j)).
template <int NPL>
__device__ __forceinline__ void frame_finish(const ProductArgs &a, int64_t f, bool rows, int half, int status,
                                             const uint64_t *W, int lane) {
  constexpr int NM = (32 * NPL + 63) / 64;
  const int nr = a.nr, nbits = a.nr * a.nc;
  const int nbytes = (nbits + 7) / 8;
  uint8_t *out = a.bits + (size_t)f * nbytes;
  for (int by = lane; by < nbytes; by += 32) {
    unsigned v = 0;
#pragma unroll
    for (int t = 0; t < 8; t++) {
      const int p = by * 8 + t;
      if (p < nbits) {
        const int i = p / nr, j = p - i * nr;
        const uint64_t word = rows     ? W[i * NM + (j >> 6)] >> (j & 63)
                              : a.diag ? W[((i - j + nr) % nr) * NM + (j >> 6)] >> (j & 63)
                                       : W[j * NM + (i >> 6)] >> (i & 63);
        v |= (unsigned)(word & 1ull) << t;
      }
    }
    out[by] = (uint8_t)v;
  }
  if (lane == 0) {
    a.half_iters[f] = half;
    a.status[f] = (uint8_t)status;
  }
  __syncwarp();
}

// ---- plain form: one launch per half iteration, then a check launch ----
template <int NPL, class SYN, bool ROWS, int MINB, bool GEN>
__global__ void __launch_bounds__(TPB, MINB) k_product_half(const DevCode rowc, const DevCode colc, const SisoParams P,
                                                         const ProductArgs a, int half) {
  extern __shared__ __align__(16) unsigned char smem[];
  using LY = Layout<NPL, SYN>;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int jm = max(rowc.jmax, colc.jmax);
  unsigned char *tl = block_tail(smem, LY::warp_bytes);
  init_block_lock(tl, P);
  Scratch<NPL, SYN> sc;
  bind_scratch(sc, smem, warp, LY::warp_bytes, tl + TAIL_BYTES, tl);
  const DevCode &code = ROWS ? rowc : colc;  // the code of this half's words
  const int n = ROWS ? a.nc : a.nr;          // words per frame in this half
  const int64_t items = a.n_frames * n;
  const int64_t nwarps = (int64_t)gridDim.x * WARPS_PER_BLOCK;
  tally_clear(sc.tally(), lane);
  for (int64_t it = (int64_t)blockIdx.x * WARPS_PER_BLOCK + warp; it < items; it += nwarps) {
    const int64_t f = it / n;
    const int wd = (int)(it - f * n);
    const int32_t fs = __ldg(a.fstate + f);
    if (fs != F_RUN && fs != F_BAD_PENDING) continue;  // finished frames only: a flag raised during
                                                        // this half must not change which words run
    const int q = product_word<NPL, SYN, false, GEN>(code, P, a, sc, f, wd, half, lane);
    if (lane == 0 && q < 0) atomicExch(a.fstate + f, (int32_t)F_BAD_PENDING);
  }
  tally_flush(sc.tally(), a.wsum, a.xf_count, lane);
}

// One warp per frame.
template <int NPL, class SYN>
__global__ void __launch_bounds__(TPB) k_product_check(const DevCode rowc, const DevCode colc, const ProductArgs a,
                                                       int half) {
  constexpr int NM = (32 * NPL + 63) / 64;
  constexpr int NT = 32 * NPL;
  __shared__ uint64_t words_s[WARPS_PER_BLOCK][NT * NM];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t nwarps = (int64_t)gridDim.x * WARPS_PER_BLOCK;
  const bool rows = (half & 1) != 0;
  const DevCode &wc = rows ? rowc : colc, &xc = rows ? colc : rowc;
  const int n = xc.n;  // words of the last half
  for (int64_t f = (int64_t)blockIdx.x * WARPS_PER_BLOCK + warp; f < a.n_frames; f += nwarps) {
    const int32_t st = a.fstate[f];
    if (st != F_RUN && st != F_BAD_PENDING) continue;
    uint64_t *W = words_s[warp];
    for (int x = lane; x < n * NM; x += 32) W[x] = a.hb[(size_t)f * a.hbw * NM + x];
    __syncwarp();
    const bool ok = a.diag ? frame_valid_diag<NPL>(wc, W, rows, lane) : frame_valid<NPL>(wc, xc, W, lane);
    const bool bad = st == F_BAD_PENDING;
    const bool finish = bad || ok || half >= a.max_half;
    if (lane == 0) {
      a.par_queries[f] += a.hmax[f];
      a.hmax[f] = 0;
    }
    if (!finish) {
      if (lane == 0 && a.active) atomicAdd(a.active, 1);
      __syncwarp();
      continue;
    }
    frame_finish<NPL>(a, f, rows, half, bad ? 2 : (ok ? 0 : 1), W, lane);
    if (lane == 0) a.fstate[f] = bad ? F_BAD : (ok ? F_DECODED : F_MAXIT);
    __syncwarp();
  }
}

// ---- persistent forms: one launch decodes the whole batch ----

// Draw a word ticket and wait until its slot of the frame-half list is
// filled.  A filled slot holds +(e + 1) for an odd half of list entry e and
// -(e + 1) for an even one: the slot itself says which half it is, so a
// ticket that the half skips (codes of different lengths) is recognised even
// after the frame has moved on to its next half.  Returns 1 with *f1 = the
// signed slot value, or 0 when the list is done (every frame finished or
// parked) or the launch's error word *err_w is set.  The wait backs off
// exponentially and gives up after max_spin microseconds of sleep, setting
// the error word.  All reads of shared state are made by lane 0 and
// broadcast, so the whole warp takes the same branch.
// Lane 0 of a warp publishes and observes the list with release/acquire
// operations at GPU scope; __syncwarp orders the other lanes' accesses before
// (release) or after (acquire) lane 0's, so no lane runs a full fence per
// word (1-2% faster than a __threadfence on both sides).
__device__ __forceinline__ int32_t ld_acquire_gpu(const volatile int32_t *p) {
  int32_t v;
  asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ int32_t atom_add_acq_rel_gpu(int32_t *p, int32_t x) {
  int32_t old;
  asm volatile("atom.acq_rel.gpu.global.add.s32 %0, [%1], %2;" : "=r"(old) : "l"(p), "r"(x) : "memory");
  return old;
}

__device__ __forceinline__ int sched_take(int32_t *ctrl_w, int32_t *err_w, const volatile int32_t *queue,
                                          int64_t nslots, int64_t frames, int slot_n, int max_spin, int lane,
                                          int *slot_out, int *word_out, int *f1_out, int *waited) {
  volatile int32_t *ctrl = ctrl_w;  // [0] slots reserved, [1] word tickets, [2] finished frames
  const volatile int32_t *err = err_w;
  int ticket = 0;
  if (lane == 0) ticket = atomicAdd(ctrl_w + 1, 1);
  ticket = __shfl_sync(FULL, ticket, 0);
  const int slot = ticket / slot_n;
  int f1 = 0, st = 0;  // st: 0 wait, 1 work, 2 stop
  long long slept = 0;
  unsigned nap = 64;
  for (;;) {
    if (lane == 0) {
      if (*err != 0) {
        st = 2;
      } else if (slot < nslots && (f1 = ld_acquire_gpu(queue + slot)) != 0) {
        st = 1;
      } else if (ctrl[2] >= frames) {
        st = 2;  // every frame finished: this ticket has no work
      } else {
        st = 0;
      }
    }
    st = __shfl_sync(FULL, st, 0);
    if (st != 0) break;
    *waited = 1;
    if (slept > (long long)max_spin * 1000) {
      if (lane == 0) atomicExch(err_w, 1);
      st = 2;
      break;
    }
    __nanosleep(nap);
    slept += nap;
    if (nap < 8192) nap <<= 1;
  }
  if (st == 2) return 0;
  *slot_out = slot;
  *word_out = ticket - slot * slot_n;
  *f1_out = __shfl_sync(FULL, f1, 0);
  __syncwarp();  // after lane 0's acquire: the warp reads the frame's state for this half
  return 1;
}

// After the last word of a half of frame f (list entry f + 1 in the launch's
// index space `gf`): check the frame and finish it, park it (a serving epoch
// ran out: its state stays for the next launch) or append its next half.
template <int NPL, bool GEN>
__device__ __forceinline__ void frame_after_half(const DevCode &wc, const DevCode &xc, const ProductArgs &a,
                                                 int32_t *ctrl, int32_t *queue_w, int64_t f, int64_t gf, int half,
                                                 uint64_t *W, int lane) {
  constexpr int NM = (32 * NPL + 63) / 64;
  const int n = xc.n;  // words of this half
  __syncwarp();  // after lane 0's acquire of the frame's word count: the other words' results
  __threadfence();
  const bool rows = (half & 1) != 0;
  const int hbw = GEN ? a.hbw : n;
  for (int x = lane; x < n * NM; x += 32) W[x] = ld_state<true>(a.hb + (size_t)f * hbw * NM + x);
  __syncwarp();
  const bool ok = (GEN && a.diag) ? frame_valid_diag<NPL>(wc, W, rows, lane) : frame_valid<NPL>(wc, xc, W, lane);
  int bad = 0, stop = 0;
  if (lane == 0) {
    bad = __ldcg(a.bad + f);
    a.par_queries[f] += __ldcg(a.hmax + f);
    a.hmax[f] = 0;
    stop = a.half_stop ? __ldcg(a.half_stop + f) : a.max_half;
  }
  bad = __shfl_sync(FULL, bad, 0);
  stop = __shfl_sync(FULL, stop, 0);
  if (bad || ok || half >= a.max_half) {
    frame_finish<NPL>(a, f, rows, half, bad ? 2 : (ok ? 0 : 1), W, lane);
    __threadfence();
    if (lane == 0) atomicAdd(ctrl + 2, 1);
  } else if (half >= stop) {
    if (lane == 0) {  // parked: resumes at half + 1 in a later launch
      a.half_cur[f] = half + 1;
      a.done_words[f] = 0;
      __threadfence();
      atomicAdd(ctrl + 2, 1);
    }
  } else if (lane == 0) {
    a.half_cur[f] = half + 1;
    a.done_words[f] = 0;
    __threadfence();
    const int t = atomicAdd(ctrl + 0, 1);  // < nslots: every frame appends at most max_half - 1 times
    const int e = (int)(gf + 1);
    atomicExch(queue_w + t, ((half + 1) & 1) ? e : -e);  // the sign gives the half's parity
  }
  __syncwarp();
}

// Frame-halves are appended to a list (a.queue[s] = +-(frame + 1) once slot s
// is filled, negative for an even half); the first F slots hold every
// frame's current half.  Warps draw global word tickets T: slot T / slot_n,
// word T mod slot_n, one atomic per word.  The
// warp that completes a frame's last word of a half runs the frame check and
// either finishes the frame or appends it for its next half.  A warp whose
// slot is not filled yet waits with exponential back-off; all waits are
// bounded (a.max_spin microseconds of accumulated sleep without progress):
// the kernel then records an error and every warp returns.  GEN: two codes or
// wrapped diagonals (the code of a word is chosen per half); otherwise a
// square product code whose words all use rowc, with no per-word selection
// of a code (selecting one of two parameter structs at run time makes the
// compiler copy it to local memory).
template <int NPL, class SYN, int MINB, bool GEN, bool LANES = false>
__global__ void __launch_bounds__(TPB, MINB) k_product_persistent(const DevCode rowc, const DevCode colc,
                                                               const SisoParams P, const ProductArgs a) {
  extern __shared__ __align__(16) unsigned char smem[];
  using LY = Layout<NPL, SYN>;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int jm = max(rowc.jmax, colc.jmax);
  unsigned char *tl = block_tail(smem, LY::warp_bytes);
  init_block_lock(tl, P);
  Scratch<NPL, SYN> sc;
  bind_scratch(sc, smem, warp, LY::warp_bytes, block_dp_area(smem, LY::warp_bytes, a.dp_area, a.dp_stride), tl);
  const int slot_n = GEN ? max(a.nr, a.nc) : rowc.n;  // tickets per list slot: the most words in a half
  const int64_t nslots = a.n_frames * (int64_t)a.max_half;  // a frame has at most max_half halves
  tally_clear(sc.tally(), lane);
  if (lane == 0) atomicAdd(a.ctrl + 4, 1);  // one more active warp
  int waited = 0;
  for (;;) {
    // Drain: a warp leaves once the unfinished frames cannot use it (each has
    // at most slot_n words in flight), so the SMs go to other work sharing
    // the GPU (the parallel kernels of the mixed form); the warps that stay
    // can always take every word that becomes available.  Decided before a
    // ticket is drawn (a drawn ticket is always decoded), and only once the
    // warp has had to wait for work: while the list runs ahead of the
    // tickets the check is skipped.
    int leave = 0;
    if (waited && lane == 0) {
      const int64_t need = (a.n_frames - (int64_t)__ldcg(a.ctrl + 2)) * slot_n;
      if ((int64_t)__ldcg(a.ctrl + 4) - 1 >= need) {
        if ((int64_t)atomicSub(a.ctrl + 4, 1) - 1 >= need)
          leave = 1;
        else
          atomicAdd(a.ctrl + 4, 1);
      }
    }
    if (__shfl_sync(FULL, leave, 0)) {
      // this block has begun to leave: a decoder launched as a programmatic
      // dependent of this one may start (no effect otherwise)
      asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
      break;
    }
    int slot, w, f1;
    if (!sched_take(a.ctrl, a.ctrl + 3, a.queue, nslots, a.n_frames, slot_n, a.max_spin, lane, &slot, &w, &f1,
                    &waited))
      break;
    const bool rows = f1 > 0;                      // the slot's half is odd: a row half
    int64_t li = (int64_t)(f1 > 0 ? f1 : -f1) - 1;  // list index
    const DevCode &code = GEN ? (rows ? rowc : colc) : rowc, &xcode = GEN ? (rows ? colc : rowc) : rowc;
    const int n = xcode.n;  // words in this half
    // a ticket past this half's words (codes of different lengths); decided
    // from the slot, since the frame may already be in its next half
    if (GEN && w >= n) continue;
    int64_t f = a.frame_list ? (int64_t)a.frame_list[li] : li;
    int half = 0;  // the slot's half: the frame cannot leave it before this word is done
    if (lane == 0) half = __ldcg(a.half_cur + f);
    half = __shfl_sync(FULL, half, 0);
    if (lane == 0) reinterpret_cast<WordCtx *>(sc.W())->li = li;
    const int q = product_word<NPL, SYN, true, GEN, LANES>(code, P, a, sc, f, w, half, lane);
    {
      const volatile WordCtx *vc = reinterpret_cast<const volatile WordCtx *>(sc.W());
      f = vc->f;
      li = vc->li;
      half = vc->half;
    }
    if (lane == 0 && q < 0) atomicExch(a.bad + f, 1);
    __syncwarp();  // every lane's L_E and hard decision, then lane 0 releases them
    int done = 0;
    if (lane == 0) done = atom_add_acq_rel_gpu(a.done_words + f, 1);  // acquire: the frame's other words
    done = __shfl_sync(FULL, done, 0);
    if (done != n - 1) continue;
    frame_after_half<NPL, GEN>(code, xcode, a, a.ctrl, a.queue, f, li, half, sc.W(), lane);
  }
  tally_flush(sc.tally(), a.wsum, a.xf_count, lane);
}

// list and counters of the persistent form: every frame queued for half 1
static __global__ void k_persistent_init(const ProductArgs a) {
  const int64_t F = a.n_frames;
  const int64_t slots = F * (int64_t)a.max_half;
  int32_t *queue = a.queue;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < slots; i += (int64_t)gridDim.x * blockDim.x) {
    if (i >= F) queue[i] = 0;
    if (i < F) {
      int64_t f = i;
      bool fresh = true;
      if (a.frame_list) {
        const int32_t e = a.frame_list[i];
        fresh = e < 0;
        f = fresh ? -(int64_t)e - 1 : (int64_t)e;
        if (fresh) a.frame_list[i] = (int32_t)f;
      }
      if (fresh) {
        a.half_cur[f] = 1;
        a.bad[f] = 0;
        a.queries[f] = 0;
        a.par_queries[f] = 0;
        if (a.frame_list) a.status[f] = 255;  // in progress until the frame finishes
      }
      a.done_words[f] = 0;
      a.hmax[f] = 0;
      if (a.half_stop) a.half_stop[f] = a.half_cur[f] + a.epoch_halves - 1;
      queue[i] = (a.half_cur[f] & 1) ? (int32_t)(i + 1) : -(int32_t)(i + 1);  // signed by the half's parity
    }
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    a.ctrl[0] = (int32_t)F;  // next slot to reserve
    a.ctrl[1] = 0;           // word tickets drawn
    a.ctrl[2] = 0;           // frames finished
    a.ctrl[3] = 0;           // error
    a.ctrl[4] = 0;           // active warps
  }
}

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------
inline int sm_count() {
  static int sms = 0;
  if (!sms) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (sms <= 0) sms = 1;
  }
  return sms;
}

template <class K>
inline int grid_for(K kernel, int smem, int64_t warps_needed) {
  int occ = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kernel, TPB, smem);
  if (occ < 1) occ = 1;
  int64_t blocks = (warps_needed + WARPS_PER_BLOCK - 1) / WARPS_PER_BLOCK;
  int64_t cap = (int64_t)sm_count() * occ;
  if (blocks > cap) blocks = cap;
  if (blocks < 1) blocks = 1;
  return (int)blocks;
}

// The schedule a launch runs: the code's, except that the 12-block kernels
// (40 registers, more spills per word) are used only when the launch has more
// words than the 8-block grid has warps; a smaller batch gains nothing from
// the extra warps and decodes each word faster at 64 registers.
inline int launch_minb(int minb, int64_t words) {
  return (minb == 12 && words > (int64_t)sm_count() * 8 * WARPS_PER_BLOCK) ? 12 : 8;
}

template <class K>
inline cudaError_t set_smem(K kernel, int smem) {
  if (smem > 48 * 1024) return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  return cudaSuccess;
}

template <int NPL, class SYN>
cudaError_t launch_decode(const DevCode &code, const SisoParams &P, const DecodeArgs &a, cudaStream_t s) {
  if (a.n_words <= 0) return cudaSuccess;
  const int smem = block_scratch_bytes<NPL, SYN>(code.jmax);
  const bool eight = launch_minb(code.minb, a.n_words) == 8, lanes = code.ord_lanes && P.thr <= 0.f;
  auto kern = lanes ? (eight ? k_decode<NPL, SYN, 8, true> : k_decode<NPL, SYN, 12, true>)
                    : (eight ? k_decode<NPL, SYN, 8, false> : k_decode<NPL, SYN, 12, false>);
  cudaError_t e = set_smem(kern, smem);
  if (e != cudaSuccess) return e;
  const int grid = grid_for(kern, smem, a.n_words);
  kern<<<grid, TPB, smem, s>>>(code, P, a);
  return cudaGetLastError();
}

template <int NPL, class SYN>
cudaError_t launch_trace(const DevCode &code, const float *lam, int max_q, uint64_t *out, int32_t *count,
                         int32_t *c_out, cudaStream_t s) {
  const int smem = block_scratch_bytes<NPL, SYN>(code.jmax);
  auto kern = k_trace<NPL, SYN>;
  cudaError_t e = set_smem(kern, smem);
  if (e != cudaSuccess) return e;
  kern<<<1, 32, smem, s>>>(code, lam, max_q, out, count, c_out);
  return cudaGetLastError();
}

template <int NPL, class SYN, bool GEN>
cudaError_t launch_product_half(const DevCode &rowc, const DevCode &colc, const SisoParams &P, const ProductArgs &a,
                                int half, cudaStream_t s) {
  const int smem = block_scratch_bytes<NPL, SYN>(std::max(rowc.jmax, colc.jmax));
  const int64_t items = a.n_frames * ((half & 1) ? a.nc : a.nr);
  const int minb = launch_minb(rowc.minb, items);
  if (half & 1) {
    auto kern = minb == 8 ? k_product_half<NPL, SYN, true, 8, GEN> : k_product_half<NPL, SYN, true, 12, GEN>;
    cudaError_t e = set_smem(kern, smem);
    if (e != cudaSuccess) return e;
    kern<<<grid_for(kern, smem, items), TPB, smem, s>>>(rowc, colc, P, a, half);
  } else {
    auto kern = minb == 8 ? k_product_half<NPL, SYN, false, 8, GEN> : k_product_half<NPL, SYN, false, 12, GEN>;
    cudaError_t e = set_smem(kern, smem);
    if (e != cudaSuccess) return e;
    kern<<<grid_for(kern, smem, items), TPB, smem, s>>>(rowc, colc, P, a, half);
  }
  return cudaGetLastError();
}

template <int NPL, class SYN>
cudaError_t launch_product_check(const DevCode &rowc, const DevCode &colc, const ProductArgs &a, int half,
                                 cudaStream_t s) {
  auto kern = k_product_check<NPL, SYN>;
  kern<<<grid_for(kern, 0, a.n_frames), TPB, 0, s>>>(rowc, colc, a, half);
  return cudaGetLastError();
}

template <int NPL, class SYN>
cudaError_t launch_product_init(const DevCode &code, const ProductArgs &a, cudaStream_t s) {
  (void)code;
  cudaError_t e = cudaMemsetAsync(a.fstate, 0, sizeof(int32_t) * a.n_frames, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(a.hmax, 0, sizeof(int32_t) * a.n_frames, s);
  if (e == cudaSuccess && a.queries) e = cudaMemsetAsync(a.queries, 0, sizeof(int64_t) * a.n_frames, s);
  if (e == cudaSuccess && a.par_queries) e = cudaMemsetAsync(a.par_queries, 0, sizeof(int64_t) * a.n_frames, s);
  return e;
}

template <int NPL, class SYN, bool GEN>
cudaError_t launch_product_persistent(const DevCode &rowc, const DevCode &colc, const SisoParams &P,
                                      const ProductArgs &a, cudaStream_t s, int part) {
  if (a.n_frames <= 0) return cudaSuccess;
  cudaError_t e = cudaSuccess;
  if (part == PERSISTENT_ALL || part == PERSISTENT_INIT) {
    k_persistent_init<<<(int)std::min<int64_t>((a.n_frames + 255) / 256, 4096), 256, 0, s>>>(a);
    e = cudaGetLastError();
    if (e != cudaSuccess || part == PERSISTENT_INIT) return e;
  }
  // with a global remaining-mass region only the warps' areas are shared memory
  const int smem = a.dp_area ? WARPS_PER_BLOCK * Layout<NPL, SYN>::warp_bytes + TAIL_BYTES
                             : block_scratch_bytes<NPL, SYN>(std::max(rowc.jmax, colc.jmax));
  const int64_t words = a.n_frames * std::max(a.nr, a.nc);  // the most words of one half
  // the lanes-enumerated order: the square geometry only (GEN reads the table)
  const bool eight = launch_minb(rowc.minb, words) == 8, lanes = !GEN && rowc.ord_lanes && P.thr <= 0.f;
  auto kern = lanes ? (eight ? k_product_persistent<NPL, SYN, 8, GEN, !GEN> : k_product_persistent<NPL, SYN, 12, GEN, !GEN>)
                    : (eight ? k_product_persistent<NPL, SYN, 8, GEN> : k_product_persistent<NPL, SYN, 12, GEN>);
  e = set_smem(kern, smem);
  if (e != cudaSuccess) return e;
  int occ = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, TPB, smem);
  if (occ < 1) occ = 1;
  // every block resident at once, no more warps than words of the batch
  const int64_t want = (words + WARPS_PER_BLOCK - 1) / WARPS_PER_BLOCK;
  int64_t cap = (int64_t)sm_count() * occ;
  if (a.grid_cap > 0 && a.grid_cap < cap) cap = a.grid_cap;
  if (a.dp_area && a.dp_blocks < cap) cap = a.dp_blocks;  // one slice of the region per block
  const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(cap, want));
  if (part == PERSISTENT_DECODE_PDL) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(TPB);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kern, rowc, colc, P, a);
  }
  kern<<<grid, TPB, smem, s>>>(rowc, colc, P, a);
  return cudaGetLastError();
}

#define SG_INSTANTIATE(NPL, SYN)                                                                                 \
  template cudaError_t launch_decode<NPL, SYN>(const DevCode &, const SisoParams &, const DecodeArgs &,          \
                                               cudaStream_t);                                                    \
  template cudaError_t launch_trace<NPL, SYN>(const DevCode &, const float *, int, uint64_t *, int32_t *,        \
                                              int32_t *, cudaStream_t);                                          \
  template cudaError_t launch_product_half<NPL, SYN, false>(const DevCode &, const DevCode &, const SisoParams &, \
                                                            const ProductArgs &, int, cudaStream_t);             \
  template cudaError_t launch_product_check<NPL, SYN>(const DevCode &, const DevCode &, const ProductArgs &, int, \
                                                      cudaStream_t);                                             \
  template cudaError_t launch_product_init<NPL, SYN>(const DevCode &, const ProductArgs &, cudaStream_t);           \
  template cudaError_t launch_product_persistent<NPL, SYN, false>(const DevCode &, const DevCode &,              \
                                                                  const SisoParams &, const ProductArgs &,       \
                                                                  cudaStream_t, int);

// Launchers of the general geometry (two codes, or wrapped diagonals), in
// translation units of their own so that they compile in parallel.
#define SG_INSTANTIATE_GEN(NPL, SYN)                                                                             \
  template cudaError_t launch_product_half<NPL, SYN, true>(const DevCode &, const DevCode &, const SisoParams &,  \
                                                           const ProductArgs &, int, cudaStream_t);              \
  template cudaError_t launch_product_persistent<NPL, SYN, true>(const DevCode &, const DevCode &,               \
                                                                 const SisoParams &, const ProductArgs &,        \
                                                                 cudaStream_t, int);

}  // namespace sg
