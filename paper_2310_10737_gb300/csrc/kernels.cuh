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

template <int NPL, class SYN>
__host__ __device__ inline int warp_scratch_bytes(int jmax) {
  return Layout<NPL, SYN>::bytes(jmax);
}

// ---------------------------------------------------------------------------
template <int NPL, class SYN>
__global__ void __launch_bounds__(TPB, 6) k_decode(const DevCode code, const SisoParams P, const DecodeArgs a,
                                                int wbytes) {
  extern __shared__ __align__(16) unsigned char smem[];
  constexpr int NM = (32 * NPL + 63) / 64;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  Scratch<NPL, SYN> sc;
  sc.bind(smem + warp * wbytes);
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
    siso_word<NPL, SYN>(code, P, sc, lam, lane, lapp, res, &used_xf);
    const bool empty = res.nhit == 0;
#pragma unroll
    for (int k = 0; k < NPL; k++) {
      const int i = lane + 32 * k;
      if (i < n) {
        if (a.llr_app) a.llr_app[base + i] = lapp[k];
        if (a.llr_ext) a.llr_ext[base + i] = empty ? 0.f : __fsub_rn(lapp[k], lam[k]);
        if (a.hard) a.hard[base + i] = lapp[k] < 0.f ? 1 : 0;
      }
    }
    if (lane == 0) {
      if (a.p_miss) a.p_miss[w] = res.pmiss;
      if (a.queries) a.queries[w] = res.queries;
      if (a.list_count) a.list_count[w] = res.nhit;
      if (used_xf && a.xf_count) atomicAdd(a.xf_count, 1);
      if (a.wsum) atomicAdd(a.wsum, (unsigned long long)res.wsum);
    }
    if (a.list_words || a.list_app) {
      for (int l = lane; l < P.L; l += 32) {
        if (a.list_words)
#pragma unroll
          for (int wd = 0; wd < NM; wd++)
            a.list_words[((size_t)w * P.L + l) * NM + wd] = l < res.nhit ? sc.cw[l * NM + wd] : 0ull;
        if (a.list_app) a.list_app[(size_t)w * P.L + l] = l < res.nhit ? sc.wl[l] : 0.f;
      }
    }
    __syncwarp();
  }
}

template <int NPL, class SYN>
__global__ void k_trace(const DevCode code, const float *lam_in, int max_q, uint64_t *out, int32_t *count,
                        int32_t *c_out, int wbytes) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int lane = threadIdx.x & 31;
  Scratch<NPL, SYN> sc;
  sc.bind(smem);
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

// Per-warp tallies flushed to the global counters once, when the warp exits.
struct WarpTally {
  unsigned long long wsum = 0;  // summed pattern weights
  int xf = 0;                   // words that took the extended-range path
  __device__ void flush(const ProductArgs &a, int lane) const {
    if (lane != 0) return;
    if (a.wsum && wsum) atomicAdd(a.wsum, wsum);
    if (a.xf_count && xf) atomicAdd(a.xf_count, xf);
  }
};

// One component word of frame f in half `half` (rows when odd): lambda =
// L_Ch + fl32(alpha L_E) (L_A = 0 in the first half), SOGRAND, then L_E and
// the hard decision of L_APP are stored and the query counters updated.
// Returns the word's query count (-1: non-finite input).
template <int NPL, class SYN, bool COHERENT>
__device__ __forceinline__ int product_word(const DevCode &code, const SisoParams &P, const ProductArgs &a,
                                            const Scratch<NPL, SYN> &sc, int64_t f, int wd, int half, int lane,
                                            WarpTally &tally) {
  constexpr int NM = (32 * NPL + 63) / 64;
#ifdef SG_PHASE_PROFILE
  const long long t0 = clock64();
#endif
  const int n = code.n;
  const bool rows = (half & 1) != 0;
  const size_t fb = (size_t)f * n * n;
  float lam[NPL];
#pragma unroll
  for (int k = 0; k < NPL; k++) {
    const int i = lane + 32 * k;
    float x = 0.f;
    if (i < n) {
      const size_t pos = fb + (rows ? (size_t)wd * n + i : (size_t)i * n + wd);
      x = __ldg(a.llr_ch + pos);
      if (half > 1) x = __fadd_rn(x, __fmul_rn(a.alpha, ld_state<COHERENT>(a.le + pos)));  // L_A = alpha L_E
    }
    lam[k] = x;
  }
  float lapp[NPL];
  WordResult res;
  int used_xf = 0;
  siso_word<NPL, SYN>(code, P, sc, lam, lane, lapp, res, &used_xf);
  const bool empty = res.nhit == 0;
  unsigned hb[NPL];
#pragma unroll
  for (int k = 0; k < NPL; k++) {
    const int i = lane + 32 * k;
    if (i < n) {
      const size_t pos = fb + (rows ? (size_t)wd * n + i : (size_t)i * n + wd);
      a.le[pos] = (empty || res.queries < 0) ? 0.f : __fsub_rn(lapp[k], lam[k]);
    }
    hb[k] = __ballot_sync(FULL, i < n && lapp[k] < 0.f);
  }
  if (lane == 0) {
    uint64_t *dst = a.hb + ((size_t)f * n + wd) * NM;
#pragma unroll
    for (int wd2 = 0; wd2 < NM; wd2++) {
      uint64_t v = hb[2 * wd2];
      if (2 * wd2 + 1 < NPL) v |= (uint64_t)hb[2 * wd2 + 1] << 32;
      dst[wd2] = v;
    }
    if (res.queries >= 0) {
      atomicAdd(reinterpret_cast<unsigned long long *>(a.queries + f), (unsigned long long)res.queries);
      atomicMax(a.hmax + f, res.queries);
      tally.wsum += (unsigned long long)res.wsum;
    }
    tally.xf += used_xf;
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

// Hard decision of frame f after a half: W holds its n words (rows after an
// odd half, columns after an even one).  Every word of this orientation is a
// codeword iff parity(word & H row t) = 0 for all t; every word of the other
// orientation is a codeword iff, for every t, the XOR of the words selected
// by H row t is zero (bit-sliced, no transpose).  Warp-uniform result.
template <int NPL>
__device__ __forceinline__ bool frame_valid(const DevCode &code, const uint64_t *W, int lane) {
  constexpr int NM = (32 * NPL + 63) / 64;
  const int n = code.n, m = code.m;
  bool ok = true;
#pragma unroll
  for (int k = 0; k < NPL; k++) {
    const int wd = lane + 32 * k;
    if (wd < n) {
      for (int t = 0; t < m && ok; t++) {
        int p = 0;
#pragma unroll
        for (int x = 0; x < NM; x++) p ^= __popcll(W[wd * NM + x] & __ldg(code.hrow + t * NM + x));
        if (p & 1) ok = false;
      }
    }
  }
  ok = __all_sync(FULL, ok);
  for (int t = 0; t < m && ok; t++) {
    uint64_t acc[NM];
#pragma unroll
    for (int x = 0; x < NM; x++) acc[x] = 0;
#pragma unroll
    for (int k = 0; k < NPL; k++) {
      const int wd = lane + 32 * k;
      if (wd < n && ((__ldg(code.hrow + t * NM + (wd >> 6)) >> (wd & 63)) & 1ull))
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

// Write the frame's decision as row-major bits and its status.  R is scratch
// for the row words (n * NM).
template <int NPL>
__device__ __forceinline__ void frame_finish(const DevCode &code, const ProductArgs &a, int64_t f, bool rows,
                                             int half, int status, const uint64_t *W, uint64_t *R, int lane) {
  constexpr int NM = (32 * NPL + 63) / 64;
  const int n = code.n;
  const uint64_t *src = W;
  if (!rows) {
#pragma unroll
    for (int k = 0; k < NPL; k++) {
      const int i = lane + 32 * k;
      if (i < n) {
        uint64_t r[NM];
#pragma unroll
        for (int x = 0; x < NM; x++) r[x] = 0;
        for (int j = 0; j < n; j++) {
          const uint64_t bit = (W[j * NM + (i >> 6)] >> (i & 63)) & 1ull;
#pragma unroll
          for (int x = 0; x < NM; x++)
            if ((j >> 6) == x) r[x] |= bit << (j & 63);
        }
#pragma unroll
        for (int x = 0; x < NM; x++) R[i * NM + x] = r[x];
      }
    }
    __syncwarp();
    src = R;
  }
  const int nbytes = (n * n + 7) / 8;
  uint8_t *out = a.bits + (size_t)f * nbytes;
  for (int by = lane; by < nbytes; by += 32) {
    unsigned v = 0;
#pragma unroll
    for (int t = 0; t < 8; t++) {
      const int p = by * 8 + t;
      if (p < n * n) {
        const int i = p / n, j = p - i * n;
        v |= (unsigned)((src[i * NM + (j >> 6)] >> (j & 63)) & 1ull) << t;
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
template <int NPL, class SYN, bool ROWS>
__global__ void __launch_bounds__(TPB, 6) k_product_half(const DevCode code, const SisoParams P, const ProductArgs a,
                                                      int half, int wbytes) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  Scratch<NPL, SYN> sc;
  sc.bind(smem + warp * wbytes);
  const int n = code.n;
  const int64_t items = a.n_frames * n;
  const int64_t nwarps = (int64_t)gridDim.x * WARPS_PER_BLOCK;
  WarpTally tally;
  for (int64_t it = (int64_t)blockIdx.x * WARPS_PER_BLOCK + warp; it < items; it += nwarps) {
    const int64_t f = it / n;
    const int wd = (int)(it - f * n);
    const int32_t fs = __ldg(a.fstate + f);
    if (fs != F_RUN && fs != F_BAD_PENDING) continue;  // finished frames only: a flag raised during
                                                        // this half must not change which words run
    const int q = product_word<NPL, SYN, false>(code, P, a, sc, f, wd, half, lane, tally);
    if (lane == 0 && q < 0) atomicExch(a.fstate + f, (int32_t)F_BAD_PENDING);
  }
  tally.flush(a, lane);
}

// One warp per frame.
template <int NPL, class SYN>
__global__ void __launch_bounds__(TPB) k_product_check(const DevCode code, const ProductArgs a, int half) {
  constexpr int NM = (32 * NPL + 63) / 64;
  constexpr int NT = 32 * NPL;
  __shared__ uint64_t words_s[WARPS_PER_BLOCK][NT * NM];
  __shared__ uint64_t rows_s[WARPS_PER_BLOCK][NT * NM];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int n = code.n;
  const int64_t nwarps = (int64_t)gridDim.x * WARPS_PER_BLOCK;
  const bool rows = (half & 1) != 0;
  for (int64_t f = (int64_t)blockIdx.x * WARPS_PER_BLOCK + warp; f < a.n_frames; f += nwarps) {
    const int32_t st = a.fstate[f];
    if (st != F_RUN && st != F_BAD_PENDING) continue;
    uint64_t *W = words_s[warp];
    for (int x = lane; x < n * NM; x += 32) W[x] = a.hb[(size_t)f * n * NM + x];
    __syncwarp();
    const bool ok = frame_valid<NPL>(code, W, lane);
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
    frame_finish<NPL>(code, a, f, rows, half, bad ? 2 : (ok ? 0 : 1), W, rows_s[warp], lane);
    if (lane == 0) a.fstate[f] = bad ? F_BAD : (ok ? F_DECODED : F_MAXIT);
    __syncwarp();
  }
}

// ---- persistent form: one launch decodes the whole batch ----
// Frame-halves are appended to a list (a.queue[s] = frame + 1 once slot s is
// filled); the first F slots hold every frame's first half.  Warps draw
// global word tickets T: slot T / n, word T mod n, one atomic per word.  The
// warp that completes a frame's last word of a half runs the frame check and
// either finishes the frame or appends it for its next half.  A warp whose
// slot is not filled yet waits with exponential back-off; all waits are
// bounded (a.max_spin microseconds of accumulated sleep without progress):
// the kernel then records an error and every warp returns.
template <int NPL, class SYN>
__global__ void __launch_bounds__(TPB, 6) k_product_persistent(const DevCode code, const SisoParams P,
                                                               const ProductArgs a, int wbytes) {
  extern __shared__ __align__(16) unsigned char smem[];
  constexpr int NM = (32 * NPL + 63) / 64;
  constexpr int NT = 32 * NPL;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  Scratch<NPL, SYN> sc;
  sc.bind(smem + warp * wbytes);
  const int n = code.n;
  const int64_t F = a.n_frames;
  volatile int32_t *ctrl = a.ctrl;  // [0] slots reserved, [1] word tickets, [2] finished frames, [3] error
  const int64_t nslots = F * (int64_t)a.max_half;  // a frame has at most max_half halves
  const volatile int32_t *queue = a.queue;
  uint64_t *W = reinterpret_cast<uint64_t *>(sc.tail);
  uint64_t *R = W + NT * NM;
  // Every read of shared scheduling state is made by lane 0 and broadcast, so
  // the whole warp always takes the same branch.
  WarpTally tally;
  for (;;) {
    int ticket = 0;
    if (lane == 0) ticket = atomicAdd(a.ctrl + 1, 1);
    ticket = __shfl_sync(FULL, ticket, 0);
    const int slot = ticket / n, w = ticket - slot * n;
    int f1 = 0, st = 0;  // st: 0 wait, 1 work, 2 stop
    long long slept = 0;
    unsigned nap = 64;
    for (;;) {
      if (lane == 0) {
        if (ctrl[3] != 0) {
          st = 2;
        } else if (slot < nslots && (f1 = queue[slot]) != 0) {
          st = 1;
        } else if (ctrl[2] >= F) {
          st = 2;  // every frame finished: this ticket has no work
        } else {
          st = 0;
        }
      }
      st = __shfl_sync(FULL, st, 0);
      if (st != 0) break;
      if (slept > (long long)a.max_spin * 1000) {
        if (lane == 0) atomicExch(a.ctrl + 3, 1);
        st = 2;
        break;
      }
      __nanosleep(nap);
      slept += nap;
      if (nap < 8192) nap <<= 1;
    }
    if (st == 2) break;
    const int64_t f = (int64_t)__shfl_sync(FULL, f1, 0) - 1;
    __threadfence();  // acquire: the frame's state for this half
    int half = 0;
    if (lane == 0) half = __ldcg(a.half_cur + f);
    half = __shfl_sync(FULL, half, 0);
    const int q = product_word<NPL, SYN, true>(code, P, a, sc, f, w, half, lane, tally);
    if (lane == 0 && q < 0) atomicExch(a.bad + f, 1);
    __threadfence();  // release this word's L_E and hard decision
    __syncwarp();
    int done = 0;
    if (lane == 0) done = atomicAdd(a.done_words + f, 1);
    done = __shfl_sync(FULL, done, 0);
    if (done != n - 1) continue;
    // last word of this half: check the frame
    __threadfence();
    const bool rows = (half & 1) != 0;
    for (int x = lane; x < n * NM; x += 32) W[x] = ld_state<true>(a.hb + (size_t)f * n * NM + x);
    __syncwarp();
    const bool ok = frame_valid<NPL>(code, W, lane);
    int bad = 0;
    if (lane == 0) {
      bad = __ldcg(a.bad + f);
      a.par_queries[f] += __ldcg(a.hmax + f);
      a.hmax[f] = 0;
    }
    bad = __shfl_sync(FULL, bad, 0);
    if (bad || ok || half >= a.max_half) {
      frame_finish<NPL>(code, a, f, rows, half, bad ? 2 : (ok ? 0 : 1), W, R, lane);
      __threadfence();
      if (lane == 0) atomicAdd(a.ctrl + 2, 1);
    } else if (lane == 0) {
      a.half_cur[f] = half + 1;
      a.done_words[f] = 0;
      __threadfence();
      const int t = atomicAdd(a.ctrl + 0, 1);  // < nslots: every frame appends at most max_half - 1 times
      atomicExch(a.queue + t, (int)(f + 1));
    }
    __syncwarp();
  }
  tally.flush(a, lane);
}

// list and counters of the persistent form: every frame queued for half 1
static __global__ void k_persistent_init(const ProductArgs a) {
  const int64_t F = a.n_frames;
  const int64_t slots = F * (int64_t)a.max_half;
  int32_t *queue = a.queue;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < slots; i += (int64_t)gridDim.x * blockDim.x) {
    queue[i] = i < F ? (int32_t)(i + 1) : 0;
    if (i < F) {
      a.half_cur[i] = 1;
      a.done_words[i] = 0;
      a.bad[i] = 0;
      a.hmax[i] = 0;
      a.queries[i] = 0;
      a.par_queries[i] = 0;
    }
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    a.ctrl[0] = (int32_t)F;  // next slot to reserve
    a.ctrl[1] = 0;           // word tickets drawn
    a.ctrl[2] = 0;           // frames finished
    a.ctrl[3] = 0;           // error
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

template <class K>
inline cudaError_t set_smem(K kernel, int smem) {
  if (smem > 48 * 1024) return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  return cudaSuccess;
}

template <int NPL, class SYN>
cudaError_t launch_decode(const DevCode &code, const SisoParams &P, const DecodeArgs &a, cudaStream_t s) {
  if (a.n_words <= 0) return cudaSuccess;
  const int wb = warp_scratch_bytes<NPL, SYN>(code.jmax);
  const int smem = wb * WARPS_PER_BLOCK;
  auto kern = k_decode<NPL, SYN>;
  cudaError_t e = set_smem(kern, smem);
  if (e != cudaSuccess) return e;
  const int grid = grid_for(kern, smem, a.n_words);
  kern<<<grid, TPB, smem, s>>>(code, P, a, wb);
  return cudaGetLastError();
}

template <int NPL, class SYN>
cudaError_t launch_trace(const DevCode &code, const float *lam, int max_q, uint64_t *out, int32_t *count,
                         int32_t *c_out, cudaStream_t s) {
  const int wb = warp_scratch_bytes<NPL, SYN>(code.jmax);
  auto kern = k_trace<NPL, SYN>;
  cudaError_t e = set_smem(kern, wb);
  if (e != cudaSuccess) return e;
  kern<<<1, 32, wb, s>>>(code, lam, max_q, out, count, c_out, wb);
  return cudaGetLastError();
}

template <int NPL, class SYN>
cudaError_t launch_product_half(const DevCode &code, const SisoParams &P, const ProductArgs &a, int half,
                                cudaStream_t s) {
  const int wb = warp_scratch_bytes<NPL, SYN>(code.jmax);
  const int smem = wb * WARPS_PER_BLOCK;
  const int64_t items = a.n_frames * code.n;
  if (half & 1) {
    auto kern = k_product_half<NPL, SYN, true>;
    cudaError_t e = set_smem(kern, smem);
    if (e != cudaSuccess) return e;
    kern<<<grid_for(kern, smem, items), TPB, smem, s>>>(code, P, a, half, wb);
  } else {
    auto kern = k_product_half<NPL, SYN, false>;
    cudaError_t e = set_smem(kern, smem);
    if (e != cudaSuccess) return e;
    kern<<<grid_for(kern, smem, items), TPB, smem, s>>>(code, P, a, half, wb);
  }
  return cudaGetLastError();
}

template <int NPL, class SYN>
cudaError_t launch_product_check(const DevCode &code, const ProductArgs &a, int half, cudaStream_t s) {
  auto kern = k_product_check<NPL, SYN>;
  kern<<<grid_for(kern, 0, a.n_frames), TPB, 0, s>>>(code, a, half);
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

template <int NPL, class SYN>
cudaError_t launch_product_persistent(const DevCode &code, const SisoParams &P, const ProductArgs &a, cudaStream_t s) {
  if (a.n_frames <= 0) return cudaSuccess;
  k_persistent_init<<<(int)std::min<int64_t>((a.n_frames + 255) / 256, 4096), 256, 0, s>>>(a);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const int wb = warp_scratch_bytes<NPL, SYN>(code.jmax);
  const int smem = wb * WARPS_PER_BLOCK;
  auto kern = k_product_persistent<NPL, SYN>;
  e = set_smem(kern, smem);
  if (e != cudaSuccess) return e;
  int occ = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, TPB, smem);
  if (occ < 1) occ = 1;
  // every block resident at once, no more warps than words of the batch
  const int64_t want = (a.n_frames * code.n + WARPS_PER_BLOCK - 1) / WARPS_PER_BLOCK;
  const int grid = (int)std::max<int64_t>(1, std::min<int64_t>((int64_t)sm_count() * occ, want));
  kern<<<grid, TPB, smem, s>>>(code, P, a, wb);
  return cudaGetLastError();
}

#define SG_INSTANTIATE(NPL, SYN)                                                                                 \
  template cudaError_t launch_decode<NPL, SYN>(const DevCode &, const SisoParams &, const DecodeArgs &,          \
                                               cudaStream_t);                                                    \
  template cudaError_t launch_trace<NPL, SYN>(const DevCode &, const float *, int, uint64_t *, int32_t *,        \
                                              int32_t *, cudaStream_t);                                          \
  template cudaError_t launch_product_half<NPL, SYN>(const DevCode &, const SisoParams &, const ProductArgs &,   \
                                                     int, cudaStream_t);                                         \
  template cudaError_t launch_product_check<NPL, SYN>(const DevCode &, const ProductArgs &, int, cudaStream_t); \
  template cudaError_t launch_product_init<NPL, SYN>(const DevCode &, const ProductArgs &, cudaStream_t);           \
  template cudaError_t launch_product_persistent<NPL, SYN>(const DevCode &, const SisoParams &, const ProductArgs &, \
                                                           cudaStream_t);

}  // namespace sg
