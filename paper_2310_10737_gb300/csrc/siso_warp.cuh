// siso_warp.cuh -- one warp decodes one component word with soft-output GRAND.
//
// arXiv 2310.10737 (SOGRAND):
//   Sec. III-B  GRAND query loop, membership H x = 0, even-code parity skip;
//   Sec. IV     Corollary: APP of every list word and of "not in the list",
//               phi = (2^k-1)/(2^n-1) (parity class: 2^(n-1) in place of 2^n);
//   Sec. V-B    SISO in/out (L_Ch + L_A -> L_APP, L_E) and eq. LLRi.
// Query order: 1-line ORBGRAND (cited by the paper), cost(z) = sum of the
// reliability ranks in z + c |z|, ties by Hamming weight then lexicographic
// rank vector; c from an exact integer least-squares line through the sorted
// reliabilities quantised to 1/256.
//
// Warp mapping: lane l holds bits l, l+32, ... (NPL per lane).  The word's
// |lambda| are bitonic-sorted across the warp (64-bit keys |lambda|:index so
// ties fall to the lower index) and the H columns are permuted into rank order
// in shared memory.  The query order depends only on (n, c, parity class), so
// it is read from a flattened table: every chunk of 32 consecutive queries is
// one coalesced 512-byte copy (cp.async into the warp's shared slots, issued
// while the previous chunk is tested), lane j takes query q0 + j, XORs its pattern's
// H columns into the syndrome of y and reports a hit; __ballot_sync + __ffs
// keep the hits in query order, so list, stop point and query count are those
// of a sequential decoder.
//
// Remaining mass.  The Corollary needs the mass of the unqueried patterns of
// the parity class, i.e. the class total minus the queried mass.  Every
// pattern mass is the product of per-rank factors t_e = exp(-|lambda_e|)
// (one FP32 value per rank), and the queried masses are formed and summed in
// double-float (an unevaluated pair of floats: Knuth's TwoSum and the
// FMA-based exact product), so the difference is exact for those factors up
// to about 2^-46 of the operands.  It is taken in FP32 when the remainder is
// at least 2% of the operands, in double-float when it is at least 2^-26 of
// them; below that (the list has taken nearly all the mass) the kernel sums
// the unqueried patterns directly (all terms positive): patterns of cost above
// the stop level C* by a dynamic programme over the ranks (cost-indexed,
// parity-split, a pattern is added to the tail the moment one more rank lifts
// it over C*), plus the unqueried rest of level C* from the table.  There the
// masses are cost-scaled by exp(gamma * cost) so that every factor stays <= 1;
// if the scaled total still falls below 2^-60 (all dominant terms underflow)
// or overflows, the same computation is redone in an extended-range float
// (FP32 mantissa + int exponent).
#pragma once
#include <cuda_runtime.h>
#include <math_constants.h>

#include <cstdint>

#include "sg_common.h"

namespace sg {

#ifdef SG_PHASE_PROFILE
// [0] prologue cycles [1] query-loop cycles [2] remainder cycles [3] soft-output
// cycles [4] words [5] query chunks [6] - [7] DP ranks [8] XF fallbacks [9] smem DP
// Every translation unit has its own copy of the counters (no relocatable
// device code), so each registers a reader that sogrand_debug_phase sums.
__device__ unsigned long long g_phase[16];
#define SG_PROF(i, v) atomicAdd(&g_phase[i], (unsigned long long)(v))
typedef int (*PhaseReader)(unsigned long long *acc, int reset);
void phase_register(PhaseReader r);
namespace {
int phase_read_here(unsigned long long *acc, int reset) {
  unsigned long long v[16];
  if (cudaMemcpyFromSymbol(v, g_phase, sizeof(v)) != cudaSuccess) return 1;
  for (int i = 0; i < 16; i++) acc[i] += v[i];
  if (reset) {
    unsigned long long z[16] = {0};
    if (cudaMemcpyToSymbol(g_phase, z, sizeof(z)) != cudaSuccess) return 1;
  }
  return 0;
}
struct PhaseHook {
  PhaseHook() { phase_register(phase_read_here); }
} phase_hook_;
}  // namespace
#else
#define SG_PROF(i, v) ((void)0)
#endif

constexpr unsigned FULL = 0xffffffffu;
constexpr float LOG2E_F = 1.4426950408889634f;
constexpr float LN2_F = 0.6931471805599453f;

__host__ __device__ constexpr int align16(int x) { return (x + 15) & ~15; }

// ----------------------------------------------------------------------------
// double-float: value = h + l, |l| <= ulp(h) / 2 after df_norm.  Rounded
// intrinsics keep the compiler from contracting the error terms.
// ----------------------------------------------------------------------------
struct DF {
  float h, l;
};
__device__ __forceinline__ DF df_two_sum(float a, float b) {  // Knuth: s + err == a + b exactly
  const float s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  return {s, __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb))};
}
__device__ __forceinline__ DF df_norm(float h, float l) {  // |h| >= |l| (Dekker's fast two-sum)
  const float s = __fadd_rn(h, l);
  return {s, __fsub_rn(l, __fsub_rn(s, h))};
}
__device__ __forceinline__ DF df_add(DF a, DF b) {
  const DF s = df_two_sum(a.h, b.h), t = df_two_sum(a.l, b.l);
  const DF r = df_norm(s.h, __fadd_rn(s.l, t.h));
  return df_norm(r.h, __fadd_rn(r.l, t.l));
}
// a + b for a, b >= 0 (no cancellation: one TwoSum on the high parts)
__device__ __forceinline__ DF df_add_pos(DF a, DF b) {
  const DF s = df_two_sum(a.h, b.h);
  return df_norm(s.h, __fadd_rn(s.l, __fadd_rn(a.l, b.l)));
}
__device__ __forceinline__ DF df_mul(DF a, DF b) {  // the FMA gives the exact error of a.h * b.h
  const float p = __fmul_rn(a.h, b.h);
  return df_norm(p, fmaf(a.h, b.l, fmaf(a.l, b.h, fmaf(a.h, b.h, -p))));
}
__device__ __forceinline__ DF df_mul_f(DF a, float b) {
  const float p = __fmul_rn(a.h, b);
  return df_norm(p, fmaf(a.l, b, fmaf(a.h, b, -p)));
}
// running sum of nonnegative terms: the low part collects the exact rounding errors
__device__ __forceinline__ void df_acc(DF &a, DF x) {
  const DF s = df_two_sum(a.h, x.h);
  a.h = s.h;
  a.l = __fadd_rn(a.l, __fadd_rn(s.l, x.l));
}
// The warp butterflies that run once per word are loops, not unrolled: the
// kernel's per-word path is long and instruction fetch is its first stall, so
// a smaller path is faster (these three loops: 7% for eBCH(64,57)).
__device__ __forceinline__ DF df_warp_sum(DF x) {  // x >= 0; lane 0's result broadcast (warp-uniform)
  x = df_norm(x.h, x.l);
#pragma unroll 1
  for (int d = 16; d > 0; d >>= 1)
    x = df_add_pos(x, DF{__shfl_xor_sync(0xffffffffu, x.h, d), __shfl_xor_sync(0xffffffffu, x.l, d)});
  return {__shfl_sync(0xffffffffu, x.h, 0), __shfl_sync(0xffffffffu, x.l, 0)};
}

// ----------------------------------------------------------------------------
// extended-range float: value = m * 2^e, m in [1, 2) (or 0)
// ----------------------------------------------------------------------------
struct XF {
  float m;
  int e;
};
constexpr int XF_ZERO_E = -(1 << 29);

__device__ __forceinline__ XF xf_zero() { return {0.f, XF_ZERO_E}; }
__device__ __forceinline__ XF xf_one() { return {1.f, 0}; }
__device__ __forceinline__ XF xf_norm(float m, int e) {
  if (m == 0.f) return xf_zero();
  int b = __float_as_int(m);
  int ex = ((b >> 23) & 0xff) - 127;
  return {__int_as_float((b & 0x807fffff) | (127 << 23)), e + ex};
}
__device__ __forceinline__ XF xf_mul(XF a, XF b) { return xf_norm(a.m * b.m, a.e + b.e); }
__device__ __forceinline__ XF xf_add(XF a, XF b) {
  if (a.e < b.e) {
    XF t = a;
    a = b;
    b = t;
  }
  int d = b.e - a.e;
  if (d < -40) return a;
  float m = a.m + b.m * __int_as_float((127 + d) << 23);
  return xf_norm(m, a.e);
}
__device__ __forceinline__ XF xf_from_log2(float x) {
  if (!(x > -1e30f)) return xf_zero();
  float f = floorf(x);
  return xf_norm(exp2f(x - f), (int)f);
}
__device__ __forceinline__ float xf_log2(XF a) { return a.m == 0.f ? -CUDART_INF_F : (float)a.e + log2f(a.m); }

// Number policies for the remaining-mass computation.
struct FOps {  // plain FP32, cost-scaled
  using T = float;
  static __device__ __forceinline__ T zero() { return 0.f; }
  static __device__ __forceinline__ T one() { return 1.f; }
  static __device__ __forceinline__ T add(T a, T b) { return a + b; }
  static __device__ __forceinline__ T mul(T a, T b) { return a * b; }
  static __device__ __forceinline__ T fma(T a, T b, T c) { return fmaf(a, b, c); }
  static __device__ __forceinline__ T from_log2(float x) { return exp2f(x); }
  static __device__ __forceinline__ T from_float(float x) { return x; }
  static __device__ __forceinline__ T shfl(T a, int src) { return __shfl_sync(FULL, a, src); }
  static __device__ __forceinline__ T shfl_down(T a, int d) { return __shfl_down_sync(FULL, a, d); }
  static __device__ __forceinline__ T shfl_xor(T a, int d) { return __shfl_xor_sync(FULL, a, d); }
};
struct XOps {  // extended range, unscaled
  using T = XF;
  static __device__ __forceinline__ T zero() { return xf_zero(); }
  static __device__ __forceinline__ T one() { return xf_one(); }
  static __device__ __forceinline__ T add(T a, T b) { return xf_add(a, b); }
  static __device__ __forceinline__ T mul(T a, T b) { return xf_mul(a, b); }
  static __device__ __forceinline__ T fma(T a, T b, T c) { return xf_add(xf_mul(a, b), c); }
  static __device__ __forceinline__ T from_log2(float x) { return xf_from_log2(x); }
  static __device__ __forceinline__ T from_float(float x) { return xf_norm(x, 0); }
  static __device__ __forceinline__ T shfl(T a, int src) {
    return {__shfl_sync(FULL, a.m, src), __shfl_sync(FULL, a.e, src)};
  }
  static __device__ __forceinline__ T shfl_down(T a, int d) {
    return {__shfl_down_sync(FULL, a.m, d), __shfl_down_sync(FULL, a.e, d)};
  }
  static __device__ __forceinline__ T shfl_xor(T a, int d) {
    return {__shfl_xor_sync(FULL, a.m, d), __shfl_xor_sync(FULL, a.e, d)};
  }
};

// ----------------------------------------------------------------------------
// per-warp shared-memory scratch
// ----------------------------------------------------------------------------
// H column and mass factor t = exp(-|lambda|) of one reliability rank, read
// together in the query loop
template <class SYN>
struct RankRec {
  SYN h;
  float t;
};

// Shared memory of a block: one area per warp (below), then a tail: the lock
// word of the block's remaining-mass area with the lock's poll limit (16
// bytes) and one 16-byte tally slot per warp (summed pattern weights,
// extended-range words), flushed to global counters when the warp exits; then
// (unless the launch puts it in global memory) the remaining-mass area for the
// whole block (the cost DP, needed by about 1% of component decodings or
// fewer).
constexpr int TAIL_BYTES = 16 + 16 * WARPS_PER_BLOCK;

template <int NPL, class SYN>
struct Layout {
  static constexpr int NT = 32 * NPL;
  static constexpr int NM = (NT + 63) / 64;
  static constexpr int o_l2 = 0;                                      // float[NT] |lambda| log2(e), by rank
  static constexpr int o_al = o_l2 + 4 * NT;                          // float[NT] |lambda|, by rank
  static constexpr int o_hr = o_al + 4 * NT;  // RankRec[NT + 1] H column + mass factor, by rank; [n] neutral
  static constexpr int o_cw = align16(o_hr + (int)sizeof(RankRec<SYN>) * (NT + 1));  // u64[LMAX][NM] listed codewords
  static constexpr int o_lp = o_cw + 8 * LMAX * NM;                   // float[LMAX] log p(z)/p(0)
  static constexpr int o_wl = o_lp + 4 * LMAX;                        // float[LMAX] APP of each listed word
  static constexpr int o_perm = o_wl + 4 * LMAX;                      // u8[NT] rank -> bit
  static constexpr int o_w = align16(o_perm + NT);                    // u64[NT][NM] words of a frame (check)
  // During a word the frame-check area is free: its first 32 bytes hold the
  // word's context (product kernels) and then float[NT] the word's lambda.
  // (A separate area would cost 1 KB per block, which moved the shared-memory
  // carveout of the 8-block schedule up a step and shrank L1 by a quarter.)
  static constexpr int o_lam = o_w + 32;
  static_assert(32 + 4 * NT + 4 * (NPL + 1) <= 8 * NT * NM, "lambda and the word head fit in the frame-check area");
  static constexpr int o_pf = align16(o_w + 8 * NT * NM);             // uint4[32] the next chunk of order entries
  static constexpr int warp_bytes = o_pf + 16 * 32;
  // block area (sized for the 8-byte XF policy): sfac[NT+1], fu[NT+1], fb[NT+1], ek[J] (float), he[J], ho[J]
  static __host__ __device__ int dp_bytes(int jm) { return align16(24 * (NT + 1) + 20 * jm + 32); }
  // a block of WARPS_PER_BLOCK warps: their areas, the tail and the remaining-mass area
  static __host__ __device__ int block_bytes(int jm) { return WARPS_PER_BLOCK * warp_bytes + TAIL_BYTES + dp_bytes(jm); }
};

// A warp's view of the block's scratch: its own area, the block's tail
// (lock word and tally slots, shared memory) and the block's remaining-mass
// area (shared or global memory).  Only the base addresses are kept; every
// array is a fixed offset from them.
template <int NPL, class SYN>
struct Scratch {
  using LY = Layout<NPL, SYN>;
  unsigned char *base;  // this warp's area
  unsigned char *dp;    // the block's remaining-mass area
  unsigned char *tl;    // the block's tail: lock word and poll limit, then the warps' tally slots
  __device__ void bind(unsigned char *warp_area, unsigned char *dp_area, unsigned char *tail_area) {
    base = warp_area;
    dp = dp_area;
    tl = tail_area;
  }
  __device__ float *l2() const { return reinterpret_cast<float *>(base + LY::o_l2); }
  __device__ float *al() const { return reinterpret_cast<float *>(base + LY::o_al); }
  __device__ RankRec<SYN> *hr() const { return reinterpret_cast<RankRec<SYN> *>(base + LY::o_hr); }
  __device__ uint64_t *cw() const { return reinterpret_cast<uint64_t *>(base + LY::o_cw); }
  __device__ float *lp() const { return reinterpret_cast<float *>(base + LY::o_lp); }
  __device__ float *wl() const { return reinterpret_cast<float *>(base + LY::o_wl); }
  __device__ uint8_t *perm() const { return base + LY::o_perm; }
  __device__ uint4 *pf() const { return reinterpret_cast<uint4 *>(base + LY::o_pf); }
  __device__ uint64_t *W() const { return reinterpret_cast<uint64_t *>(base + LY::o_w); }
  // lambda by bit, kept here during the search and read back (volatile) for
  // the soft output, so that it holds no registers while the search runs
  __device__ float *lamv() const { return reinterpret_cast<float *>(base + LY::o_lam); }
  __device__ float lam_at(int i) const { return *reinterpret_cast<const volatile float *>(base + LY::o_lam + 4 * i); }
  // the word's hard decision words (NPL) and 1-line parameter, after lambda
  __device__ unsigned *headv() const { return reinterpret_cast<unsigned *>(base + LY::o_lam + 4 * LY::NT); }
  __device__ unsigned head_at(int k) const { return *reinterpret_cast<const volatile unsigned *>(base + LY::o_lam + 4 * LY::NT + 4 * k); }
  __device__ unsigned char *tail() const { return dp; }
  __device__ int *lock() const { return reinterpret_cast<int *>(tl); }
  // this warp's tally slot: [0] summed pattern weights, [1] extended-range words
  __device__ unsigned long long *tally() const {
    return reinterpret_cast<unsigned long long *>(tl + 16) + 2 * (threadIdx.x >> 5);
  }
};

// The block's remaining-mass area is taken by one warp at a time.  Its holder
// runs a bounded computation that waits for nothing, so the wait ends; the
// bound (lock[1] polls, about 4 s by default) only keeps a broken state from
// spinning for ever: the warp then proceeds without the lock and reports it
// (returns false).
__device__ __forceinline__ bool dp_lock(int *lock, int lane) {
  int ok = 1;
  if (lane == 0) {
    unsigned nap = 32;
    long long tries = 0;
    const long long limit = *reinterpret_cast<volatile int *>(lock + 1);
    while (atomicCAS(lock, 0, 1) != 0) {
      if (++tries > limit) {
        ok = 0;
        break;
      }
      __nanosleep(nap);
      if (nap < 1024) nap <<= 1;
    }
  }
  ok = __shfl_sync(0xffffffffu, ok, 0);
  __threadfence_block();
  return ok != 0;
}
__device__ __forceinline__ void dp_unlock(int *lock, bool held, int lane) {
  __syncwarp();
  __threadfence_block();
  if (lane == 0 && held) atomicExch(lock, 0);
}

// ----------------------------------------------------------------------------
// warp helpers
// ----------------------------------------------------------------------------
// Bitonic sort of the warp's 32 * NPL keys, ascending, lane l holding sorted
// positions l NPL .. l NPL + NPL - 1 (blocked).  The exchanges at distance
// j < NPL stay inside a lane's registers, so fewer stages need shuffles (15
// of 21 for 64 keys, 15 of 28 for 128; 20 and 25 when lane l held positions
// l, l + 32, ...: 1-3% faster per word, most for 128-bit codes).  The stages
// run as loops rather than unrolled: the sort is straight-line work done once
// per word, and its unrolled form (about 20 stages of shuffles) made the
// kernel's code large enough that warps in other phases of their words
// stalled on instruction fetch (measured 4-10% slower for codes of 64 and 128
// bits).
template <int NPL>
__device__ __forceinline__ void warp_bitonic_sort_blocked(uint64_t (&v)[NPL], int lane) {
  constexpr int N = 32 * NPL;
#pragma unroll 1
  for (int size = 2; size <= N; size <<= 1) {
#pragma unroll 1
    for (int j = size >> 1; j >= NPL; j >>= 1) {
      const int lj = j / NPL;  // partner lane: lane ^ lj, same register
#pragma unroll
      for (int k = 0; k < NPL; k++) {
        const uint64_t o = __shfl_xor_sync(FULL, v[k], lj);
        const int p = lane * NPL + k;
        const bool asc = (p & size) == 0;
        const bool lower = (lane & lj) == 0;
        v[k] = (lower == asc) ? (v[k] < o ? v[k] : o) : (v[k] < o ? o : v[k]);
      }
    }
    if constexpr (NPL > 1) {
#pragma unroll
      for (int j = NPL / 2; j > 0; j >>= 1) {
        if (j <= (size >> 1)) {
#pragma unroll
          for (int k = 0; k < NPL; k++) {
            if ((k & j) == 0) {
              const int kp = k | j;
              const bool asc = ((lane * NPL + k) & size) == 0;
              const uint64_t a = v[k], b = v[kp];
              const bool sw = asc ? (a > b) : (a < b);
              v[k] = sw ? b : a;
              v[kp] = sw ? a : b;
            }
          }
        }
      }
    }
  }
}

__device__ __forceinline__ int64_t warp_sum_i64(int64_t x) {
#pragma unroll
  for (int d = 16; d > 0; d >>= 1) x += __shfl_xor_sync(FULL, x, d);
  return x;
}

__device__ __forceinline__ float warp_min_f(float x) {
#pragma unroll
  for (int d = 16; d > 0; d >>= 1) x = fminf(x, __shfl_xor_sync(FULL, x, d));
  return x;
}

// floor(v * 256 + 1/2) for v >= 0, saturating at 2^20 - 1.  Exact in FP32:
// v * 256 is a power-of-two scaling, and below the saturation point x + 1/2
// needs no rounding (x < 2^20 has an ulp of at most 2^-4).
__device__ __forceinline__ int64_t quant256(float v) {
  const float x = v * 256.f;
  if (!(x < 1048576.f)) return (1 << 20) - 1;
  return (int64_t)min((int)floorf(x + 0.5f), (1 << 20) - 1);
}

// 1-line ORBGRAND parameter: intercept/slope of the least-squares line through
// (r, a_r), r = 1..n, rounded half up, clamped to [0, c_max]; 0 if the slope
// is not positive.  All lanes get the same value.
__device__ __forceinline__ int one_line_c(int64_t sy, int64_t sxy, int n, int c_max) {
  int64_t sx = (int64_t)n * (n + 1) / 2;
  int64_t sxx = (int64_t)n * (n + 1) * (2 * n + 1) / 6;
  int64_t D = (int64_t)n * sxx - sx * sx;
  int64_t Nb = (int64_t)n * sxy - sx * sy;
  if (Nb <= 0) return 0;
  int64_t num = sy * D - Nb * sx;
  int64_t top = 2 * num + (int64_t)n * Nb;
  if (top < 0) return 0;
  // floor(top / den) clamped to c_max: an FP32 estimate (the hardware
  // reciprocal: a few ulp) corrected with exact integer products (the
  // quotient that matters is at most c_max <= 128)
  const int64_t den = 2 * (int64_t)n * Nb;
  if (top >= (int64_t)(c_max + 1) * den) return c_max;
  int64_t c = (int64_t)__fdividef((float)top, (float)den);
  c = c < 0 ? 0 : (c > c_max ? c_max : c);
  while (c > 0 && c * den > top) c--;
  while (c < c_max && (c + 1) * den <= top) c++;
  return (int)c;
}

// rank k (0-based position in the pattern) of a table entry: byte k + 1
template <int K>
__device__ __forceinline__ int ent_rank(const uint4 &e) {
  constexpr int B = K + 1;
  const unsigned wd = (B >> 2) == 0 ? e.x : (B >> 2) == 1 ? e.y : (B >> 2) == 2 ? e.z : e.w;
  return (wd >> (8 * (B & 3))) & 0xff;
}

// XOR of the rank-ordered H columns of a pattern and its mass relative to
// p(0), the product of its ranks' factors, in double-float (0 for the zero
// pattern).  The loop runs to the warp's largest weight; a shorter pattern's
// extra bytes name the neutral record hr[n] (H column 0, factor 1: the XOR
// and the products are exact no-ops).  Ranks go in pairs: both records are
// loaded before either is used (two shared-memory loads in flight, half the
// branches), and the pair's second rank past the weight is the neutral
// record (2-3% faster than one rank at a time; fours were slower).
template <class SYN>
__device__ __forceinline__ SYN ent_syndrome(const uint4 &e, int w, int wmax, const RankRec<SYN> *hr, DF &mass) {
  SYN s = 0;
  float mh = 1.f, ml = 0.f;
  const auto mul = [&](float t) {
    const float p = __fmul_rn(mh, t);
    ml = fmaf(ml, t, fmaf(mh, t, -p));
    mh = p;
  };
#define SG_R2(K)                                       \
  if (K < wmax) {                                      \
    const RankRec<SYN> v0 = hr[ent_rank<K>(e)];        \
    const RankRec<SYN> v1 = hr[ent_rank<K + 1>(e)];    \
    s ^= v0.h ^ v1.h;                                  \
    mul(v0.t);                                         \
    mul(v1.t);                                         \
  }
  SG_R2(0) SG_R2(2) SG_R2(4) SG_R2(6) SG_R2(8) SG_R2(10) SG_R2(12)
#undef SG_R2
  if (14 < wmax) {
    const RankRec<SYN> v = hr[ent_rank<14>(e)];
    s ^= v.h;
    mul(v.t);
  }
  mass = w > 0 ? DF{mh, ml} : DF{0.f, 0.f};
  return s;
}

// sum over the pattern's ranks of a per-rank float
__device__ __forceinline__ float ent_sum(const uint4 &e, int w, const float *x) {
  float s = 0.f;
#define SG_S(K) \
  if (K < w) s += x[ent_rank<K>(e)];
  SG_S(0) SG_S(1) SG_S(2) SG_S(3) SG_S(4) SG_S(5) SG_S(6) SG_S(7)
  SG_S(8) SG_S(9) SG_S(10) SG_S(11) SG_S(12) SG_S(13) SG_S(14)
#undef SG_S
  return s;
}

// ----------------------------------------------------------------------------
// remaining mass: tail over cost > Cs (DP) + unqueried rest of level Cs
// ----------------------------------------------------------------------------
// Register form of the rank DP for Cs < 32 * SLOTS: lane l holds the head
// masses of cost j = 32 s + l (s < SLOTS) for both parities; the shift by
// d_e = e + 1 + c is a shuffle from lane (l - d) mod 32 plus a slot select.
template <class Ops, int SLOTS>
__device__ __forceinline__ void dp_regs(int Cs, int c, int R0, int cls, const typename Ops::T *sfac,
                                        const typename Ops::T *fu, const typename Ops::T *fb, const float *ek,
                                        typename Ops::T g_even, typename Ops::T g_odd, int lane,
                                        typename Ops::T &acc) {
  using T = typename Ops::T;
  constexpr bool SCALED = sizeof(T) == 4;
  T he[SLOTS], ho[SLOTS];
#pragma unroll
  for (int t = 0; t < SLOTS; t++) {
    he[t] = (t == 0 && lane == 0) ? Ops::one() : Ops::zero();
    ho[t] = Ops::zero();
  }
  for (int e = 0; e < R0; e++) {
    const int d = e + 1 + c;
    const T s = sfac[e];
    const T Fb = fb[e + 1];
    const T F1u = Ops::add(Ops::one(), fu[e + 1]);
    const int dq = d >> 5, dr = d & 31;
    const int src = (lane - dr) & 31;
    const int back = dq + (lane < dr ? 1 : 0);  // source slot = sl - back
    T she[SLOTS], sho[SLOTS];
#pragma unroll
    for (int t = 0; t < SLOTS; t++) {
      she[t] = Ops::shfl(he[t], src);
      sho[t] = Ops::shfl(ho[t], src);
    }
#pragma unroll
    for (int sl = 0; sl < SLOTS; sl++) {
      const int j = sl * 32 + lane;
      if (j <= Cs) {
        if (j > Cs - d) {
          T w = s;
          if constexpr (SCALED) w = Ops::mul(w, Ops::from_float(ek[j + d - Cs]));
          T term;
          if (cls == 0)
            term = Ops::add(Ops::mul(he[sl], Fb), Ops::mul(ho[sl], F1u));
          else if (cls == 1)
            term = Ops::add(Ops::mul(he[sl], F1u), Ops::mul(ho[sl], Fb));
          else
            term = Ops::mul(Ops::add(he[sl], ho[sl]), Ops::add(F1u, Fb));
          acc = Ops::fma(w, term, acc);
        }
        if (j >= d) {
          const int ss = sl - back;
          T pe = Ops::zero(), po = Ops::zero();
#pragma unroll
          for (int t = 0; t < SLOTS; t++)
            if (t == ss) {
              pe = she[t];
              po = sho[t];
            }
          he[sl] = Ops::fma(s, po, he[sl]);
          ho[sl] = Ops::fma(s, pe, ho[sl]);
        }
      }
    }
#ifdef SG_PHASE_PROFILE
    if (lane == 0) SG_PROF(7, 1);
#endif
  }
  // high ranks (d_e > Cs) joined to every head pattern
#pragma unroll
  for (int sl = 0; sl < SLOTS; sl++) {
    const int j = sl * 32 + lane;
    if (j <= Cs) {
      T w = Ops::one();
      if constexpr (SCALED) w = Ops::from_float(ek[j]);
      T term;
      if (cls == 0)
        term = Ops::add(Ops::mul(he[sl], g_even), Ops::mul(ho[sl], g_odd));
      else if (cls == 1)
        term = Ops::add(Ops::mul(he[sl], g_odd), Ops::mul(ho[sl], g_even));
      else
        term = Ops::mul(Ops::add(he[sl], ho[sl]), Ops::add(g_even, g_odd));
      acc = Ops::fma(w, term, acc);
    }
  }
}

// Shared-memory form of the same DP for large stop levels (out of line: rare).
template <class Ops>
__device__ __noinline__ void dp_smem(int Cs, int c, int R0, int cls, const typename Ops::T *sfac, const typename Ops::T *fu,
                        const typename Ops::T *fb, const float *ek, typename Ops::T g_even, typename Ops::T g_odd,
                        typename Ops::T *he, typename Ops::T *ho, int lane, typename Ops::T &acc) {
  using T = typename Ops::T;
  constexpr bool SCALED = sizeof(T) == 4;
  for (int j = lane; j <= Cs; j += 32) {
    he[j] = j == 0 ? Ops::one() : Ops::zero();
    ho[j] = Ops::zero();
  }
  __syncwarp();
  const int nslot = (Cs + 32) >> 5;
  for (int e = 0; e < R0; e++) {
    const int d = e + 1 + c;
    const T s = sfac[e];
    const T Fb = fb[e + 1];
    const T F1u = Ops::add(Ops::one(), fu[e + 1]);
    // slots from the top, so every read of he/ho[j - d] sees the values
    // before this rank (a slot's reads are separated from its writes)
    for (int sl = nslot - 1; sl >= 0; sl--) {
      const int j = sl * 32 + lane;
      T ne = Ops::zero(), no = Ops::zero();
      const bool inr = j <= Cs;
      const bool upd = inr && j >= d;
      if (inr) {
        const T hej = he[j], hoj = ho[j];
        if (j > Cs - d) {
          T w = s;
          if constexpr (SCALED) w = Ops::mul(w, Ops::from_float(ek[j + d - Cs]));
          T term;
          if (cls == 0)
            term = Ops::add(Ops::mul(hej, Fb), Ops::mul(hoj, F1u));
          else if (cls == 1)
            term = Ops::add(Ops::mul(hej, F1u), Ops::mul(hoj, Fb));
          else
            term = Ops::mul(Ops::add(hej, hoj), Ops::add(F1u, Fb));
          acc = Ops::fma(w, term, acc);
        }
        if (upd) {
          ne = Ops::fma(s, ho[j - d], hej);
          no = Ops::fma(s, he[j - d], hoj);
        }
      }
      __syncwarp();
      if (upd) {
        he[j] = ne;
        ho[j] = no;
      }
      __syncwarp();
    }
  }
  for (int j = lane; j <= Cs; j += 32) {
    T w = Ops::one();
    if constexpr (SCALED) w = Ops::from_float(ek[j]);
    T term;
    if (cls == 0)
      term = Ops::add(Ops::mul(he[j], g_even), Ops::mul(ho[j], g_odd));
    else if (cls == 1)
      term = Ops::add(Ops::mul(he[j], g_odd), Ops::mul(ho[j], g_even));
    else
      term = Ops::mul(Ops::add(he[j], ho[j]), Ops::add(g_even, g_odd));
    acc = Ops::fma(w, term, acc);
  }
  __syncwarp();
}

// The (scaled) remaining mass summed over the warp.  With FOps every mass
// carries the factor 2^(g2 * Cs) (g2 = gamma log2 e); with XOps g2 = 0.
// `qs` is the order-table index of the last queried pattern.
template <class Ops, int NPL, class SYN>
__device__ __noinline__ typename Ops::T remaining_scaled(const Scratch<NPL, SYN> &sc, const DevOrder &O, int tb, int tc, int qs,
                                            int n, int c, int cls, int Cs, float g2, int lane) {
  using T = typename Ops::T;
  constexpr int NT = 32 * NPL;
  T *sfac = reinterpret_cast<T *>(sc.tail());
  T *fu = sfac + NT + 1;
  T *fb = fu + NT + 1;
  float *ek = reinterpret_cast<float *>(fb + NT + 1);
  T *he = reinterpret_cast<T *>(ek + align16(4 * (Cs + 1)) / 4);
  T *ho = he + (Cs + 1);
  constexpr bool SCALED = sizeof(T) == 4;
  const int R0 = min(max(Cs - c, 0), n);  // ranks e < R0 can sit inside a pattern of cost <= Cs
  const float g2Cs = g2 * (float)Cs;

  // --- unqueried rest of level Cs (the table stores every level completely)
  T acc = Ops::zero();
  for (int q0 = qs + 1; q0 < tc; q0 += 32) {
    const int q = q0 + lane;
    bool in = false;
    if (q < tc) in = __ldg(O.cost + tb + q) == (uint16_t)Cs;
    if (in) {
      const uint4 e = __ldg(O.ent + tb + q);
      const float s2 = ent_sum(e, e.x & 0xff, sc.l2());
      acc = Ops::add(acc, Ops::from_log2(g2Cs - s2));
    }
    if (!__all_sync(FULL, in)) break;  // costs are nondecreasing
  }

  // --- per-rank factors and suffix products F_e = prod_{e' >= e} (1 + y t_e')
  //     kept as (u, b) = (even part - 1, odd part); lanes own ranks
  //     lane*NPL .. lane*NPL+NPL-1.
  {
    T lu[NPL], lb[NPL];
    T u = Ops::zero(), b = Ops::zero();
#pragma unroll
    for (int k = NPL - 1; k >= 0; k--) {
      const int e = lane * NPL + k;
      T t = Ops::zero();
      if (e < n) {
        t = Ops::from_log2(-sc.l2()[e]);
        // factor used by the tail: low ranks t * 2^(g2 d_e), high ranks t * 2^(g2 Cs)
        const float d = (float)(e + 1 + c);
        sfac[e] = Ops::from_log2((e < R0 ? g2 * d : g2Cs) - sc.l2()[e]);
      }
      const T nu = Ops::fma(b, t, u);
      const T nb = Ops::fma(u, t, Ops::add(b, t));
      u = nu;
      b = nb;
      lu[k] = u;
      lb[k] = b;
    }
    T su = u, sb = b;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      const T ou = Ops::shfl_down(su, d), ob = Ops::shfl_down(sb, d);
      if (lane + d < 32) {
        const T nu = Ops::add(Ops::add(su, ou), Ops::fma(su, ou, Ops::mul(sb, ob)));
        const T nb = Ops::add(Ops::add(sb, ob), Ops::fma(su, ob, Ops::mul(sb, ou)));
        su = nu;
        sb = nb;
      }
    }
    T xu = Ops::shfl_down(su, 1), xb = Ops::shfl_down(sb, 1);
    if (lane == 31) {
      xu = Ops::zero();
      xb = Ops::zero();
    }
#pragma unroll
    for (int k = 0; k < NPL; k++) {
      const int e = lane * NPL + k;
      if (e < n) {
        fu[e] = Ops::add(Ops::add(lu[k], xu), Ops::fma(lu[k], xu, Ops::mul(lb[k], xb)));
        fb[e] = Ops::add(Ops::add(lb[k], xb), Ops::fma(lu[k], xb, Ops::mul(lb[k], xu)));
      }
    }
    if (lane == 0) {
      fu[n] = Ops::zero();
      fb[n] = Ops::zero();
    }
  }
  if constexpr (SCALED)
    for (int j = lane; j <= Cs; j += 32) ek[j] = exp2f(-g2 * (float)j);
  __syncwarp();

  // --- high ranks (d_e > Cs): G_P = sum_e sfac_e * F_{e+1} (parity of the
  //     pattern {e} + any higher subset), reduced over the warp
  T g_even = Ops::zero(), g_odd = Ops::zero();
  for (int e = R0 + lane; e < n; e += 32) {
    const T s = sfac[e];
    g_odd = Ops::fma(s, Ops::add(Ops::one(), fu[e + 1]), g_odd);
    g_even = Ops::fma(s, fb[e + 1], g_even);
  }
#pragma unroll
  for (int d = 16; d > 0; d >>= 1) {
    g_even = Ops::add(g_even, Ops::shfl_xor(g_even, d));
    g_odd = Ops::add(g_odd, Ops::shfl_xor(g_odd, d));
  }

  // --- low ranks in ascending order: tail contributions and the cost DP
  bool done = false;
  if constexpr (SCALED) {
    if (Cs < 64) {
      dp_regs<Ops, 2>(Cs, c, R0, cls, sfac, fu, fb, ek, g_even, g_odd, lane, acc);
      done = true;
    } else if (Cs < 128) {
      dp_regs<Ops, 4>(Cs, c, R0, cls, sfac, fu, fb, ek, g_even, g_odd, lane, acc);
      done = true;
    }
  }
  if (!done) {
#ifdef SG_PHASE_PROFILE
    if (lane == 0) SG_PROF(9, 1);
#endif
    dp_smem<Ops>(Cs, c, R0, cls, sfac, fu, fb, ek, g_even, g_odd, he, ho, lane, acc);
  }
#pragma unroll
  for (int d = 16; d > 0; d >>= 1) acc = Ops::add(acc, Ops::shfl_xor(acc, d));
  __syncwarp();
  return acc;
}

// Extended-range evaluation (out of line: only when every FP32-scaled term
// of the dominant part underflows).
template <int NPL, class SYN>
__device__ __noinline__ float remaining_log2_xf(const Scratch<NPL, SYN> &sc, const DevOrder &O, int tb, int tc, int qs,
                                                int n, int c, int cls, int Cs, int lane) {
  const XF x = remaining_scaled<XOps, NPL, SYN>(sc, O, tb, tc, qs, n, c, cls, Cs, 0.f, lane);
  return __shfl_sync(FULL, xf_log2(x), 0);
}

// Class total of the nonzero patterns in double-float: prod_e (1 + y t_e) as
// (even part - 1, odd part), lanes own ranks lane*NPL .. lane*NPL+NPL-1, then
// a butterfly over the warp; lane 0's result is broadcast.  Every term is
// nonnegative, so the additions need no cancellation handling.
template <int NPL, class SYN>
__device__ __noinline__ DF class_total_df(const Scratch<NPL, SYN> &sc, int n, int cls, int lane) {
  DF u = {0.f, 0.f}, b = {0.f, 0.f};
#pragma unroll
  for (int k = 0; k < NPL; k++) {
    const int e = lane * NPL + k;
    if (e < n) {
      const float t = sc.hr()[e].t;
      const DF nu = df_add_pos(u, df_mul_f(b, t));
      const DF nb = df_add_pos(df_add_pos(b, DF{t, 0.f}), df_mul_f(u, t));
      u = nu;
      b = nb;
    }
  }
#pragma unroll 1
  for (int d = 16; d > 0; d >>= 1) {
    const DF ou = {__shfl_xor_sync(FULL, u.h, d), __shfl_xor_sync(FULL, u.l, d)};
    const DF ob = {__shfl_xor_sync(FULL, b.h, d), __shfl_xor_sync(FULL, b.l, d)};
    const DF nu = df_add_pos(df_add_pos(u, ou), df_add_pos(df_mul(u, ou), df_mul(b, ob)));
    const DF nb = df_add_pos(df_add_pos(b, ob), df_add_pos(df_mul(u, ob), df_mul(b, ou)));
    u = nu;
    b = nb;
  }
  const DF E = cls == 0 ? u : (cls == 1 ? b : df_add_pos(u, b));
  return {__shfl_sync(FULL, E.h, 0), __shfl_sync(FULL, E.l, 0)};
}

// The unqueried patterns summed directly: the cost DP of remaining_scaled
// under the block's lock.  Out of line: the DP runs for 0.04-0.9% of the
// component words, and as a call it keeps the two call sites of
// remaining_log2 short (1-1.5% faster than inline for eBCH(32,26), (64,51)
// and (128,120) at 7 blocks per SM; within 1% for eBCH(64,57)).
template <int NPL, class SYN>
__device__ __noinline__ float remaining_log2_dp(const Scratch<NPL, SYN> &sc, const DevOrder &O, int tb, int tc,
                                                int qs, int n, int c, int cls, int lane, int *used_xf) {
#ifdef SG_PHASE_PROFILE
  if (lane == 0) SG_PROF(6, 1);
#endif
  const int Cs = __ldg(O.cost + tb + qs);
  const int R0 = min(max(Cs - c, 0), n);
  float g = CUDART_INF_F;
  for (int e = lane; e < R0; e += 32) g = fminf(g, sc.l2()[e] / (float)(e + 1 + c));
  g = __shfl_sync(FULL, warp_min_f(g), 0);
  if (!(g < CUDART_INF_F)) g = 0.f;
  const bool held = dp_lock(sc.lock(), lane);
  float out;
  const float tot = __shfl_sync(FULL, remaining_scaled<FOps, NPL, SYN>(sc, O, tb, tc, qs, n, c, cls, Cs, g, lane), 0);
  if (tot >= 0x1p-60f && tot < CUDART_INF_F) {
    out = log2f(tot) - g * (float)Cs;
  } else {
    if (used_xf) *used_xf |= 1;
#ifdef SG_PHASE_PROFILE
    if (lane == 0) SG_PROF(8, 1);
#endif
    out = remaining_log2_xf<NPL, SYN>(sc, O, tb, tc, qs, n, c, cls, Cs, lane);
  }
  dp_unlock(sc.lock(), held, lane);
  if (!held && used_xf) *used_xf |= 2;
  return out;
}

// log2 of the remaining (unqueried) mass relative to p(0^n|r); warp-uniform.
// *used_xf (if given) gets bit 0 when the extended-range sum was needed and
// bit 1 when the block's remaining-mass area could not be locked.
// tq is the queried mass of the nonzero patterns (double-float, summed over
// the warp, the same value in every lane).  The class total minus tq is used
// when it is well conditioned: in FP32 when the difference is at least 2% of
// the operands (FP32 rounding of about 4e-6 of them moves it by at most 2e-4
// relative), in double-float when it is at least 2^-26 of them (rounding of a
// few 2^-46 moves it by at most about 1e-5 relative).  Otherwise the
// unqueried patterns are summed directly.
template <int NPL, class SYN>
__device__ float remaining_log2(const Scratch<NPL, SYN> &sc, const DevOrder &O, int tb, int tc, int qs, int n, int c,
                                int cls, int lane, DF tq, int *used_xf) {
  // class total of the nonzero patterns: prod_e (1 + y t_e) as (even - 1, odd)
  {
    float u = 0.f, b = 0.f;
#pragma unroll
    for (int k = 0; k < NPL; k++) {
      const int e = lane * NPL + k;
      if (e < n) {
        const float t = sc.hr()[e].t;
        const float nu = fmaf(b, t, u), nb = fmaf(u, t, b + t);
        u = nu;
        b = nb;
      }
    }
#pragma unroll 1
    for (int d = 16; d > 0; d >>= 1) {
      const float ou = __shfl_xor_sync(FULL, u, d), ob = __shfl_xor_sync(FULL, b, d);
      const float nu = (u + ou) + fmaf(u, ou, b * ob);
      const float nb = (b + ob) + fmaf(u, ob, b * ou);
      u = nu;
      b = nb;
    }
    // the butterfly's fused products round differently per lane: take lane
    // 0's value so the branch below is warp-uniform
    u = __shfl_sync(FULL, u, 0);
    b = __shfl_sync(FULL, b, 0);
    const float enz = cls == 0 ? u : (cls == 1 ? b : u + b);
    const float tqf = tq.h + tq.l;
    const float r = enz - tqf;
    const bool in_range = enz > 0x1p-60f && enz < 0x1p60f;
    // the hardware log2 (about 2^-22 relative): far inside the soft output's tolerance
    if (in_range && r > 0.02f * (enz + tqf)) return __log2f(r);
    if (in_range) {
      const DF E = class_total_df<NPL, SYN>(sc, n, cls, lane);
      const DF R = df_add(E, DF{-tq.h, -tq.l});
#ifdef SG_PHASE_PROFILE
      if (lane == 0) SG_PROF(R.h > 0x1p-26f * (E.h + tq.h) ? 12 : 13, 1);
#endif
      if (R.h > 0x1p-26f * (E.h + tq.h)) return __log2f(R.h + R.l);
    }
#ifdef SG_PHASE_PROFILE
    if (!in_range && lane == 0) SG_PROF(15, 1);
#endif
  }
  return remaining_log2_dp<NPL, SYN>(sc, O, tb, tc, qs, n, c, cls, lane, used_xf);
}

// numerically safe log(exp(a) + exp(b)) (natural log, -inf aware)
__device__ __forceinline__ float lse(float a, float b) {
  const float mx = fmaxf(a, b), mn = fminf(a, b);
  if (mx == -CUDART_INF_F) return mx;
  return mx + log1pf(expf(mn - mx));
}
__device__ __forceinline__ float softplus(float z) { return fmaxf(z, 0.f) + log1pf(expf(-fabsf(z))); }

// ----------------------------------------------------------------------------
// one word
// ----------------------------------------------------------------------------
template <int NPL, class SYN>
struct WordHead {
  unsigned yb[NPL];  // hard decision, bits lane + 32k
  int par;           // parity of y
  SYN s0;            // syndrome of y
  int c;             // 1-line parameter
};

// Hard decision, parity, syndrome of y, reliability ranks (scratch al/l2/
// perm/hs) and the 1-line parameter.  Returns false (and leaves the head
// undefined) if any input is not finite.
template <int NPL, class SYN>
__device__ bool siso_prologue(const DevCode &code, const Scratch<NPL, SYN> &sc, const float (&lam)[NPL], int lane,
                              WordHead<NPL, SYN> &h) {
  const int n = code.n;
  bool bad = false;
#pragma unroll
  for (int k = 0; k < NPL; k++)
    if (lane + 32 * k < n && !isfinite(lam[k])) bad = true;
  if (__any_sync(FULL, bad)) return false;

  int par = 0;
  SYN s0p = 0;
#pragma unroll
  for (int k = 0; k < NPL; k++) {
    const int i = lane + 32 * k;
    const bool one = (i < n) && lam[k] < 0.f;  // lambda = 0 -> bit 0
    h.yb[k] = __ballot_sync(FULL, one);
    par ^= __popc(h.yb[k]) & 1;
    if (one) s0p ^= (SYN)__ldg(code.hcol + i);
  }
  h.par = par;
  if (sizeof(SYN) == 4) {
    h.s0 = (SYN)__reduce_xor_sync(FULL, (unsigned)s0p);
  } else {
    const unsigned lo_ = __reduce_xor_sync(FULL, (unsigned)(uint64_t)s0p);
    const unsigned hi_ = __reduce_xor_sync(FULL, (unsigned)((uint64_t)s0p >> 32));
    h.s0 = (SYN)(((uint64_t)hi_ << 32) | lo_);
  }

  // reliability ranks: sort (|lambda|, index) ascending
  uint64_t key[NPL];
#pragma unroll
  for (int k = 0; k < NPL; k++) {
    const int i = lane + 32 * k;
    key[k] = i < n ? (((uint64_t)__float_as_uint(fabsf(lam[k])) << 32) | (uint64_t)i) : ~0ull;
  }
  warp_bitonic_sort_blocked<NPL>(key, lane);
  int64_t sy = 0, sxy = 0;
#pragma unroll
  for (int k = 0; k < NPL; k++) {
    const int e = lane * NPL + k;  // sorted position (blocked layout)
    if (e < n) {
      const float a = __uint_as_float((unsigned)(key[k] >> 32));
      const int idx = (int)(key[k] & 0xffffffffu);
      const float l2v = __fmul_rn(a, LOG2E_F);
      sc.al()[e] = a;
      sc.l2()[e] = l2v;
      sc.perm()[e] = (uint8_t)idx;
      sc.hr()[e] = RankRec<SYN>{(SYN)__ldg(code.hcol + idx), exp2f(-l2v)};
      const int64_t qa = quant256(a);
      sy += qa;
      sxy += qa * (e + 1);
    }
  }
  // sy < 2^27 fits one 32-bit reduction; sxy < 2^34 is split at bit 24
  sy = (int64_t)__reduce_add_sync(FULL, (unsigned)sy);
  sxy = ((int64_t)__reduce_add_sync(FULL, (unsigned)(sxy >> 24)) << 24) +
        (int64_t)__reduce_add_sync(FULL, (unsigned)(sxy & 0xffffff));
  h.c = one_line_c(sy, sxy, n, code.c_max);
  if (lane == 0) sc.hr()[n] = RankRec<SYN>{(SYN)0, 1.f};  // neutral record for unused entry bytes
  __syncwarp();
  return true;
}

// rank mask (bit r = rank r + 1) of a table entry
template <int NM>
__device__ __forceinline__ void ent_mask(const uint4 &e, uint64_t (&m)[NM]) {
  const int w = e.x & 0xff;
#pragma unroll
  for (int x = 0; x < NM; x++) m[x] = 0;
#define SG_M(K)                                           \
  if (K < w) {                                            \
    const int r = ent_rank<K>(e);                         \
    _Pragma("unroll") for (int x = 0; x < NM; x++) {      \
      if ((r >> 6) == x) m[x] |= 1ull << (r & 63);        \
    }                                                     \
  }
  SG_M(0) SG_M(1) SG_M(2) SG_M(3) SG_M(4) SG_M(5) SG_M(6) SG_M(7)
  SG_M(8) SG_M(9) SG_M(10) SG_M(11) SG_M(12) SG_M(13) SG_M(14)
#undef SG_M
}

// ----------------------------------------------------------------------------
// the query order enumerated by the lanes (instead of read from the table)
// ----------------------------------------------------------------------------
// 1-line ORBGRAND (Sec. III-B) queries the patterns in order of cost = sum of
// ranks + c * weight; the patterns of one cost and weight w are the
// partitions of m = cost - c w into w distinct parts <= n (rank sets), taken
// in lexicographic order of the ascending rank vector.  Pattern o of such a
// group is found part by part: with the parts so far summing to m - m', wl
// parts left and each part above the last one (at least a0), part a is taken
// if o is below the number of ways to finish after it, and otherwise o drops
// by that number and a grows.  The ways to finish after a are the
// (wl - 1)-subsets of {a+1..n} with sum m' - a, i.e. (subtracting a from
// each) the (wl - 1)-subsets of {1..n-a} with sum m' - wl a, read from the
// table of subset counts.  The last two parts follow in closed form: the
// pairs {a, m' - a} in order of a, from max(a0, m' - n).  The pattern is
// written as a table entry (weight byte, 0-based rank bytes, n in the unused
// bytes) into the lane's 16-byte slot and read back.
__device__ __forceinline__ uint4 unrank_entry(const int32_t *scnt, int sc_w, int sc_m, int n, int w, int m, int o,
                                              uint4 *slot) {
  unsigned char *b = reinterpret_cast<unsigned char *>(slot);
  const unsigned nn = (unsigned)n * 0x01010101u;
  *slot = make_uint4((nn & ~0xffu) | (unsigned)w, nn, nn, nn);
  int lo = 1;
#pragma unroll 1
  for (int i = 0; i < w - 2; i++) {
    const int wl = w - i;
    int a = lo;
#pragma unroll 1
    for (; a < n; a++) {  // bounded: for an index inside the group the count is reached by a = n - 1
      const int mm = m - wl * a;
      const int cnt = mm < 0 ? 0 : __ldg(scnt + ((n - a) * sc_w + (wl - 1)) * sc_m + mm);
      if (o < cnt) break;
      o -= cnt;
    }
    b[1 + i] = (unsigned char)(a - 1);
    m -= a;
    lo = a + 1;
  }
  // (the clamps keep every rank byte a valid record index, n the neutral one,
  // whatever the arguments; for an offset inside its group they change nothing)
  if (w >= 2) {
    const int a = max(lo, m - n) + o;
    b[w - 1] = (unsigned char)min(max(a - 1, 0), n);
    b[w] = (unsigned char)min(max(m - a - 1, 0), n);
  } else if (w == 1) {
    b[1] = (unsigned char)min(max(m - 1, 0), n);
  }
  return *slot;
}

// The group window of the lane-enumerated order: the group holding query q
// (warp-uniform: its index g, start gx and record gy) and, for a chunk of 32
// queries q .. q + 31, each lane's group and its offset there, from one
// coalesced load of the next 32 group records (group starts after q are at
// least q + 1, and at most 32 of them fall in q + 1 .. q + 32) and a bit mask
// of the groups that start inside the chunk.  Order (c, class) owns groups
// g0 .. ge - 1.
struct GroupWindow {
  const uint2 *grp;
  int g, ge;
  unsigned gx, gy;
  __device__ __forceinline__ void init(const uint2 *grp_, int g0, int ge_) {
    grp = grp_;
    g = g0;
    ge = ge_;
    gx = 0u;
    gy = g < ge ? __ldg(&grp[g].y) : 0u;
  }
  // lane's pattern for query q + lane (an empty entry for lane >= lim), then
  // the window moves on to the group holding q + 32
  __device__ __forceinline__ uint4 chunk(int q, int lim, int lane, const int32_t *scnt, int sc_w, int sc_m, int n,
                                         uint4 *slot) {
    const int gi = g + 1 + lane;
    const uint2 r = gi < ge ? __ldg(grp + gi) : make_uint2(0x7fffffffu, 0u);
    const int d = (int)r.x - q;
    const unsigned starts = __reduce_or_sync(FULL, d < 32 ? 1u << d : 0u);  // groups starting in the chunk
    const unsigned upto = lane == 31 ? 0xffffffffu : ((2u << lane) - 1u);
    const int rg = __popc(starts & upto);  // groups started after q and at or before q + lane
    const unsigned sx = __shfl_sync(FULL, r.x, rg > 0 ? rg - 1 : 0);
    const unsigned sy = __shfl_sync(FULL, r.y, rg > 0 ? rg - 1 : 0);
    const unsigned my = rg > 0 ? sy : gy;
    const int mo = q + lane - (int)(rg > 0 ? sx : gx);
    uint4 e = make_uint4(0u, 0u, 0u, 0u);
    if (lane < lim) e = unrank_entry(scnt, sc_w, sc_m, n, (int)(my >> 16), (int)(my & 0xffffu), mo, slot);
    const int adv = __popc(__ballot_sync(FULL, d <= 32));
    if (adv > 0) {
      gx = __shfl_sync(FULL, r.x, adv - 1);
      gy = __shfl_sync(FULL, r.y, adv - 1);
      g += adv;
    }
    return e;
  }
};

// The canonical query order for one input (test hook): writes the first
// max_q rank masks (NM words each); returns how many were written.
template <int NPL, class SYN>
__device__ int trace_word(const DevCode &code, const Scratch<NPL, SYN> &sc, const float (&lam)[NPL], int lane,
                          int max_q, uint64_t *out, int *c_out) {
  constexpr int NM = (32 * NPL + 63) / 64;
  WordHead<NPL, SYN> h;
  if (!siso_prologue<NPL, SYN>(code, sc, lam, lane, h)) return -1;
  const DevOrder &O = code.ord;
  const int ti = h.c * O.ncls + (code.even ? h.par : 0);
  const int tb = __ldg(O.base + ti), tc = __ldg(O.count + ti);
  const int qn = min(max_q, tc);
  if (code.ord_lanes) {  // the order as the lanes enumerate it
    GroupWindow W;
    W.init(code.grp.grp, __ldg(code.grp.gbase + ti), __ldg(code.grp.gbase + ti + 1));
    for (int q0 = 0; q0 < qn; q0 += 32) {
      const uint4 e = W.chunk(q0, min(32, qn - q0), lane, code.grp.scnt, code.grp.sc_w, code.grp.sc_m, code.n,
                              sc.pf() + lane);
      if (q0 + lane < qn) {
        uint64_t m[NM];
        ent_mask<NM>(e, m);
#pragma unroll
        for (int x = 0; x < NM; x++) out[(size_t)(q0 + lane) * NM + x] = m[x];
      }
    }
  } else {
    for (int q = lane; q < qn; q += 32) {
      uint64_t m[NM];
      ent_mask<NM>(__ldg(O.ent + tb + q), m);
#pragma unroll
      for (int x = 0; x < NM; x++) out[(size_t)q * NM + x] = m[x];
    }
  }
  if (c_out && lane == 0) *c_out = h.c;
  return qn;
}

__device__ __forceinline__ float warp_sum_f(float x) {
#pragma unroll
  for (int d = 16; d > 0; d >>= 1) x += __shfl_xor_sync(FULL, x, d);
  return x;
}

// Record the hit of lane hl as list entry `slot`: the codeword y + z in bit
// order (sc.cw()) and log p(z)/p(0) = -sum |lambda| over z (sc.lp()).  The
// pattern is broadcast and lane k handles its k-th rank.
template <int NPL, class SYN>
__device__ __forceinline__ void record_hit(const Scratch<NPL, SYN> &sc, const WordHead<NPL, SYN> &h, const uint4 &e,
                                           int hl, int slot, int lane) {
  constexpr int NM = (32 * NPL + 63) / 64;
  uint4 b;
  b.x = __shfl_sync(FULL, e.x, hl);
  b.y = __shfl_sync(FULL, e.y, hl);
  b.z = __shfl_sync(FULL, e.z, hl);
  b.w = __shfl_sync(FULL, e.w, hl);
  const int w = b.x & 0xff;
  const int byte = lane + 1;  // rank k = lane sits in byte k + 1
  const unsigned wd = byte < 4 ? b.x : (byte < 8 ? b.y : (byte < 12 ? b.z : b.w));
  const bool mine = lane < w;
  const int r = mine ? (wd >> (8 * (byte & 3))) & 0xff : 0;
  const float ls = warp_sum_f(mine ? sc.al()[r] : 0.f);
  const int bi = mine ? sc.perm()[r] : 0;
#pragma unroll
  for (int k = 0; k < NPL; k++) {
    const unsigned word = __reduce_or_sync(FULL, (mine && (bi >> 5) == k) ? 1u << (bi & 31) : 0u) ^ sc.head_at(k);
    if (lane == 0) reinterpret_cast<unsigned *>(sc.cw() + slot * NM)[k] = word;
  }
  if (lane == 0) {
    if (NPL & 1) reinterpret_cast<unsigned *>(sc.cw() + slot * NM)[NPL] = 0u;  // upper half of the last u64
    sc.lp()[slot] = -ls;
  }
  __syncwarp();
}

// threshold rule: predicted probability that the list misses the codeword
__device__ __forceinline__ bool thr_reached(const float *lp, int nhit, float M, float thr) {
  float D = M;
  for (int l = 0; l < nhit; l++) D = lse(D, lp[l]);
  return expf(M - D) < thr;
}
template <int NPL, class SYN>
__device__ __forceinline__ bool thr_reached(const Scratch<NPL, SYN> &sc, int nhit, float M, float thr) {
  return thr_reached(sc.lp(), nhit, M, thr);
}

// eq. LLRi in the log domain for a bit whose linear sums underflowed (out of line: rare)
template <int NPL, class SYN>
__device__ __noinline__ float lapp_logdomain(const Scratch<NPL, SYN> &sc, int nhit, float M, float x, int i) {
  constexpr int NM = (32 * NPL + 63) / 64;
  float b0 = M - softplus(-x), b1 = M - softplus(x);
  const uint64_t bitm = 1ull << (i & 63);
  for (int l = 0; l < nhit; l++) {
    if (sc.cw()[l * NM + (i >> 6)] & bitm)
      b1 = lse(b1, sc.lp()[l]);
    else
      b0 = lse(b0, sc.lp()[l]);
  }
  return b0 - b1;
}

// The query loop when no threshold rule applies (thr = 0), out of line: its
// register allocation is its own, not shaped by the rest of the word (inline,
// the loop shared the word's registers and spilled; out of line it needs
// none, and decoding is 4-26% faster across the codes, most for the
// loop-bound eBCH(64,51)).  Same steps as the general loop in siso_word
// below: chunks of 32 queries, each lane's next entry copied ahead by
// cp.async, syndromes and double-float masses of the patterns, hits kept in
// query order until L codewords are listed or the cap is reached.
struct LoopOut {
  int q, nhit, wacc;
  DF tmass;
};
template <int NPL, class SYN>
__device__ __noinline__ LoopOut query_loop_plain(const Scratch<NPL, SYN> sc, const WordHead<NPL, SYN> &h,
                                                 const uint4 *ent, int qlim, int L, int lane) {
  int q = 0, nhit = 0, wacc = 0;
  DF tmass = {0.f, 0.f};
#ifdef SG_PHASE_PROFILE
  int nchunks = 0;
#endif
  const unsigned pf_addr = (unsigned)__cvta_generic_to_shared(sc.pf() + lane);
  if (lane < qlim) asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(pf_addr), "l"(ent + lane) : "memory");
  asm volatile("cp.async.commit_group;" ::: "memory");
  for (;;) {
    const int lim = min(32, qlim - q);
    if (lim <= 0) break;
#ifdef SG_PHASE_PROFILE
    nchunks++;
#endif
    uint4 e = make_uint4(0u, 0u, 0u, 0u);
    asm volatile("cp.async.wait_all;" ::: "memory");
    if (lane < lim) e = sc.pf()[lane];
    if (q + 32 + lane < qlim)
      asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(pf_addr), "l"(ent + q + 32 + lane) : "memory");
    asm volatile("cp.async.commit_group;" ::: "memory");
    const int w = e.x & 0xff;
    const int wmax = (int)__reduce_max_sync(FULL, (unsigned)w);
    DF mass;
    const SYN s = ent_syndrome<SYN>(e, w, wmax, sc.hr(), mass) ^ h.s0;
    const bool hit = lane < lim && s == 0;
    unsigned hm = __ballot_sync(FULL, hit);
    int stop_lane = -1;
    while (hm) {
      const int hl = __ffs(hm) - 1;
      hm &= hm - 1;
      record_hit<NPL, SYN>(sc, h, e, hl, nhit, lane);
      nhit++;
      if (nhit >= L) {
        stop_lane = hl;
        break;
      }
    }
    if (stop_lane >= 0) {
      if (lane <= stop_lane) {
        wacc += w;
        df_acc(tmass, mass);
      }
      q += stop_lane + 1;
      break;
    }
    wacc += w;
    df_acc(tmass, mass);
    q += lim;
  }
  asm volatile("cp.async.wait_all;" ::: "memory");
#ifdef SG_PHASE_PROFILE
  if (lane == 0) SG_PROF(5, nchunks);
#endif
  return LoopOut{q, nhit, wacc, tmass};
}

// The thr = 0 query loop with the order enumerated by the lanes: the same
// chunks of 32 queries, syndromes, masses and hit recording as
// query_loop_plain; lane j finds the group of query q0 + j from the group
// starts of the chunk (one coalesced load of the next 32 group records, a
// bit mask of the groups that start inside the chunk) and unranks its offset
// in that group.  The order's groups are grp[g0 .. ge - 1]; the arguments are
// plain values and pointers (a reference to the kernel's code parameter would
// make the compiler copy the parameter to local memory).
template <int NPL, class SYN>
__device__ __noinline__ LoopOut query_loop_lanes(const Scratch<NPL, SYN> sc, const WordHead<NPL, SYN> &h,
                                                 const uint2 *grp, int g0, int ge, const int32_t *scnt, int sc_w,
                                                 int sc_m, int n, int qlim, int L, int lane) {
  int q = 0, nhit = 0, wacc = 0;
  DF tmass = {0.f, 0.f};
  GroupWindow W;
  W.init(grp, g0, ge);
  uint4 *slot = sc.pf() + lane;
  for (;;) {
    const int lim = min(32, qlim - q);
    if (lim <= 0) break;
    const uint4 e = W.chunk(q, lim, lane, scnt, sc_w, sc_m, n, slot);
    const int w = e.x & 0xff;
    const int wmax = (int)__reduce_max_sync(FULL, (unsigned)w);
    DF mass;
    const SYN s = ent_syndrome<SYN>(e, w, wmax, sc.hr(), mass) ^ h.s0;
    const bool hit = lane < lim && s == 0;
    unsigned hm = __ballot_sync(FULL, hit);
    int stop_lane = -1;
    while (hm) {
      const int hl = __ffs(hm) - 1;
      hm &= hm - 1;
      record_hit<NPL, SYN>(sc, h, e, hl, nhit, lane);
      nhit++;
      if (nhit >= L) {
        stop_lane = hl;
        break;
      }
    }
    if (stop_lane >= 0) {
      if (lane <= stop_lane) {
        wacc += w;
        df_acc(tmass, mass);
      }
      q += stop_lane + 1;
      break;
    }
    wacc += w;
    df_acc(tmass, mass);
    q += lim;
  }
  return LoopOut{q, nhit, wacc, tmass};
}

// The thr = 0 query loop of a word: patterns from the order table, or
// enumerated by the lanes (LANES, kernels of their own).
template <int NPL, class SYN, bool LANES>
__device__ __forceinline__ LoopOut query_loop(const Scratch<NPL, SYN> &sc, const WordHead<NPL, SYN> &h,
                                              const DevCode &code, int ti, int tb, int qlim, int L, int lane) {
  if constexpr (LANES)
    return query_loop_lanes<NPL, SYN>(sc, h, code.grp.grp, __ldg(code.grp.gbase + ti), __ldg(code.grp.gbase + ti + 1),
                                      code.grp.scnt, code.grp.sc_w, code.grp.sc_m, code.n, qlim, L, lane);
  else
    return query_loop_plain<NPL, SYN>(sc, h, code.ord.ent + tb, qlim, L, lane);
}

// lam[k] is bit lane + 32k of the SISO input lambda = fl32(L_Ch + L_A)
// (the caller loads it; entries past n are ignored).  On return lapp[k] holds
// L_APP for the same bits, res the per-word results; the list (in query
// order) is left in the scratch: sc.cw() (codewords, natural bit order),
// sc.lp() (log p(z)/p(0)) and sc.wl() (APP of each word).  *flags (if given)
// collects the remaining-mass flags (bit 0: extended range; bit 1: the
// block's remaining-mass area could not be locked).
template <int NPL, class SYN, bool LANES = false>
__device__ void siso_word(const DevCode &code, const SisoParams &P, const Scratch<NPL, SYN> &sc,
                          const float (&lam)[NPL], int lane, float (&lapp)[NPL], WordResult &res,
                          int *flags = nullptr) {
  constexpr int NT = 32 * NPL;
  constexpr int NM = (NT + 63) / 64;
  const int n = code.n;
#ifdef SG_PHASE_PROFILE
  const long long t0 = clock64();
#endif
#pragma unroll
  for (int k = 0; k < NPL; k++) sc.lamv()[lane + 32 * k] = lam[k];  // each lane reads back its own
  WordHead<NPL, SYN> h;
  if (!siso_prologue<NPL, SYN>(code, sc, lam, lane, h)) {
#pragma unroll
    for (int k = 0; k < NPL; k++) lapp[k] = lam[k];
    res.queries = -1;
    res.nhit = 0;
    res.pmiss = 1.f;
    res.logD = 0.f;
    res.wsum = 0;
    return;
  }
#ifdef SG_PHASE_PROFILE
  const long long t1 = clock64();
  int nchunks = 0;
#endif

  // query loop over the flattened order of (c, class)
  const DevOrder &O = code.ord;
  const int cls = code.even ? h.par : -1;
  const int ti = h.c * O.ncls + (code.even ? h.par : 0);
  if (lane == 0) {
#pragma unroll
    for (int k = 0; k < NPL; k++) sc.headv()[k] = h.yb[k];
    sc.headv()[NPL] = (unsigned)h.c;
  }
  __syncwarp();
  const int tb = __ldg(O.base + ti), tc = __ldg(O.count + ti);
  const int qlim = min(P.cap, tc);
  int q = 0, nhit = 0;
  float lr2 = 0.f;  // log2 remaining mass (set when the search stops)
  bool have_lr2 = false;
  int wacc = 0;       // this lane's share of the summed pattern weights
  DF tmass = {0.f, 0.f};  // this lane's share of the queried mass (nonzero patterns)
  // each lane's entry of the next chunk is copied into its 16-byte slot of the
  // warp's shared area while the current chunk is tested (cp.async: no
  // registers held, the L2 latency overlaps the chunk's work)
  if (P.thr <= 0.f) {  // no threshold rule: the out-of-line loop
    const LoopOut lo = query_loop<NPL, SYN, LANES>(sc, h, code, ti, tb, qlim, P.L, lane);
    q = lo.q;
    nhit = lo.nhit;
    wacc = lo.wacc;
    tmass = lo.tmass;
  } else {  // with the threshold rule checked at every new list word
    const unsigned pf_addr = (unsigned)__cvta_generic_to_shared(sc.pf() + lane);
    if (lane < qlim)
      asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(pf_addr), "l"(O.ent + tb + lane) : "memory");
    asm volatile("cp.async.commit_group;" ::: "memory");
    for (;;) {
      const int lim = min(32, qlim - q);
      if (lim <= 0) break;
#ifdef SG_PHASE_PROFILE
      nchunks++;
#endif
      uint4 e = make_uint4(0u, 0u, 0u, 0u);
      asm volatile("cp.async.wait_all;" ::: "memory");
      if (lane < lim) e = sc.pf()[lane];  // after the wait (a compiler barrier): this lane's own slot
      if (q + 32 + lane < qlim)
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(pf_addr), "l"(O.ent + tb + q + 32 + lane) : "memory");
      asm volatile("cp.async.commit_group;" ::: "memory");
      const int w = e.x & 0xff;
      const int wmax = (int)__reduce_max_sync(FULL, (unsigned)w);
      DF mass;
      const SYN s = ent_syndrome<SYN>(e, w, wmax, sc.hr(), mass) ^ h.s0;
      const bool hit = lane < lim && s == 0;
      unsigned hm = __ballot_sync(FULL, hit);
      int stop_lane = -1;
      while (hm) {
        const int hl = __ffs(hm) - 1;
        hm &= hm - 1;
        record_hit<NPL, SYN>(sc, h, e, hl, nhit, lane);
        nhit++;
        if (nhit >= P.L) {
          stop_lane = hl;
          break;
        }
        if (P.thr > 0.f) {
          DF part = tmass;
          if (lane <= hl) df_acc(part, mass);
          const DF tq = df_warp_sum(part);
          const float r2 = remaining_log2<NPL, SYN>(sc, O, tb, tc, q + hl, n, (int)sc.head_at(NPL), cls, lane, tq, flags);
          if (thr_reached(sc, nhit, r2 * LN2_F + code.log_phi, P.thr)) {
            stop_lane = hl;
            lr2 = r2;
            have_lr2 = true;
            break;
          }
        }
      }
      if (stop_lane >= 0) {
        if (lane <= stop_lane) {
          wacc += w;
          df_acc(tmass, mass);
        }
        q += stop_lane + 1;
        break;
      }
      wacc += w;  // lanes past lim hold an empty entry
      df_acc(tmass, mass);
      q += lim;
    }
    // a copy for a chunk that was not needed may still be in flight: wait for
    // it, so that it cannot land in the slot after the next word's first copy
    asm volatile("cp.async.wait_all;" ::: "memory");
  }
  // the whole parity class has been queried: nothing remains
  const bool exhausted = q >= tc && tc == O.class_size;
  __syncwarp();
#ifdef SG_PHASE_PROFILE
  const long long t2 = clock64();
#endif

  // soft output (Corollary + eq. LLRi)
  if (!have_lr2)
    lr2 = (exhausted || P.forney) ? -CUDART_INF_F
                    : remaining_log2<NPL, SYN>(sc, O, tb, tc, q - 1, n, (int)sc.head_at(NPL), cls, lane, df_warp_sum(tmass),
                                               flags);
#ifdef SG_PHASE_PROFILE
  const long long t3 = clock64();
#endif
  const float M = lr2 * LN2_F + code.log_phi;  // log (R phi), natural
  res.wsum = (int32_t)__reduce_add_sync(FULL, (unsigned)wacc);
  res.queries = q;
  res.nhit = nhit;
  if (nhit == 0) {
#pragma unroll
    for (int k = 0; k < NPL; k++) lapp[k] = sc.lam_at(lane + 32 * k);
    res.pmiss = 1.f;
    res.logD = M;
  } else {
    // log(R phi + sum_l p_l), all relative to p(0): max plus log of a sum.
    // The hardware exponential and logarithm (relative errors near 2^-21 over
    // these ranges) keep L_APP within about 1e-5 of the exact formula, far
    // inside the soft output's tolerance; no decision is taken on them.
    float mx = M;
    for (int l = 0; l < nhit; l++) mx = fmaxf(mx, sc.lp()[l]);
    float sum = M == -CUDART_INF_F ? 0.f : __expf(M - mx);
    for (int l = 0; l < nhit; l++) sum += __expf(sc.lp()[l] - mx);
    const float D = mx + __logf(sum);
    res.logD = D;
    const float pm = M == -CUDART_INF_F ? 0.f : __expf(M - D);
    res.pmiss = pm;
    // APP of each listed word (list weights relative to the normaliser)
    if (lane < nhit) sc.wl()[lane] = __expf(sc.lp()[lane] - D);
    __syncwarp();
    // eq. LLRi: the miss term, then each listed word adds its APP to the side
    // of its bit; a list word's bit mask is read once for all the lane's bits
    float a0[NPL], a1[NPL];
#pragma unroll
    for (int k = 0; k < NPL; k++) {
      const float x = sc.lam_at(lane + 32 * k);
      // sigma(x) and sigma(-x) without cancellation
      const float ex = __expf(-fabsf(x));
      const float sp = __fdividef(1.f, 1.f + ex), sn = ex * sp;  // sigma(|x|), sigma(-|x|)
      a0[k] = pm * (x >= 0.f ? sp : sn);                          // miss term, bit 0
      a1[k] = pm * (x >= 0.f ? sn : sp);                          // miss term, bit 1
    }
    for (int l = 0; l < nhit; l++) {
      const float wlv = sc.wl()[l];
#pragma unroll
      for (int k = 0; k < NPL; k++) {
        const int i = lane + 32 * k;
        if ((sc.cw()[l * NM + (i >> 6)] >> (i & 63)) & 1ull)
          a1[k] += wlv;
        else
          a0[k] += wlv;
      }
    }
#pragma unroll
    for (int k = 0; k < NPL; k++) {
      // both sums lie in (1e-30, 1 + 1e-6]: __fdividef's range
      lapp[k] = (a0[k] > 1e-30f && a1[k] > 1e-30f)
                    ? __logf(__fdividef(a0[k], a1[k]))
                    : lapp_logdomain<NPL, SYN>(sc, nhit, M, sc.lam_at(lane + 32 * k), lane + 32 * k);
    }
  }
#ifdef SG_PHASE_PROFILE
  const long long t4 = clock64();
  if (lane == 0) {
    SG_PROF(0, t1 - t0);
    SG_PROF(1, t2 - t1);
    SG_PROF(2, t3 - t2);
    SG_PROF(3, t4 - t3);
    SG_PROF(4, 1);
    SG_PROF(5, nchunks);
  }
#endif
}

}  // namespace sg
