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
// ties fall to the lower index), the H columns are permuted into rank order
// in shared memory, and every chunk of 32 consecutive queries is spread over
// the 32 lanes: lane j takes query q0 + j, XORs its pattern's H columns into
// the syndrome of y and reports a hit; __ballot_sync + __ffs keep the hits in
// query order, so list, stop point and query count are those of a sequential
// decoder.
//
// Remaining mass.  The Corollary needs 1 - sum_{j <= q_L} p(z^j).  In FP32
// that difference cancels catastrophically as soon as the queried mass
// dominates, so the kernel sums the unqueried patterns directly (all terms
// positive): patterns of cost above the stop level C* by a dynamic programme
// over the ranks (cost-indexed, parity-split, a pattern is added to the tail
// the moment one more rank lifts it over C*), plus the unqueried rest of
// level C* by enumeration.  Masses are cost-scaled by exp(gamma * cost) so
// that every factor stays <= 1; if the scaled total still falls below 2^-60
// (all dominant terms underflow) or overflows, the same computation is redone
// in an extended-range float (FP32 mantissa + int exponent).
#pragma once
#include <cuda_runtime.h>
#include <math_constants.h>

#include <cstdint>

#include "sg_common.h"

namespace sg {

constexpr unsigned FULL = 0xffffffffu;
constexpr float LOG2E_F = 1.4426950408889634f;
constexpr float LN2_F = 0.6931471805599453f;

__host__ __device__ constexpr int align16(int x) { return (x + 15) & ~15; }

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
__device__ __forceinline__ XF xf_shfl_down(XF a, int d) {
  return {__shfl_down_sync(FULL, a.m, d), __shfl_down_sync(FULL, a.e, d)};
}
__device__ __forceinline__ XF xf_shfl_xor(XF a, int d) {
  return {__shfl_xor_sync(FULL, a.m, d), __shfl_xor_sync(FULL, a.e, d)};
}

// Number policies for the remaining-mass computation.
struct FOps {  // plain FP32, cost-scaled
  using T = float;
  static __device__ __forceinline__ T zero() { return 0.f; }
  static __device__ __forceinline__ T one() { return 1.f; }
  static __device__ __forceinline__ T add(T a, T b) { return a + b; }
  static __device__ __forceinline__ T mul(T a, T b) { return a * b; }
  static __device__ __forceinline__ T from_log2(float x) { return exp2f(x); }
  static __device__ __forceinline__ T from_float(float x) { return x; }
  static __device__ __forceinline__ T shfl_down(T a, int d) { return __shfl_down_sync(FULL, a, d); }
  static __device__ __forceinline__ T shfl_xor(T a, int d) { return __shfl_xor_sync(FULL, a, d); }
};
struct XOps {  // extended range, unscaled
  using T = XF;
  static __device__ __forceinline__ T zero() { return xf_zero(); }
  static __device__ __forceinline__ T one() { return xf_one(); }
  static __device__ __forceinline__ T add(T a, T b) { return xf_add(a, b); }
  static __device__ __forceinline__ T mul(T a, T b) { return xf_mul(a, b); }
  static __device__ __forceinline__ T from_log2(float x) { return xf_from_log2(x); }
  static __device__ __forceinline__ T from_float(float x) { return xf_norm(x, 0); }
  static __device__ __forceinline__ T shfl_down(T a, int d) { return xf_shfl_down(a, d); }
  static __device__ __forceinline__ T shfl_xor(T a, int d) { return xf_shfl_xor(a, d); }
};

// ----------------------------------------------------------------------------
// per-warp shared-memory scratch
// ----------------------------------------------------------------------------
template <int NPL, class SYN>
struct Layout {
  static constexpr int NT = 32 * NPL;
  static constexpr int NM = (NT + 63) / 64;
  static constexpr int o_l2 = 0;                                      // float[NT] |lambda| log2(e), by rank
  static constexpr int o_al = o_l2 + 4 * NT;                          // float[NT] |lambda|, by rank
  static constexpr int o_hs = o_al + 4 * NT;                          // SYN[NT] H column, by rank
  static constexpr int o_zm = align16(o_hs + (int)sizeof(SYN) * NT);  // u64[LMAX][NM] hit rank masks
  static constexpr int o_cw = o_zm + 8 * LMAX * NM;                   // u64[LMAX][NM] hit codewords
  static constexpr int o_lp = o_cw + 8 * LMAX * NM;                   // float[LMAX] log p(z)/p(0)
  static constexpr int o_perm = o_lp + 4 * LMAX;                      // u8[NT] rank -> bit
  static constexpr int o_tail = align16(o_perm + NT);
  // tail area (sized for the 8-byte XF policy): sfac[NT], fu[NT+1], fb[NT+1], he[J], ho[J], ek[J]
  static __host__ __device__ int bytes(int jm) { return align16(o_tail + 8 * (3 * NT + 2) + 20 * jm + 16); }
};

template <int NPL, class SYN>
struct Scratch {
  using LY = Layout<NPL, SYN>;
  float *l2, *al;
  SYN *hs;
  uint64_t *zm, *cw;
  float *lp;
  uint8_t *perm;
  unsigned char *tail;
  __device__ void bind(unsigned char *base) {
    l2 = reinterpret_cast<float *>(base + LY::o_l2);
    al = reinterpret_cast<float *>(base + LY::o_al);
    hs = reinterpret_cast<SYN *>(base + LY::o_hs);
    zm = reinterpret_cast<uint64_t *>(base + LY::o_zm);
    cw = reinterpret_cast<uint64_t *>(base + LY::o_cw);
    lp = reinterpret_cast<float *>(base + LY::o_lp);
    perm = base + LY::o_perm;
    tail = base + LY::o_tail;
  }
};

// ----------------------------------------------------------------------------
// warp helpers
// ----------------------------------------------------------------------------
template <int NPL>
__device__ __forceinline__ void warp_bitonic_sort(uint64_t (&v)[NPL], int lane) {
  constexpr int N = 32 * NPL;
#pragma unroll
  for (int size = 2; size <= N; size <<= 1) {
#pragma unroll
    for (int j = size >> 1; j > 0; j >>= 1) {
      if (j >= 32) {
        const int kj = j >> 5;
#pragma unroll
        for (int k = 0; k < NPL; k++) {
          const int kp = k ^ kj;
          if (kp > k) {
            const bool asc = ((k * 32 + lane) & size) == 0;
            uint64_t a = v[k], b = v[kp];
            bool sw = asc ? (a > b) : (a < b);
            v[k] = sw ? b : a;
            v[kp] = sw ? a : b;
          }
        }
      } else {
#pragma unroll
        for (int k = 0; k < NPL; k++) {
          uint64_t o = __shfl_xor_sync(FULL, v[k], j);
          const bool asc = ((k * 32 + lane) & size) == 0;
          const bool lower = (lane & j) == 0;
          v[k] = (lower == asc) ? (v[k] < o ? v[k] : o) : (v[k] < o ? o : v[k]);
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

// floor(v * 256 + 1/2) for v >= 0 (exact, integer arithmetic), saturating at 2^20 - 1.
__device__ __forceinline__ int64_t quant256(float v) {
  const int64_t AMAX = (1 << 20) - 1;
  uint32_t b = __float_as_uint(v);
  int ex = (b >> 23) & 0xff;
  uint32_t mant = (b & 0x7fffffu) | (ex ? 0x800000u : 0u);
  int sh = 142 - (ex ? ex : 1);
  if (sh <= 0) return AMAX;
  if (sh > 40) return 0;
  int64_t a = ((int64_t)mant + ((int64_t)1 << (sh - 1))) >> sh;
  return a > AMAX ? AMAX : a;
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
  int64_t c = top / (2 * (int64_t)n * Nb);
  return (int)(c > c_max ? c_max : c);
}

// ----------------------------------------------------------------------------
// query-order walk over (cost level, Hamming weight) groups  (warp-uniform)
// ----------------------------------------------------------------------------
struct Walk {
  DevTables T;
  int n, c, w0, step, nw;
  int C, wi, pos, gsize, gbase, a, b;
  bool done;

  __device__ __forceinline__ int wt(int i) const { return w0 + i * step; }
  __device__ __forceinline__ int lo(int i) const {
    int w = wt(i);
    return w * (w + 1) / 2 + c * w;
  }
  __device__ __forceinline__ int hi(int i) const {
    int w = wt(i);
    return w * (2 * n - w + 1) / 2 + c * w;
  }
  __device__ __forceinline__ void load() {
    int w = wt(wi);
    int li = C - c * w - w * (w + 1) / 2;
    if (li < 0 || li >= __ldg(T.lnum + w)) {
      gsize = 0;
      gbase = 0;
    } else {
      int base = __ldg(T.lbase + w) + li;
      gsize = __ldg(T.lcnt + base);
      gbase = __ldg(T.sbase + w) + __ldg(T.loff + base);
    }
    pos = 0;
  }
  __device__ __forceinline__ void settle() {
    for (;;) {
      while (a < nw && hi(a) < C) a++;
      while (b + 1 < nw && lo(b + 1) <= C) b++;
      if (a <= b) break;
      if (b + 1 < nw) {
        C = lo(b + 1);
        continue;
      }
      done = true;
      return;
    }
    wi = a;
    load();
  }
  __device__ void init(const DevTables &t, int n_, int c_, bool even, int par) {
    T = t;
    n = n_;
    c = c_;
    w0 = even ? par : 0;
    step = even ? 2 : 1;
    int top = t.wtop < n + 1 ? t.wtop : n + 1;
    nw = top > w0 ? (top - w0 + step - 1) / step : 0;
    a = 0;
    b = -1;
    done = nw == 0;
    if (!done) {
      C = lo(0);
      settle();
    }
  }
  __device__ __forceinline__ void advance() {
    if (wi < b) {
      wi++;
      load();
      return;
    }
    C++;
    settle();
  }
  // jump to group (C_, wi_) with pos_ patterns of it already consumed
  __device__ void seek(int C_, int wi_, int pos_) {
    C = C_;
    a = 0;
    b = -1;
    done = false;
    while (a < nw && hi(a) < C) a++;
    while (b + 1 < nw && lo(b + 1) <= C) b++;
    wi = wi_;
    load();
    pos = pos_;
  }
  // Hand the next patterns (at most `limit`, and only of level Cfix when
  // Cfix >= 0) to lanes 0..count-1.  Lane j receives its pattern index and
  // the walk position just after it.
  __device__ __forceinline__ int assign(int limit, int lane, int Cfix, int &pidx, int &lC, int &lwi, int &lpos) {
    int base = 0;
    while (base < limit && !done) {
      if (Cfix >= 0 && C != Cfix) break;
      int take = gsize - pos;
      if (take > limit - base) take = limit - base;
      int rel = lane - base;
      if (rel >= 0 && rel < take) {
        pidx = gbase + pos + rel;
        lC = C;
        lwi = wi;
        lpos = pos + rel + 1;
      }
      base += take;
      pos += take;
      if (pos >= gsize) advance();
    }
    return base;
  }
};

template <int NM>
__device__ __forceinline__ void load_mask(const DevTables &T, int pidx, uint64_t (&mk)[NM]) {
  const uint64_t *p = T.pat + (size_t)pidx * NM;
  if (NM == 1) {
    mk[0] = __ldg(p);
  } else {
    ulonglong2 v = __ldg(reinterpret_cast<const ulonglong2 *>(p));
    mk[0] = v.x;
    mk[NM - 1] = v.y;
  }
}

// ----------------------------------------------------------------------------
// remaining mass: tail over cost > Cs (DP) + unqueried rest of level Cs
// ----------------------------------------------------------------------------
// Returns the (scaled) remaining mass summed over the warp.  With FOps the
// masses carry the factor 2^(g2 * Cs) (g2 = gamma log2 e); with XOps g2 = 0.
template <class Ops, int NPL, class SYN>
__device__ typename Ops::T remaining_scaled(const Scratch<NPL, SYN> &sc, Walk W, int n, int cls, int Cs, int wis,
                                            int poss, float g2, int lane) {
  using T = typename Ops::T;
  constexpr int NT = 32 * NPL;
  constexpr int NM = (NT + 63) / 64;
  const int c = W.c;
  T *sfac = reinterpret_cast<T *>(sc.tail);
  T *fu = sfac + NT;
  T *fb = fu + NT + 1;
  T *he = fb + NT + 1;
  T *ho = he + (Cs + 1);
  float *ek = reinterpret_cast<float *>(ho + (Cs + 1));
  constexpr bool SCALED = sizeof(T) == 4;
  const int R0 = min(max(Cs - c, 0), n);  // ranks e < R0 can sit inside a pattern of cost <= Cs
  const float g2Cs = g2 * (float)Cs;

  // --- unqueried rest of level Cs
  T acc = Ops::zero();
  {
    Walk R = W;
    R.seek(Cs, wis, poss);
    if (R.pos >= R.gsize) R.advance();
    while (!R.done && R.C == Cs) {
      int pidx = 0, lC, lwi, lpos;
      int cnt = R.assign(32, lane, Cs, pidx, lC, lwi, lpos);
      if (lane < cnt) {
        uint64_t mk[NM];
        load_mask<NM>(W.T, pidx, mk);
        float s2 = 0.f;
#pragma unroll
        for (int wd = 0; wd < NM; wd++) {
          uint64_t x = mk[wd];
          while (x) {
            int r = __ffsll((long long)x) - 1 + 64 * wd;
            x &= x - 1;
            s2 += sc.l2[r];
          }
        }
        acc = Ops::add(acc, Ops::from_log2(g2Cs - s2));
      }
      if (cnt == 0) break;
    }
  }

  // --- per-rank factors and suffix products F_e = prod_{e' >= e} (1 + y t_e')
  //     kept as (u, b) = (even part - 1, odd part); lanes own ranks
  //     lane*NPL .. lane*NPL+NPL-1.
  {
    T lu[NPL], lb[NPL];
    T u = Ops::zero(), b = Ops::zero();
#pragma unroll
    for (int k = NPL - 1; k >= 0; k--) {
      int e = lane * NPL + k;
      T t = Ops::zero();
      if (e < n) {
        t = Ops::from_log2(-sc.l2[e]);
        // factor used by the tail: low ranks t * 2^(g2 d_e), high ranks t * 2^(g2 Cs)
        float d = (float)(e + 1 + c);
        sfac[e] = Ops::from_log2((e < R0 ? g2 * d : g2Cs) - sc.l2[e]);
      }
      T nu = Ops::add(u, Ops::mul(b, t));
      T nb = Ops::add(Ops::add(b, t), Ops::mul(u, t));
      u = nu;
      b = nb;
      lu[k] = u;
      lb[k] = b;
    }
    // inclusive suffix scan of the block products over lanes
    T su = u, sb = b;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      T ou = Ops::shfl_down(su, d), ob = Ops::shfl_down(sb, d);
      if (lane + d < 32) {
        T nu = Ops::add(Ops::add(su, ou), Ops::add(Ops::mul(su, ou), Ops::mul(sb, ob)));
        T nb = Ops::add(Ops::add(sb, ob), Ops::add(Ops::mul(su, ob), Ops::mul(sb, ou)));
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
      int e = lane * NPL + k;
      if (e <= n) {
        T fu_ = Ops::add(Ops::add(lu[k], xu), Ops::add(Ops::mul(lu[k], xu), Ops::mul(lb[k], xb)));
        T fb_ = Ops::add(Ops::add(lb[k], xb), Ops::add(Ops::mul(lu[k], xb), Ops::mul(lb[k], xu)));
        if (e < n) {
          fu[e] = fu_;
          fb[e] = fb_;
        }
      }
    }
    if (lane == 0) {
      fu[n] = Ops::zero();
      fb[n] = Ops::zero();
    }
  }
  // cost DP init and the 2^(-g2 k) table
  for (int j = lane; j <= Cs; j += 32) {
    he[j] = j == 0 ? Ops::one() : Ops::zero();
    ho[j] = Ops::zero();
    if constexpr (SCALED) ek[j] = exp2f(-g2 * (float)j);
  }
  __syncwarp();

  // --- high ranks (d_e > Cs): G_P = sum_e sfac_e * F_{e+1} (parity of
  //     pattern {e} + higher subset), reduced over the warp
  T g_even = Ops::zero(), g_odd = Ops::zero();
  for (int e = R0 + lane; e < n; e += 32) {
    T s = sfac[e];
    T one_u = Ops::add(Ops::one(), fu[e + 1]);
    g_odd = Ops::add(g_odd, Ops::mul(s, one_u));
    g_even = Ops::add(g_even, Ops::mul(s, fb[e + 1]));
  }
#pragma unroll
  for (int d = 16; d > 0; d >>= 1) {
    g_even = Ops::add(g_even, Ops::shfl_xor(g_even, d));
    g_odd = Ops::add(g_odd, Ops::shfl_xor(g_odd, d));
  }

  // --- low ranks in ascending order: tail contributions, then DP update.
  //     Entry slots are walked from the top so that every read of
  //     he/ho[j - d] sees the values before this rank (reads of a slot are
  //     separated from its writes by __syncwarp).
  const int nslot = (Cs + 32) >> 5;
  for (int e = 0; e < R0; e++) {
    const int d = e + 1 + c;
    const T s = sfac[e];
    const T Fb = fb[e + 1];
    const T F1u = Ops::add(Ops::one(), fu[e + 1]);
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
          acc = Ops::add(acc, Ops::mul(w, term));
        }
        if (upd) {
          ne = Ops::add(hej, Ops::mul(s, ho[j - d]));
          no = Ops::add(hoj, Ops::mul(s, he[j - d]));
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
  // high ranks joined to every head pattern
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
    acc = Ops::add(acc, Ops::mul(w, term));
  }
#pragma unroll
  for (int d = 16; d > 0; d >>= 1) acc = Ops::add(acc, Ops::shfl_xor(acc, d));
  __syncwarp();
  return acc;
}

// log2 of the remaining (unqueried) mass relative to p(0^n|r); warp-uniform.
template <int NPL, class SYN>
__device__ float remaining_log2(const Scratch<NPL, SYN> &sc, const Walk &W, int n, int cls, int Cs, int wis, int poss,
                                int lane, int *used_xf) {
  const int c = W.c;
  const int R0 = min(max(Cs - c, 0), n);
  float g = CUDART_INF_F;
  for (int e = lane; e < R0; e += 32) g = fminf(g, sc.l2[e] / (float)(e + 1 + c));
  g = warp_min_f(g);
  if (!(g < CUDART_INF_F)) g = 0.f;
  float tot = remaining_scaled<FOps, NPL, SYN>(sc, W, n, cls, Cs, wis, poss, g, lane);
  if (tot >= 0x1p-60f && tot < CUDART_INF_F) return log2f(tot) - g * (float)Cs;
  if (used_xf) *used_xf = 1;
  XF x = remaining_scaled<XOps, NPL, SYN>(sc, W, n, cls, Cs, wis, poss, 0.f, lane);
  return xf_log2(x);
}

// numerically safe log(exp(a) + exp(b)) (natural log, -inf aware)
__device__ __forceinline__ float lse(float a, float b) {
  float mx = fmaxf(a, b), mn = fminf(a, b);
  if (mx == -CUDART_INF_F) return mx;
  return mx + log1pf(expf(mn - mx));
}
__device__ __forceinline__ float softplus(float z) { return fmaxf(z, 0.f) + log1pf(expf(-fabsf(z))); }

// ----------------------------------------------------------------------------
// one word
// ----------------------------------------------------------------------------
// Per-word state after the prologue (warp-uniform except yb).
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
    unsigned lo_ = __reduce_xor_sync(FULL, (unsigned)(uint64_t)s0p);
    unsigned hi_ = __reduce_xor_sync(FULL, (unsigned)((uint64_t)s0p >> 32));
    h.s0 = (SYN)(((uint64_t)hi_ << 32) | lo_);
  }

  // reliability ranks: sort (|lambda|, index) ascending
  uint64_t key[NPL];
#pragma unroll
  for (int k = 0; k < NPL; k++) {
    const int i = lane + 32 * k;
    key[k] = i < n ? (((uint64_t)__float_as_uint(fabsf(lam[k])) << 32) | (uint64_t)i) : ~0ull;
  }
  warp_bitonic_sort<NPL>(key, lane);
  int64_t sy = 0, sxy = 0;
#pragma unroll
  for (int k = 0; k < NPL; k++) {
    const int e = k * 32 + lane;
    if (e < n) {
      const float a = __uint_as_float((unsigned)(key[k] >> 32));
      const int idx = (int)(key[k] & 0xffffffffu);
      sc.al[e] = a;
      sc.l2[e] = a * LOG2E_F;
      sc.perm[e] = (uint8_t)idx;
      sc.hs[e] = (SYN)__ldg(code.hcol + idx);
      const int64_t qa = quant256(a);
      sy += qa;
      sxy += qa * (e + 1);
    }
  }
  sy = warp_sum_i64(sy);
  sxy = warp_sum_i64(sxy);
  h.c = one_line_c(sy, sxy, n, code.c_max);
  __syncwarp();
  return true;
}

// The canonical query order for one input (test hook): writes the first
// max_q rank masks; returns how many were written.
template <int NPL, class SYN>
__device__ int trace_word(const DevCode &code, const Scratch<NPL, SYN> &sc, const float (&lam)[NPL], int lane,
                          int max_q, uint64_t *out, int *c_out) {
  constexpr int NM = (32 * NPL + 63) / 64;
  WordHead<NPL, SYN> h;
  if (!siso_prologue<NPL, SYN>(code, sc, lam, lane, h)) return -1;
  Walk W;
  W.init(code.tab, code.n, h.c, code.even != 0, h.par);
  int q = 0;
  while (!W.done && q < max_q) {
    int limit = min(32, max_q - q);
    int pidx = 0, lC, lwi, lpos;
    const int nv = W.assign(limit, lane, -1, pidx, lC, lwi, lpos);
    if (lane < nv) {
      uint64_t mk[NM];
      load_mask<NM>(code.tab, pidx, mk);
#pragma unroll
      for (int wd = 0; wd < NM; wd++) out[(size_t)(q + lane) * NM + wd] = mk[wd];
    }
    q += nv;
    if (nv == 0) break;
  }
  if (c_out && lane == 0) *c_out = h.c;
  return q;
}

// lam[k] is bit lane + 32k of the SISO input lambda = fl32(L_Ch + L_A)
// (the caller loads it; entries past n are ignored).  On return lapp[k] holds
// L_APP for the same bits, res the per-word results; the list (in query
// order) is left in the scratch: sc.cw (codewords, natural bit order) and
// sc.lp (log p(z)/p(0)).
template <int NPL, class SYN>
__device__ void siso_word(const DevCode &code, const SisoParams &P, const Scratch<NPL, SYN> &sc,
                          const float (&lam)[NPL], int lane, float (&lapp)[NPL], WordResult &res,
                          int *xf_count = nullptr) {
  constexpr int NT = 32 * NPL;
  constexpr int NM = (NT + 63) / 64;
  const int n = code.n;

  WordHead<NPL, SYN> h;
  if (!siso_prologue<NPL, SYN>(code, sc, lam, lane, h)) {
#pragma unroll
    for (int k = 0; k < NPL; k++) lapp[k] = lam[k];
    res.queries = -1;
    res.nhit = 0;
    res.pmiss = 1.f;
    res.logD = 0.f;
    return;
  }

  // query loop
  Walk W;
  W.init(code.tab, n, h.c, code.even != 0, h.par);
  const int cls = code.even ? h.par : -1;
  int q = 0, nhit = 0;
  int sC = 0, swi = 0, spos = 0;
  bool exhausted = false;
  float lr2 = 0.f;  // log2 remaining mass (set when the search stops)
  bool have_lr2 = false;
  for (;;) {
    if (W.done) {
      exhausted = true;
      break;
    }
    int limit = P.cap - q;
    if (limit > 32) limit = 32;
    int pidx = 0, lC = 0, lwi = 0, lpos = 0;
    const int nv = W.assign(limit, lane, -1, pidx, lC, lwi, lpos);
    bool hit = false;
    uint64_t mk[NM];
#pragma unroll
    for (int wd = 0; wd < NM; wd++) mk[wd] = 0;
    if (lane < nv) {
      load_mask<NM>(code.tab, pidx, mk);
      SYN s = h.s0;
#pragma unroll
      for (int wd = 0; wd < NM; wd++) {
        uint64_t x = mk[wd];
        while (x) {
          const int r = __ffsll((long long)x) - 1 + 64 * wd;
          x &= x - 1;
          s ^= sc.hs[r];
        }
      }
      hit = s == 0;
    }
    unsigned hm = __ballot_sync(FULL, hit);
    int stop_lane = -1;
    while (hm) {
      const int hl = __ffs(hm) - 1;
      hm &= hm - 1;
      if (lane == hl) {
        // record the list entry: codeword in bit order and log mass
        uint64_t cw[NM];
#pragma unroll
        for (int wd = 0; wd < NM; wd++) cw[wd] = 0;
        float ls = 0.f;
#pragma unroll
        for (int wd = 0; wd < NM; wd++) {
          uint64_t x = mk[wd];
          while (x) {
            const int r = __ffsll((long long)x) - 1 + 64 * wd;
            x &= x - 1;
            ls += sc.al[r];
            const int bi = sc.perm[r];
#pragma unroll
            for (int w2 = 0; w2 < NM; w2++)
              if ((bi >> 6) == w2) cw[w2] ^= 1ull << (bi & 63);
          }
        }
#pragma unroll
        for (int wd = 0; wd < NM; wd++) {
          uint64_t yw = 0;
#pragma unroll
          for (int hh = 0; hh < 2; hh++) {
            const int kk = wd * 2 + hh;
            if (kk < NPL) yw |= (uint64_t)h.yb[kk] << (32 * hh);
          }
          sc.cw[nhit * NM + wd] = cw[wd] ^ yw;
          sc.zm[nhit * NM + wd] = mk[wd];
        }
        sc.lp[nhit] = -ls;
      }
      nhit++;
      if (nhit >= P.L) {
        stop_lane = hl;
        break;
      }
      if (P.thr > 0.f) {
        __syncwarp();
        const int hC = __shfl_sync(FULL, lC, hl), hwi = __shfl_sync(FULL, lwi, hl), hpos = __shfl_sync(FULL, lpos, hl);
        const float r2 = remaining_log2<NPL, SYN>(sc, W, n, cls, hC, hwi, hpos, lane, xf_count);
        const float M = r2 * LN2_F + code.log_phi;
        float D = M;
        for (int l = 0; l < nhit; l++) D = lse(D, sc.lp[l]);
        if (expf(M - D) < P.thr) {
          stop_lane = hl;
          lr2 = r2;
          have_lr2 = true;
          break;
        }
      }
    }
    if (stop_lane >= 0) {
      q += stop_lane + 1;
      sC = __shfl_sync(FULL, lC, stop_lane);
      swi = __shfl_sync(FULL, lwi, stop_lane);
      spos = __shfl_sync(FULL, lpos, stop_lane);
      if (W.done && stop_lane == nv - 1) exhausted = true;
      break;
    }
    q += nv;
    if (q >= P.cap) {
      sC = __shfl_sync(FULL, lC, nv - 1);
      swi = __shfl_sync(FULL, lwi, nv - 1);
      spos = __shfl_sync(FULL, lpos, nv - 1);
      if (W.done) exhausted = true;
      break;
    }
  }
  __syncwarp();

  // soft output (Corollary + eq. LLRi), natural log domain
  if (!have_lr2)
    lr2 = exhausted ? -CUDART_INF_F : remaining_log2<NPL, SYN>(sc, W, n, cls, sC, swi, spos, lane, xf_count);
  const float M = lr2 * LN2_F + code.log_phi;  // log (R phi)
  res.queries = q;
  res.nhit = nhit;
  if (nhit == 0) {
#pragma unroll
    for (int k = 0; k < NPL; k++) lapp[k] = lam[k];
    res.pmiss = 1.f;
    res.logD = M;
    return;
  }
  float D = M;
  for (int l = 0; l < nhit; l++) D = lse(D, sc.lp[l]);
  res.logD = D;
  res.pmiss = M == -CUDART_INF_F ? 0.f : expf(M - D);
#pragma unroll
  for (int k = 0; k < NPL; k++) {
    const int i = lane + 32 * k;
    const float x = lam[k];
    float a0 = M - softplus(-x);  // M + log sigma(x)
    float a1 = M - softplus(x);   // M + log sigma(-x)
    for (int l = 0; l < nhit; l++) {
      const bool bit = (sc.cw[l * NM + (i >> 6)] >> (i & 63)) & 1ull;
      if (bit)
        a1 = lse(a1, sc.lp[l]);
      else
        a0 = lse(a0, sc.lp[l]);
    }
    lapp[k] = a0 - a1;
  }
}

}  // namespace sg
