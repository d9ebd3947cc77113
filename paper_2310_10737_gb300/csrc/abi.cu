// abi.cu -- host side of libsogrand: the C ABI declared in include/sogrand.h,
// code objects, query-order tables, argument checks and kernel dispatch.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <new>
#include <vector>

#include "launch.h"
#include "siso_warp.cuh"
#include "sogrand.h"

struct sogrand_code {
  int n = 0, k = 0, m = 0, even = 0, c_max = 0, nm = 1;
  float log_phi = 0.f;
  int device = 0;
  uint64_t *d_hcol = nullptr;  // [n]
  uint64_t *d_hrow = nullptr;  // [m][nm]
  void *d_tab = nullptr;
  sg::DevTables tab{};
  int jmax = 1;
  int64_t tab_cap = 0;
  std::mutex mu;
};

namespace {

constexpr int64_t DEFAULT_CAP = 10000;
constexpr int64_t MAX_CAP = int64_t(1) << 24;
constexpr int64_t SAT = int64_t(1) << 60;

inline int64_t sat_add(int64_t a, int64_t b) { return (a > SAT - b) ? SAT : a + b; }

// log(2^a - 1)
double log_pow2m1(int a) { return a * std::log(2.0) + std::log1p(-std::ldexp(1.0, -a)); }

// ---------------------------------------------------------------------------
// query-order tables
// ---------------------------------------------------------------------------
struct HostTables {
  std::vector<uint64_t> pat;
  std::vector<int32_t> sbase, lbase, lnum, lcnt, loff;
  int wtop = 0, nm = 1, jmax = 1;
};

// cnt[w][m] = number of w-subsets of {1..n} with sum m (saturating), w <= wlim
struct SubsetCounts {
  int n, wlim, M;
  std::vector<int64_t> v;
  int64_t at(int w, int64_t m) const {
    if (w < 0 || w > wlim || m < 0 || m > M) return 0;
    return v[(size_t)w * (M + 1) + m];
  }
  SubsetCounts(int n_, int wlim_) : n(n_), wlim(wlim_), M(n_ * (n_ + 1) / 2) {
    v.assign((size_t)(wlim + 1) * (M + 1), 0);
    v[0] = 1;
    for (int x = 1; x <= n; x++) {
      for (int w = std::min(x, wlim); w >= 1; w--) {
        int64_t *dst = &v[(size_t)w * (M + 1)];
        const int64_t *src = &v[(size_t)(w - 1) * (M + 1)];
        const int mtop = std::min(M, w * (2 * x - w + 1) / 2);
        for (int m = mtop; m >= x; m--) dst[m] = sat_add(dst[m], src[m - x]);
      }
    }
  }
};

// append, in lexicographic order of the ascending rank vector, every
// w-subset of {lo..n} with sum `rest` to the partial mask
void emit_subsets(int n, int w, int lo, int64_t rest, uint64_t m0, uint64_t m1, int nm, std::vector<uint64_t> &out) {
  if (w == 0) {
    if (rest == 0) {
      out.push_back(m0);
      if (nm == 2) out.push_back(m1);
    }
    return;
  }
  for (int r = lo; r <= n; r++) {
    const int64_t left = rest - r;
    const int64_t k = w - 1;
    if (left < k * r + k * (k + 1) / 2) break;       // the k smallest ranks above r already exceed it
    if (left > k * n - k * (k - 1) / 2) continue;    // the k largest ranks cannot reach it
    uint64_t a = m0, b = m1;
    if (r <= 64)
      a |= 1ull << (r - 1);
    else
      b |= 1ull << (r - 65);
    emit_subsets(n, w - 1, r + 1, left, a, b, nm, out);
  }
}

int build_tables(int n, int64_t cap, int c_max, HostTables &T) {
  const int wlim = std::min(n, sg::WMAXT - 1);
  SubsetCounts N(n, wlim);
  T.nm = (n + 63) / 64;
  // weights that can be reached within `cap` queries for some c >= 0
  // (c = 0 reaches each weight earliest) in any parity class
  int wtop = 1;
  for (int K = 0; K < 3; K++) {  // 0 even, 1 odd, 2 all
    std::vector<int64_t> pre(N.M + 2, 0);
    for (int m = 0; m <= N.M; m++) {
      int64_t s = 0;
      for (int w = 0; w <= wlim; w++)
        if (K == 2 || (w & 1) == K) s = sat_add(s, N.at(w, m));
      pre[m + 1] = sat_add(pre[m], s);
    }
    for (int w = 0; w <= wlim; w++) {
      if (K != 2 && (w & 1) != K) continue;
      if (pre[w * (w + 1) / 2] <= cap) wtop = std::max(wtop, w + 1);
    }
  }
  T.wtop = wtop;
  T.sbase.assign(wtop, 0);
  T.lbase.assign(wtop, 0);
  T.lnum.assign(wtop, 0);
  int64_t total = 0;
  for (int w = 0; w < wtop; w++) {
    T.sbase[w] = (int32_t)total;
    T.lbase[w] = (int32_t)T.lcnt.size();
    const int mlo = w * (w + 1) / 2, mhi = w * (2 * n - w + 1) / 2;
    int64_t off = 0;
    for (int m = mlo; m <= mhi && off <= cap; m++) {
      const int64_t cnt = N.at(w, m);
      if (cnt >= (int64_t(1) << 30) || off + cnt >= (int64_t(1) << 30)) return SOGRAND_ENOMEM;
      T.lcnt.push_back((int32_t)cnt);
      T.loff.push_back((int32_t)off);
      const size_t before = T.pat.size();
      emit_subsets(n, w, 1, m, 0ull, 0ull, T.nm, T.pat);
      if ((int64_t)(T.pat.size() - before) != cnt * T.nm) return SOGRAND_EINVAL;  // internal consistency
      off += cnt;
    }
    T.lnum[w] = (int32_t)(T.lcnt.size() - T.lbase[w]);
    total += off;
    if (total >= (int64_t(1) << 27)) return SOGRAND_ENOMEM;
  }
  // largest cost level a search of at most `cap` queries can stop on
  // (nondecreasing in c, so evaluated at c_max), per parity class
  int64_t cmax_all = 0;
  for (int K = 0; K < 3; K++) {
    int64_t cum = 0, C = 0, last = 0;
    const int64_t Ctop = (int64_t)c_max * n + (int64_t)n * (n + 1) / 2;
    for (C = 0; C <= Ctop; C++) {
      int64_t s = 0;
      for (int w = 0; w < wtop; w++) {
        if (K != 2 && (w & 1) != K) continue;
        s = sat_add(s, N.at(w, C - (int64_t)c_max * w));
      }
      if (s) last = C;
      cum = sat_add(cum, s);
      if (cum >= cap) break;
    }
    cmax_all = std::max(cmax_all, std::min(C, Ctop) > last ? std::min(C, Ctop) : last);
  }
  if (cmax_all > 60000) return SOGRAND_ENOMEM;
  T.jmax = (int)cmax_all + 2;
  return SOGRAND_OK;
}

int upload_tables(sogrand_code *c, const HostTables &T, int64_t cap) {
  const size_t bpat = T.pat.size() * sizeof(uint64_t);
  const size_t nw = T.sbase.size(), nl = T.lcnt.size();
  const size_t bint = (3 * nw + 2 * nl) * sizeof(int32_t);
  const size_t bytes = ((bpat + 255) & ~size_t(255)) + bint + 16;
  void *mem = nullptr;
  if (cudaMalloc(&mem, bytes) != cudaSuccess) return SOGRAND_ENOMEM;
  char *p = (char *)mem;
  uint64_t *dpat = (uint64_t *)p;
  int32_t *di = (int32_t *)(p + ((bpat + 255) & ~size_t(255)));
  std::vector<int32_t> ints;
  ints.reserve(3 * nw + 2 * nl);
  ints.insert(ints.end(), T.sbase.begin(), T.sbase.end());
  ints.insert(ints.end(), T.lbase.begin(), T.lbase.end());
  ints.insert(ints.end(), T.lnum.begin(), T.lnum.end());
  ints.insert(ints.end(), T.lcnt.begin(), T.lcnt.end());
  ints.insert(ints.end(), T.loff.begin(), T.loff.end());
  if ((bpat && cudaMemcpy(dpat, T.pat.data(), bpat, cudaMemcpyHostToDevice) != cudaSuccess) ||
      cudaMemcpy(di, ints.data(), ints.size() * sizeof(int32_t), cudaMemcpyHostToDevice) != cudaSuccess) {
    cudaFree(mem);
    return SOGRAND_ECUDA;
  }
  if (c->d_tab) {
    cudaDeviceSynchronize();  // no decode may still read the old tables
    cudaFree(c->d_tab);
  }
  c->d_tab = mem;
  c->tab.pat = dpat;
  c->tab.sbase = di;
  c->tab.lbase = di + nw;
  c->tab.lnum = di + 2 * nw;
  c->tab.lcnt = di + 3 * nw;
  c->tab.loff = di + 3 * nw + nl;
  c->tab.wtop = T.wtop;
  c->tab.nm = T.nm;
  c->jmax = T.jmax;
  c->tab_cap = cap;
  return SOGRAND_OK;
}

int reserve_locked(sogrand_code *c, int64_t cap) {
  if (cap <= c->tab_cap) return SOGRAND_OK;
  HostTables T;
  int rc;
  try {
    rc = build_tables(c->n, cap, c->c_max, T);
  } catch (const std::bad_alloc &) {
    return SOGRAND_ENOMEM;
  }
  if (rc != SOGRAND_OK) return rc;
  return upload_tables(c, T, cap);
}

sg::DevCode dev_code(const sogrand_code *c) {
  sg::DevCode d{};
  d.n = c->n;
  d.k = c->k;
  d.m = c->m;
  d.even = c->even;
  d.c_max = c->c_max;
  d.log_phi = c->log_phi;
  d.hcol = c->d_hcol;
  d.hrow = c->d_hrow;
  d.tab = c->tab;
  d.jmax = c->jmax;
  return d;
}

// GF(2) rank test: is the all-ones vector in the row space of H?
bool ones_in_rowspace(int n, int m, const uint8_t *H) {
  std::vector<std::vector<uint8_t>> A(m + 1, std::vector<uint8_t>(n));
  for (int t = 0; t < m; t++)
    for (int i = 0; i < n; i++) A[t][i] = H[(size_t)t * n + i] & 1;
  auto rank = [n](std::vector<std::vector<uint8_t>> M) {
    int r = 0;
    for (int col = 0; col < n && r < (int)M.size(); col++) {
      int piv = -1;
      for (int i = r; i < (int)M.size(); i++)
        if (M[i][col]) {
          piv = i;
          break;
        }
      if (piv < 0) continue;
      std::swap(M[r], M[piv]);
      for (int i = 0; i < (int)M.size(); i++)
        if (i != r && M[i][col])
          for (int j = 0; j < n; j++) M[i][j] ^= M[r][j];
      r++;
    }
    return r;
  };
  std::vector<std::vector<uint8_t>> Hm(A.begin(), A.begin() + m);
  const int r0 = rank(Hm);
  for (int i = 0; i < n; i++) A[m][i] = 1;
  return rank(A) == r0;
}

#define SG_DISPATCH(code, CALL)                                            \
  do {                                                                     \
    const int npl_ = (code)->n <= 32 ? 1 : ((code)->n <= 64 ? 2 : 4);      \
    const bool s32_ = (code)->m <= 32;                                     \
    if (npl_ == 1 && s32_) {                                               \
      constexpr int NPL = 1;                                               \
      using SYN = uint32_t;                                                \
      CALL;                                                                \
    } else if (npl_ == 1) {                                                \
      constexpr int NPL = 1;                                               \
      using SYN = uint64_t;                                                \
      CALL;                                                                \
    } else if (npl_ == 2 && s32_) {                                        \
      constexpr int NPL = 2;                                               \
      using SYN = uint32_t;                                                \
      CALL;                                                                \
    } else if (npl_ == 2) {                                                \
      constexpr int NPL = 2;                                               \
      using SYN = uint64_t;                                                \
      CALL;                                                                \
    } else if (s32_) {                                                     \
      constexpr int NPL = 4;                                               \
      using SYN = uint32_t;                                                \
      CALL;                                                                \
    } else {                                                               \
      constexpr int NPL = 4;                                               \
      using SYN = uint64_t;                                                \
      CALL;                                                                \
    }                                                                      \
  } while (0)

int ensure_cap(sogrand_code *c, int64_t cap) {
  std::lock_guard<std::mutex> g(c->mu);
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev != c->device) return SOGRAND_EINVAL;
  return reserve_locked(c, cap);
}

}  // namespace

namespace sg {
int scratch_bytes(int npl, int syn_bytes, int jmax) {
  if (npl == 1) return syn_bytes == 4 ? Layout<1, uint32_t>::bytes(jmax) : Layout<1, uint64_t>::bytes(jmax);
  if (npl == 2) return syn_bytes == 4 ? Layout<2, uint32_t>::bytes(jmax) : Layout<2, uint64_t>::bytes(jmax);
  return syn_bytes == 4 ? Layout<4, uint32_t>::bytes(jmax) : Layout<4, uint64_t>::bytes(jmax);
}
}  // namespace sg

extern "C" {

const char *sogrand_strerror(int err) {
  switch (err) {
    case SOGRAND_OK: return "ok";
    case SOGRAND_EINVAL: return "invalid argument";
    case SOGRAND_ENOMEM: return "out of memory";
    case SOGRAND_ECUDA: return "CUDA runtime error";
    case SOGRAND_ETIMEOUT: return "bounded device wait timed out";
    case SOGRAND_EUNSUPPORTED: return "unsupported configuration";
    default: return "unknown error";
  }
}

int sogrand_code_create(int n, int k, const uint8_t *H, int even, sogrand_code **out) {
  if (!out) return SOGRAND_EINVAL;
  *out = nullptr;
  if (n < 2 || n > sg::NMAX || k < 1 || k >= n || n - k > 64 || !H || (even != 0 && even != 1))
    return SOGRAND_EINVAL;
  const int m = n - k;
  for (int i = 0; i < m * n; i++)
    if (H[i] > 1) return SOGRAND_EINVAL;
  if (even && !ones_in_rowspace(n, m, H)) return SOGRAND_EINVAL;
  sogrand_code *c = new (std::nothrow) sogrand_code();
  if (!c) return SOGRAND_ENOMEM;
  c->n = n;
  c->k = k;
  c->m = m;
  c->even = even;
  c->c_max = n;
  c->nm = (n + 63) / 64;
  c->log_phi = (float)(log_pow2m1(k) - log_pow2m1(even ? n - 1 : n));
  cudaGetDevice(&c->device);
  std::vector<uint64_t> hcol(n, 0), hrow((size_t)m * c->nm, 0);
  for (int t = 0; t < m; t++)
    for (int i = 0; i < n; i++)
      if (H[(size_t)t * n + i]) {
        hcol[i] |= 1ull << t;
        hrow[(size_t)t * c->nm + (i >> 6)] |= 1ull << (i & 63);
      }
  if (cudaMalloc(&c->d_hcol, n * sizeof(uint64_t)) != cudaSuccess ||
      cudaMalloc(&c->d_hrow, hrow.size() * sizeof(uint64_t)) != cudaSuccess) {
    sogrand_code_destroy(c);
    return SOGRAND_ENOMEM;
  }
  if (cudaMemcpy(c->d_hcol, hcol.data(), n * sizeof(uint64_t), cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(c->d_hrow, hrow.data(), hrow.size() * sizeof(uint64_t), cudaMemcpyHostToDevice) != cudaSuccess) {
    sogrand_code_destroy(c);
    return SOGRAND_ECUDA;
  }
  int rc = reserve_locked(c, DEFAULT_CAP);
  if (rc != SOGRAND_OK) {
    sogrand_code_destroy(c);
    return rc;
  }
  *out = c;
  return SOGRAND_OK;
}

void sogrand_code_destroy(sogrand_code *c) {
  if (!c) return;
  if (c->d_hcol) cudaFree(c->d_hcol);
  if (c->d_hrow) cudaFree(c->d_hrow);
  if (c->d_tab) cudaFree(c->d_tab);
  delete c;
}

int sogrand_code_reserve(sogrand_code *c, int64_t cap) {
  if (!c || cap < 1 || cap > MAX_CAP) return SOGRAND_EINVAL;
  return ensure_cap(c, cap);
}

int sogrand_code_info(const sogrand_code *c, int *n, int *k) {
  if (!c) return SOGRAND_EINVAL;
  if (n) *n = c->n;
  if (k) *k = c->k;
  return SOGRAND_OK;
}

int sogrand_decode(sogrand_code *c, int64_t n_words, const float *llr_ch, const float *llr_a, int L, int64_t cap,
                   float thr, uint8_t *hard, float *llr_app, float *llr_ext, float *p_miss, int64_t *queries,
                   uint64_t *list_words, float *list_app, int32_t *list_count, void *stream) {
  if (!c || n_words < 0 || L < 1 || L > sg::LMAX || cap < 1 || cap > MAX_CAP || !(thr >= 0.f && thr < 1.f))
    return SOGRAND_EINVAL;
  if (n_words > 0 && !llr_ch) return SOGRAND_EINVAL;
  if (n_words == 0) return SOGRAND_OK;
  int rc = ensure_cap(c, cap);
  if (rc != SOGRAND_OK) return rc;
  sg::DevCode d = dev_code(c);
  sg::SisoParams P{L, (int32_t)cap, thr};
  sg::DecodeArgs a{n_words, llr_ch, llr_a, hard, llr_app, llr_ext, p_miss, queries, list_words, list_app, list_count,
                   nullptr};
  cudaError_t e;
  SG_DISPATCH(c, e = (sg::launch_decode<NPL, SYN>(d, P, a, (cudaStream_t)stream)));
  return e == cudaSuccess ? SOGRAND_OK : SOGRAND_ECUDA;
}

int product_decode_ex(sogrand_code *rc_, const sogrand_code *cc_, int64_t F, const float *llr_ch, int L, int64_t cap,
                      float thr, float alpha, int max_iter, uint8_t *bits, int32_t *half_iters, uint8_t *status,
                      int64_t *queries, int64_t *par_queries, int32_t *xf_words, void *stream) {
  if (!rc_ || !cc_ || F < 0 || L < 1 || L > sg::LMAX || cap < 1 || cap > MAX_CAP || !(thr >= 0.f && thr < 1.f) ||
      !(alpha > 0.f && alpha < 1e6f) || max_iter < 1 || max_iter > 1000)
    return SOGRAND_EINVAL;
  if (rc_ != cc_) return SOGRAND_EUNSUPPORTED;
  sogrand_code *c = rc_;
  if (c->n - 1 < 63 && cap >= (int64_t(1) << (c->n - 1))) return SOGRAND_EINVAL;
  if (F == 0) return SOGRAND_OK;
  if (!llr_ch || !bits) return SOGRAND_EINVAL;
  int rc = ensure_cap(c, cap);
  if (rc != SOGRAND_OK) return rc;
  cudaStream_t s = (cudaStream_t)stream;
  const int n = c->n, nm = c->nm;
  // scratch, stream-ordered
  const size_t b_le = (size_t)F * n * n * sizeof(float);
  const size_t b_hb = (size_t)F * n * nm * sizeof(uint64_t);
  const size_t b_i32 = (size_t)F * sizeof(int32_t);
  const size_t b_i64 = (size_t)F * sizeof(int64_t);
  auto al = [](size_t x) { return (x + 255) & ~size_t(255); };
  // every sub-buffer starts on a 256-byte boundary (64-bit atomics need 8)
  const size_t total = al(b_le) + al(b_hb) + 2 * al(b_i32) + (half_iters ? 0 : al(b_i32)) +
                       (queries ? 0 : al(b_i64)) + (par_queries ? 0 : al(b_i64)) + (status ? 0 : al((size_t)F)) + 256;
  char *mem = nullptr;
  if (cudaMallocAsync((void **)&mem, total, s) != cudaSuccess) return SOGRAND_ENOMEM;
  char *p = mem;
  auto take = [&p, &al](size_t bytes) {
    char *r = p;
    p += al(bytes);
    return r;
  };
  sg::ProductArgs a{};
  a.n_frames = F;
  a.llr_ch = llr_ch;
  a.alpha = alpha;
  a.max_half = 2 * max_iter;
  a.le = (float *)take(b_le);
  a.hb = (uint64_t *)take(b_hb);
  a.fstate = (int32_t *)take(b_i32);
  a.hmax = (int32_t *)take(b_i32);
  a.bits = bits;
  a.half_iters = half_iters ? half_iters : (int32_t *)take(b_i32);
  a.queries = queries ? queries : (int64_t *)take(b_i64);
  a.par_queries = par_queries ? par_queries : (int64_t *)take(b_i64);
  a.status = status ? status : (uint8_t *)take((size_t)F);
  a.active = (int32_t *)take(sizeof(int32_t));
  a.xf_count = xf_words;
  sg::DevCode d = dev_code(c);
  sg::SisoParams P{L, (int32_t)cap, thr};
  cudaError_t e = cudaSuccess;
  SG_DISPATCH(c, e = (sg::launch_product_init<NPL, SYN>(d, a, s)));
  for (int h = 1; h <= a.max_half && e == cudaSuccess; h++) {
    SG_DISPATCH(c, e = (sg::launch_product_half<NPL, SYN>(d, P, a, h, s)));
    if (e != cudaSuccess) break;
    e = cudaMemsetAsync(a.active, 0, sizeof(int32_t), s);
    if (e != cudaSuccess) break;
    SG_DISPATCH(c, e = (sg::launch_product_check<NPL, SYN>(d, a, h, s)));
    if (e != cudaSuccess) break;
    int32_t act = 1;
    e = cudaMemcpyAsync(&act, a.active, sizeof(int32_t), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e == cudaSuccess && act == 0) break;
  }
  cudaError_t e2 = cudaFreeAsync(mem, s);
  if (e != cudaSuccess || e2 != cudaSuccess) return SOGRAND_ECUDA;
  return SOGRAND_OK;
}

int product_decode(sogrand_code *row_code, const sogrand_code *col_code, int64_t n_frames, const float *llr_ch, int L,
                   int64_t cap, float thr, float alpha, int max_iter, uint8_t *bits, int32_t *half_iters,
                   uint8_t *status, int64_t *queries, void *stream) {
  return product_decode_ex(row_code, col_code, n_frames, llr_ch, L, cap, thr, alpha, max_iter, bits, half_iters,
                           status, queries, nullptr, nullptr, stream);
}

int sogrand_trace_patterns(sogrand_code *c, const float *llr, int64_t max_q, uint64_t *patterns_out, int64_t *n_out,
                           int32_t *c_out) {
  if (!c || !llr || max_q < 1 || max_q > MAX_CAP || !patterns_out || !n_out) return SOGRAND_EINVAL;
  int rc = ensure_cap(c, max_q);
  if (rc != SOGRAND_OK) return rc;
  const int n = c->n, nm = c->nm;
  float *dl = nullptr;
  uint64_t *dout = nullptr;
  int32_t *dcnt = nullptr;
  if (cudaMalloc(&dl, n * sizeof(float)) != cudaSuccess || cudaMalloc(&dout, max_q * nm * sizeof(uint64_t)) != cudaSuccess ||
      cudaMalloc(&dcnt, 2 * sizeof(int32_t)) != cudaSuccess) {
    cudaFree(dl);
    cudaFree(dout);
    cudaFree(dcnt);
    return SOGRAND_ENOMEM;
  }
  cudaError_t e = cudaMemcpy(dl, llr, n * sizeof(float), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemset(dcnt, 0, 2 * sizeof(int32_t));
  sg::DevCode d = dev_code(c);
  if (e == cudaSuccess) SG_DISPATCH(c, e = (sg::launch_trace<NPL, SYN>(d, dl, (int)max_q, dout, dcnt, dcnt + 1, 0)));
  int32_t h[2] = {0, 0};
  if (e == cudaSuccess) e = cudaMemcpy(h, dcnt, 2 * sizeof(int32_t), cudaMemcpyDeviceToHost);
  if (e == cudaSuccess && h[0] > 0)
    e = cudaMemcpy(patterns_out, dout, (size_t)h[0] * nm * sizeof(uint64_t), cudaMemcpyDeviceToHost);
  cudaFree(dl);
  cudaFree(dout);
  cudaFree(dcnt);
  if (e != cudaSuccess) return SOGRAND_ECUDA;
  if (h[0] < 0) return SOGRAND_EINVAL;  // non-finite input
  *n_out = h[0];
  if (c_out) *c_out = h[1];
  return SOGRAND_OK;
}

}  // extern "C"
