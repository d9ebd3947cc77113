// abi.cu -- host side of libsogrand: the C ABI declared in include/sogrand.h,
// code objects, query-order tables, argument checks and kernel dispatch.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <memory>
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
  sg::DevOrder ord{};
  sg::DevGroups grp{};
  int jmax = 1;
  int minb = 12;  // schedule: resident blocks per SM (8 or 12), see sogrand_code_tune
  int dp_global = 1;  // schedule: the batched forms keep the remaining-mass area in global memory
  int ord_lanes = 0;  // 1: lanes enumerate the query order instead of reading the order table
  int64_t tab_cap = 0;
  int64_t tab_bytes = 0;
  std::mutex mu;
};

namespace {

constexpr int64_t DEFAULT_CAP = 10000;
constexpr int64_t MAX_CAP = int64_t(1) << 24;
constexpr int64_t SAT = int64_t(1) << 60;

inline int64_t sat_add(int64_t a, int64_t b) { return (a > SAT - b) ? SAT : a + b; }

// Limits of the bounded device waits (sogrand_set_wait_limits), read when a
// decode is launched: a persistent launch's warps give up after this much
// accumulated back-off without work; a warp gives up on the block's
// remaining-mass lock after lock_polls polls.
std::atomic<int64_t> g_queue_wait_us{2000000};
std::atomic<int64_t> g_lock_polls{int64_t(1) << 22};
std::atomic<int> g_lock_preheld{0};

sg::SisoParams siso_params(int L, int64_t cap, float thr, int forney = 0) {
  sg::SisoParams P{L, (int32_t)cap, thr};
  P.forney = forney;
  P.lock_polls = (int32_t)g_lock_polls.load();
  P.lock_preheld = g_lock_preheld.load();
  return P;
}

// log(2^a - 1)
double log_pow2m1(int a) { return a * std::log(2.0) + std::log1p(-std::ldexp(1.0, -a)); }

// ---------------------------------------------------------------------------
// query-order tables
// ---------------------------------------------------------------------------
struct HostTables {
  std::vector<uint4> ent;       // weight byte + rank bytes, per (c, class) order, concatenated
  std::vector<uint16_t> cost;   // cost of each entry
  std::vector<int32_t> base, count;
  int ncls = 1, class_size = 0, jmax = 1;
  // groups (one cost, one weight) of every order and the subset counts that
  // unrank a pattern within its group (on-lane enumeration)
  std::vector<uint2> grp;       // x: first entry within the order; y: m | w << 16
  std::vector<int32_t> gbase;   // first group of order (c, class); one extra end entry
  std::vector<int32_t> scnt;    // [N = 0..n][w < sc_w][m < sc_m]
  int sc_w = 1, sc_m = 1;
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

// Append, in lexicographic order of the ascending rank vector, every subset
// of {lo..n} with `left` more elements and sum `rest` (ranks 1-based here,
// stored 0-based in bytes 1..w of the entry; bytes past w hold n, the index
// of a neutral rank record: H column 0, mass factor 1).
void emit_subsets(int n, int w, int depth, int lo, int64_t rest, uint8_t *bytes, std::vector<uint4> &out) {
  const int left = w - depth;
  if (left == 0) {
    if (rest == 0) {
      uint4 e;
      std::memcpy(&e, bytes, 16);
      out.push_back(e);
    }
    return;
  }
  for (int r = lo; r <= n; r++) {
    const int64_t rem = rest - r;
    const int64_t k = left - 1;
    if (rem < k * r + k * (k + 1) / 2) break;     // the k smallest ranks above r already exceed it
    if (rem > k * n - k * (k - 1) / 2) continue;  // the k largest ranks cannot reach it
    bytes[1 + depth] = (uint8_t)(r - 1);
    emit_subsets(n, w, depth + 1, r + 1, rem, bytes, out);
  }
  bytes[1 + depth] = (uint8_t)n;
}

int build_tables(int n, int64_t cap, int c_max, bool even, HostTables &T) {
  const int wlim = std::min(n, sg::WMAXT - 1);
  SubsetCounts N(n, wlim);
  const int ncls = even ? 2 : 1;
  // weights reachable within `cap` queries for some c >= 0 (c = 0 reaches
  // each weight earliest) in any class
  int wtop = 1;
  for (int K = 0; K < ncls; K++) {
    std::vector<int64_t> pre(N.M + 2, 0);
    for (int m = 0; m <= N.M; m++) {
      int64_t s = 0;
      for (int w = 0; w <= wlim; w++)
        if (!even || (w & 1) == K) s = sat_add(s, N.at(w, m));
      pre[m + 1] = sat_add(pre[m], s);
    }
    for (int w = 0; w <= wlim; w++) {
      if (even && (w & 1) != K) continue;
      if (pre[w * (w + 1) / 2] <= cap) wtop = std::max(wtop, w + 1);
    }
  }
  if (wtop - 1 > sg::WENT) return SOGRAND_EUNSUPPORTED;
  // per-weight streams: every w-subset in (logistic weight, lexicographic)
  // order, complete levels while the level starts within the first `cap`
  std::vector<std::vector<uint4>> stream(wtop);
  std::vector<std::vector<int64_t>> loff(wtop);  // level start, indexed by m - mmin(w); one extra end entry
  for (int w = 0; w < wtop; w++) {
    const int mlo = w * (w + 1) / 2, mhi = w * (2 * n - w + 1) / 2;
    int64_t off = 0;
    uint8_t bytes[16];
    std::memset(bytes, n, sizeof(bytes));
    bytes[0] = (uint8_t)w;
    for (int m = mlo; m <= mhi && off <= cap; m++) {
      const int64_t cnt = N.at(w, m);
      if (off + cnt >= (int64_t(1) << 28)) return SOGRAND_ENOMEM;
      loff[w].push_back(off);
      emit_subsets(n, w, 0, 1, m, bytes, stream[w]);
      off += cnt;
      if ((int64_t)stream[w].size() != off) return SOGRAND_EINVAL;  // internal consistency
    }
    loff[w].push_back(off);
  }
  // merged order for every (c, class)
  T.ncls = ncls;
  const int nb = even ? n - 1 : n;
  T.class_size = nb >= 31 ? INT32_MAX : (1 << nb);
  T.base.assign((size_t)(c_max + 1) * ncls, 0);
  T.count.assign((size_t)(c_max + 1) * ncls, 0);
  int maxcost = 0, maxm = 0;
  for (int c = 0; c <= c_max; c++) {
    for (int K = 0; K < ncls; K++) {
      const size_t start = T.ent.size();
      T.gbase.push_back((int32_t)T.grp.size());
      const int64_t Ctop = (int64_t)c * n + (int64_t)n * (n + 1) / 2;
      for (int64_t C = 0; C <= Ctop && (int64_t)(T.ent.size() - start) < cap; C++) {
        for (int w = 0; w < wtop; w++) {
          if (even && (w & 1) != K) continue;
          const int64_t m = C - (int64_t)c * w;
          const int64_t mlo = w * (w + 1) / 2;
          if (m < mlo) break;
          const int64_t li = m - mlo;
          if (li + 1 >= (int64_t)loff[w].size()) continue;  // past the stored levels (beyond the cap)
          const int64_t a = loff[w][li], b = loff[w][li + 1];
          if (b == a) continue;
          if (C > 65535) return SOGRAND_EUNSUPPORTED;
          T.grp.push_back(make_uint2((unsigned)(T.ent.size() - start), (unsigned)m | ((unsigned)w << 16)));
          maxm = std::max(maxm, (int)m);
          T.ent.insert(T.ent.end(), stream[w].begin() + a, stream[w].begin() + b);
          T.cost.insert(T.cost.end(), (size_t)(b - a), (uint16_t)C);
          maxcost = std::max(maxcost, (int)C);
        }
        if (T.ent.size() >= (size_t(1) << 30)) return SOGRAND_ENOMEM;
      }
      T.base[(size_t)c * ncls + K] = (int32_t)start;
      T.count[(size_t)c * ncls + K] = (int32_t)(T.ent.size() - start);
    }
  }
  T.jmax = maxcost + 2;
  T.gbase.push_back((int32_t)T.grp.size());
  // scnt[N][w][m]: w-subsets of {1..N} with sum m (N = 0..n, w < sc_w, m <= the
  // largest group sum), saturated at INT32_MAX: unranking only subtracts a
  // count smaller than the index it reduces, which is below the group's size
  T.sc_w = wtop;
  T.sc_m = maxm + 1;
  const size_t plane = (size_t)T.sc_w * T.sc_m;
  T.scnt.assign((size_t)(n + 1) * plane, 0);
  T.scnt[0] = 1;
  for (int N = 1; N <= n; N++) {
    const int32_t *prev = &T.scnt[(size_t)(N - 1) * plane];
    int32_t *cur = &T.scnt[(size_t)N * plane];
    for (int w = 0; w < T.sc_w; w++)
      for (int m = 0; m < T.sc_m; m++) {
        int64_t v = prev[(size_t)w * T.sc_m + m];
        if (w >= 1 && m >= N) v += prev[(size_t)(w - 1) * T.sc_m + (m - N)];
        cur[(size_t)w * T.sc_m + m] = (int32_t)std::min<int64_t>(v, INT32_MAX);
      }
  }
  return SOGRAND_OK;
}

int upload_tables(sogrand_code *c, const HostTables &T, int64_t cap) {
  auto al = [](size_t x) { return (x + 255) & ~size_t(255); };
  const size_t be = T.ent.size() * sizeof(uint4), bc = T.cost.size() * sizeof(uint16_t);
  const size_t bi = T.base.size() * sizeof(int32_t);
  const size_t bg = T.grp.size() * sizeof(uint2), bgb = T.gbase.size() * sizeof(int32_t);
  const size_t bs = T.scnt.size() * sizeof(int32_t);
  const size_t bytes = al(be) + al(bc) + 2 * al(bi) + al(bg) + al(bgb) + al(bs);
  void *mem = nullptr;
  if (cudaMalloc(&mem, bytes) != cudaSuccess) return SOGRAND_ENOMEM;
  char *p = (char *)mem;
  uint4 *dent = (uint4 *)p;
  uint16_t *dcost = (uint16_t *)(p + al(be));
  int32_t *dbase = (int32_t *)(p + al(be) + al(bc));
  int32_t *dcount = (int32_t *)(p + al(be) + al(bc) + al(bi));
  uint2 *dgrp = (uint2 *)(p + al(be) + al(bc) + 2 * al(bi));
  int32_t *dgbase = (int32_t *)((char *)dgrp + al(bg));
  int32_t *dscnt = (int32_t *)((char *)dgbase + al(bgb));
  if (cudaMemcpy(dgrp, T.grp.data(), bg, cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(dgbase, T.gbase.data(), bgb, cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(dscnt, T.scnt.data(), bs, cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(dent, T.ent.data(), be, cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(dcost, T.cost.data(), bc, cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(dbase, T.base.data(), bi, cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(dcount, T.count.data(), bi, cudaMemcpyHostToDevice) != cudaSuccess) {
    cudaFree(mem);
    return SOGRAND_ECUDA;
  }
  if (c->d_tab) {
    cudaDeviceSynchronize();  // no decode may still read the old tables
    cudaFree(c->d_tab);
  }
  c->d_tab = mem;
  c->ord.ent = dent;
  c->ord.cost = dcost;
  c->ord.base = dbase;
  c->ord.count = dcount;
  c->ord.ncls = T.ncls;
  c->ord.class_size = T.class_size;
  c->grp.grp = dgrp;
  c->grp.gbase = dgbase;
  c->grp.scnt = dscnt;
  c->grp.sc_w = T.sc_w;
  c->grp.sc_m = T.sc_m;
  c->jmax = T.jmax;
  c->tab_cap = cap;
  c->tab_bytes = (int64_t)bytes;
  return SOGRAND_OK;
}

int reserve_locked(sogrand_code *c, int64_t cap) {
  if (cap <= c->tab_cap) return SOGRAND_OK;
  HostTables T;
  int rc;
  try {
    rc = build_tables(c->n, cap, c->c_max, c->even != 0, T);
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
  d.ord = c->ord;
  d.jmax = c->jmax;
  d.minb = c->minb;
  d.dp_global = c->dp_global;
  d.ord_lanes = c->ord_lanes;
  d.grp = c->grp;
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

// ---------------------------------------------------------------------------
// device scratch: one stream-ordered memory pool per device, owned by the
// library.  It keeps its memory between calls (release threshold: never), so
// the per-frame L_E state (4 n^2 bytes a frame, gigabytes for a large batch)
// is not unmapped and mapped again on every decode.  sogrand_release_cached
// hands the idle memory back.
// ---------------------------------------------------------------------------
constexpr int MAX_DEV = 64;
std::mutex g_pool_mu;
cudaMemPool_t g_pool[MAX_DEV] = {};

cudaError_t scratch_alloc(char **p, size_t bytes, cudaStream_t s) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= MAX_DEV) return cudaErrorInvalidDevice;
  cudaMemPool_t pool = nullptr;
  {
    std::lock_guard<std::mutex> g(g_pool_mu);
    if (!g_pool[dev]) {
      cudaMemPoolProps pp{};
      pp.allocType = cudaMemAllocationTypePinned;
      pp.handleTypes = cudaMemHandleTypeNone;
      pp.location.type = cudaMemLocationTypeDevice;
      pp.location.id = dev;
      e = cudaMemPoolCreate(&g_pool[dev], &pp);
      if (e != cudaSuccess) {
        g_pool[dev] = nullptr;
        return e;
      }
      uint64_t keep = UINT64_MAX;
      e = cudaMemPoolSetAttribute(g_pool[dev], cudaMemPoolAttrReleaseThreshold, &keep);
      if (e != cudaSuccess) return e;
    }
    pool = g_pool[dev];
  }
  return cudaMallocFromPoolAsync((void **)p, bytes, pool, s);
}

// Row and column codes of a product code: the same code, or two codes of the
// same kernel class (bits per lane and syndrome width), which one
// instantiation of the product kernels decodes.
int pair_check(const sogrand_code *r, const sogrand_code *c) {
  if (r == c) return SOGRAND_OK;
  auto npl = [](int n) { return n <= 32 ? 1 : (n <= 64 ? 2 : 4); };
  if (npl(r->n) != npl(c->n) || (r->m > 32) != (c->m > 32) || r->device != c->device) return SOGRAND_EUNSUPPORTED;
  return SOGRAND_OK;
}

int ensure_cap(sogrand_code *c, int64_t cap) {
  std::lock_guard<std::mutex> g(c->mu);
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev != c->device) return SOGRAND_EINVAL;
  return reserve_locked(c, cap);
}

}  // namespace

#ifdef SG_PHASE_PROFILE
namespace sg {
std::vector<PhaseReader> &phase_readers() {
  static std::vector<PhaseReader> v;
  return v;
}
void phase_register(PhaseReader r) { phase_readers().push_back(r); }
}  // namespace sg
#endif

// Accessors for the serving loop (server.cu), which sees codes only through these.
namespace sgi {
sg::DevCode dev_code_of(const sogrand_code *c) { return dev_code(c); }
int code_n(const sogrand_code *c) { return c->n; }
int code_nm(const sogrand_code *c) { return c->nm; }
int code_m(const sogrand_code *c) { return c->m; }
int ensure_code_cap(sogrand_code *c, int64_t cap) { return ensure_cap(c, cap); }
cudaError_t launch_persistent_for(const sogrand_code *c, const sg::SisoParams &P, const sg::ProductArgs &a,
                                  cudaStream_t s) {
  const sg::DevCode d = dev_code(c);
  cudaError_t e = cudaSuccess;
  SG_DISPATCH(c, e = (sg::launch_product_persistent<NPL, SYN, false>(d, d, P, a, s)));
  return e;
}
sg::SisoParams siso_params_of(int L, int64_t cap, float thr) { return siso_params(L, cap, thr); }
int32_t queue_wait_us() { return (int32_t)g_queue_wait_us.load(); }
int code_dp_global(const sogrand_code *c) { return c->dp_global; }
int dp_slice(const sogrand_code *c) {
  return sg::dp_slice_bytes(c->n <= 32 ? 1 : (c->n <= 64 ? 2 : 4), c->m > 32 ? 8 : 4, c->jmax);
}
int sm_count_of_device() {
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  return sms > 0 ? sms : 1;
}
}  // namespace sgi

namespace sg {
int dp_area_bytes(int npl, int syn_bytes, int jmax) {
  if (npl == 1) return syn_bytes == 4 ? Layout<1, uint32_t>::dp_bytes(jmax) : Layout<1, uint64_t>::dp_bytes(jmax);
  if (npl == 2) return syn_bytes == 4 ? Layout<2, uint32_t>::dp_bytes(jmax) : Layout<2, uint64_t>::dp_bytes(jmax);
  return syn_bytes == 4 ? Layout<4, uint32_t>::dp_bytes(jmax) : Layout<4, uint64_t>::dp_bytes(jmax);
}
int dp_slice_bytes(int npl, int syn_bytes, int jmax) { return (dp_area_bytes(npl, syn_bytes, jmax) + 127) & ~127; }
}  // namespace sg

extern "C" {

int sogrand_release_cached(void) {
  std::lock_guard<std::mutex> g(g_pool_mu);
  for (int d = 0; d < MAX_DEV; d++)
    if (g_pool[d] && cudaMemPoolTrimTo(g_pool[d], 0) != cudaSuccess) return SOGRAND_ECUDA;
  return SOGRAND_OK;
}

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
  // default schedule until tuned: 12 blocks per SM (40 registers) for codes
  // of up to 64 bits, else 8 (64 registers)
  c->minb = n <= 64 ? 12 : 8;
  // and the remaining-mass area in global memory for the others (they gain L1)
  c->dp_global = (n <= 64 && m <= 8) ? 0 : 1;
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

int sogrand_code_tables(const sogrand_code *c, int64_t *query_cap, int64_t *bytes) {
  if (!c) return SOGRAND_EINVAL;
  std::lock_guard<std::mutex> g(const_cast<sogrand_code *>(c)->mu);
  if (query_cap) *query_cap = c->tab_cap;
  if (bytes) *bytes = c->tab_bytes;
  return SOGRAND_OK;
}

int sogrand_set_wait_limits(int64_t queue_wait_us, int64_t lock_polls, int lock_preheld) {
  if (queue_wait_us > INT32_MAX || lock_polls > INT32_MAX || lock_preheld > 1) return SOGRAND_EINVAL;
  if (queue_wait_us >= 0) g_queue_wait_us.store(queue_wait_us);
  if (lock_polls >= 0) g_lock_polls.store(lock_polls);
  if (lock_preheld >= 0) g_lock_preheld.store(lock_preheld);
  return SOGRAND_OK;
}

}  // extern "C"

namespace {
int decode_words(sogrand_code *c, int64_t n_words, const float *llr_ch, const float *llr_a, int L, int64_t cap,
                 float thr, int forney, uint8_t *hard, float *llr_app, float *llr_ext, float *p_miss, int64_t *queries,
                 uint64_t *list_words, float *list_app, int32_t *list_count, void *stream) {
  if (!c || n_words < 0 || L < 1 || L > sg::LMAX || cap < 1 || cap > MAX_CAP || !(thr >= 0.f && thr < 1.f) ||
      (forney && thr > 0.f))
    return SOGRAND_EINVAL;
  if (n_words > 0 && !llr_ch) return SOGRAND_EINVAL;
  if (n_words == 0) return SOGRAND_OK;
  int rc = ensure_cap(c, cap);
  if (rc != SOGRAND_OK) return rc;
  sg::DevCode d = dev_code(c);
  sg::SisoParams P = siso_params(L, cap, thr, forney);
  sg::DecodeArgs a{n_words, llr_ch, llr_a, hard, llr_app, llr_ext, p_miss, queries, list_words, list_app, list_count,
                   nullptr};
  cudaError_t e;
  SG_DISPATCH(c, e = (sg::launch_decode<NPL, SYN>(d, P, a, (cudaStream_t)stream)));
  return e == cudaSuccess ? SOGRAND_OK : SOGRAND_ECUDA;
}
}  // namespace

extern "C" {

int sogrand_decode(sogrand_code *c, int64_t n_words, const float *llr_ch, const float *llr_a, int L, int64_t cap,
                   float thr, uint8_t *hard, float *llr_app, float *llr_ext, float *p_miss, int64_t *queries,
                   uint64_t *list_words, float *list_app, int32_t *list_count, void *stream) {
  return decode_words(c, n_words, llr_ch, llr_a, L, cap, thr, 0, hard, llr_app, llr_ext, p_miss, queries, list_words,
                      list_app, list_count, stream);
}

int sogrand_decode_forney(sogrand_code *c, int64_t n_words, const float *llr_ch, const float *llr_a, int L,
                          int64_t cap, uint8_t *hard, float *llr_app, float *llr_ext, float *p_miss, int64_t *queries,
                          uint64_t *list_words, float *list_app, int32_t *list_count, void *stream) {
  return decode_words(c, n_words, llr_ch, llr_a, L, cap, 0.f, 1, hard, llr_app, llr_ext, p_miss, queries, list_words,
                      list_app, list_count, stream);
}

int product_decode_ex(sogrand_code *rc_, const sogrand_code *cc_, int64_t F, const float *llr_ch, int L, int64_t cap,
                      float thr, float alpha, int max_iter, uint8_t *bits, int32_t *half_iters, uint8_t *status,
                      int64_t *queries, product_decode_stats *stats, void *stream) {
  int64_t *par_queries = stats ? stats->par_queries : nullptr;
  if (stats && stats->timing_ms) stats->timing_ms[0] = stats->timing_ms[1] = 0.f;
  if (stats && stats->launches) stats->launches[0] = 0;
  if (!rc_ || !cc_ || F < 0 || L < 1 || L > sg::LMAX || cap < 1 || cap > MAX_CAP || !(thr >= 0.f && thr < 1.f) ||
      !(alpha > 0.f && alpha < 1e6f) || max_iter < 1 || max_iter > 1000)
    return SOGRAND_EINVAL;
  int rc = pair_check(rc_, cc_);
  if (rc != SOGRAND_OK) return rc;
  sogrand_code *c = rc_, *cc = const_cast<sogrand_code *>(cc_);
  for (const sogrand_code *x : {(const sogrand_code *)c, cc_})
    if (x->n - 1 < 63 && cap >= (int64_t(1) << (x->n - 1))) return SOGRAND_EINVAL;
  if (F == 0) return SOGRAND_OK;
  if (!llr_ch || !bits) return SOGRAND_EINVAL;
  rc = ensure_cap(c, cap);
  if (rc == SOGRAND_OK && cc != c) rc = ensure_cap(cc, cap);
  if (rc != SOGRAND_OK) return rc;
  cudaStream_t s = (cudaStream_t)stream;
  const int nr = c->n, nc = cc->n, nm = c->nm, hbw = std::max(nr, nc);
  // scratch, stream-ordered
  const size_t b_le = (size_t)F * nr * nc * sizeof(float);
  const size_t b_hb = (size_t)F * hbw * nm * sizeof(uint64_t);
  const size_t b_i32 = (size_t)F * sizeof(int32_t);
  const size_t b_i64 = (size_t)F * sizeof(int64_t);
  auto al = [](size_t x) { return (x + 255) & ~size_t(255); };
  // every sub-buffer starts on a 256-byte boundary (64-bit atomics need 8)
  const size_t total = al(b_le) + al(b_hb) + 2 * al(b_i32) + (half_iters ? 0 : al(b_i32)) +
                       (queries ? 0 : al(b_i64)) + (par_queries ? 0 : al(b_i64)) + (status ? 0 : al((size_t)F)) + 256;
  char *mem = nullptr;
  if (scratch_alloc(&mem, total, s) != cudaSuccess) return SOGRAND_ENOMEM;
  char *p = mem;
  auto take = [&p, &al](size_t bytes) {
    char *r = p;
    p += al(bytes);
    return r;
  };
  sg::ProductArgs a{};
  a.n_frames = F;
  a.nr = nr;
  a.nc = nc;
  a.hbw = hbw;
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
  a.xf_count = stats ? stats->xf_words : nullptr;
  a.wsum = stats ? reinterpret_cast<unsigned long long *>(stats->weight_sum) : nullptr;
  sg::DevCode d = dev_code(c), dcol = dev_code(cc);
  const bool gen = cc != c || a.nr != a.nc;  // not the square product of one code
  sg::SisoParams P = siso_params(L, cap, thr);
  cudaError_t e = cudaSuccess;
  const bool timed = stats && stats->timing_ms;
  cudaEvent_t ev[3] = {nullptr, nullptr, nullptr};
  if (timed)
    for (int i = 0; i < 3 && e == cudaSuccess; i++) e = cudaEventCreate(&ev[i]);
  int launches = 0;
  float t_half = 0.f, t_check = 0.f;
  if (e == cudaSuccess) SG_DISPATCH(c, e = (sg::launch_product_init<NPL, SYN>(d, a, s)));
  float *le_trace = stats ? stats->le_trace : nullptr;
  int32_t *wq_trace = stats ? stats->word_queries : nullptr;
  const size_t nn = (size_t)nr * nc;
  for (int h = 1; h <= a.max_half && e == cudaSuccess; h++) {
    // teacher-forcing traces: this half's per-word query counts go straight to
    // their slice; the L_E state is copied after the half
    a.wq = wq_trace ? wq_trace + (size_t)(h - 1) * F * hbw : nullptr;
    if (timed) e = cudaEventRecord(ev[0], s);
    if (e == cudaSuccess)
      SG_DISPATCH(c, e = (gen ? sg::launch_product_half<NPL, SYN, true>(d, dcol, P, a, h, s)
                              : sg::launch_product_half<NPL, SYN, false>(d, dcol, P, a, h, s)));
    if (e != cudaSuccess) break;
    launches++;
    if (le_trace)
      e = cudaMemcpyAsync(le_trace + (size_t)(h - 1) * F * nn, a.le, (size_t)F * nn * sizeof(float),
                          cudaMemcpyDeviceToDevice, s);
    if (e != cudaSuccess) break;
    if (timed) e = cudaEventRecord(ev[1], s);
    if (e == cudaSuccess) e = cudaMemsetAsync(a.active, 0, sizeof(int32_t), s);
    if (e == cudaSuccess) SG_DISPATCH(c, e = (sg::launch_product_check<NPL, SYN>(d, dcol, a, h, s)));
    if (e != cudaSuccess) break;
    launches++;
    if (timed) e = cudaEventRecord(ev[2], s);
    int32_t act = 1;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&act, a.active, sizeof(int32_t), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e == cudaSuccess && timed) {
      float x = 0.f, y = 0.f;
      e = cudaEventElapsedTime(&x, ev[0], ev[1]);
      if (e == cudaSuccess) e = cudaEventElapsedTime(&y, ev[1], ev[2]);
      t_half += x;
      t_check += y;
    }
    if (e == cudaSuccess && act == 0) break;
  }
  for (int i = 0; i < 3; i++)
    if (ev[i]) cudaEventDestroy(ev[i]);
  cudaError_t e2 = cudaFreeAsync(mem, s);
  if (stats && stats->timing_ms) {
    stats->timing_ms[0] = t_half;
    stats->timing_ms[1] = t_check;
  }
  if (stats && stats->launches) stats->launches[0] = launches;
  if (e != cudaSuccess || e2 != cudaSuccess) return SOGRAND_ECUDA;
  return SOGRAND_OK;
}

}  // extern "C"

namespace {

// Argument checks shared by the batched entry points.
int persistent_check(const sogrand_code *rc_, const sogrand_code *cc_, int64_t F, int L, int64_t cap, float thr,
                     float alpha, int max_iter) {
  if (!rc_ || !cc_ || F < 0 || L < 1 || L > sg::LMAX || cap < 1 || cap > MAX_CAP || !(thr >= 0.f && thr < 1.f) ||
      !(alpha > 0.f && alpha < 1e6f) || max_iter < 1 || max_iter > 1000)
    return SOGRAND_EINVAL;
  const int prc = pair_check(rc_, cc_);
  if (prc != SOGRAND_OK) return prc;
  for (const sogrand_code *x : {rc_, cc_})
    if (x->n - 1 < 63 && cap >= (int64_t(1) << (x->n - 1))) return SOGRAND_EINVAL;
  // word tickets (slots x the larger n, plus one per idle warp) are 32-bit
  if (F * 2 * (int64_t)max_iter * std::max(rc_->n, cc_->n) >= (int64_t(1) << 31) - (int64_t(1) << 22))
    return SOGRAND_EINVAL;
  return SOGRAND_OK;
}

inline size_t al256(size_t x) { return (x + 255) & ~size_t(255); }

// Scratch of one batched decode of F frames: L_E state, hard decisions, the
// per-frame counters, the frame-half list, room for every optional output and
// the control words.  Every sub-buffer starts on a 256-byte boundary.
size_t persistent_scratch_bytes(int64_t F, int nr, int nc, int nm, int max_iter) {
  const size_t b_i32 = (size_t)F * sizeof(int32_t), b_i64 = (size_t)F * sizeof(int64_t);
  return al256((size_t)F * nr * nc * sizeof(float)) + al256((size_t)F * std::max(nr, nc) * nm * sizeof(uint64_t)) +
         5 * al256(b_i32) +
         al256((size_t)F * 2 * max_iter * sizeof(int32_t)) + 2 * al256(b_i64) + al256((size_t)F) +
         al256(8 * sizeof(int32_t));
}

// The global remaining-mass region of a persistent launch: one slice per
// resident block (at most 8 blocks per SM in either schedule).
inline int npl_of_n(int n) { return n <= 32 ? 1 : (n <= 64 ? 2 : 4); }
int dp_slice_of(const sogrand_code *rc, const sogrand_code *cc) {
  return sg::dp_slice_bytes(npl_of_n(rc->n), rc->m > 32 ? 8 : 4, std::max(rc->jmax, cc->jmax));
}
size_t dp_region_bytes(const sogrand_code *rc, const sogrand_code *cc) {
  return al256((size_t)sgi::sm_count_of_device() * sg::MAX_BLOCKS_PER_SM * dp_slice_of(rc, cc));
}

// Queue set-up and the persistent kernel for F frames on stream s (nothing
// is waited for).  Outputs that are null go to the scratch.  *err_dev is the
// device word that holds the kernel's timeout flag afterwards.
cudaError_t persistent_enqueue(sogrand_code *c, const sogrand_code *cc, int64_t F, const float *llr_ch,
                               const sg::SisoParams &P, float alpha, int max_iter, uint8_t *bits, int32_t *half_iters,
                               uint8_t *status, int64_t *queries, int64_t *par_queries, unsigned long long *wsum,
                               int32_t *xf, char *mem, cudaStream_t s, int32_t **err_dev, int diag = 0,
                               int part = sg::PERSISTENT_ALL) {
  const int nr = c->n, nc = cc->n, nm = c->nm, hbw = std::max(nr, nc);
  char *p = mem;
  auto take = [&p](size_t bytes) {
    char *r = p;
    p += al256(bytes);
    return r;
  };
  const size_t b_i32 = (size_t)F * sizeof(int32_t), b_i64 = (size_t)F * sizeof(int64_t);
  sg::ProductArgs a{};
  a.n_frames = F;
  a.nr = nr;
  a.nc = nc;
  a.hbw = hbw;
  a.diag = diag;
  a.llr_ch = llr_ch;
  a.alpha = alpha;
  a.max_half = 2 * max_iter;
  a.le = (float *)take((size_t)F * nr * nc * sizeof(float));
  a.hb = (uint64_t *)take((size_t)F * hbw * nm * sizeof(uint64_t));
  a.hmax = (int32_t *)take(b_i32);
  a.half_cur = (int32_t *)take(b_i32);
  a.done_words = (int32_t *)take(b_i32);
  a.bad = (int32_t *)take(b_i32);
  a.queue = (int32_t *)take((size_t)F * 2 * max_iter * sizeof(int32_t));
  int32_t *hi_s = (int32_t *)take(b_i32);
  int64_t *q_s = (int64_t *)take(b_i64);
  int64_t *pq_s = (int64_t *)take(b_i64);
  uint8_t *st_s = (uint8_t *)take((size_t)F);
  a.ctrl = (int32_t *)take(8 * sizeof(int32_t));
  a.bits = bits;
  a.half_iters = half_iters ? half_iters : hi_s;
  a.queries = queries ? queries : q_s;
  a.par_queries = par_queries ? par_queries : pq_s;
  a.status = status ? status : st_s;
  a.max_spin = (int32_t)g_queue_wait_us.load();  // back-off without any work before giving up
  // the blocks' remaining-mass areas: the region that follows the scratch
  // (or shared memory, as the code's schedule says)
  a.dp_area = c->dp_global ? (unsigned char *)(mem + al256(persistent_scratch_bytes(F, nr, nc, nm, max_iter))) : nullptr;
  a.dp_stride = dp_slice_of(c, cc);
  a.dp_blocks = sgi::sm_count_of_device() * sg::MAX_BLOCKS_PER_SM;
  a.xf_count = xf;
  a.wsum = wsum;
  *err_dev = a.ctrl + 3;
  sg::DevCode d = dev_code(c), dcol = dev_code(cc);
  const bool gen = cc != c || a.diag || a.nr != a.nc;  // not the square product of one code
  cudaError_t e = cudaSuccess;
  SG_DISPATCH(c, e = (gen ? sg::launch_product_persistent<NPL, SYN, true>(d, dcol, P, a, s, part)
                          : sg::launch_product_persistent<NPL, SYN, false>(d, dcol, P, a, s, part)));
  return e;
}

}  // namespace

extern "C" {

}  // extern "C"

namespace {
// The batched form for a product code (diag = 0) or a QC-GLDPC (diag = 1).
int persistent_decode(sogrand_code *rc_, const sogrand_code *cc_, int diag, int64_t F, const float *llr_ch, int L,
                      int64_t cap, float thr, float alpha, int max_iter, uint8_t *bits, int32_t *half_iters,
                      uint8_t *status, int64_t *queries, product_decode_stats *stats, void *stream) {
  if (stats && stats->timing_ms) stats->timing_ms[0] = stats->timing_ms[1] = 0.f;
  if (stats && stats->launches) stats->launches[0] = 0;
  int rc = persistent_check(rc_, cc_, F, L, cap, thr, alpha, max_iter);
  if (rc != SOGRAND_OK) return rc;
  if (F == 0) return SOGRAND_OK;
  if (!llr_ch || !bits) return SOGRAND_EINVAL;
  sogrand_code *c = rc_, *cc = const_cast<sogrand_code *>(cc_);
  rc = ensure_cap(c, cap);
  if (rc == SOGRAND_OK && cc != c) rc = ensure_cap(cc, cap);
  if (rc != SOGRAND_OK) return rc;
  cudaStream_t s = (cudaStream_t)stream;
  char *mem = nullptr;
  if (scratch_alloc(&mem, al256(persistent_scratch_bytes(F, c->n, cc->n, c->nm, max_iter)) + dp_region_bytes(c, cc), s) !=
      cudaSuccess)
    return SOGRAND_ENOMEM;
  const sg::SisoParams P = siso_params(L, cap, thr);
  const bool timed = stats && stats->timing_ms;
  cudaEvent_t ev[2] = {nullptr, nullptr};
  cudaError_t e = cudaSuccess;
  if (timed)
    for (int i = 0; i < 2 && e == cudaSuccess; i++) e = cudaEventCreate(&ev[i]);
  if (e == cudaSuccess && timed) e = cudaEventRecord(ev[0], s);
  int32_t *err_dev = nullptr;
  if (e == cudaSuccess)
    e = persistent_enqueue(c, cc, F, llr_ch, P, alpha, max_iter, bits, half_iters, status, queries,
                           stats ? stats->par_queries : nullptr,
                           stats ? reinterpret_cast<unsigned long long *>(stats->weight_sum) : nullptr,
                           stats ? stats->xf_words : nullptr, mem, s, &err_dev, diag);
  if (e == cudaSuccess && timed) e = cudaEventRecord(ev[1], s);
  int32_t err = 0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&err, err_dev, sizeof(int32_t), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e == cudaSuccess && timed) {
    float x = 0.f;
    e = cudaEventElapsedTime(&x, ev[0], ev[1]);
    stats->timing_ms[0] = x;
  }
  for (int i = 0; i < 2; i++)
    if (ev[i]) cudaEventDestroy(ev[i]);
  if (stats && stats->launches) stats->launches[0] = 2;  // queue set-up + the persistent kernel
  cudaError_t e2 = cudaFreeAsync(mem, s);
  if (e != cudaSuccess || e2 != cudaSuccess) return SOGRAND_ECUDA;
  return err ? SOGRAND_ETIMEOUT : SOGRAND_OK;
}
}  // namespace

extern "C" {

int product_decode_persistent(sogrand_code *rc_, const sogrand_code *cc_, int64_t F, const float *llr_ch, int L,
                              int64_t cap, float thr, float alpha, int max_iter, uint8_t *bits, int32_t *half_iters,
                              uint8_t *status, int64_t *queries, product_decode_stats *stats, void *stream) {
  return persistent_decode(rc_, cc_, 0, F, llr_ch, L, cap, thr, alpha, max_iter, bits, half_iters, status, queries,
                           stats, stream);
}

int gldpc_decode(sogrand_code *code, int64_t F, const float *llr_ch, int L, int64_t cap, float thr, float alpha,
                 int max_iter, uint8_t *bits, int32_t *half_iters, uint8_t *status, int64_t *queries,
                 product_decode_stats *stats, void *stream) {
  return persistent_decode(code, code, 1, F, llr_ch, L, cap, thr, alpha, max_iter, bits, half_iters, status, queries,
                           stats, stream);
}

int sogrand_code_schedule(sogrand_code *c, int minb, int *current) {
  if (!c || (minb != 0 && minb != 8 && minb != 12)) return SOGRAND_EINVAL;
  if (minb) c->minb = minb;
  if (current) *current = c->minb;
  return SOGRAND_OK;
}

int sogrand_code_dp_area(sogrand_code *c, int where, int *current) {
  if (!c || where < -1 || where > 1) return SOGRAND_EINVAL;
  if (where >= 0) c->dp_global = where;
  if (current) *current = c->dp_global;
  return SOGRAND_OK;
}

int sogrand_code_order_source(sogrand_code *c, int source, int *current) {
  if (!c || source < -1 || source > 1) return SOGRAND_EINVAL;
  if (source >= 0) c->ord_lanes = source;
  if (current) *current = c->ord_lanes;
  return SOGRAND_OK;
}

int sogrand_code_tune(sogrand_code *c, int64_t F, const float *llr_ch, int L, int64_t cap, float thr, float alpha,
                      int max_iter, int *chosen, float *ms_out, void *stream) {
  int rc = persistent_check(c, c, F, L, cap, thr, alpha, max_iter);
  if (rc != SOGRAND_OK) return rc;
  if (F < 1 || !llr_ch) return SOGRAND_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  const size_t nb = ((size_t)c->n * c->n + 7) / 8;
  char *bits = nullptr;
  if (scratch_alloc(&bits, al256((size_t)F * nb), s) != cudaSuccess) return SOGRAND_ENOMEM;
  // every (blocks per SM, remaining-mass area) pair
  const int cand[4] = {8, 8, 12, 12}, cdp[4] = {0, 1, 0, 1};
  float best = 0.f, ms[2] = {0.f, 0.f};
  int pick = c->minb, pick_dp = c->dp_global;
  const int keep = c->minb, keep_dp = c->dp_global;
  for (int i = 0; i < 4 && rc == SOGRAND_OK; i++) {
    c->minb = cand[i];
    c->dp_global = cdp[i];
    float t = 0.f;
    for (int rep = 0; rep < 2 && rc == SOGRAND_OK; rep++) {  // the first run warms caches and the pool
      float tm[2] = {0.f, 0.f};
      product_decode_stats st{nullptr, nullptr, nullptr, tm, nullptr};
      rc = product_decode_persistent(c, c, F, llr_ch, L, cap, thr, alpha, max_iter, (uint8_t *)bits, nullptr,
                                     nullptr, nullptr, &st, stream);
      t = tm[0];
    }
    const int j = i / 2;
    if (i % 2 == 0 || t < ms[j]) ms[j] = t;  // the better placement for this block count
    if (rc == SOGRAND_OK && (i == 0 || t < best)) {
      best = t;
      pick = cand[i];
      pick_dp = cdp[i];
    }
  }
  c->minb = rc == SOGRAND_OK ? pick : keep;
  c->dp_global = rc == SOGRAND_OK ? pick_dp : keep_dp;
  if (cudaFreeAsync(bits, s) != cudaSuccess && rc == SOGRAND_OK) rc = SOGRAND_ECUDA;
  if (rc == SOGRAND_OK) {
    if (chosen) *chosen = pick;
    if (ms_out) {
      ms_out[0] = ms[0];
      ms_out[1] = ms[1];
    }
  }
  return rc;
}

int product_decode_host(sogrand_code *rc_, const sogrand_code *cc_, int64_t F, const float *llr_ch, int L,
                        int64_t cap, float thr, float alpha, int max_iter, uint8_t *bits, int32_t *half_iters,
                        uint8_t *status, int64_t *queries, void *stream) {
  int rc = persistent_check(rc_, cc_, F, L, cap, thr, alpha, max_iter);
  if (rc != SOGRAND_OK) return rc;
  if (F == 0) return SOGRAND_OK;
  if (!llr_ch || !bits) return SOGRAND_EINVAL;
  sogrand_code *c = rc_, *cc = const_cast<sogrand_code *>(cc_);
  rc = ensure_cap(c, cap);
  if (rc == SOGRAND_OK && cc != c) rc = ensure_cap(cc, cap);
  if (rc != SOGRAND_OK) return rc;
  cudaStream_t s = (cudaStream_t)stream;
  const int nr = c->n, nc = cc->n, nm = c->nm;
  const size_t in_f = (size_t)nr * nc * sizeof(float), nb = ((size_t)nr * nc + 7) / 8;
  // Chunks of the batch move through three stages on their own streams:
  // copy in (h2d), decode (two streams taking chunks in turn, so the tail of
  // one chunk overlaps the start of the next), copy out (d2h).  Events order
  // the stages of each chunk; all streams start after the caller's stream.
  // Chunk sizes: 2048 frames first, doubling up to a quarter of the batch,
  // so that decoding starts after a short copy and each later copy takes
  // less time than the decoding of the chunk before it (about every other
  // call the copy in runs at ~15 GB/s instead of ~210 GB/s on a GB300), with
  // few chunks, since each adds a launch tail.
  const int64_t cmax = std::max<int64_t>(2048, (F + 3) / 4);
  std::vector<int64_t> starts;
  for (int64_t f0 = 0, ck = std::min<int64_t>(2048, F); f0 < F; f0 += ck, ck = std::min(2 * ck, cmax))
    starts.push_back(f0);
  starts.push_back(F);
  const int64_t K = (int64_t)starts.size() - 1;
  int64_t chunk = 0;
  for (int64_t k = 0; k < K; k++) chunk = std::max(chunk, starts[k + 1] - starts[k]);
  const size_t b_in = al256((size_t)F * in_f), b_bits = al256((size_t)F * nb);
  const size_t b_out = b_in + b_bits + al256((size_t)F * 4) + al256((size_t)F) + al256((size_t)F * 8);
  const size_t b_scr = al256(persistent_scratch_bytes(chunk, nr, nc, nm, max_iter)) + dp_region_bytes(c, cc);
  char *mem = nullptr;
  if (scratch_alloc(&mem, b_out + 2 * b_scr + al256((size_t)K * sizeof(int32_t)), s) != cudaSuccess)
    return SOGRAND_ENOMEM;
  float *d_in = (float *)mem;
  uint8_t *d_bits = (uint8_t *)(mem + b_in);
  int32_t *d_hi = (int32_t *)(mem + b_in + b_bits);
  uint8_t *d_st = (uint8_t *)(mem + b_in + b_bits + al256((size_t)F * 4));
  int64_t *d_q = (int64_t *)(mem + b_in + b_bits + al256((size_t)F * 4) + al256((size_t)F));
  int32_t *d_err = (int32_t *)(mem + b_out + 2 * b_scr);  // one timeout flag per chunk
  const sg::SisoParams P = siso_params(L, cap, thr);
  cudaStream_t st[4] = {nullptr, nullptr, nullptr, nullptr};  // h2d, decode x2, d2h
  std::vector<cudaEvent_t> ev;
  cudaError_t e = cudaSuccess;
  for (int i = 0; i < 4 && e == cudaSuccess; i++) e = cudaStreamCreateWithFlags(&st[i], cudaStreamNonBlocking);
  auto event = [&ev, &e]() {
    cudaEvent_t x = nullptr;
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&x, cudaEventDisableTiming);
    if (x) ev.push_back(x);
    return x;
  };
  cudaEvent_t start = event();
  if (e == cudaSuccess) e = cudaMemsetAsync(d_err, 0, (size_t)K * sizeof(int32_t), s);
  if (e == cudaSuccess) e = cudaEventRecord(start, s);
  for (int i = 0; i < 4 && e == cudaSuccess; i++) e = cudaStreamWaitEvent(st[i], start, 0);
  for (int64_t k = 0; k < K && e == cudaSuccess; k++) {
    const int64_t f0 = starts[k], Fk = starts[k + 1] - starts[k];
    if (Fk <= 0) break;
    cudaStream_t sd = st[1 + (k & 1)];
    cudaEvent_t in_done = event(), dec_done = event();
    if (e == cudaSuccess)
      e = cudaMemcpyAsync((char *)d_in + f0 * in_f, (const char *)llr_ch + f0 * in_f, Fk * in_f,
                          cudaMemcpyHostToDevice, st[0]);
    if (e == cudaSuccess) e = cudaEventRecord(in_done, st[0]);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(sd, in_done, 0);
    int32_t *err_k = nullptr;
    if (e == cudaSuccess)
      e = persistent_enqueue(c, cc, Fk, (const float *)((const char *)d_in + f0 * in_f), P, alpha, max_iter,
                             d_bits + f0 * nb, d_hi + f0, d_st + f0, d_q + f0, nullptr, nullptr, nullptr,
                             mem + b_out + (k & 1) * b_scr, sd, &err_k);
    if (e == cudaSuccess) e = cudaMemcpyAsync(d_err + k, err_k, sizeof(int32_t), cudaMemcpyDeviceToDevice, sd);
    if (e == cudaSuccess) e = cudaEventRecord(dec_done, sd);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(st[3], dec_done, 0);
    if (e == cudaSuccess) e = cudaMemcpyAsync(bits + f0 * nb, d_bits + f0 * nb, Fk * nb, cudaMemcpyDeviceToHost, st[3]);
    if (e == cudaSuccess && half_iters)
      e = cudaMemcpyAsync(half_iters + f0, d_hi + f0, Fk * 4, cudaMemcpyDeviceToHost, st[3]);
    if (e == cudaSuccess && status) e = cudaMemcpyAsync(status + f0, d_st + f0, Fk, cudaMemcpyDeviceToHost, st[3]);
    if (e == cudaSuccess && queries)
      e = cudaMemcpyAsync(queries + f0, d_q + f0, Fk * 8, cudaMemcpyDeviceToHost, st[3]);
  }
  std::vector<int32_t> err((size_t)K, 0);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(err.data(), d_err, (size_t)K * sizeof(int32_t), cudaMemcpyDeviceToHost, st[3]);
  // the caller's stream resumes after every stage
  for (int i = 0; i < 4 && st[i]; i++) {
    cudaEvent_t x = event();
    if (e == cudaSuccess) e = cudaEventRecord(x, st[i]);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(s, x, 0);
  }
  cudaError_t e2 = cudaFreeAsync(mem, s);
  cudaError_t e3 = cudaStreamSynchronize(s);
  for (cudaEvent_t x : ev) cudaEventDestroy(x);
  for (int i = 0; i < 4; i++)
    if (st[i]) cudaStreamDestroy(st[i]);
  if (e != cudaSuccess || e2 != cudaSuccess || e3 != cudaSuccess) return SOGRAND_ECUDA;
  for (int64_t k = 0; k < K; k++)
    if (err[k]) return SOGRAND_ETIMEOUT;
  return SOGRAND_OK;
}

}  // extern "C"

namespace {
// The mixed form as one CUDA graph, captured on one stream: the list set-up
// of every group, then a persistent decoder kernel per group (each the
// single-code batched kernel of its code, with its own frame-half list) in a
// chain of programmatic dependent launches, launched with one cudaGraphLaunch.
// A decoder's warps leave as soon as its unfinished frames cannot use them,
// and once every block of it has begun to leave the next group's decoder may
// start: its blocks take the SMs that the tail frees, so no SM idles while
// any code has work, and two codes' kernels share an SM only in that tail
// (on parallel branches they shared SMs throughout and competed for the
// instruction cache, the kernel's first stall: about 1% slower than the
// per-code launches in sequence).
int mixed_graph_decode(int n_groups, const sogrand_frame_group *groups, int L, int64_t cap, float thr, float alpha,
                       int max_iter, product_decode_stats *stats, cudaStream_t s) {
  std::vector<int> live;
  for (int g = 0; g < n_groups; g++)
    if (groups[g].n_frames > 0) live.push_back(g);
  const int k = (int)live.size();
  // scratch of every group's batched decode, with its remaining-mass region
  std::vector<size_t> off(k + 1, 0);
  for (int x = 0; x < k; x++) {
    const sogrand_frame_group &G = groups[live[x]];
    off[x + 1] = off[x] + al256(persistent_scratch_bytes(G.n_frames, G.code->n, G.code->n, G.code->nm, max_iter)) +
                 dp_region_bytes(G.code, G.code);
  }
  char *mem = nullptr;
  if (scratch_alloc(&mem, off[k] + 256, s) != cudaSuccess) return SOGRAND_ENOMEM;
  const sg::SisoParams P = siso_params(L, cap, thr);
  std::vector<int32_t *> err_dev(k, nullptr);  // each decoder's timeout flag
  cudaStream_t cs = nullptr;
  std::vector<cudaEvent_t> ev;
  cudaError_t e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  if (e == cudaSuccess) e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
  if (e == cudaSuccess) {
    for (int pass = 0; pass < 2; pass++) {
      for (int x = 0; x < k && e == cudaSuccess; x++) {
        const sogrand_frame_group &G = groups[live[x]];
        const int part = pass == 0 ? sg::PERSISTENT_INIT : (x == 0 ? sg::PERSISTENT_DECODE : sg::PERSISTENT_DECODE_PDL);
        e = persistent_enqueue(G.code, G.code, G.n_frames, G.llr_ch, P, alpha, max_iter, G.bits, G.half_iters,
                               G.status, G.queries, nullptr,
                               stats ? reinterpret_cast<unsigned long long *>(stats->weight_sum) : nullptr,
                               stats ? stats->xf_words : nullptr, mem + off[x], cs, &err_dev[x], 0, part);
      }
    }
    const cudaError_t ec = cudaStreamEndCapture(cs, &graph);
    if (e == cudaSuccess) e = ec;
  }
  if (e == cudaSuccess) e = cudaGraphInstantiate(&exec, graph, 0);
  const bool timed = stats && stats->timing_ms;
  cudaEvent_t t0 = nullptr, t1 = nullptr;  // timed events (the others have timing disabled)
  if (e == cudaSuccess && timed) {
    e = cudaEventCreate(&t0);
    if (e == cudaSuccess) e = cudaEventCreate(&t1);
  }
  if (t0) ev.push_back(t0);
  if (t1) ev.push_back(t1);
  if (e == cudaSuccess && timed) e = cudaEventRecord(t0, s);
  if (e == cudaSuccess) e = cudaGraphLaunch(exec, s);
  if (e == cudaSuccess && timed) e = cudaEventRecord(t1, s);
  // the timeout flags, read after the whole graph (every decoder) has finished
  std::vector<int32_t> err(k, 0);
  for (int x = 0; x < k && e == cudaSuccess; x++)
    e = cudaMemcpyAsync(&err[x], err_dev[x], sizeof(int32_t), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e == cudaSuccess && timed) {
    float ms = 0.f;
    e = cudaEventElapsedTime(&ms, t0, t1);
    stats->timing_ms[0] = ms;
  }
  if (stats && stats->launches) stats->launches[0] = 1;  // one graph launch (an init and a decoder kernel per code)
  if (exec) cudaGraphExecDestroy(exec);
  if (graph) cudaGraphDestroy(graph);
  for (cudaEvent_t x : ev) cudaEventDestroy(x);
  if (cs) cudaStreamDestroy(cs);
  const cudaError_t e2 = cudaFreeAsync(mem, s);
  if (e != cudaSuccess || e2 != cudaSuccess) return SOGRAND_ECUDA;
  for (int32_t x : err)
    if (x) return SOGRAND_ETIMEOUT;
  return SOGRAND_OK;
}
}  // namespace

extern "C" {

int product_decode_mixed(int n_groups, const sogrand_frame_group *groups, int L, int64_t cap, float thr, float alpha,
                         int max_iter, product_decode_stats *stats, void *stream) {
  if (stats && stats->timing_ms) stats->timing_ms[0] = stats->timing_ms[1] = 0.f;
  if (stats && stats->launches) stats->launches[0] = 0;
  if (n_groups < 1 || n_groups > SOGRAND_MIX_MAX_GROUPS || !groups) return SOGRAND_EINVAL;
  int64_t total = 0;
  for (int g = 0; g < n_groups; g++) {
    const sogrand_frame_group &G = groups[g];
    int rc = persistent_check(G.code, G.code, G.n_frames, L, cap, thr, alpha, max_iter);
    if (rc != SOGRAND_OK) return rc;
    if (G.n_frames > 0 && (!G.llr_ch || !G.bits)) return SOGRAND_EINVAL;
    total += G.n_frames;
  }
  if (total == 0) return SOGRAND_OK;
  for (int g = 0; g < n_groups; g++) {
    int rc = ensure_cap(groups[g].code, cap);
    if (rc != SOGRAND_OK) return rc;
  }
  return mixed_graph_decode(n_groups, groups, L, cap, thr, alpha, max_iter, stats, (cudaStream_t)stream);
}

int product_decode(sogrand_code *row_code, const sogrand_code *col_code, int64_t n_frames, const float *llr_ch, int L,
                   int64_t cap, float thr, float alpha, int max_iter, uint8_t *bits, int32_t *half_iters,
                   uint8_t *status, int64_t *queries, void *stream) {
  return product_decode_ex(row_code, col_code, n_frames, llr_ch, L, cap, thr, alpha, max_iter, bits, half_iters,
                           status, queries, nullptr, stream);
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

// ---------------------------------------------------------------------------
// product_decode_noalloc: product decoding for callers that may not allocate
// ---------------------------------------------------------------------------
// The scratch of the turbo decoder (extrinsic state, hard decisions, frame
// flags) lives in this fixed device array instead of stream-ordered
// allocations.  Every GPU that loads the library holds it until the process
// exits.  Host code only sees a stand-in for the array's name, so its device
// address is taken once per device with cudaGetSymbolAddress and passed to
// the kernels as a plain pointer.
static __device__ __align__(256) unsigned char g_noalloc_scratch[SOGRAND_NOALLOC_SCRATCH_BYTES];

namespace {
constexpr int NOALLOC_MAX_DEVICES = 64;
std::mutex g_noalloc_mu;
void *g_noalloc_ptr[NOALLOC_MAX_DEVICES] = {nullptr};
}  // namespace

extern "C" {

int product_decode_noalloc(sogrand_code *rc_, const sogrand_code *cc_, int64_t F, const float *llr_ch, int L,
                           int64_t cap, float thr, float alpha, int max_iter, uint8_t *bits, int32_t *half_iters,
                           uint8_t *status, int64_t *queries, void *stream) {
  if (!rc_ || !cc_ || F < 0 || L < 1 || L > sg::LMAX || cap < 1 || cap > MAX_CAP || !(thr >= 0.f && thr < 1.f) ||
      !(alpha > 0.f && alpha < 1e6f) || max_iter < 1 || max_iter > 1000)
    return SOGRAND_EINVAL;
  if (rc_ != cc_) return SOGRAND_EUNSUPPORTED;
  sogrand_code *c = rc_;
  if (c->n - 1 < 63 && cap >= (int64_t(1) << (c->n - 1))) return SOGRAND_EINVAL;
  if (F == 0) return SOGRAND_OK;
  if (!llr_ch || !bits || !half_iters || !status || !queries) return SOGRAND_EINVAL;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return SOGRAND_ECUDA;
  if (dev != c->device || dev < 0 || dev >= NOALLOC_MAX_DEVICES) return SOGRAND_EINVAL;
  {
    // the query-order tables must already cover the cap: growing them allocates
    std::lock_guard<std::mutex> g(c->mu);
    if (cap > c->tab_cap) return SOGRAND_EINVAL;
  }
  const int n = c->n, nm = c->nm;
  // bound F before any product with it (a huge F must not wrap the size below)
  if (F > (int64_t)(SOGRAND_NOALLOC_SCRATCH_BYTES / (4 * n * n + 8 * n * nm + 16))) return SOGRAND_EINVAL;
  auto al = [](size_t x) { return (x + 255) & ~size_t(255); };
  const size_t b_le = (size_t)F * n * n * sizeof(float), b_hb = (size_t)F * n * nm * sizeof(uint64_t);
  const size_t b_i32 = (size_t)F * sizeof(int32_t), b_i64 = (size_t)F * sizeof(int64_t);
  const size_t need = al(b_le) + al(b_hb) + 2 * al(b_i32) + al(b_i64);
  if (need > (size_t)SOGRAND_NOALLOC_SCRATCH_BYTES) return SOGRAND_EINVAL;  // too many frames for the fixed scratch
  void *base = nullptr;
  {
    std::lock_guard<std::mutex> g(g_noalloc_mu);
    if (!g_noalloc_ptr[dev]) {
      // device address of the array on the current device (set-up, once per device)
      if (cudaGetSymbolAddress(&g_noalloc_ptr[dev], g_noalloc_scratch) != cudaSuccess) {
        g_noalloc_ptr[dev] = nullptr;
        return SOGRAND_ECUDA;
      }
    }
    base = g_noalloc_ptr[dev];
  }
  char *p = (char *)base;
  auto take = [&p, &al](size_t bytes) {
    char *r = p;
    p += al(bytes);
    return r;
  };
  cudaStream_t s = (cudaStream_t)stream;
  sg::ProductArgs a{};
  a.n_frames = F;
  a.nr = a.nc = a.hbw = c->n;
  a.llr_ch = llr_ch;
  a.alpha = alpha;
  a.max_half = 2 * max_iter;
  a.le = (float *)take(b_le);
  a.hb = (uint64_t *)take(b_hb);
  a.fstate = (int32_t *)take(b_i32);
  a.hmax = (int32_t *)take(b_i32);
  a.par_queries = (int64_t *)take(b_i64);
  a.active = nullptr;
  a.bits = bits;
  a.half_iters = half_iters;
  a.status = status;
  a.queries = queries;
  sg::DevCode d = dev_code(c);
  sg::SisoParams P = siso_params(L, cap, thr);
  // frame flags, per-half maxima and counters start at zero on every call
  // (the array keeps the previous call's contents)
  cudaError_t e = cudaSuccess;
  SG_DISPATCH(c, e = (sg::launch_product_init<NPL, SYN>(d, a, s)));
  // every half iteration is launched; the kernels skip frames that finished,
  // so the host never waits on the device
  for (int h = 1; h <= a.max_half && e == cudaSuccess; h++) {
    SG_DISPATCH(c, e = (sg::launch_product_half<NPL, SYN, false>(d, d, P, a, h, s)));
    if (e == cudaSuccess) SG_DISPATCH(c, e = (sg::launch_product_check<NPL, SYN>(d, d, a, h, s)));
  }
  return e == cudaSuccess ? SOGRAND_OK : SOGRAND_ECUDA;
}

#ifdef SG_PHASE_PROFILE
// phase counters of the profiling build (not part of the public ABI): the sum
// over the translation units that registered a reader
int sogrand_debug_phase(unsigned long long *out, int reset) {
  for (int i = 0; i < 16; i++) out[i] = 0;
  int bad = 0;
  for (sg::PhaseReader r : sg::phase_readers()) bad |= r(out, reset);
  return bad ? SOGRAND_ECUDA : 0;
}
#endif

}  // extern "C"
