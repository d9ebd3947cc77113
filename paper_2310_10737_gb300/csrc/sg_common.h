// sg_common.h -- types shared by the host and device halves of libsogrand.
// Internal to the library; the public interface is include/sogrand.h.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>

namespace sg {

constexpr int NMAX = 128;      // longest component code
constexpr int LMAX = 16;       // longest list a decode may request
constexpr int WMAXT = 64;      // most Hamming weights a query-order table may reach
constexpr int WENT = 15;       // most ranks one table entry holds
constexpr int WARPS_PER_BLOCK = 4;
// Schedules: the per-word kernels are compiled for 8 resident blocks per SM
// (64 registers a thread) and for 12 (40 registers); a launch never has more
// than MAX_BLOCKS_PER_SM blocks resident on an SM.
constexpr int MAX_BLOCKS_PER_SM = 12;

// Query order of one code, flattened per 1-line parameter c and parity class.
// For every c in [0, c_max] and class (the parity of y for an even code, or
// the single class of all patterns) the patterns are stored in query order:
// increasing cost = sum of ranks + c * weight, ties by weight, then by the
// ascending rank vector in lexicographic order.  Each order is stored up to
// the query cap it was built for and then to the end of that cost level.
struct DevOrder {
  const uint4 *ent;       // [total] byte 0: Hamming weight w; bytes 1..w: ranks (0-based, ascending)
  const uint16_t *cost;   // [total] cost of each pattern
  const int32_t *base;    // [(c_max+1) * ncls] first entry of order (c, class)
  const int32_t *count;   // [(c_max+1) * ncls] entries stored for (c, class)
  int32_t ncls;           // 2 for an even code (class = parity of y), else 1
  int32_t class_size;     // patterns in one class (saturated): count == class_size means the whole class
};

// The same orders as groups, for lanes that enumerate their patterns instead
// of reading DevOrder::ent (DevCode::ord_lanes): a group is the run of
// patterns of one cost and one Hamming weight w, i.e. the w-subsets of the
// ranks {1..n} with rank sum m = cost - c w, in lexicographic order.  (A
// struct apart from DevOrder, which the kernels copy to local memory when
// they pass it to out-of-line functions.)
struct DevGroups {
  const uint2 *grp;       // [groups] x: first entry of the group within its order; y: m | w << 16
  const int32_t *gbase;   // [(c_max+1) * ncls + 1] first group of order (c, class)
  const int32_t *scnt;    // [(n+1) * sc_w * sc_m] w-subsets of {1..N} with sum m at (N, w, m), saturated
  int32_t sc_w, sc_m;     // extents of scnt in w and m
};

struct DevCode {
  int32_t n, k, m;       // length, dimension, parity checks (m = n - k)
  int32_t even;          // 1: even code, search restricted to the parity of y
  int32_t c_max;         // clamp of the 1-line parameter
  float log_phi;         // log((2^k-1)/(2^(n-1)-1)) (even) or log((2^k-1)/(2^n-1))
  const uint64_t *hcol;  // [n] syndrome contribution of bit i (bit t = H[t][i])
  const uint64_t *hrow;  // [m][nm] rows of H as bit masks over the n positions
  DevOrder ord;
  int32_t jmax;          // largest stored cost + 2 (bounds the remaining-mass DP)
  int32_t minb;          // schedule: resident blocks per SM the kernels are compiled for (8 or 12)
  int32_t dp_global;     // schedule: the batched forms keep the remaining-mass area in global memory
  int32_t ord_lanes;     // 1: the lanes enumerate the query order (loop without the threshold rule)
  DevGroups grp;         // the order's groups (used with ord_lanes)
};

struct SisoParams {
  int32_t L;
  int32_t cap;
  float thr;
  int32_t forney = 0;            // 1: Forney's list-only normalisation (the mass outside the list taken as 0)
  int32_t lock_polls = 1 << 22;  // polls of the block's remaining-mass lock before a warp gives up on it
  int32_t lock_preheld = 0;      // 1: blocks start with that lock taken (test of the bound)
};

// Per-word results that the callers write out.
struct WordResult {
  int32_t queries;       // -1: invalid input
  int32_t nhit;
  float pmiss;
  float logD;            // log(sum of list masses + R phi), relative to p(0)
  int32_t wsum;          // sum of the Hamming weights of the queried patterns
};

}  // namespace sg
