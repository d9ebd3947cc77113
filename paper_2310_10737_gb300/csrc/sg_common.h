// sg_common.h -- types shared by the host and device halves of libsogrand.
// Internal to the library; the public interface is include/sogrand.h.
#pragma once
#include <cstdint>

namespace sg {

constexpr int NMAX = 128;      // longest component code
constexpr int LMAX = 16;       // longest list a decode may request
constexpr int WMAXT = 64;      // most Hamming-weight streams a pattern table holds
constexpr int WARPS_PER_BLOCK = 4;

// Query-order tables of one code length (built on the host, resident on the
// device).  Stream w holds every w-subset of the reliability ranks {1..n}
// in increasing logistic weight (sum of ranks) and, within one logistic
// weight, in lexicographic order of the ascending rank vector, truncated
// after the first level whose offset exceeds the query cap it was built for.
struct DevTables {
  const uint64_t *pat;   // [total][nm] rank masks (bit r-1 = rank r)
  const int32_t *sbase;  // [wtop] first pattern of stream w
  const int32_t *lbase;  // [wtop] first level record of stream w
  const int32_t *lnum;   // [wtop] number of stored levels of stream w
  const int32_t *lcnt;   // level sizes
  const int32_t *loff;   // level offsets within the stream
  int32_t wtop;          // streams 0..wtop-1 exist
  int32_t nm;            // 64-bit words per mask
};

struct DevCode {
  int32_t n, k, m;       // length, dimension, parity checks (m = n - k)
  int32_t even;          // 1: even code, search restricted to the parity of y
  int32_t c_max;         // clamp of the 1-line parameter
  float log_phi;         // log((2^k-1)/(2^(n-1)-1)) (even) or log((2^k-1)/(2^n-1))
  const uint64_t *hcol;  // [n] syndrome contribution of bit i (bit t = H[t][i])
  const uint64_t *hrow;  // [m][nm] rows of H as bit masks over the n positions
  DevTables tab;
  int32_t jmax;          // largest cost level the remaining-mass DP may need, + 1
};

struct SisoParams {
  int32_t L;
  int32_t cap;
  float thr;
};

// Per-word results that the callers write out.
struct WordResult {
  int32_t queries;       // -1: invalid input
  int32_t nhit;
  float pmiss;
  float logD;            // log(sum of list masses + R phi), relative to p(0)
};

}  // namespace sg
