// peak.cu -- integer-pipe throughput probe: the denominator of the decoder's
// roofline.  The decoder's work is 32-bit integer and logic instructions
// (XOR of H columns, compares, ballots, byte extracts), so its ceiling is the
// rate at which the SMs retire such instructions, measured here with a loop
// of independent LOP3 (three-input XOR) and IADD (add) chains per thread.
#include <cuda_runtime.h>

#include <cstdint>

#include "sogrand.h"

namespace {

constexpr int CHAINS = 8;          // independent dependency chains per thread
constexpr int OPS_PER_STEP = 2;    // one lop3 + one add per chain per step
constexpr int UNROLL = 8;          // steps per loop trip
constexpr int PEAK_TPB = 256;

__global__ void __launch_bounds__(PEAK_TPB) k_int_peak(uint32_t *sink, int trips, uint32_t seed) {
  uint32_t x[CHAINS];
#pragma unroll
  for (int j = 0; j < CHAINS; j++) x[j] = (threadIdx.x + 977u * j) ^ seed;
  const uint32_t b = seed * 2654435761u, c = seed ^ 0x9e3779b9u;
  for (int t = 0; t < trips; t++) {
#pragma unroll
    for (int u = 0; u < UNROLL; u++) {
#pragma unroll
      for (int j = 0; j < CHAINS; j++) {
        asm volatile("lop3.b32 %0, %0, %1, %2, 0x96;" : "+r"(x[j]) : "r"(b), "r"(c));
        asm volatile("add.u32 %0, %0, %1;" : "+r"(x[j]) : "r"(c));
      }
    }
  }
  uint32_t acc = 0;
#pragma unroll
  for (int j = 0; j < CHAINS; j++) acc ^= x[j];
  if (acc == 0x5ca1ab1eu) sink[blockIdx.x] = acc;  // keeps the chains live; practically never taken
}

}  // namespace

extern "C" int sogrand_int_peak(int64_t trips, double *ops_per_s, double *ms_out, void *stream) {
  if (trips < 1 || trips > (int64_t(1) << 30) || !ops_per_s) return SOGRAND_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  int dev = 0, sms = 0, occ = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_int_peak, PEAK_TPB, 0) != cudaSuccess)
    return SOGRAND_ECUDA;
  const int grid = sms * (occ > 0 ? occ : 1);
  uint32_t *sink = nullptr;
  cudaEvent_t ev[2] = {nullptr, nullptr};
  cudaError_t e = cudaMalloc(&sink, (size_t)grid * sizeof(uint32_t));
  for (int i = 0; i < 2 && e == cudaSuccess; i++) e = cudaEventCreate(&ev[i]);
  if (e == cudaSuccess) {
    k_int_peak<<<grid, PEAK_TPB, 0, s>>>(sink, 1, 12345u);  // warm-up
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaEventRecord(ev[0], s);
  if (e == cudaSuccess) {
    k_int_peak<<<grid, PEAK_TPB, 0, s>>>(sink, (int)trips, 12345u);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaEventRecord(ev[1], s);
  if (e == cudaSuccess) e = cudaEventSynchronize(ev[1]);
  float ms = 0.f;
  if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, ev[0], ev[1]);
  for (int i = 0; i < 2; i++)
    if (ev[i]) cudaEventDestroy(ev[i]);
  if (sink) cudaFree(sink);
  if (e != cudaSuccess || ms <= 0.f) return SOGRAND_ECUDA;
  const double ops = (double)grid * PEAK_TPB * (double)trips * UNROLL * CHAINS * OPS_PER_STEP;
  *ops_per_s = ops / (ms * 1e-3);
  if (ms_out) *ms_out = ms;
  return SOGRAND_OK;
}
