// Throughput probes of the benchmark: the practical ceilings the selection
// kernels are measured against.  A measurement aid, not part of the method
// and not part of libgbar's C ABI: this file builds libgbar_probe.so, which
// only the benchmark and its test load.
//
//   mode GBAR_PROBE_PHILOX         every thread evaluates n Philox4x32-10
//                                  blocks (the selection's counter layout,
//                                  tag 0) and folds their words together: the
//                                  integer multiply-add bound of trial
//                                  generation.
//   mode GBAR_PROBE_PHILOX_GATHER  the same blocks, each with its two trials'
//                                  candidates j = mulhi(w, M), the two
//                                  gathers table[j] and the FP32 acceptance
//                                  test: the bound of trial generation plus
//                                  random gathers from a table of M floats
//                                  (L1- or L2-resident depending on M).
//
// One warp-instruction stream per thread, no work claiming, no early exit:
// every round is independent, so these reach what the hardware sustains for
// the same arithmetic and access pattern.
#include <algorithm>
#include <cstdint>

#include "device.cuh"

#define GBAR_PROBE_PHILOX 0
#define GBAR_PROBE_PHILOX_GATHER 1

namespace {

constexpr int kProbeThreads = 256;

template <int MODE>
__global__ void __launch_bounds__(kProbeThreads) k_probe(uint32_t n, uint32_t k0, uint32_t k1,
                                                         const float* __restrict__ table, uint32_t M,
                                                         float T, uint32_t* out) {
  const uint32_t tid = blockIdx.x * blockDim.x + threadIdx.x;
  uint32_t acc = 0;
  for (uint32_t i = 0; i < n; i += 2) {
    uint4 w[2];
#pragma unroll
    for (int u = 0; u < 2; ++u) w[u] = gbar::philox10(make_uint4(i + u, tid, 7u, 0u), k0, k1);
    if constexpr (MODE == GBAR_PROBE_PHILOX) {
#pragma unroll
      for (int u = 0; u < 2; ++u) acc ^= w[u].x ^ w[u].y ^ w[u].z ^ w[u].w;
    } else {
      float x[4];
#pragma unroll
      for (int u = 0; u < 2; ++u) {
        x[2 * u] = __ldg(table + gbar::candidate(w[u].x, M));
        x[2 * u + 1] = __ldg(table + gbar::candidate(w[u].z, M));
      }
#pragma unroll
      for (int t = 0; t < 4; ++t) {
        const uint32_t wu = (t & 1) ? w[t >> 1].w : w[t >> 1].y;
        acc += gbar::accept_f32(wu, T, x[t]) ? 1u : 0u;
      }
    }
  }
  out[tid] = acc;
}

inline bool aligned4(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 3u) == 0; }

}  // namespace

// Launches SM count x threads_per_sm / 256 blocks of 256 threads; every
// thread evaluates blocks_per_thread Philox blocks (even, > 0).  d_table [M]
// FP32 (gather mode; 0 < M < 2^31); d_out [out_words] uint32, one word per
// launched thread.  The caller times the launch and divides the Philox
// blocks, SM count x threads_per_sm x blocks_per_thread, by the time.
// Returns 0, -1 (bad argument), -2 (misaligned pointer) or -3 (CUDA error).
extern "C" int gbar_probe_throughput(int mode, const float* d_table, uint32_t M,
                                     uint32_t blocks_per_thread, uint32_t threads_per_sm,
                                     uint32_t* d_out, size_t out_words, void* stream) {
  if (mode != GBAR_PROBE_PHILOX && mode != GBAR_PROBE_PHILOX_GATHER) return -1;
  if (blocks_per_thread == 0 || (blocks_per_thread & 1u) || threads_per_sm == 0 ||
      threads_per_sm % kProbeThreads || !d_out)
    return -1;
  if (mode == GBAR_PROBE_PHILOX_GATHER && (!d_table || M == 0 || M >= (1u << 31))) return -1;
  if (!aligned4(d_out) || !aligned4(d_table)) return -2;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return -3;
  const uint64_t grid = (uint64_t)std::max(1, sms) * (threads_per_sm / kProbeThreads);
  if (grid * kProbeThreads > out_words || grid >= (1ull << 31)) return -1;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (mode == GBAR_PROBE_PHILOX)
    k_probe<GBAR_PROBE_PHILOX><<<(uint32_t)grid, kProbeThreads, 0, s>>>(blocks_per_thread, 1u, 2u,
                                                                         d_table, M, 1.0f, d_out);
  else
    k_probe<GBAR_PROBE_PHILOX_GATHER><<<(uint32_t)grid, kProbeThreads, 0, s>>>(
        blocks_per_thread, 1u, 2u, d_table, M, 1.0f, d_out);
  return cudaGetLastError() == cudaSuccess ? 0 : -3;
}
