// Throughput probes: the practical ceilings the selection kernels are
// measured against.  Not part of the method; the benchmark times them with
// CUDA events.
//
//   mode AR_PROBE_PHILOX         every thread evaluates n Philox4x32-10 blocks
//                                (the selection's counter layout, tag 0) and
//                                folds their words together: the integer
//                                multiply-add bound of trial generation.
//   mode AR_PROBE_PHILOX_GATHER  the same blocks, each with its two trials'
//                                candidates j = mulhi(w, M), the two gathers
//                                table[j] and the FP32 acceptance test: the
//                                bound of trial generation plus random
//                                gathers from a table of M floats (L1- or
//                                L2-resident depending on M).
//
// One warp-instruction stream per thread, no work claiming, no early exit:
// every round is independent, so these reach what the hardware sustains for
// the same arithmetic and access pattern.
#include <algorithm>

#include "device.cuh"
#include "host.hpp"

namespace gbar {
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
    for (int u = 0; u < 2; ++u) w[u] = philox10(make_uint4(i + u, tid, 7u, 0u), k0, k1);
    if constexpr (MODE == AR_PROBE_PHILOX) {
#pragma unroll
      for (int u = 0; u < 2; ++u) acc ^= w[u].x ^ w[u].y ^ w[u].z ^ w[u].w;
    } else {
      float x[4];
#pragma unroll
      for (int u = 0; u < 2; ++u) {
        x[2 * u] = __ldg(table + candidate(w[u].x, M));
        x[2 * u + 1] = __ldg(table + candidate(w[u].z, M));
      }
#pragma unroll
      for (int t = 0; t < 4; ++t) {
        const uint32_t wu = (t & 1) ? w[t >> 1].w : w[t >> 1].y;
        acc += accept_f32(wu, T, x[t]) ? 1u : 0u;
      }
    }
  }
  out[tid] = acc;
}

}  // namespace
}  // namespace gbar

using namespace gbar;

extern "C" int ar_probe_throughput(int mode, const float* d_table, uint32_t M,
                                   uint32_t blocks_per_thread, uint32_t threads_per_sm,
                                   uint32_t* d_out, size_t out_words, void* stream) {
  if (mode != AR_PROBE_PHILOX && mode != AR_PROBE_PHILOX_GATHER) return AR_ERR_ARG;
  if (blocks_per_thread == 0 || (blocks_per_thread & 1u) || threads_per_sm == 0 ||
      threads_per_sm % kProbeThreads || !d_out)
    return AR_ERR_ARG;
  if (mode == AR_PROBE_PHILOX_GATHER && (!d_table || M == 0 || M >= (1u << 31))) return AR_ERR_ARG;
  if (!aligned(d_out, 4) || !aligned(d_table, 4)) return AR_ERR_ALIGN;
  const DeviceInfo& dev = device_info();
  const uint64_t grid = (uint64_t)std::max(1, dev.sm_count) * (threads_per_sm / kProbeThreads);
  if (grid * kProbeThreads > out_words || grid >= (1ull << 31)) return AR_ERR_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (mode == AR_PROBE_PHILOX)
    k_probe<AR_PROBE_PHILOX><<<(uint32_t)grid, kProbeThreads, 0, s>>>(blocks_per_thread, 1u, 2u,
                                                                       d_table, M, 1.0f, d_out);
  else
    k_probe<AR_PROBE_PHILOX_GATHER><<<(uint32_t)grid, kProbeThreads, 0, s>>>(
        blocks_per_thread, 1u, 2u, d_table, M, 1.0f, d_out);
  return check_launch();
}
