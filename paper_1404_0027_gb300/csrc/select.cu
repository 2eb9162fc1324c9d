// ar_select_k: K independent AR selections from one propensity vector
// (Section "A GPU acceptance-rejection algorithm": K next reactions selected
// in parallel; Section "Test and validation": K realizations sharing one D).
//
// Every CTA stages alpha in shared memory (converted once to the comparison
// precision when that loses nothing the comparison uses) and, when no bound
// is given, reduces the exact maximum itself from that copy -- the bound
// reduction fused into the selection kernel.  Warps then run the warp-level
// selection engine of select.cuh over contiguous ranges of selection ids,
// with 1, 2 or 4 Philox blocks per lane per round as the expected trials per
// selection (M T / sum of the staged copy) are few, moderate or many.
// Vectors larger than the shared-memory budget are gathered from global
// memory (they stay L2-resident: 2^20 FP32 propensities are 4 MB of a
// 129 MB L2).
#include "device.cuh"
#include "host.hpp"
#include "select.cuh"

namespace gbar {
namespace {

constexpr int kNT = 512;

constexpr int kWarps = kNT / 32;
constexpr size_t kScratch = (size_t)kWarps * 64 * sizeof(uint32_t);

struct SelParams {
  const void* alpha;
  const double* bound;
  int32_t* idx;
  ar_stats* stats;
  uint32_t* status;
  unsigned long long cap;
  uint32_t M;
  uint32_t K;
  uint32_t spw;  // selections per warp
  uint32_t sel_base;
  uint32_t b;
  uint32_t k0, k1;
};

__host__ __device__ inline size_t align16(size_t x) { return (x + 15) & ~size_t(15); }

// TS: source element type; TA: staged element type; CMP: comparison.
template <typename TS, typename TA, int CMP, bool SMEM>
__global__ void __launch_bounds__(kNT) k_select(const SelParams p) {
  extern __shared__ __align__(16) unsigned char smem[];
  const uint32_t M = p.M;
  TA* s_alpha = reinterpret_cast<TA*>(smem);
  uint32_t* scr = reinterpret_cast<uint32_t*>(smem + (SMEM ? align16((size_t)M * sizeof(TA)) : 0)) +
                  (threadIdx.x >> 5) * 64;
  const TS* g_alpha = static_cast<const TS*>(p.alpha);
  __shared__ unsigned long long s_max[kWarps];
  __shared__ unsigned long long s_umax[kWarps];
  __shared__ float s_sum[kWarps];

  // 1. stage alpha (and its maximum when no bound is given)
  unsigned long long smax = 0, umax = 0;  // bit-pattern maxima of the staged values
  float ssum = 0.f;  // rough total: sets the Philox blocks per lane per round
  if (SMEM) {
    for (uint32_t i = threadIdx.x; i < M; i += kNT) {
      const TS x = __ldg(g_alpha + i);
      TA y;
      if constexpr (sizeof(TA) == sizeof(TS)) y = x;
      else y = __double2float_rn(x);
      s_alpha[i] = y;
      ssum += (float)y;
      if (p.bound == nullptr) {
        if constexpr (sizeof(TA) == 4) {
          const uint32_t bits = __float_as_uint(y);
          const unsigned long long sb = (int32_t)bits < 0 ? 0ull : bits;
          smax = sb > smax ? sb : smax;
          umax = bits > umax ? bits : umax;
        } else {
          const unsigned long long bits = (unsigned long long)__double_as_longlong(y);
          const unsigned long long sb = (long long)bits < 0 ? 0ull : bits;
          smax = sb > smax ? sb : smax;
          umax = bits > umax ? bits : umax;
        }
      }
    }
  }
  double T = 0.0;
  bool bad_alpha = false;
  if (p.bound == nullptr) {
    smax = warp_max_u64(smax);
    umax = warp_max_u64(umax);
    if ((threadIdx.x & 31) == 0) {
      s_max[threadIdx.x >> 5] = smax;
      s_umax[threadIdx.x >> 5] = umax;
    }
    __syncthreads();
    smax = 0;
    umax = 0;
#pragma unroll
    for (int w = 0; w < kWarps; ++w) {
      smax = s_max[w] > smax ? s_max[w] : smax;
      umax = s_umax[w] > umax ? s_umax[w] : umax;
    }
    if constexpr (sizeof(TA) == 4) {
      bad_alpha = smax >= 0x7f800000ull || umax > 0x80000000ull;
      T = (double)__uint_as_float((uint32_t)smax);
    } else {
      bad_alpha = smax >= 0x7ff0000000000000ull || umax > 0x8000000000000000ull;
      T = __longlong_as_double((long long)smax);
    }
  } else {
    T = *p.bound;
    __syncthreads();
  }
  // Philox blocks per lane per round, from the expected trials per selection
  // M T / sum (staged vectors; 2 otherwise): many blocks per round amortise
  // the round's ballots when acceptance is rare, few waste little when it is
  // frequent.  The results do not depend on it.
  int U = 2;
  if (SMEM) {
    ssum = warp_sum_f32(ssum);
    if ((threadIdx.x & 31) == 0) s_sum[threadIdx.x >> 5] = ssum;
    __syncthreads();
    float tot = 0.f;
#pragma unroll
    for (int w = 0; w < kWarps; ++w) tot += s_sum[w];
    const float E = (float)M * (float)T / tot;
    if (E <= 4.f) U = 1;
    else if (E > 48.f) U = 4;
  }

  // 2. bound checks (identical in every CTA)
  uint32_t st = 0;
  const float Tf = __double2float_rn(T);
  if (bad_alpha) st = AR_STATUS_BAD_ALPHA;
  else if (!(T >= 0.0) || isinf(T) || (CMP == AR_CMP_F32 && isinf(Tf))) st = AR_STATUS_BAD_BOUND;
  else if (T == 0.0 || M == 0) st = AR_STATUS_ALL_ZERO;

  // 3. selections
  const uint32_t gw = blockIdx.x * kWarps + (threadIdx.x >> 5);
  const unsigned long long q64 = (unsigned long long)gw * p.spw;
  if (q64 < p.K) {
    const uint32_t q = (uint32_t)q64;
    const uint32_t q_end = (uint32_t)min((unsigned long long)p.K, q64 + p.spw);
    if (st) {
      warp_fill(q, q_end, (int32_t)M, p.idx);
      if ((threadIdx.x & 31) == 0 && blockIdx.x == 0 && (threadIdx.x >> 5) == 0)
        atomicOr(p.status, st);
    } else {
      SelCounters c;
      auto run_select = [&](int u, uint32_t q0, uint32_t q1, const auto& acc, SelCounters& cc) {
        if (u == 1)
          warp_select<1>(q0, q1, p.sel_base, M, p.b, p.k0, p.k1, p.cap, acc, p.idx, scr, cc);
        else if (u == 4)
          warp_select<4>(q0, q1, p.sel_base, M, p.b, p.k0, p.k1, p.cap, acc, p.idx, scr, cc);
        else
          warp_select<2>(q0, q1, p.sel_base, M, p.b, p.k0, p.k1, p.cap, acc, p.idx, scr, cc);
      };
      if constexpr (CMP == AR_CMP_F32) {
        auto acc = [&](uint32_t j, uint32_t w) -> bool {
          float a;
          if constexpr (SMEM) a = (float)s_alpha[j];
          else if constexpr (sizeof(TS) == 4) a = __ldg(g_alpha + j);
          else a = __double2float_rn(__ldg(g_alpha + j));
          return accept_f32(w, Tf, a);
        };
        run_select(U, q, q_end, acc, c);
      } else {
        const F64Bound tb = f64_bound(T);  // the FP64 test with its FP32 pre-filter
        auto acc = [&](uint32_t j, uint32_t w) -> bool {
          if constexpr (SMEM) return accept_f64(w, tb, s_alpha[j]);
          else return accept_f64(w, tb, __ldg(g_alpha + j));
        };
        run_select(U, q, q_end, acc, c);
      }
      flush_counters(c, p.stats);
      if (c.capped) {
        if ((threadIdx.x & 31) == 0) atomicOr(p.status, AR_STATUS_TRIAL_CAP);
      }
    }
  }
}

template <typename TS, typename TA, int CMP, bool SMEM>
int launch(const SelParams& p, size_t smem, int sm_count, cudaStream_t s) {
  auto kern = k_select<TS, TA, CMP, SMEM>;
  static int configured_smem[64] = {0};
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 64 && configured_smem[dev] < (int)smem) {
    const cudaError_t e =
        cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) {
      set_cuda_error(e);
      return AR_ERR_CUDA;
    }
    configured_smem[dev] = (int)smem;
  }
  int per_sm = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kNT, smem);
  if (per_sm < 1) per_sm = 1;
  // Spread the selections over every resident warp, at least one each.
  const unsigned long long w_max = (unsigned long long)sm_count * per_sm * kWarps;
  SelParams q = p;
  q.spw = (uint32_t)((p.K + w_max - 1) / w_max);
  if (q.spw < 1) q.spw = 1;
  const unsigned long long warps = (p.K + q.spw - 1) / q.spw;
  const unsigned grid = (unsigned)((warps + kWarps - 1) / kWarps);
  kern<<<grid, kNT, smem, s>>>(q);
  return check_launch();
}

}  // namespace
}  // namespace gbar

using namespace gbar;

extern "C" size_t ar_select_k_smem_limit(void) {
  const DeviceInfo& d = device_info();
  const size_t lim = d.max_smem_optin > 0 ? (size_t)d.max_smem_optin : (size_t)(227 * 1024);
  return lim - kScratch;
}

extern "C" int ar_select_k(const void* d_alpha, int dtype, int64_t M, const double* d_bound,
                           int64_t K, uint64_t seed, uint64_t sel_offset, uint32_t realization,
                           int cmp, uint64_t trial_cap, int32_t* d_idx, ar_stats* d_stats,
                           uint32_t* d_status, void* stream) {
  if (!valid_dtype(dtype) || !valid_cmp(cmp) || M < 0 || M >= (1ll << 31) || K < 0)
    return AR_ERR_ARG;
  if (trial_cap < 1 || trial_cap > (1ull << 32)) return AR_ERR_ARG;
  if (sel_offset + (uint64_t)K > (1ull << 32)) return AR_ERR_ARG;
  if (K == 0) return AR_OK;
  if (!d_idx || !d_status || (M > 0 && !d_alpha)) return AR_ERR_ARG;
  if (!aligned(d_alpha, dtype_size(dtype)) || !aligned(d_idx, 4) || !aligned(d_status, 4) ||
      !aligned(d_bound, 8) || !aligned(d_stats, 8))
    return AR_ERR_ALIGN;
  const DeviceInfo& dev = device_info();
  // staged element: FP32 unless both the data and the comparison are FP64
  const size_t es = (dtype == AR_F64 && cmp == AR_CMP_F64) ? 8 : 4;
  const bool fits = (size_t)M * es <= ar_select_k_smem_limit();
  if (!d_bound && !fits) return AR_ERR_ARG;
  SelParams p{};
  p.alpha = d_alpha;
  p.bound = d_bound;
  p.idx = d_idx;
  p.stats = d_stats;
  p.status = d_status;
  p.cap = trial_cap;
  p.M = (uint32_t)M;
  p.K = (uint32_t)K;
  p.sel_base = (uint32_t)sel_offset;
  p.b = realization;
  p.k0 = (uint32_t)(seed & 0xffffffffu);
  p.k1 = (uint32_t)(seed >> 32);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const size_t smem = (fits ? align16((size_t)M * es) : 0) + kScratch;
  const int sms = dev.sm_count > 0 ? dev.sm_count : 1;
  if (dtype == AR_F32) {
    if (cmp == AR_CMP_F32)
      return fits ? launch<float, float, AR_CMP_F32, true>(p, smem, sms, s)
                  : launch<float, float, AR_CMP_F32, false>(p, smem, sms, s);
    return fits ? launch<float, float, AR_CMP_F64, true>(p, smem, sms, s)
                : launch<float, float, AR_CMP_F64, false>(p, smem, sms, s);
  }
  if (cmp == AR_CMP_F32)
    return fits ? launch<double, float, AR_CMP_F32, true>(p, smem, sms, s)
                : launch<double, double, AR_CMP_F32, false>(p, smem, sms, s);
  return fits ? launch<double, double, AR_CMP_F64, true>(p, smem, sms, s)
              : launch<double, double, AR_CMP_F64, false>(p, smem, sms, s);
}
