// ar_select_batched: thousands of realizations with uneven M_b and K_b in one
// persistent launch.  The paper runs K realizations as K thread blocks of M
// threads (Section "A GPU acceptance-rejection algorithm"; a 1D grid limited
// to 65536 blocks, Section "Implementation"; several blocks per realization
// when M exceeds a block, Discussion).
//
// Here every warp of a persistent grid is an independent worker: it claims a
// realization from a global queue (in the order a plan chose, largest first,
// so the last claims are the cheap ones), streams its propensities once from
// HBM with coalesced loads -- computing the exact maximum (the threshold T)
// on bit patterns and an exact fixed-point sum -- and then runs the
// warp-level selection engine of select.cuh on its K_b selections.  The
// engine's gathers hit the realization's lines in L1 (read-only loads), so no
// staging copy or CTA-wide barrier is needed, and warps never wait for one
// another: a warp that finishes early claims the next realization.
#include <algorithm>
#include <cmath>
#include <numeric>
#include <vector>

#include "device.cuh"
#include "host.hpp"
#include "select.cuh"

namespace gbar {
namespace {

constexpr int kWarps = 16;  // warps per CTA
constexpr int kNT = kWarps * 32;
constexpr int kCtasPerSm = 2;
constexpr uint32_t kFxBlock = 16384;  // per-lane fixed-point block (< 2^14 terms of < 2^48)

struct BatchWork {
  uint32_t queue;  // next position of the processing order to claim
  uint32_t done;   // CTAs finished
  uint32_t pad[2];
};

struct BatchParams {
  const uint32_t* order;  // processing order (plan), NULL: 0..B-1
  const unsigned char* alpha;
  const int64_t* offsets;
  const int64_t* out_offsets;
  double* bound_sum;
  int32_t* idx;
  ar_stats* stats;
  uint32_t* status;
  BatchWork* work;
  unsigned long long cap;
  uint32_t B;
  uint32_t sel_base;
  uint32_t b_base;
  uint32_t k0, k1;
};

// Warp reduction of one realization: exact maximum (on bit patterns),
// validity, and the FP64-grade sum.  Every lane returns T and the sum.
template <typename TS>
__device__ __forceinline__ void warp_bound(const TS* __restrict__ a, uint32_t M, double& T,
                                           double& sum, bool& bad) {
  const uint32_t lane = threadIdx.x & 31u;
  if constexpr (sizeof(TS) == 4) {
    const uint32_t* u = reinterpret_cast<const uint32_t*>(a);
    MaxF32 mx;
    uint32_t i = lane;
    for (; i + 96 < M; i += 128) {
      const uint32_t x0 = __ldg(u + i), x1 = __ldg(u + i + 32), x2 = __ldg(u + i + 64),
                     x3 = __ldg(u + i + 96);
      mx.add(x0);
      mx.add(x1);
      mx.add(x2);
      mx.add(x3);
    }
    for (; i < M; i += 32) mx.add(__ldg(u + i));
    mx.smax = warp_max_i32(mx.smax);
    mx.umax = warp_max_u32(mx.umax);
    bad = mx.bad();
    const uint32_t mb = mx.value_bits();
    T = (double)__uint_as_float(mb);
    const int e_ref = fx_eref(mb);
    // second pass (L1 hits): exact per lane, in blocks of kFxBlock elements
    double lane_sum = 0.0;
    FxSum fx;
    uint32_t in_block = 0;
    i = lane;
    for (; i + 96 < M; i += 128) {
      const uint32_t x0 = __ldg(u + i), x1 = __ldg(u + i + 32), x2 = __ldg(u + i + 64),
                     x3 = __ldg(u + i + 96);
      fx.add(x0, e_ref);
      fx.add(x1, e_ref);
      fx.add(x2, e_ref);
      fx.add(x3, e_ref);
      if ((in_block += 4) >= kFxBlock) {
        lane_sum = __dadd_rn(lane_sum, fx.to_double(e_ref));
        fx = FxSum();
        in_block = 0;
      }
    }
    for (; i < M; i += 32) fx.add(__ldg(u + i), e_ref);
    if (M < 65536u) {
      // fewer than 2^16 terms of < 2^48 in the whole warp: exact integer sum
      fx.warp_reduce();
      sum = fx.to_double(e_ref);
    } else {
      lane_sum = __dadd_rn(lane_sum, fx.to_double(e_ref));
      sum = warp_sum_f64(lane_sum);
    }
  } else {
    const unsigned long long* u = reinterpret_cast<const unsigned long long*>(a);
    MaxF64 mx;
    double s = 0.0;
    for (uint32_t i = lane; i < M; i += 32) {
      const unsigned long long x = __ldg(u + i);
      mx.add(x);
      s = __dadd_rn(s, __longlong_as_double((long long)x));
    }
    mx.smax = warp_max_i64(mx.smax);
    mx.umax = warp_max_u64(mx.umax);
    bad = mx.bad();
    T = __longlong_as_double((long long)mx.value_bits());
    sum = warp_sum_f64(s);
  }
}

template <typename TS, int CMP>
__global__ void __launch_bounds__(kNT, kCtasPerSm) k_batched(const BatchParams p) {
  __shared__ uint32_t s_scr[kWarps * 64];
  const uint32_t lane = threadIdx.x & 31u;
  uint32_t* scr = s_scr + (threadIdx.x >> 5) * 64;
  SelCounters cnt;
  uint32_t status_acc = 0;
  for (;;) {
    uint32_t i = 0;
    if (lane == 0) i = atomicAdd(&p.work->queue, 1u);
    i = __shfl_sync(kFull, i, 0);
    if (i >= p.B) break;
    const uint32_t b = p.order ? __ldg(p.order + i) : i;
    int64_t v = 0;
    if (lane < 2) v = __ldg(p.offsets + b + lane);
    else if (lane < 4) v = __ldg(p.out_offsets + b + lane - 2);
    const int64_t a0 = __shfl_sync(kFull, v, 0), a1 = __shfl_sync(kFull, v, 1);
    const int64_t o0 = __shfl_sync(kFull, v, 2), o1 = __shfl_sync(kFull, v, 3);
    const uint32_t K = o1 > o0 ? (uint32_t)(o1 - o0) : 0u;
    int32_t* idx = p.idx + o0;
    uint32_t st = 0;
    uint32_t M = 0;
    if (a1 < a0 || a1 - a0 >= (1ll << 31)) {
      st = AR_STATUS_UNSUPPORTED;
      M = a1 < a0 ? 0u : 0x7fffffffu;
    } else {
      M = (uint32_t)(a1 - a0);
    }
    const TS* a = reinterpret_cast<const TS*>(p.alpha) + a0;
    double T = 0.0, sum = 0.0;
    if (!st) {
      bool bad = false;
      warp_bound<TS>(a, M, T, sum, bad);
      if (bad) st = AR_STATUS_BAD_ALPHA;
      else if (T == 0.0) st = AR_STATUS_ALL_ZERO;
      else if (CMP == AR_CMP_F32 && isinf(__double2float_rn(T))) st = AR_STATUS_BAD_BOUND;
    }
    if (lane == 0) {
      double* o = p.bound_sum + 2 * (size_t)b;
      o[0] = T;
      o[1] = sum;
    }
    if (st) {
      status_acc |= st;
      warp_fill(0, K, (int32_t)M, idx);
      continue;
    }
    const uint32_t bid = p.b_base + b;
    if constexpr (CMP == AR_CMP_F32) {
      const float Tf = __double2float_rn(T);
      auto acc = [&](uint32_t j, uint32_t w) -> bool {
        float x;
        if constexpr (sizeof(TS) == 4) x = __ldg(a + j);
        else x = __double2float_rn(__ldg(a + j));
        return accept_f32(w, Tf, x);
      };
      warp_select(0u, K, p.sel_base, M, bid, p.k0, p.k1, p.cap, acc, idx, scr, cnt);
    } else {
      auto acc = [&](uint32_t j, uint32_t w) -> bool {
        return accept_f64(w, T, (double)__ldg(a + j));
      };
      warp_select(0u, K, p.sel_base, M, bid, p.k0, p.k1, p.cap, acc, idx, scr, cnt);
    }
  }
  if (cnt.capped) status_acc |= AR_STATUS_TRIAL_CAP;
  flush_counters(cnt, p.stats);
  status_acc = __reduce_or_sync(kFull, status_acc);
  if (lane == 0 && status_acc) atomicOr(p.status, status_acc);
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    if (atomicAdd(&p.work->done, 1u) == gridDim.x - 1u) {
      // every CTA has left the claim loop: return the queue to zero
      p.work->queue = 0u;
      p.work->done = 0u;
      __threadfence();
    }
  }
}

template <typename TS, int CMP>
int launch(const BatchParams& p, cudaStream_t s) {
  auto kern = k_batched<TS, CMP>;
  int per_sm = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kNT, 0);
  if (per_sm < 1) per_sm = 1;
  const DeviceInfo& d = device_info();
  const uint64_t sms = (uint64_t)(d.sm_count > 0 ? d.sm_count : 1);
  // no more CTAs than needed to give every realization its own warp
  const uint64_t need = ((uint64_t)p.B + kWarps - 1) / kWarps;
  const unsigned grid = (unsigned)std::min<uint64_t>(sms * (uint64_t)per_sm, need);
  kern<<<grid, kNT, 0, s>>>(p);
  return check_launch();
}

}  // namespace
}  // namespace gbar

using namespace gbar;

// The processing order of a batch: realizations sorted by an estimate of
// their cost, largest first, so that the work still unclaimed near the end
// of a launch is the cheapest (longest-processing-time-first list
// scheduling over the persistent warps).
struct ar_plan {
  int device;
  int64_t B;
  uint32_t* d_order;
};

extern "C" int ar_plan_create(const int64_t* h_offsets, const int64_t* h_out_offsets, int64_t B,
                              ar_plan** out) {
  if (!out || B <= 0 || B >= (1ll << 31) || !h_offsets || !h_out_offsets) return AR_ERR_ARG;
  *out = nullptr;
  // cost model: one streaming pass over M_b plus K_b selections whose trial
  // count grows like log M_b for spread-out propensities
  std::vector<double> cost(B);
  for (int64_t b = 0; b < B; ++b) {
    const int64_t M = h_offsets[b + 1] - h_offsets[b];
    const int64_t K = h_out_offsets[b + 1] - h_out_offsets[b];
    if (M < 0 || K < 0) return AR_ERR_ARG;
    cost[b] = 0.4 * (double)M + 1.7 * (double)K * (0.6 + std::log((double)std::max<int64_t>(M, 2)));
  }
  std::vector<uint32_t> order(B);
  std::iota(order.begin(), order.end(), 0u);
  std::stable_sort(order.begin(), order.end(),
                   [&](uint32_t x, uint32_t y) { return cost[x] > cost[y]; });
  auto* p = new ar_plan();
  p->device = device_info().device;
  p->B = B;
  p->d_order = nullptr;
  cudaError_t e = cudaMalloc(&p->d_order, sizeof(uint32_t) * (size_t)B);
  if (e == cudaSuccess)
    e = cudaMemcpy(p->d_order, order.data(), sizeof(uint32_t) * (size_t)B, cudaMemcpyHostToDevice);
  if (e != cudaSuccess) {
    set_cuda_error(e);
    cudaFree(p->d_order);
    delete p;
    return AR_ERR_CUDA;
  }
  *out = p;
  return AR_OK;
}

extern "C" void ar_plan_destroy(ar_plan* plan) {
  if (!plan) return;
  int cur = 0;
  cudaGetDevice(&cur);
  if (cur != plan->device) cudaSetDevice(plan->device);
  cudaFree(plan->d_order);
  if (cur != plan->device) cudaSetDevice(cur);
  delete plan;
}

extern "C" size_t ar_select_batched_workspace_size(int64_t B) {
  (void)B;
  return sizeof(BatchWork);
}

extern "C" int ar_select_batched(const void* d_alpha_cat, int dtype, const int64_t* d_offsets,
                                 const int64_t* d_out_offsets, int64_t B, uint64_t seed,
                                 uint64_t sel_offset, uint32_t realization_base, int cmp,
                                 uint64_t trial_cap, const ar_plan* plan, double* d_bound_sum,
                                 int32_t* d_idx, ar_stats* d_stats, uint32_t* d_status,
                                 void* d_work, size_t work_bytes, void* stream) {
  if (!valid_dtype(dtype) || !valid_cmp(cmp) || B < 0 || B >= (1ll << 31)) return AR_ERR_ARG;
  if (trial_cap < 1 || trial_cap > (1ull << 32)) return AR_ERR_ARG;
  if (B == 0) return AR_OK;
  if (!d_alpha_cat || !d_offsets || !d_out_offsets || !d_bound_sum || !d_idx || !d_status)
    return AR_ERR_ARG;
  if (!aligned(d_alpha_cat, dtype_size(dtype)) || !aligned(d_offsets, 8) ||
      !aligned(d_out_offsets, 8) || !aligned(d_bound_sum, 8) || !aligned(d_idx, 4) ||
      !aligned(d_status, 4) || !aligned(d_stats, 8))
    return AR_ERR_ALIGN;
  if (!d_work || work_bytes < ar_select_batched_workspace_size(B)) return AR_ERR_WORKSPACE;
  if (!aligned(d_work, 16)) return AR_ERR_ALIGN;
  if ((uint64_t)realization_base + (uint64_t)B > (1ull << 32)) return AR_ERR_ARG;
  if (sel_offset >= (1ull << 32)) return AR_ERR_ARG;
  if (plan) {
    int dev = 0;
    cudaGetDevice(&dev);
    if (plan->B != B || plan->device != dev) return AR_ERR_ARG;
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  BatchParams p{};
  p.order = plan ? plan->d_order : nullptr;
  p.alpha = static_cast<const unsigned char*>(d_alpha_cat);
  p.offsets = d_offsets;
  p.out_offsets = d_out_offsets;
  p.bound_sum = d_bound_sum;
  p.idx = d_idx;
  p.stats = d_stats;
  p.status = d_status;
  p.work = static_cast<BatchWork*>(d_work);
  p.cap = trial_cap;
  p.B = (uint32_t)B;
  p.sel_base = (uint32_t)sel_offset;
  p.b_base = realization_base;
  p.k0 = (uint32_t)(seed & 0xffffffffu);
  p.k1 = (uint32_t)(seed >> 32);
  if (dtype == AR_F32)
    return cmp == AR_CMP_F32 ? launch<float, AR_CMP_F32>(p, s) : launch<float, AR_CMP_F64>(p, s);
  return cmp == AR_CMP_F32 ? launch<double, AR_CMP_F32>(p, s) : launch<double, AR_CMP_F64>(p, s);
}
