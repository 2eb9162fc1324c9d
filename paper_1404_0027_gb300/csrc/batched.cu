// ar_select_batched: thousands of realizations with uneven M_b and K_b in one
// persistent launch.  The paper runs K realizations as K thread blocks of M
// threads (Section "A GPU acceptance-rejection algorithm"; 1D grid limited to
// 65536 blocks, Section "Implementation"; several blocks per realization when
// M exceeds a block, Discussion).  Here a grid of one CTA per SM pulls
// realizations from a work queue; each realization's propensities are
// streamed once from HBM into shared memory by the tensor memory accelerator
// (cp.async.bulk completing on an mbarrier) while the previous realization
// is being selected from (double buffering); the CTA reduces the exact
// maximum (the threshold T) and the FP64-grade sum, then its warps run the
// warp-level AR selection engine on the K_b selections.
#include "device.cuh"
#include "host.hpp"
#include "select.cuh"

namespace gbar {
namespace {

constexpr int kNT = 512;
constexpr int kWarps = kNT / 32;
constexpr uint32_t kBufBytes = 64u * 1024u;        // one realization slot
constexpr uint32_t kSlotBytes = kBufBytes + 16u;   // + realignment
constexpr size_t kScratch = (size_t)kWarps * 64 * sizeof(uint32_t);
constexpr size_t kSmem = 2 * (size_t)kSlotBytes + kScratch;
constexpr uint32_t kWaitPolls = 1u << 16;          // bounded mbarrier wait (~6 s at most)

// Work queue in the caller's workspace.  It must be zero before the first
// call; the last CTA to finish returns it to zero, so a call is one launch.
struct BatchWork {
  uint32_t queue;  // next realization to claim
  uint32_t done;   // CTAs finished
  uint32_t pad[2];
};

struct BatchParams {
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

__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void* src, uint32_t bytes,
                                         uint32_t bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
      ::"r"(dst), "l"(src), "r"(bytes), "r"(bar)
      : "memory");
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes)
               : "memory");
}

// Realization descriptor held in shared memory while it is in flight.
struct Slot {
  int64_t a_begin;     // element offset in alpha_cat
  uint32_t M;
  uint32_t b;          // batch index (B = none)
  uint32_t shift;      // byte offset of element 0 inside the slot
  uint32_t in_smem;    // 1: staged in shared memory; 0: read from global
};

// Issues the load of realization b into slot `slot` (thread 0 only).
template <typename TS>
__device__ void issue_load(const BatchParams& p, uint32_t b, Slot& sl, unsigned char* buf,
                           uint32_t bar) {
  sl.b = b;
  if (b >= p.B) {
    sl.M = 0;
    sl.in_smem = 0;
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
    return;
  }
  const int64_t a0 = p.offsets[b], a1 = p.offsets[b + 1];
  sl.a_begin = a0;
  sl.M = (uint32_t)(a1 - a0);
  const uintptr_t g0 = (uintptr_t)(p.alpha + a0 * (int64_t)sizeof(TS));
  const uintptr_t g1 = g0 + (uintptr_t)sl.M * sizeof(TS);
  sl.shift = (uint32_t)(g0 & 15u);
  sl.in_smem = (uint64_t)sl.M * sizeof(TS) <= kBufBytes;
  const uintptr_t lo = (g0 + 15u) & ~uintptr_t(15);
  const uintptr_t hi = g1 & ~uintptr_t(15);
  if (sl.in_smem && hi > lo) {
    const uint32_t total = (uint32_t)(hi - lo);
    mbar_expect_tx(bar, total);
    const uint32_t dst0 = (uint32_t)__cvta_generic_to_shared(buf) + (uint32_t)(lo - (g0 & ~uintptr_t(15)));
    for (uint32_t off = 0; off < total; off += 32768u) {
      const uint32_t n = total - off < 32768u ? total - off : 32768u;
      bulk_g2s(dst0 + off, (const void*)(lo + off), n, bar);
    }
  } else {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
  }
}

template <typename TS, int CMP>
__global__ void __launch_bounds__(kNT, 1) k_batched(const BatchParams p) {
  extern __shared__ __align__(128) unsigned char smem[];
  unsigned char* buf[2] = {smem, smem + kSlotBytes};
  uint32_t* scr = reinterpret_cast<uint32_t*>(smem + 2 * kSlotBytes) + (threadIdx.x >> 5) * 64;
  __shared__ __align__(8) uint64_t bars[2];
  __shared__ Slot slots[2];
  __shared__ unsigned long long s_r0[kWarps], s_r1[kWarps];
  __shared__ float s_r2[kWarps];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint32_t bar0 = (uint32_t)__cvta_generic_to_shared(&bars[0]);
  const uint32_t bar1 = (uint32_t)__cvta_generic_to_shared(&bars[1]);

  if (threadIdx.x == 0) {
    mbar_init(bar0, 1);
    mbar_init(bar1, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    const uint32_t b = atomicAdd(&p.work->queue, 1u);
    issue_load<TS>(p, b, slots[0], buf[0], bar0);
  }
  __syncthreads();

  SelCounters cnt;
  uint32_t status_acc = 0;
  for (uint32_t it = 0;; ++it) {
    const uint32_t cur = it & 1u;
    const Slot sl = slots[cur];
    if (sl.b >= p.B) break;
    if (threadIdx.x == 0) {
      const uint32_t nb = atomicAdd(&p.work->queue, 1u);
      issue_load<TS>(p, nb, slots[cur ^ 1u], buf[cur ^ 1u], cur ? bar0 : bar1);
    }
    const bool landed = mbar_wait(&bars[cur], (it >> 1) & 1u, kWaitPolls);
    if (__syncthreads_or(!landed)) {
      if (threadIdx.x == 0) atomicOr(p.status, AR_STATUS_TIMEOUT);
      break;
    }
    const TS* g_alpha = reinterpret_cast<const TS*>(p.alpha) + sl.a_begin;
    const TS* a = sl.in_smem ? reinterpret_cast<const TS*>(buf[cur] + sl.shift) : g_alpha;
    const uint32_t M = sl.M;
    if (sl.in_smem) {
      // Elements outside the 16-byte aligned range moved by the bulk copy:
      // [0, head) and [tail, M) (all of them when no aligned block exists).
      const int64_t g0 = (int64_t)(uintptr_t)g_alpha;
      const int64_t g1 = g0 + (int64_t)M * (int64_t)sizeof(TS);
      const int64_t lo = (g0 + 15) & ~int64_t(15), hi = g1 & ~int64_t(15);
      int64_t head = (lo - g0) / (int64_t)sizeof(TS);
      int64_t tail = (hi - g0) / (int64_t)sizeof(TS);
      if (hi <= lo) head = tail = M;  // no bulk copy was issued: load everything
      if (head > M) head = M;
      if (tail < head) tail = head;
      TS* w = reinterpret_cast<TS*>(buf[cur] + sl.shift);
      for (int64_t i = threadIdx.x; i < head; i += kNT) w[i] = g_alpha[i];
      for (int64_t i = tail + threadIdx.x; i < M; i += kNT) w[i] = g_alpha[i];
    }
    __syncthreads();

    // ---- bound: exact maximum and FP64-grade sum ------------------------
    double T;
    bool bad;
    if constexpr (sizeof(TS) == 4) {
      MaxF32 mx;
      for (uint32_t i = threadIdx.x; i < M; i += kNT) mx.add(__float_as_uint(a[i]));
      mx.smax = warp_max_i32(mx.smax);
      mx.umax = warp_max_u32(mx.umax);
      if (lane == 0) {
        s_r0[warp] = (unsigned long long)(uint32_t)mx.smax;
        s_r1[warp] = mx.umax;
      }
      __syncthreads();
      int32_t sm = INT32_MIN;
      uint32_t um = 0;
#pragma unroll
      for (int w = 0; w < kWarps; ++w) {
        sm = max(sm, (int32_t)(uint32_t)s_r0[w]);
        um = max(um, (uint32_t)s_r1[w]);
      }
      mx.smax = sm;
      mx.umax = um;
      bad = mx.bad();
      const uint32_t mbits = mx.value_bits();
      T = (double)__uint_as_float(mbits);
      const int e_ref = fx_eref(mbits);
      FxSum fx;
      for (uint32_t i = threadIdx.x; i < M; i += kNT) fx.add(__float_as_uint(a[i]), e_ref);
      fx.warp_reduce();
      __syncthreads();  // s_r* reuse
      if (lane == 0) {
        s_r0[warp] = fx.a1;
        s_r1[warp] = fx.a2;
        s_r2[warp] = fx.a3;
      }
      __syncthreads();
      if (warp == 0) {
        FxSum f;
        if (lane < kWarps) {
          f.a1 = s_r0[lane];
          f.a2 = s_r1[lane];
          f.a3 = s_r2[lane];
        }
        f.warp_reduce();
        if (lane == 0) {
          double* o = p.bound_sum + 2 * (size_t)sl.b;
          o[0] = T;
          o[1] = f.to_double(e_ref);
        }
      }
    } else {
      MaxF64 mx;
      double sum = 0.0;
      for (uint32_t i = threadIdx.x; i < M; i += kNT) {
        const double x = a[i];
        mx.add((unsigned long long)__double_as_longlong(x));
        sum = __dadd_rn(sum, x);
      }
      mx.smax = warp_max_i64(mx.smax);
      mx.umax = warp_max_u64(mx.umax);
      sum = warp_sum_f64(sum);
      if (lane == 0) {
        s_r0[warp] = (unsigned long long)mx.smax;
        s_r1[warp] = mx.umax;
      }
      __shared__ double s_sum[kWarps];
      if (lane == 0) s_sum[warp] = sum;
      __syncthreads();
      long long sm = INT64_MIN;
      unsigned long long um = 0;
      double tot = 0.0;
#pragma unroll
      for (int w = 0; w < kWarps; ++w) {
        sm = max(sm, (long long)s_r0[w]);
        um = max(um, s_r1[w]);
      }
      if (warp == 0) {
        tot = lane < kWarps ? s_sum[lane] : 0.0;
        tot = warp_sum_f64(tot);
      }
      mx.smax = sm;
      mx.umax = um;
      bad = mx.bad();
      T = __longlong_as_double((long long)mx.value_bits());
      if (threadIdx.x == 0) {
        double* o = p.bound_sum + 2 * (size_t)sl.b;
        o[0] = T;
        o[1] = tot;
      }
    }
    uint32_t st = 0;
    if (bad) st = AR_STATUS_BAD_ALPHA;
    else if (T == 0.0) st = AR_STATUS_ALL_ZERO;
    const float Tf = __double2float_rn(T);
    if (CMP == AR_CMP_F32 && !st && isinf(Tf)) st = AR_STATUS_BAD_BOUND;

    // ---- selections ------------------------------------------------------
    const int64_t o0 = p.out_offsets[sl.b];
    const uint32_t Kb = (uint32_t)(p.out_offsets[sl.b + 1] - o0);
    int32_t* idx = p.idx + o0;
    const uint32_t per = (Kb + kWarps - 1) / kWarps;
    const uint32_t q = min(Kb, per * (uint32_t)warp);
    const uint32_t q_end = min(Kb, q + per);
    if (st) {
      status_acc |= st;
      warp_fill(q, q_end, (int32_t)M, idx);
    } else if (q < q_end) {
      const uint32_t bid = p.b_base + sl.b;
      if constexpr (CMP == AR_CMP_F32) {
        auto acc = [&](uint32_t j, uint32_t w) -> bool {
          float x;
          if constexpr (sizeof(TS) == 4) x = a[j];
          else x = __double2float_rn(a[j]);
          return accept_f32(w, Tf, x);
        };
        warp_select(q, q_end, p.sel_base, M, bid, p.k0, p.k1, p.cap, acc, idx, scr, cnt);
      } else {
        auto acc = [&](uint32_t j, uint32_t w) -> bool { return accept_f64(w, T, (double)a[j]); };
        warp_select(q, q_end, p.sel_base, M, bid, p.k0, p.k1, p.cap, acc, idx, scr, cnt);
      }
    }
    __syncthreads();  // slot `cur` is free for the load issued next iteration
  }
  if (cnt.capped) status_acc |= AR_STATUS_TRIAL_CAP;
  flush_counters(cnt, p.stats);
  status_acc = __reduce_or_sync(kFull, status_acc);
  if (lane == 0 && status_acc) atomicOr(p.status, status_acc);
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    if (atomicAdd(&p.work->done, 1u) == gridDim.x - 1u) {
      // every CTA has left the claim loop
      p.work->queue = 0u;
      p.work->done = 0u;
      __threadfence();
    }
  }
}

template <typename TS, int CMP>
int launch(const BatchParams& p, cudaStream_t s) {
  auto kern = k_batched<TS, CMP>;
  static bool configured[64] = {false};
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 64 && !configured[dev]) {
    const cudaError_t e =
        cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmem);
    if (e != cudaSuccess) {
      set_cuda_error(e);
      return AR_ERR_CUDA;
    }
    configured[dev] = true;
  }
  const DeviceInfo& d = device_info();
  const unsigned sms = (unsigned)(d.sm_count > 0 ? d.sm_count : 1);
  const unsigned grid = sms < p.B ? sms : p.B;
  kern<<<grid, kNT, kSmem, s>>>(p);
  return check_launch();
}

}  // namespace
}  // namespace gbar

using namespace gbar;

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
  (void)plan;
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
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  BatchWork* wk = static_cast<BatchWork*>(d_work);
  BatchParams p{};
  p.alpha = static_cast<const unsigned char*>(d_alpha_cat);
  p.offsets = d_offsets;
  p.out_offsets = d_out_offsets;
  p.bound_sum = d_bound_sum;
  p.idx = d_idx;
  p.stats = d_stats;
  p.status = d_status;
  p.work = wk;
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
