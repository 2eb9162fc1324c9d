// ar_bound: threshold T = max_j alpha_j (exact) and alpha_0 = sum_j alpha_j
// (FP64-grade) of one propensity vector.  Paper: the threshold of Section
// "Election step" (T_w = w max alpha, w = 1, in Section "Quality of the
// selection of the reaction indexes"); alpha_0 of Section "The Stochastic
// Simulation Algorithm"; the reduction of Section "A GPU acceptance-rejection
// algorithm" (a classical GPU reduction, extended to several blocks when M
// exceeds one block, Discussion).
//
// One pass over HBM: each CTA keeps its chunk in registers, reduces the
// maximum on bit patterns (integer max), then accumulates the chunk in exact
// fixed point relative to its own maximum (FP32 input) or in FP64 (FP64
// input).  Multi-CTA launches finish in the last CTA to arrive, which
// combines the per-CTA partials in CTA order (deterministic) and returns the
// workspace header to zero, so a call is a single kernel launch.
#include "device.cuh"
#include "host.hpp"

namespace gbar {
namespace {

constexpr int kNT = 512;
constexpr int kEptF32 = 16;  // chunk 8192 elements (< 2^15, the fixed-point headroom)
constexpr int kEptF64 = 8;   // chunk 4096 elements

struct BoundWork {
  uint32_t counter;
  uint32_t status;
  uint32_t pad[2];
  // followed by unsigned long long maxbits[G]; double sums[G];
};

__device__ __forceinline__ unsigned long long* work_max(BoundWork* w) {
  return reinterpret_cast<unsigned long long*>(w + 1);
}
__device__ __forceinline__ double* work_sum(BoundWork* w, int G) {
  return reinterpret_cast<double*>(work_max(w) + G);
}

// Last-CTA combination of per-CTA partials.  Returns in thread 0.
__device__ void combine_partials(BoundWork* wk, int G, bool f64, double* out,
                                 uint32_t* status) {
  __shared__ unsigned long long s_m[kNT / 32];
  __shared__ double s_s[kNT / 32];
  __threadfence();
  unsigned long long m = 0;
  double s = 0.0;
  for (int i = threadIdx.x; i < G; i += kNT) {
    const unsigned long long mi = __ldcg(work_max(wk) + i);
    m = mi > m ? mi : m;
    s = __dadd_rn(s, __ldcg(work_sum(wk, G) + i));
  }
  m = warp_max_u64(m);
  s = warp_sum_f64(s);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (lane == 0) {
    s_m[warp] = m;
    s_s[warp] = s;
  }
  __syncthreads();
  if (warp == 0) {
    m = lane < kNT / 32 ? s_m[lane] : 0ull;
    s = lane < kNT / 32 ? s_s[lane] : 0.0;
    m = warp_max_u64(m);
    s = warp_sum_f64(s);
    if (lane == 0) {
      const uint32_t st = __ldcg(&wk->status);
      double mx = f64 ? __longlong_as_double((long long)m) : (double)__uint_as_float((uint32_t)m);
      if (st & AR_STATUS_BAD_ALPHA) atomicOr(status, AR_STATUS_BAD_ALPHA);
      else if (m == 0) atomicOr(status, AR_STATUS_ALL_ZERO);
      out[0] = mx;
      out[1] = s;
      // every other CTA has published: return the workspace to zero
      wk->counter = 0u;
      wk->status = 0u;
      __threadfence();
    }
  }
}

// Per-CTA epilogue shared by both dtypes: single-CTA launches write the
// result, multi-CTA launches publish a partial and the last CTA combines.
__device__ void finish_cta(unsigned long long max_bits, bool bad, double partial,
                           bool f64, double* out, uint32_t* status, BoundWork* wk) {
  __shared__ bool s_last;
  if (gridDim.x == 1) {
    if (threadIdx.x == 0) {
      out[0] = f64 ? __longlong_as_double((long long)max_bits)
                   : (double)__uint_as_float((uint32_t)max_bits);
      out[1] = partial;
      if (bad) atomicOr(status, AR_STATUS_BAD_ALPHA);
      else if (max_bits == 0) atomicOr(status, AR_STATUS_ALL_ZERO);
    }
    return;
  }
  const int G = gridDim.x;
  if (threadIdx.x == 0) {
    work_max(wk)[blockIdx.x] = max_bits;
    work_sum(wk, G)[blockIdx.x] = partial;
    if (bad) atomicOr(&wk->status, AR_STATUS_BAD_ALPHA);
    __threadfence();
    const uint32_t ticket = atomicAdd(&wk->counter, 1u);
    s_last = ticket == (uint32_t)(G - 1);
  }
  __syncthreads();
  if (s_last) combine_partials(wk, G, f64, out, status);
}

__global__ void __launch_bounds__(kNT) k_bound_f32(const float* __restrict__ a, int64_t M,
                                                   double* out, uint32_t* status,
                                                   BoundWork* wk) {
  __shared__ int32_t s_smax[kNT / 32];
  __shared__ uint32_t s_umax[kNT / 32];
  __shared__ unsigned long long s_a1[kNT / 32], s_a2[kNT / 32];
  __shared__ float s_a3[kNT / 32];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t base = (int64_t)blockIdx.x * (kNT * kEptF32);
  uint32_t v[kEptF32];
  MaxF32 mx;
#pragma unroll
  for (int k = 0; k < kEptF32; ++k) {
    const int64_t i = base + (int64_t)k * kNT + threadIdx.x;
    v[k] = i < M ? __float_as_uint(__ldg(a + i)) : 0u;
    mx.add(v[k]);
  }
  mx.smax = warp_max_i32(mx.smax);
  mx.umax = warp_max_u32(mx.umax);
  if (lane == 0) {
    s_smax[warp] = mx.smax;
    s_umax[warp] = mx.umax;
  }
  __syncthreads();
  if (threadIdx.x < 32) {
    int32_t sm = threadIdx.x < kNT / 32 ? s_smax[threadIdx.x] : INT32_MIN;
    uint32_t um = threadIdx.x < kNT / 32 ? s_umax[threadIdx.x] : 0u;
    sm = warp_max_i32(sm);
    um = warp_max_u32(um);
    if (threadIdx.x == 0) {
      s_smax[0] = sm;
      s_umax[0] = um;
    }
  }
  __syncthreads();
  mx.smax = s_smax[0];
  mx.umax = s_umax[0];
  const uint32_t max_bits = mx.value_bits();
  const int e_ref = fx_eref(max_bits);
  FxSum fx;
#pragma unroll
  for (int k = 0; k < kEptF32; ++k) fx.add(v[k], e_ref);
  fx.warp_reduce();
  if (lane == 0) {
    s_a1[warp] = fx.a1;
    s_a2[warp] = fx.a2;
    s_a3[warp] = fx.a3;
  }
  __syncthreads();
  double partial = 0.0;
  if (threadIdx.x < 32) {
    FxSum f;
    if (threadIdx.x < kNT / 32) {
      f.a1 = s_a1[threadIdx.x];
      f.a2 = s_a2[threadIdx.x];
      f.a3 = s_a3[threadIdx.x];
    }
    f.warp_reduce();
    partial = f.to_double(e_ref);
  }
  finish_cta(max_bits, mx.bad(), partial, false, out, status, wk);
}

__global__ void __launch_bounds__(kNT) k_bound_f64(const double* __restrict__ a, int64_t M,
                                                   double* out, uint32_t* status,
                                                   BoundWork* wk) {
  __shared__ long long s_smax[kNT / 32];
  __shared__ unsigned long long s_umax[kNT / 32];
  __shared__ double s_sum[kNT / 32];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t base = (int64_t)blockIdx.x * (kNT * kEptF64);
  MaxF64 mx;
  double sum = 0.0;
#pragma unroll
  for (int k = 0; k < kEptF64; ++k) {
    const int64_t i = base + (int64_t)k * kNT + threadIdx.x;
    const double x = i < M ? __ldg(a + i) : 0.0;
    mx.add((unsigned long long)__double_as_longlong(x));
    sum = __dadd_rn(sum, x);
  }
  mx.smax = warp_max_i64(mx.smax);
  mx.umax = warp_max_u64(mx.umax);
  sum = warp_sum_f64(sum);
  if (lane == 0) {
    s_smax[warp] = mx.smax;
    s_umax[warp] = mx.umax;
    s_sum[warp] = sum;
  }
  __syncthreads();
  double partial = 0.0;
  if (threadIdx.x < 32) {
    long long sm = threadIdx.x < kNT / 32 ? s_smax[threadIdx.x] : INT64_MIN;
    unsigned long long um = threadIdx.x < kNT / 32 ? s_umax[threadIdx.x] : 0ull;
    double s = threadIdx.x < kNT / 32 ? s_sum[threadIdx.x] : 0.0;
    sm = warp_max_i64(sm);
    um = warp_max_u64(um);
    s = warp_sum_f64(s);
    mx.smax = sm;
    mx.umax = um;
    partial = s;
  }
  // thread 0 holds the CTA result
  finish_cta(mx.value_bits(), mx.bad(), partial, true, out, status, wk);
}

inline int64_t chunk_of(int dtype) { return dtype == AR_F64 ? kNT * kEptF64 : kNT * kEptF32; }

}  // namespace
}  // namespace gbar

using namespace gbar;

extern "C" size_t ar_bound_workspace_size(int64_t M, int dtype) {
  if (M <= 0 || !valid_dtype(dtype)) return 0;
  const int64_t G = (M + chunk_of(dtype) - 1) / chunk_of(dtype);
  return G <= 1 ? 0 : sizeof(BoundWork) + (size_t)G * 16;
}

extern "C" int ar_bound(const void* d_alpha, int dtype, int64_t M, double* d_bound_sum,
                        uint32_t* d_status, void* d_work, size_t work_bytes, void* stream) {
  if (M < 0 || !valid_dtype(dtype) || !d_bound_sum || !d_status || (M > 0 && !d_alpha))
    return AR_ERR_ARG;
  if (!aligned(d_alpha, dtype_size(dtype)) || !aligned(d_bound_sum, 8) || !aligned(d_status, 4))
    return AR_ERR_ALIGN;
  const int64_t G64 = M == 0 ? 1 : (M + chunk_of(dtype) - 1) / chunk_of(dtype);
  if (G64 > (1ll << 30)) return AR_ERR_UNSUPPORTED;
  const int G = (int)G64;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  BoundWork* wk = nullptr;
  if (G > 1) {
    if (!d_work) return AR_ERR_WORKSPACE;
    if (work_bytes < ar_bound_workspace_size(M, dtype)) return AR_ERR_WORKSPACE;
    if (!aligned(d_work, 16)) return AR_ERR_ALIGN;
    wk = static_cast<BoundWork*>(d_work);
  }
  if (dtype == AR_F32)
    k_bound_f32<<<G, kNT, 0, s>>>(static_cast<const float*>(d_alpha), M, d_bound_sum, d_status, wk);
  else
    k_bound_f64<<<G, kNT, 0, s>>>(static_cast<const double*>(d_alpha), M, d_bound_sum, d_status, wk);
  return check_launch();
}

// ---------------------------------------------------------------------------
// ar_bound_noalloc: the same reduction for callers that cannot allocate
// device memory.  Its multi-CTA scratch (the arrival counter, a status word
// and one (max, sum) partial per CTA) lives in a file-scope device array
// instead of a caller-provided workspace.  Every GPU that loads this library
// holds one copy of the array until the process exits.
// ---------------------------------------------------------------------------
namespace gbar {
namespace {
constexpr int kNoAllocMaxCtas = 4096;
constexpr size_t kNoAllocScratchBytes = sizeof(BoundWork) + (size_t)kNoAllocMaxCtas * 16;
static_assert((int64_t)kNoAllocMaxCtas * kNT * kEptF32 == AR_BOUND_NOALLOC_MAX_M_F32, "limit");
static_assert((int64_t)kNoAllocMaxCtas * kNT * kEptF64 == AR_BOUND_NOALLOC_MAX_M_F64, "limit");
}  // namespace
}  // namespace gbar

static __device__ __align__(256) unsigned char g_bound_noalloc_scratch[gbar::kNoAllocScratchBytes];

extern "C" int ar_bound_noalloc(const void* d_alpha, int dtype, int64_t M, double* d_bound_sum,
                                uint32_t* d_status, void* stream) {
  // Every check that can reject the call comes before anything is enqueued.
  if (M < 0 || !valid_dtype(dtype) || !d_bound_sum || !d_status || (M > 0 && !d_alpha))
    return AR_ERR_ARG;
  const int64_t limit = dtype == AR_F64 ? AR_BOUND_NOALLOC_MAX_M_F64 : AR_BOUND_NOALLOC_MAX_M_F32;
  if (M > limit) return AR_ERR_UNSUPPORTED;
  if (!aligned(d_alpha, dtype_size(dtype)) || !aligned(d_bound_sum, 8) || !aligned(d_status, 4))
    return AR_ERR_ALIGN;
  // The host-side name of the array is only a stand-in for it: ask the
  // runtime for its device address in the current device's context.  This
  // is done on every call (it allocates nothing), so the address is never
  // stale after a device reset or under another context.  The first call
  // on a device may load the library's device code: make it before any
  // stream capture.
  void* scratch = nullptr;
  cudaError_t e = cudaGetSymbolAddress(&scratch, g_bound_noalloc_scratch);
  if (e != cudaSuccess) {
    set_cuda_error(e);
    return AR_ERR_CUDA;
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (M > chunk_of(dtype)) {
    // The array keeps what the previous call left in it.  A complete
    // multi-CTA call returns the counter and status word to zero itself, but
    // clearing them here makes this call independent of how the previous one
    // ended (for instance one that overlapped another call, which races).
    e = cudaMemsetAsync(scratch, 0, sizeof(BoundWork), s);
    if (e != cudaSuccess) {
      set_cuda_error(e);
      return AR_ERR_CUDA;
    }
  }
  return ar_bound(d_alpha, dtype, M, d_bound_sum, d_status, scratch, kNoAllocScratchBytes, stream);
}
