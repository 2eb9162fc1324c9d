// The two comparators of the paper's method, on the GPU:
//
//   ar_select_paper  the paper's own GPU rule (Sections "Election step" and
//       "Selection step"; the Results' pseudo-code): every reaction j draws
//       u_j in [0, T), is eligible when u_j < D_j (D_j != 0) with rate
//       R_j = u_j / D_j, and the selection is argmin R (lowest j on ties), or
//       the rejection sentinel M when no rate is below 1.  FP32 throughout,
//       as the paper's arrays are float.  The paper runs one block of M
//       threads per selection; here a warp takes a selection at a time, each
//       lane two reactions per Philox block, and the argmin is two warp
//       min-reductions (rate, then index).
//   ar_select_it  the direct method's inverse transform (Section "The
//       Stochastic Simulation Algorithm"): j is the smallest index whose
//       running sum exceeds u alpha_0.  The running sums are the sequential
//       FP64 sums in index order, computed once per call by one thread (the
//       dependence the paper argues against), then every selection is a
//       binary search.
#include <algorithm>

#include "device.cuh"
#include "host.hpp"

namespace gbar {
namespace {

constexpr int kPW = 8;  // warps per CTA (paper rule)
constexpr int kPNT = kPW * 32;

struct PaperParams {
  const float* D;
  uint32_t M;
  const double* bound;
  uint32_t K;
  uint32_t sel_base, b;
  uint32_t k0, k1;
  int32_t* idx;
  unsigned long long* rejections;
};

// order-preserving key of an FP32 value (-0 taken as +0)
__device__ __forceinline__ uint32_t fkey(float x) {
  const uint32_t u = __float_as_uint(__fadd_rn(x, 0.0f));
  return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}

template <bool SMEM>
__global__ void __launch_bounds__(kPNT) k_paper(const PaperParams p) {
  extern __shared__ float s_D[];
  const uint32_t lane = threadIdx.x & 31u;
  const float* D = p.D;
  if constexpr (SMEM) {
    for (uint32_t j = threadIdx.x; j < p.M; j += kPNT) s_D[j] = p.D[j];
    __syncthreads();
    D = s_D;
  }
  const float T = __double2float_rn(*p.bound);
  const uint32_t npairs = (p.M + 1u) >> 1;
  const uint32_t one_key = fkey(1.0f);
  unsigned long long rej = 0;
  for (uint32_t s = blockIdx.x * kPW + (threadIdx.x >> 5); s < p.K; s += gridDim.x * kPW) {
    uint32_t best = 0xffffffffu, arg = 0xffffffffu;  // (key of R, j)
    for (uint32_t c = lane; c < npairs; c += 32) {
      const uint4 w = philox10(make_uint4(c, p.sel_base + s, p.b, 3u), p.k0, p.k1);
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const uint32_t j = 2u * c + (uint32_t)h;
        if (j >= p.M) break;
        const uint32_t wb = h ? w.w : w.y;
        const float uT = __fmul_rn(__fmul_rn(__uint2float_rn(wb >> 8), 0x1p-24f), T);
        const float d = D[j];
        float R = __int_as_float(0x7f800000);  // ineligible: +inf
        if (uT < d && d != 0.0f) R = __fdiv_rn(uT, d);
        const uint32_t k = fkey(R);
        if (k < best) {  // j ascends within a lane: the first minimum is kept
          best = k;
          arg = j;
        }
      }
    }
    const uint32_t kmin = __reduce_min_sync(kFull, best);
    const uint32_t jmin = __reduce_min_sync(kFull, best == kmin ? arg : 0xffffffffu);
    if (lane == 0) {
      const bool ok = p.M > 0 && kmin < one_key;  // min R < 1
      p.idx[s] = ok ? (int32_t)jmin : (int32_t)p.M;
      if (!ok) ++rej;
    }
  }
  if (lane == 0 && rej && p.rejections) atomicAdd(p.rejections, rej);
}

// ---- inverse transform ------------------------------------------------------
struct ItHeader {
  double a0;
  int64_t last_nz;
  uint32_t status;
  uint32_t pad[3];
};

template <typename TS>
__global__ void k_it_scan(const TS* __restrict__ a, int64_t M, ItHeader* hdr, double* c,
                          uint32_t* d_status) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  double run = 0.0, mx = 0.0;
  int64_t last = -1;
  uint32_t st = 0;
  for (int64_t j = 0; j < M; ++j) {
    const double x = (double)a[j];
    if (!(x >= 0.0) || isinf(x)) st |= AR_STATUS_BAD_ALPHA;
    if (x > mx) mx = x;
    if (x > 0.0) last = j;
    run = __dadd_rn(run, x);
    c[j] = run;
  }
  if (!(st & AR_STATUS_BAD_ALPHA) && mx == 0.0) st |= AR_STATUS_ALL_ZERO;
  hdr->a0 = run;
  hdr->last_nz = last;
  hdr->status = st;
  if (st) atomicOr(d_status, st);
}

struct ItParams {
  const ItHeader* hdr;
  const double* c;
  int64_t M;
  uint32_t K;
  uint32_t sel_base, b;
  uint32_t k0, k1;
  int32_t* idx;
};

__global__ void __launch_bounds__(256) k_it_select(const ItParams p) {
  const double a0 = p.hdr->a0;
  const int64_t last = p.hdr->last_nz;
  const bool monotone = !(p.hdr->status & AR_STATUS_BAD_ALPHA);
  for (uint32_t s = blockIdx.x * blockDim.x + threadIdx.x; s < p.K; s += gridDim.x * blockDim.x) {
    if (!(a0 > 0.0)) {
      p.idx[s] = (int32_t)p.M;
      continue;
    }
    const uint4 w = philox10(make_uint4(0u, p.sel_base + s, p.b, 2u), p.k0, p.k1);
    const unsigned long long m = ((unsigned long long)w.x << 21) | (unsigned long long)(w.y >> 11);
    const double target = __dmul_rn(__ull2double_rn(m) * 0x1p-53, a0);
    int64_t pick = last;
    if (monotone) {
      // running sums are non-decreasing: first c_j > target by bisection
      int64_t lo = 0, hi = p.M;
      while (lo < hi) {
        const int64_t mid = lo + ((hi - lo) >> 1);
        if (__ldg(p.c + mid) > target) hi = mid;
        else lo = mid + 1;
      }
      if (lo < p.M) pick = lo;
    } else {
      for (int64_t j = 0; j < p.M; ++j)
        if (__ldg(p.c + j) > target) {
          pick = j;
          break;
        }
    }
    p.idx[s] = (int32_t)pick;
  }
}

}  // namespace
}  // namespace gbar

using namespace gbar;

extern "C" int ar_select_paper(const float* d_D, int64_t M, const double* d_bound, int64_t K,
                               uint64_t seed, uint64_t sel_offset, uint32_t realization,
                               int32_t* d_idx, unsigned long long* d_rejections, void* stream) {
  if (M < 0 || M >= (1ll << 31) || K < 0 || sel_offset + (uint64_t)K > (1ull << 32))
    return AR_ERR_ARG;
  if (K == 0) return AR_OK;
  if ((M > 0 && !d_D) || !d_bound || !d_idx) return AR_ERR_ARG;
  if (!aligned(d_D, 4) || !aligned(d_bound, 8) || !aligned(d_idx, 4) || !aligned(d_rejections, 8))
    return AR_ERR_ALIGN;
  const DeviceInfo& dev = device_info();
  PaperParams p{};
  p.D = d_D;
  p.M = (uint32_t)M;
  p.bound = d_bound;
  p.K = (uint32_t)K;
  p.sel_base = (uint32_t)sel_offset;
  p.b = realization;
  p.k0 = (uint32_t)(seed & 0xffffffffu);
  p.k1 = (uint32_t)(seed >> 32);
  p.idx = d_idx;
  p.rejections = d_rejections;
  const uint32_t sms = (uint32_t)std::max(1, dev.sm_count);
  const uint32_t need = (uint32_t)((K + kPW - 1) / kPW);
  const size_t smem = (size_t)M * sizeof(float);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (smem <= 48 * 1024) {
    const uint32_t grid = std::max(1u, std::min(need, sms * 8u));
    k_paper<true><<<grid, kPNT, smem, s>>>(p);
  } else {
    const uint32_t grid = std::max(1u, std::min(need, sms * 8u));
    k_paper<false><<<grid, kPNT, 0, s>>>(p);
  }
  return check_launch();
}

extern "C" size_t ar_select_it_workspace_size(int64_t M) {
  if (M < 0) return 0;
  return sizeof(ItHeader) + sizeof(double) * (size_t)std::max<int64_t>(M, 1);
}

extern "C" int ar_select_it(const void* d_alpha, int dtype, int64_t M, int64_t K, uint64_t seed,
                            uint64_t sel_offset, uint32_t realization, int32_t* d_idx,
                            uint32_t* d_status, void* d_work, size_t work_bytes, void* stream) {
  if (!valid_dtype(dtype) || M < 0 || M >= (1ll << 31) || K < 0 ||
      sel_offset + (uint64_t)K > (1ull << 32))
    return AR_ERR_ARG;
  if ((M > 0 && !d_alpha) || !d_status || (K > 0 && !d_idx)) return AR_ERR_ARG;
  if (!d_work || work_bytes < ar_select_it_workspace_size(M)) return AR_ERR_WORKSPACE;
  if (!aligned(d_alpha, dtype_size(dtype)) || !aligned(d_idx, 4) || !aligned(d_status, 4) ||
      !aligned(d_work, 16))
    return AR_ERR_ALIGN;
  auto* hdr = static_cast<ItHeader*>(d_work);
  double* c = reinterpret_cast<double*>(static_cast<unsigned char*>(d_work) + sizeof(ItHeader));
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (dtype == AR_F32)
    k_it_scan<float><<<1, 32, 0, s>>>(static_cast<const float*>(d_alpha), M, hdr, c, d_status);
  else
    k_it_scan<double><<<1, 32, 0, s>>>(static_cast<const double*>(d_alpha), M, hdr, c, d_status);
  int rc = check_launch();
  if (rc || K == 0) return rc;
  ItParams p{};
  p.hdr = hdr;
  p.c = c;
  p.M = M;
  p.K = (uint32_t)K;
  p.sel_base = (uint32_t)sel_offset;
  p.b = realization;
  p.k0 = (uint32_t)(seed & 0xffffffffu);
  p.k1 = (uint32_t)(seed >> 32);
  p.idx = d_idx;
  const DeviceInfo& dev = device_info();
  const uint32_t grid =
      std::max(1u, std::min((uint32_t)((K + 255) / 256), (uint32_t)std::max(1, dev.sm_count) * 8u));
  k_it_select<<<grid, 256, 0, s>>>(p);
  return check_launch();
}
