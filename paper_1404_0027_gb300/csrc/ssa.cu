// ssa_step_batched: many realizations of the Stochastic Simulation Algorithm
// (direct method, Section "The Stochastic Simulation Algorithm") advanced
// step by step on the GPU, the next reaction of every step chosen by the AR
// trial (Section "A GPU acceptance-rejection algorithm") with T = max_j a_j.
//
// One warp owns one realization for the whole call.  Its propensities live in
// the caller's FP64 array a[M] (global, L1-resident) with an FP32 copy in
// shared memory for the trial gathers; its counts X move to shared memory for
// the call when the network is small enough.  After reaction j fires, only the
// reactions that depend on a species j changes are recomputed (the
// dependency graph of Gibson & Bruck, cited in the Introduction), each as one
// FP64 rounding of c_r times the exact integer count h_r(X).  The bound is the
// exact maximum of the FP32 copies (a per-lane maximum over a strided subset:
// raised elements update it through a shared-memory maximum, and the subset
// is rescanned only when the element holding its maximum is lowered).  The total propensity a_0 is kept
// as an exact 128-bit fixed-point integer (no drift over long runs), and the
// waiting times tau = ln(1/u)/a_0 of 32 consecutive steps are computed
// together, one step per lane, because GB300 runs FP64 at a small fraction of
// its integer rate.
#include <algorithm>
#include <cmath>
#include <mutex>
#include <vector>

#include "device.cuh"
#include "host.hpp"

// ---------------------------------------------------------------------------
// Network handle (host-built, device-resident)
// ---------------------------------------------------------------------------
struct ssa_net {
  int device;
  int32_t N, M;
  int8_t* d_rtype;    // [M]
  int2* d_reac;       // [M] reactant species (A, B), -1 where unused
  double* d_rate;     // [M]
  int32_t* d_nu_ptr;  // [M+1]
  int2* d_nu;         // [nnz] (species, delta)
  int32_t* d_dep_ptr; // [M+1]
  int32_t* d_dep;     // reactions whose propensity depends on species j changes
  int32_t max_nu, max_dep;
};

namespace gbar {
namespace {

constexpr int kWarpsS = 8;
constexpr int kNTS = kWarpsS * 32;

struct SsaParams {
  const int8_t* rtype;
  const int2* reac;
  const double* rate;
  const int32_t* nu_ptr;
  const int2* nu;
  const int32_t* dep_ptr;
  const int32_t* dep;
  int32_t N, M;
  uint32_t B;
  int32_t* X;          // [B][N]
  double* a;           // [B][M] FP64 propensities (state)
  double* t;           // [B]
  unsigned long long* step;  // [B]
  int32_t* last;       // [B] nullable
  uint32_t* status;    // [B]
  unsigned long long* trials;  // [B] nullable
  long long nsteps;
  unsigned long long cap;
  uint32_t b_base;
  uint32_t k0, k1;
  uint32_t smem_stride;  // bytes of shared memory per warp
  uint32_t x_off;        // offset of the counts in a warp's shared memory (XS)
  uint32_t inc_off;      // offset of the per-lane raised maxima
  // run to a time limit, with trajectory samples (ssa_run_until)
  double t_end;
  const double* samp_t;   // [nsamp] ascending sample times
  int32_t nsamp;
  const int32_t* samp_sp; // [nspec] species recorded (NULL: 0 .. nspec-1)
  int32_t nspec;
  int32_t* traj;          // [B][nsamp][nspec]
};

// Mass-action propensity: one FP64 rounding of c times the exact count h.
__device__ __forceinline__ double propensity(const SsaParams& p, int r, const int32_t* X) {
  // every lane evaluates the same selects (no divergence over reaction types)
  const int type = __ldg(p.rtype + r);
  const int2 ab = __ldg(p.reac + r);
  const long long xa = type != 0 ? (long long)X[ab.x] : 0ll;
  const long long xb = type == 2 ? (long long)X[ab.y] : 0ll;
  long long h = 1;                                                    // 0: source
  h = type == 1 ? (xa > 0 ? xa : 0ll) : h;                            // 1: A
  h = type == 2 ? ((xa > 0 && xb > 0) ? xa * xb : 0ll) : h;           // 2: A + B
  h = type == 3 ? (xa >= 2 ? (xa * (xa - 1)) >> 1 : 0ll) : h;         // 3: 2A
  return __dmul_rn(__ldg(p.rate + r), __ll2double_rn(h));
}

// 128-bit two's-complement integers for the exact fixed-point a_0.
struct I128 {
  unsigned long long lo, hi;
};
__device__ __forceinline__ I128 add128(I128 x, I128 y) {
  I128 r;
  r.lo = x.lo + y.lo;
  r.hi = x.hi + y.hi + (r.lo < x.lo ? 1ull : 0ull);
  return r;
}
__device__ __forceinline__ I128 neg128(I128 x) {
  I128 r;
  r.lo = ~x.lo + 1ull;
  r.hi = ~x.hi + (r.lo == 0ull ? 1ull : 0ull);
  return r;
}
__device__ __forceinline__ I128 shfl_xor128(I128 x, int o) {
  x.lo = __shfl_xor_sync(kFull, x.lo, o);
  x.hi = __shfl_xor_sync(kFull, x.hi, o);
  return x;
}
__device__ __forceinline__ I128 warp_sum128(I128 x) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) x = add128(x, shfl_xor128(x, o));
  return x;
}

// floor(a * 2^S) for a finite double a >= 0, as a 128-bit integer.  Values
// whose scaled size would pass 2^120 set *ovf.
__device__ __forceinline__ I128 fix128(double a, int S, bool* ovf) {
  I128 r{0ull, 0ull};
  const unsigned long long bits = (unsigned long long)__double_as_longlong(a);
  const int e = (int)((bits >> 52) & 0x7ff);
  if (e == 0) return r;  // zero (subnormal propensities do not occur: c * h with h >= 1)
  const unsigned long long m = (bits & 0xfffffffffffffull) | 0x10000000000000ull;
  // a = m * 2^(e - 1075); scaled: m * 2^(e - 1075 + S)
  const int sh = e - 1075 + S;
  if (sh >= 0) {
    if (sh > 120 - 53) {
      *ovf = true;
      return r;
    }
    if (sh >= 64) {
      r.hi = m << (sh - 64);
    } else {
      r.lo = m << sh;
      r.hi = sh == 0 ? 0ull : (m >> (64 - sh));
    }
  } else if (sh > -64) {
    r.lo = m >> (-sh);
  }
  return r;
}

// 128-bit integer times 2^-S, rounded to double.
__device__ __forceinline__ double unfix128(I128 x, int S) {
  const double hi = __dmul_rn(__ull2double_rn(x.hi), 0x1p64);
  const double v = __dadd_rn(hi, __ull2double_rn(x.lo));
  return ldexp(v, -S);
}

// The FP64 comparison of trial word w against alpha_j: the FP32 pre-filter on
// the operand kept in shared memory, and for the rare trials it leaves open
// the FP64 test on the state array's value (written by this warp in an
// earlier step, ordered by the warp's __syncwarp).
__device__ __forceinline__ bool accept_f64_state(uint32_t w, const F64Bound& T, float op,
                                                 const double* a, int32_t j) {
  const int d = f64_filter(w, T, op);
  return d == 2 ? accept_f64_slow(w, T.T, a[j]) : d == 1;
}

// XS: the counts live in shared memory during the call (read from and
// written back to X), when the network is small enough.
template <int CMP, bool TIMED, bool XS>
__device__ __forceinline__ void ssa_warp(const SsaParams& p) {
  extern __shared__ __align__(16) unsigned char smem[];
  const uint32_t lane = threadIdx.x & 31u;
  const uint32_t warp = threadIdx.x >> 5;
  const uint32_t b = blockIdx.x * kWarpsS + warp;
  if (b >= p.B) return;
  // FP32 (or FP64) copies of the propensities for gathers and the bound,
  // then the counts (XS) and the lanes' raised maxima
  unsigned char* wsm = smem + (size_t)warp * p.smem_stride;
  // FP32 comparison: RN32 copies of the propensities; FP64 comparison: the
  // FP32 pre-filter's operands (the FP64 values are the state array a)
  float* af = reinterpret_cast<float*>(wsm);
  unsigned long long* inc = reinterpret_cast<unsigned long long*>(wsm + p.inc_off);
  uint32_t st = p.status[b];
  if (st & (AR_STATUS_ABSORBED | AR_STATUS_TRIAL_CAP | AR_STATUS_BAD_ALPHA | AR_STATUS_UNSUPPORTED))
    return;
  const int M = p.M;
  int32_t* Xg = p.X + (size_t)b * p.N;
  int32_t* X = Xg;
  if constexpr (XS) {
    X = reinterpret_cast<int32_t*>(wsm + p.x_off);
    for (int q = (int)lane; q < p.N; q += 32) X[q] = Xg[q];
    __syncwarp();
  }
  double* a = p.a + (size_t)b * M;
  const uint32_t bid = p.b_base + b;
  unsigned long long step = p.step[b];
  double t = p.t[b];
  int32_t last = p.last ? p.last[b] : -1;
  unsigned long long ntr = 0;

  // ---- propensities from X, and the scale of the fixed-point a_0
  uint32_t lmax = 0;  // per-lane max of the comparison copies (bit patterns)
  unsigned long long lmax64 = 0;
  for (int r = lane; r < M; r += 32) {
    const double v = propensity(p, r, X);
    a[r] = v;
    if constexpr (CMP == AR_CMP_F32) {
      const float f = __double2float_rn(v);
      af[r] = f;
      lmax = max(lmax, __float_as_uint(f));
    } else {
      af[r] = f64_filter_operand(v);
      lmax64 = max(lmax64, (unsigned long long)__double_as_longlong(v));
    }
  }
  unsigned long long amax_bits = warp_max_u64((unsigned long long)__double_as_longlong(
      CMP == AR_CMP_F32 ? (double)__uint_as_float(warp_max_u32(lmax))
                        : __longlong_as_double((long long)warp_max_u64(lmax64))));
  // S: a_0 < M * max * 2^S must leave 2^40 of growth room below 2^120
  const int e_max = (int)((amax_bits >> 52) & 0x7ff) - 1023;
  const int lgM = 32 - __clz((uint32_t)M);
  const int S = 120 - 40 - lgM - (e_max + 1);
  bool ovf = false;
  I128 a0x{0ull, 0ull};
  for (int r = lane; r < M; r += 32) a0x = add128(a0x, fix128(a[r], S, &ovf));
  a0x = warp_sum128(a0x);
  __syncwarp();

  // waiting-time block: lane i holds the exponential variate of step base+i
  // and, once that step has run, its fixed-point a_0
  double E = 0.0;
  I128 a0_lane{0ull, 0ull};
  int blk_fill = 32;  // force a refill before the first step
  // trajectory samples: the state at sample time t_k is the state after the
  // last reaction at a time <= t_k
  int ks = 0;
  if constexpr (TIMED)
    while (ks < p.nsamp && p.samp_t[ks] < t) ++ks;
  auto record_until = [&](double lim, bool inclusive) {
    for (; ks < p.nsamp && (inclusive ? p.samp_t[ks] <= lim : p.samp_t[ks] < lim); ++ks) {
      int32_t* dst = p.traj + ((size_t)b * (size_t)p.nsamp + (size_t)ks) * (size_t)p.nspec;
      for (int q = (int)lane; q < p.nspec; q += 32) dst[q] = X[p.samp_sp ? p.samp_sp[q] : q];
    }
  };

  auto flush_block = [&](int used) {
    // tau_i = E_i / a0_i for the used steps (lane-parallel FP64), added to t
    // in step order
    double tau = 0.0;
    if (lane < (uint32_t)used) tau = __ddiv_rn(E, unfix128(a0_lane, S));
#pragma unroll
    for (int k = 0; k < 32; ++k) {
      const double v = __shfl_sync(kFull, tau, k);
      if (k < used) t = __dadd_rn(t, v);
    }
  };

  for (long long n = 0; n < p.nsteps; ++n) {
    if (blk_fill == 32) {
      if (n > 0 && !TIMED) flush_block(32);
      // exponential variates of the next 32 steps: -ln(1 - u53), u53 from
      // counter (0, step, b, 1), words 0 and 1
      const uint4 w = philox10(make_uint4(0u, (uint32_t)(step + lane), bid, 1u), p.k0, p.k1);
      const unsigned long long m53 = ((unsigned long long)w.x << 21) | (w.y >> 11);
      const double u = __dmul_rn(__ull2double_rn(m53), 0x1p-53);
      E = -log(__dsub_rn(1.0, u));
      blk_fill = 0;
    }
    // ---- bound T = max a (exact, from the comparison copies)
    float Tf = 0.f;
    F64Bound T{};  // the FP64 comparison's bound with its FP32 pre-filter
    bool zero;
    if constexpr (CMP == AR_CMP_F32) {
      const uint32_t tb = warp_max_u32(lmax);
      Tf = __uint_as_float(tb);
      zero = tb == 0u;  // the maximum of non-negative copies, on bit patterns
    } else {
      const unsigned long long tb = warp_max_u64(lmax64);
      T = f64_bound(__longlong_as_double((long long)tb));
      zero = tb == 0ull;
    }
    if (zero) {
      st |= AR_STATUS_ABSORBED;
      if (TIMED) record_until(p.t_end, true);  // the state holds to t_end
      break;
    }
    double t_next = 0.0;
    if (TIMED) {
      // this step's waiting time first: a reaction after t_end does not fire
      const double tau = __ddiv_rn(__shfl_sync(kFull, E, blk_fill), unfix128(a0x, S));
      t_next = __dadd_rn(t, tau);
      if (t_next > p.t_end) {  // t stays at the last reaction: a resumed run is exact
        record_until(p.t_end, true);
        st |= AR_STATUS_T_END;
        break;
      }
      record_until(t_next, false);
    }
    // ---- AR selection: the whole warp tests trials 64 at a time
    const uint32_t M32 = (uint32_t)M;
    int32_t j = -1;
    unsigned long long c0 = 0;
    for (;;) {
      const unsigned long long cnt = c0 + lane;  // Philox block of trials 2cnt, 2cnt+1
      const uint4 w = philox10(make_uint4((uint32_t)cnt, (uint32_t)step, bid, 0u), p.k0, p.k1);
      const uint32_t j0 = candidate(w.x, M32), j1 = candidate(w.z, M32);
      bool a0, a1;
      if constexpr (CMP == AR_CMP_F32) {
        a0 = 2 * cnt < p.cap && accept_f32(w.y, Tf, af[j0]);
        a1 = !a0 && 2 * cnt + 1 < p.cap && accept_f32(w.w, Tf, af[j1]);
      } else {
        a0 = 2 * cnt < p.cap && accept_f64_state(w.y, T, af[j0], a, j0);
        a1 = !a0 && 2 * cnt + 1 < p.cap && accept_f64_state(w.w, T, af[j1], a, j1);
      }
      const uint32_t bal = __ballot_sync(kFull, a0 || a1);
      if (bal) {
        const uint32_t src = (uint32_t)__ffs(bal) - 1u;
        const uint32_t code = a0 ? (j0 << 1) : ((j1 << 1) | 1u);
        const uint32_t got = __shfl_sync(kFull, code, src);
        j = (int32_t)(got >> 1);
        ntr += 2 * (c0 + src) + (got & 1u) + 1;
        break;
      }
      c0 += 32;
      if (2 * c0 >= p.cap) {
        ntr += p.cap;
        break;
      }
    }
    if (j < 0) {
      st |= AR_STATUS_TRIAL_CAP;
      break;
    }
    // ---- a_0 of this step goes with its waiting time
    if (lane == (uint32_t)blk_fill) a0_lane = a0x;
    ++blk_fill;
    // ---- fire j: X += nu_j
    {
      const int q0 = __ldg(p.nu_ptr + j), q1 = __ldg(p.nu_ptr + j + 1);
      for (int q = q0 + lane; q < q1; q += 32) {
        const int2 e = __ldg(p.nu + q);
        atomicAdd(X + e.x, e.y);
      }
    }
    __syncwarp();
    // ---- recompute the dependent propensities
    {
      const int d0 = __ldg(p.dep_ptr + j), d1 = __ldg(p.dep_ptr + j + 1);
      I128 dq{0ull, 0ull};
      uint32_t rescan = 0;  // lanes whose strided maximum may have dropped
      inc[lane] = 0ull;  // the largest raised element of each lane's subset
      __syncwarp();
      for (int base = d0; base < d1; base += 32) {
        const int qi = base + (int)lane;
        const bool act = qi < d1;
        const int r = act ? __ldg(p.dep + qi) : 0;
        // the owner's maximum before this step's updates: a decrease changes
        // it only when the element held it
        const uint32_t owner = act ? ((uint32_t)r & 31u) : lane;
        const uint32_t om = __shfl_sync(kFull, lmax, owner);
        const unsigned long long om64 = __shfl_sync(kFull, lmax64, owner);
        if (act) {
          const double vn = propensity(p, r, X);
          const double vo = a[r];
          a[r] = vn;
          dq = add128(dq, add128(fix128(vn, S, &ovf), neg128(fix128(vo, S, &ovf))));
          if constexpr (CMP == AR_CMP_F32) {
            const float fo = af[r], fn = __double2float_rn(vn);
            af[r] = fn;
            if (fn < fo && __float_as_uint(fo) == om) rescan |= 1u << owner;
            if (fn > fo) atomicMax(inc + owner, (unsigned long long)__float_as_uint(fn));
          } else {
            // non-negative doubles order as their bit patterns
            const unsigned long long bo = (unsigned long long)__double_as_longlong(vo);
            const unsigned long long bn = (unsigned long long)__double_as_longlong(vn);
            af[r] = f64_filter_operand(vn);
            if (bn < bo && bo == om64) rescan |= 1u << owner;
            if (bn > bo) atomicMax(inc + owner, bn);
          }
        }
      }
      a0x = add128(a0x, warp_sum128(dq));
      __syncwarp();
      // lane maxima: rescan the strided subsets whose maximum dropped, and
      // take the maximum with the raised elements otherwise
      rescan = __reduce_or_sync(kFull, rescan);
      if (CMP == AR_CMP_F32) {
        if (rescan & (1u << lane)) {
          lmax = 0;
          for (int r = lane; r < M; r += 32) lmax = max(lmax, __float_as_uint(af[r]));
        } else {
          lmax = max(lmax, (uint32_t)inc[lane]);
        }
      } else {
        if (rescan & (1u << lane)) {
          lmax64 = 0;
          for (int r = lane; r < M; r += 32)
            lmax64 = max(lmax64, (unsigned long long)__double_as_longlong(a[r]));
        } else {
          lmax64 = max(lmax64, inc[lane]);
        }
      }
      __syncwarp();
    }
    ++step;
    last = j;
    if (TIMED) t = t_next;
  }
  // waiting times of the steps of the last, partial block
  if (!TIMED && blk_fill > 0 && blk_fill <= 32) flush_block(blk_fill);
  if (ovf) st |= AR_STATUS_UNSUPPORTED;
  if constexpr (XS) {
    __syncwarp();
    for (int q = (int)lane; q < p.N; q += 32) Xg[q] = X[q];
  }
  if (lane == 0) {
    p.t[b] = t;
    p.step[b] = step;
    p.status[b] = st;
    if (p.last) p.last[b] = last;
    if (p.trials) p.trials[b] += ntr;
  }
}

// One warp per realization, FP32 comparison.
template <bool TIMED, bool XS>
__global__ void __launch_bounds__(kNTS) k_ssa(const SsaParams p) {
  ssa_warp<AR_CMP_F32, TIMED, XS>(p);
}
// FP64 comparison: held to the FP32 step's four CTAs per SM (64 registers),
// which its shared memory (FP32 operands only) allows as well.
template <bool TIMED, bool XS>
__global__ void __launch_bounds__(kNTS, 4) k_ssa64(const SsaParams p) {
  ssa_warp<AR_CMP_F64, TIMED, XS>(p);
}

}  // namespace
}  // namespace gbar

using namespace gbar;

template <typename T>
static cudaError_t upload(T** d, const std::vector<T>& h) {
  *d = nullptr;
  if (h.empty()) return cudaSuccess;
  cudaError_t e = cudaMalloc(d, sizeof(T) * h.size());
  if (e == cudaSuccess) e = cudaMemcpy(*d, h.data(), sizeof(T) * h.size(), cudaMemcpyHostToDevice);
  return e;
}

extern "C" int ssa_net_create(int32_t N, int32_t M, const int32_t* h_rtype,
                              const int32_t* h_reactants, const double* h_rate,
                              const int32_t* h_nu_ptr, const int32_t* h_nu_species,
                              const int32_t* h_nu_delta, ssa_net** out) {
  if (!out || N <= 0 || M <= 0 || !h_rtype || !h_reactants || !h_rate || !h_nu_ptr ||
      (h_nu_ptr[M] > 0 && (!h_nu_species || !h_nu_delta)))
    return AR_ERR_ARG;
  *out = nullptr;
  std::vector<int8_t> rtype(M);
  std::vector<int2> reac(M);
  std::vector<double> rate(M);
  for (int r = 0; r < M; ++r) {
    const int t = h_rtype[r];
    const int A = h_reactants[2 * r], Bs = h_reactants[2 * r + 1];
    if (t < 0 || t > 3 || !(h_rate[r] >= 0.0) || std::isinf(h_rate[r])) return AR_ERR_ARG;
    if (t >= 1 && (A < 0 || A >= N)) return AR_ERR_ARG;
    if (t == 2 && (Bs < 0 || Bs >= N || Bs == A)) return AR_ERR_ARG;
    rtype[r] = (int8_t)t;
    reac[r] = make_int2(A, Bs);
    rate[r] = h_rate[r];
  }
  std::vector<int32_t> nu_ptr(h_nu_ptr, h_nu_ptr + M + 1);
  const int nnz = nu_ptr[M];
  if (nu_ptr[0] != 0 || nnz < 0) return AR_ERR_ARG;
  std::vector<int2> nu(nnz);
  int max_nu = 0;
  for (int r = 0; r < M; ++r) {
    if (nu_ptr[r + 1] < nu_ptr[r]) return AR_ERR_ARG;
    max_nu = std::max(max_nu, nu_ptr[r + 1] - nu_ptr[r]);
    for (int q = nu_ptr[r]; q < nu_ptr[r + 1]; ++q) {
      if (h_nu_species[q] < 0 || h_nu_species[q] >= N) return AR_ERR_ARG;
      nu[q] = make_int2(h_nu_species[q], h_nu_delta[q]);
    }
  }
  // dependency graph: reactions reading a species that reaction j changes
  std::vector<std::vector<int>> readers(N);
  for (int r = 0; r < M; ++r) {
    if (rtype[r] >= 1) readers[reac[r].x].push_back(r);
    if (rtype[r] == 2) readers[reac[r].y].push_back(r);
  }
  std::vector<int32_t> dep_ptr(M + 1, 0), dep;
  int max_dep = 0;
  for (int j = 0; j < M; ++j) {
    std::vector<int> d;
    for (int q = nu_ptr[j]; q < nu_ptr[j + 1]; ++q) {
      if (nu[q].y == 0) continue;
      const auto& rd = readers[nu[q].x];
      d.insert(d.end(), rd.begin(), rd.end());
    }
    std::sort(d.begin(), d.end());
    d.erase(std::unique(d.begin(), d.end()), d.end());
    dep.insert(dep.end(), d.begin(), d.end());
    dep_ptr[j + 1] = (int32_t)dep.size();
    max_dep = std::max(max_dep, (int)d.size());
  }
  auto* n = new ssa_net();
  n->device = device_info().device;
  n->N = N;
  n->M = M;
  n->max_nu = max_nu;
  n->max_dep = max_dep;
  cudaError_t e = upload(&n->d_rtype, rtype);
  if (e == cudaSuccess) e = upload(&n->d_reac, reac);
  if (e == cudaSuccess) e = upload(&n->d_rate, rate);
  if (e == cudaSuccess) e = upload(&n->d_nu_ptr, nu_ptr);
  if (e == cudaSuccess) e = upload(&n->d_nu, nu);
  if (e == cudaSuccess) e = upload(&n->d_dep_ptr, dep_ptr);
  if (e == cudaSuccess) e = upload(&n->d_dep, dep);
  if (e != cudaSuccess) {
    set_cuda_error(e);
    ssa_net_destroy(n);
    return AR_ERR_CUDA;
  }
  *out = n;
  return AR_OK;
}

extern "C" void ssa_net_destroy(ssa_net* n) {
  if (!n) return;
  int cur = 0;
  cudaGetDevice(&cur);
  if (cur != n->device) cudaSetDevice(n->device);
  cudaFree(n->d_rtype);
  cudaFree(n->d_reac);
  cudaFree(n->d_rate);
  cudaFree(n->d_nu_ptr);
  cudaFree(n->d_nu);
  cudaFree(n->d_dep_ptr);
  cudaFree(n->d_dep);
  if (cur != n->device) cudaSetDevice(cur);
  delete n;
}

namespace {

int ssa_launch(const ssa_net* net, int64_t B, int32_t* d_X, double* d_a, double* d_t,
               uint64_t* d_step, int64_t nsteps, uint64_t seed, uint32_t realization_base,
               int cmp, uint64_t trial_cap, int32_t* d_last, uint32_t* d_status,
               uint64_t* d_trials, SsaParams p, bool timed, void* stream) {
  if (!net || B < 0 || B >= (1ll << 31) || nsteps < 0 || !valid_cmp(cmp)) return AR_ERR_ARG;
  if (trial_cap < 1 || trial_cap > (1ull << 32)) return AR_ERR_ARG;
  if (B == 0 || nsteps == 0) return AR_OK;
  if (!d_X || !d_a || !d_t || !d_step || !d_status) return AR_ERR_ARG;
  if (!aligned(d_X, 4) || !aligned(d_a, 8) || !aligned(d_t, 8) || !aligned(d_step, 8) ||
      !aligned(d_status, 4) || !aligned(d_last, 4) || !aligned(d_trials, 8))
    return AR_ERR_ALIGN;
  if ((uint64_t)realization_base + (uint64_t)B > (1ull << 32)) return AR_ERR_ARG;
  // per warp: the comparison copies (4 bytes each for either comparison), the
  // lanes' raised maxima, the counts
  const size_t es = 4;
  const size_t inc_off = ((size_t)net->M * es + 15) & ~size_t(15);
  const size_t x_off = inc_off + 32 * sizeof(unsigned long long);
  const size_t with_x = x_off + (((size_t)net->N * 4 + 15) & ~size_t(15));
  const DeviceInfo& dev = device_info();
  const size_t limit = dev.max_smem_optin > 0 ? (size_t)dev.max_smem_optin : 227 * 1024;
  // counts in shared memory when that keeps four CTAs per SM (the
  // register limit) or does not lower the CTAs per SM at all
  const size_t sm_total = 228 * 1024, per_cta_reserved = 1024;
  auto ctas = [&](size_t stride) {
    return std::min<size_t>(4, sm_total / (stride * kWarpsS + per_cta_reserved));
  };
  const bool xs = with_x * kWarpsS <= limit && ctas(with_x) >= ctas(x_off);
  const uint32_t stride = (uint32_t)(xs ? with_x : x_off);
  const size_t smem = (size_t)stride * kWarpsS;
  if (smem > limit) return AR_ERR_UNSUPPORTED;
  p.rtype = net->d_rtype;
  p.reac = net->d_reac;
  p.rate = net->d_rate;
  p.nu_ptr = net->d_nu_ptr;
  p.nu = net->d_nu;
  p.dep_ptr = net->d_dep_ptr;
  p.dep = net->d_dep;
  p.N = net->N;
  p.M = net->M;
  p.B = (uint32_t)B;
  p.X = d_X;
  p.a = d_a;
  p.t = d_t;
  p.step = reinterpret_cast<unsigned long long*>(d_step);
  p.last = d_last;
  p.status = d_status;
  p.trials = reinterpret_cast<unsigned long long*>(d_trials);
  p.nsteps = nsteps;
  p.cap = trial_cap;
  p.b_base = realization_base;
  p.k0 = (uint32_t)(seed & 0xffffffffu);
  p.k1 = (uint32_t)(seed >> 32);
  p.smem_stride = stride;
  p.inc_off = (uint32_t)inc_off;
  p.x_off = (uint32_t)x_off;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const unsigned grid = (unsigned)((B + kWarpsS - 1) / kWarpsS);
  auto go = [&](auto kern) {
    cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    kern<<<grid, kNTS, smem, s>>>(p);
  };
  if (cmp == AR_CMP_F32) {
    if (xs) {
      if (timed) go(k_ssa<true, true>);
      else go(k_ssa<false, true>);
    } else {
      if (timed) go(k_ssa<true, false>);
      else go(k_ssa<false, false>);
    }
  } else {
    if (xs) {
      if (timed) go(k_ssa64<true, true>);
      else go(k_ssa64<false, true>);
    } else {
      if (timed) go(k_ssa64<true, false>);
      else go(k_ssa64<false, false>);
    }
  }
  return check_launch();
}

}  // namespace

extern "C" int ssa_step_batched(const ssa_net* net, int64_t B, int32_t* d_X, double* d_a,
                                double* d_t, uint64_t* d_step, int64_t nsteps, uint64_t seed,
                                uint32_t realization_base, int cmp, uint64_t trial_cap,
                                int32_t* d_last, uint32_t* d_status, uint64_t* d_trials,
                                void* stream) {
  SsaParams p{};
  return ssa_launch(net, B, d_X, d_a, d_t, d_step, nsteps, seed, realization_base, cmp,
                    trial_cap, d_last, d_status, d_trials, p, false, stream);
}

extern "C" int ssa_run_until(const ssa_net* net, int64_t B, int32_t* d_X, double* d_a,
                             double* d_t, uint64_t* d_step, double t_end, int64_t max_steps,
                             uint64_t seed, uint32_t realization_base, int cmp,
                             uint64_t trial_cap, const double* d_sample_times, int32_t nsamp,
                             const int32_t* d_sample_species, int32_t nspec, int32_t* d_traj,
                             int32_t* d_last, uint32_t* d_status, uint64_t* d_trials,
                             void* stream) {
  if (!(t_end >= 0.0) || nsamp < 0 || nspec < 0) return AR_ERR_ARG;
  if (nsamp > 0 && (!d_sample_times || !d_traj || nspec <= 0)) return AR_ERR_ARG;
  if (!net || (!d_sample_species && nspec > net->N)) return AR_ERR_ARG;
  if (!aligned(d_sample_times, 8) || !aligned(d_sample_species, 4) || !aligned(d_traj, 4))
    return AR_ERR_ALIGN;
  SsaParams p{};
  p.t_end = t_end;
  p.samp_t = d_sample_times;
  p.nsamp = nsamp;
  p.samp_sp = d_sample_species;
  p.nspec = nsamp > 0 ? nspec : 0;
  p.traj = d_traj;
  return ssa_launch(net, B, d_X, d_a, d_t, d_step, max_steps, seed, realization_base, cmp,
                    trial_cap, d_last, d_status, d_trials, p, true, stream);
}
