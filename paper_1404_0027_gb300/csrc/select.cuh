// Warp-level AR selection engine shared by the single-vector and batched
// kernels.
//
// A warp owns a queue of selections [q, q_end).  It keeps up to 32 of them
// "active", one per lane in a compact list (lane i holds the selection id and
// the next Philox counter of the i-th active selection).  Each round gives
// every active selection G = 32 >> ceil(log2(active)) lanes; lane g of a
// selection's segment evaluates the U Philox blocks t/2 = cnt + g U ..
// cnt + g U + U - 1, i.e. trials 2(cnt + g U) .. 2(cnt + g U + U) - 1, its
// lowest accepted one first.  A ballot over the lanes and a find-first-set in
// each segment pick the lowest accepted trial, so the result is the one the
// sequential AR loop of the paper (Section "A GPU acceptance-rejection
// algorithm") produces on the same stream, whatever G is.  Finished
// selections leave the list (ballot + popc compaction through shared
// memory) and queued ones join it; as the queue drains, fewer selections
// share the warp and each gets more lanes, so the tail of long geometric
// trial counts is worked on by the whole warp.
#pragma once

#include "device.cuh"

namespace gbar {

struct SelCounters {
  unsigned long long trials = 0;
  uint32_t accepted = 0;
  uint32_t capped = 0;
};

// acc(j, w) -> bool : the acceptance test of candidate j with uniform word w.
// idx[i] receives the result of local selection i (global id sel_base + i).
template <int U, class Acc>
__device__ __forceinline__ void warp_select(uint32_t q, const uint32_t q_end, const uint32_t sel_base,
                                            const uint32_t M, const uint32_t b, const uint32_t k0,
                                            const uint32_t k1, const unsigned long long cap,
                                            const Acc& acc, int32_t* __restrict__ idx,
                                            uint32_t* __restrict__ scr, SelCounters& ctr) {
  const uint32_t lane = threadIdx.x & 31u;
  const uint32_t lt_mask = (1u << lane) - 1u;
  uint32_t nA = 0;
  uint32_t my_sel = 0, my_cnt = 0;
  for (;;) {
    const uint32_t room = 32u - nA;
    const uint32_t left = q_end - q;
    const uint32_t take = room < left ? room : left;
    if (lane >= nA && lane < nA + take) {
      my_sel = q + (lane - nA);
      my_cnt = 0;
    }
    nA += take;
    q += take;
    if (nA == 0) break;
    // G = 32 >> ceil(log2(nA)) lanes per active selection; lg = log2(G).
    const uint32_t lg = 5u - (32u - __clz(nA - 1u));
    const uint32_t owner = lane >> lg;
    const uint32_t g = lane & ((1u << lg) - 1u);
    const bool valid = owner < nA;
    const uint32_t sel = __shfl_sync(kFull, my_sel, owner & 31u);
    const uint32_t cnt = __shfl_sync(kFull, my_cnt, owner & 31u) + g * U;
    uint4 w[U];
#pragma unroll
    for (int u = 0; u < U; ++u) w[u] = philox10(make_uint4(cnt + u, sel_base + sel, b, 0u), k0, k1);
    uint32_t j[2 * U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      j[2 * u] = candidate(w[u].x, M);
      j[2 * u + 1] = candidate(w[u].z, M);
    }
    int hit = -1;  // the lowest accepted trial of this lane, 0 .. 2U - 1
    uint32_t jh = 0;
    // trials of this lane below the cap: min(2U, cap - 2 cnt)
    const unsigned long long t0 = 2ull * cnt;
    const uint32_t nvalid =
        (!valid || t0 >= cap) ? 0u : (cap - t0 < 2u * U ? (uint32_t)(cap - t0) : 2u * U);
#pragma unroll
    for (int t = 2 * U - 1; t >= 0; --t) {
      const uint32_t wu = (t & 1) ? w[t >> 1].w : w[t >> 1].y;
      if ((uint32_t)t < nvalid && acc(j[t], wu)) {
        hit = t;
        jh = j[t];
      }
    }
    const uint32_t bal = __ballot_sync(kFull, hit >= 0);
    // State lane i reads its segment [i*G, i*G + G) of the ballot.
    const uint32_t seg_lo = (lane << lg) & 31u;
    const uint32_t seg_mask = lg == 5u ? kFull : ((1u << (1u << lg)) - 1u);
    const uint32_t seg = (bal >> seg_lo) & seg_mask;
    const uint32_t src = seg_lo + (uint32_t)(__ffs(seg) - 1);
    const uint32_t got_j = __shfl_sync(kFull, jh, src & 31u);
    const uint32_t got_h = (uint32_t)__shfl_sync(kFull, hit, src & 31u);
    bool done = false;
    if (lane < nA) {
      if (seg) {
        const unsigned long long t_acc =
            2ull * (my_cnt + (src - seg_lo) * U) + (unsigned long long)got_h;
        idx[my_sel] = (int32_t)got_j;
        ctr.trials += t_acc + 1ull;
        ctr.accepted += 1;
        done = true;
      } else {
        my_cnt += (1u << lg) * U;
        if (2ull * my_cnt >= cap) {
          idx[my_sel] = (int32_t)M;
          ctr.trials += cap;
          ctr.capped += 1;
          done = true;
        }
      }
    }
    const uint32_t alive = __ballot_sync(kFull, lane < nA && !done);
    const uint32_t nA2 = __popc(alive);
    if (nA2 != nA) {
      if ((alive >> lane) & 1u) {
        const uint32_t pos = __popc(alive & lt_mask);
        scr[pos] = my_sel;
        scr[32 + pos] = my_cnt;
      }
      __syncwarp();
      if (lane < nA2) {
        my_sel = scr[lane];
        my_cnt = scr[32 + lane];
      }
      __syncwarp();
    }
    nA = nA2;
  }
}

// Writes the sentinel to a warp's whole range (bound unusable / all zero).
__device__ __forceinline__ void warp_fill(uint32_t q, uint32_t q_end, int32_t v,
                                          int32_t* __restrict__ idx) {
  for (uint32_t i = q + (threadIdx.x & 31u); i < q_end; i += 32u) idx[i] = v;
}

__device__ __forceinline__ void flush_counters(SelCounters c, ar_stats* stats) {
  unsigned long long t = warp_sum_u64(c.trials);
  unsigned long long a = warp_sum_u64(c.accepted);
  unsigned long long k = warp_sum_u64(c.capped);
  if ((threadIdx.x & 31u) == 0 && stats) {
    if (t) atomicAdd(reinterpret_cast<unsigned long long*>(&stats->trials), t);
    if (a) atomicAdd(reinterpret_cast<unsigned long long*>(&stats->accepted), a);
    if (k) atomicAdd(reinterpret_cast<unsigned long long*>(&stats->capped), k);
  }
}

}  // namespace gbar
