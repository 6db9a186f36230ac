// ring.cuh -- the plane ring of a DK pass, as device functions: the shared
// memory behind the stages, the bulk copies that fill a stage with one z-plane
// tile of every array, the release count whose last warp refills the stage,
// the per-run flush of the sums into a partial-sum slot, and the lattice-wide
// slot reduction that precedes the Friedmann update.
//
// A CTA's segments form one sequence of planes (each segment adds a halo
// plane at both ends); plane g of pass p lives in stage (p * ptot + g) mod S.
// A stage holds, for every array, the plane's BY rows of the segment's y-tile
// plus one halo row on each side, each row complete in x (with MOWN the momenta,
// read at the tile's own sites only, without the halo rows).
#pragma once

#include "common.cuh"

namespace clg {

struct Ring {
  unsigned char* stages;  // S stages of stage_bytes
  uint64_t* full;         // one mbarrier per stage: all copies of the stage landed
  unsigned* released;     // warps done with each stage
  int* off;               // first plane of each segment, and the total
  double* red;            // [33][NQ] reduction scratch
  volatile int* flag;     // [0] timed out, [1] unused, [2] lattice of the last run, [3] #pending tails
  int* pend;              // lattices whose Friedmann update this CTA runs
  IssueInfo* info;        // per segment: what its refills copy
  int S;
  unsigned stage_bytes;
};

__device__ __forceinline__ Ring ring_view(unsigned char* smem, const PassArgs& P) {
  Ring R;
  R.S = P.stages;
  R.stage_bytes = P.stage_bytes_max;
  R.stages = smem;
  unsigned char* tail = smem + (size_t)R.S * R.stage_bytes;
  R.full = reinterpret_cast<uint64_t*>(tail + SM_FULL);
  R.released = reinterpret_cast<unsigned*>(tail + SM_RELEASED);
  R.off = reinterpret_cast<int*>(tail + SM_OFF);
  R.red = reinterpret_cast<double*>(tail + SM_RED);
  R.flag = reinterpret_cast<volatile int*>(tail + SM_FLAG);
  R.pend = reinterpret_cast<int*>(tail + SM_FLAG + 16);
  R.info = reinterpret_cast<IssueInfo*>(tail + SM_INFO);
  return R;
}

// Thread 0: barriers, counts, flags, plane offsets and the copy info of the
// CTA's `ns` segments starting at segs[sb].
template <int NA>
__device__ void ring_setup(const Ring& R, const PassArgs& P, int sb, int ns) {
  for (int s = 0; s < R.S; ++s) {
    mbar_init(&R.full[s], 1);
    R.released[s] = 0u;
  }
  fence_mbar_init();
  R.flag[0] = 0;
  R.flag[1] = 0;
  R.flag[2] = ns > 0 ? P.segs[sb].lat : 0;
  R.flag[3] = 0;
  R.off[0] = 0;
  for (int i = 0; i < ns; ++i) {
    const Seg& sg = P.segs[sb + i];
    const LatConst& L = P.lat[sg.lat];
    R.off[i + 1] = R.off[i] + sg.nz + 2;
    IssueInfo& in = R.info[i];
    in.z0 = sg.z0;
    in.nz = sg.nz;
    in.dir = sg.dir;
    in.ylo = sg.ytile * L.BY;
    in.N = L.N;
    in.rows = L.BY + 2;
    for (int a = 0; a < NA; ++a) {
      in.src[0][a] = L.buf[0][a];
      in.src[1][a] = L.buf[1][a];
    }
  }
}

template <typename T>
__device__ __forceinline__ const T* ring_stage(const Ring& R, int s) {
  return reinterpret_cast<const T*>(R.stages + (size_t)s * R.stage_bytes);
}

// Bulk copies of plane g (of the current pass) into stage s, issued by a
// whole warp (warp-uniform call): lane a + NA k copies run k of array a (a
// tile's rows form up to three runs where they wrap around the periodic y
// boundary).  MOWN: the odd arrays (momenta of a field/momentum layout) are
// copied without their halo rows -- the tile's own rows only, one run -- and
// each (field, momentum) pair occupies rows + (rows - 2) rows of the stage,
// the field's first.
// Stage memory is only read through the generic proxy and its reuse is
// ordered by the release count, so no proxy fence precedes the copies.
template <typename T, int NA, bool MOWN = false>
__device__ void ring_issue_warp(const Ring& R, int g, int s, int parity, int lane) {
  static_assert(3 * NA <= 32, "one lane per copy");
  int i = 0;
  while (g >= R.off[i + 1]) ++i;
  const IssueInfo& in = R.info[i];
  const int N = in.N, rows = in.rows, arr_elems = rows * N;
  const int j = g - R.off[i];
  int zp = in.dir > 0 ? in.z0 - 1 + j : in.z0 + in.nz - j;
  zp = zp < 0 ? zp + N : (zp >= N ? zp - N : zp);
  // rows ylo-1 .. ylo+rows-2 of the plane, periodic in y: r1 rows from y1, then
  // r2 rows from row 0, then (a tile as tall as the lattice wraps twice) r3 from row 0
  const int y0 = in.ylo - 1;
  const int y1 = y0 < 0 ? y0 + N : y0;
  const int r1 = min(rows, N - y1), r2 = min(rows - r1, N), r3 = rows - r1 - r2;
  const size_t stage_elems = MOWN ? (size_t)(NA / 2) * (2 * rows - 2) * N : (size_t)NA * arr_elems;
  if (lane == 0) mbar_arrive_expect_tx(&R.full[s], (uint32_t)(stage_elems * sizeof(T)));
  __syncwarp();
  if (lane < 3 * NA) {
    const int run = lane / NA, a = lane - run * NA;
    const bool own_only = MOWN && (a & 1);
    int nr = run == 0 ? r1 : (run == 1 ? r2 : r3);
    if (own_only) nr = run == 0 ? rows - 2 : 0;  // rows ylo .. ylo + BY - 1 never wrap
    if (nr > 0) {
      const int d = own_only ? 0 : (run == 0 ? 0 : (run == 1 ? r1 : r1 + r2));
      const int ys = own_only ? in.ylo : (run == 0 ? y1 : 0);
      const size_t aoff = MOWN ? (size_t)(a >> 1) * (2 * rows - 2) * N + (a & 1) * (size_t)rows * N
                               : (size_t)a * arr_elems;
      T* st = reinterpret_cast<T*>(R.stages + (size_t)s * R.stage_bytes) + aoff;
      const T* src = reinterpret_cast<const T*>(in.src[parity][a]) + (long long)zp * N * N;
      bulk_g2s(st + (size_t)d * N, src + (long long)ys * N, (uint32_t)(nr * N * sizeof(T)), &R.full[s]);
    }
  }
}

// A warp is done with plane g (in stage s); the last of the CTA's warps
// refills s with plane g + S of the same pass (which belongs in the same stage).
template <typename T, int NA, bool MOWN = false>
__device__ __forceinline__ void ring_release(const Ring& R, int g, int s, int parity, int ptot, int lane) {
  __syncwarp();
  int refill = 0;
  if (lane == 0) {
    __threadfence_block();
    const unsigned prev = atomicAdd(&R.released[s], 1u);
    if (prev == CONSUMER_WARPS - 1u) {
      R.released[s] = 0u;
      refill = g + R.S < ptot && !R.flag[0];
    }
  }
  if (__shfl_sync(0xffffffffu, refill, 0)) ring_issue_warp<T, NA, MOWN>(R, g + R.S, s, parity, lane);
  __syncwarp();
}

__device__ __forceinline__ void ring_wait(const Ring& R, int s, uint32_t par,
                                          unsigned long long limit_ns) {
  if (R.flag[0]) return;
  if (!mbar_wait_bounded(&R.full[s], par, limit_ns)) R.flag[0] = 1;
}

__device__ __forceinline__ void ring_advance(int S, int& s, uint32_t& p) {
  if (++s == S) {
    s = 0;
    p ^= 1u;
  }
}

// End of a CTA's run on a lattice (all threads): warp partials of the NUSED
// slots (accumulators acc[0..NACC), slot NQ-1 = non-finite count), a fixed
// shuffle tree over the warps per slot into P.partials, and the lattice's
// arrival count; the CTA that completes it queues the lattice's tail.
// Returns false if a wait of this CTA had timed out.
template <int NACC, int NUSED, typename T>
__device__ bool ring_flush(const Ring& R, const PassArgs& P, const Seg& sg, Acc<T> (&acc)[NACC],
                           float& nonfinite, int warp, int lane) {
  if (NUSED > 0) {
#pragma unroll
    for (int k = 0; k < NUSED; ++k) {
      double v = 0.0;
      if (k < NACC) {
        v = warp_sum(acc[k]);
      } else if (k == NQ - 1) {
        float c = nonfinite;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) c += __shfl_down_sync(0xffffffffu, c, o);
        v = (double)c;
      }
      if (lane == 0) R.red[warp * NQ + k] = v;
    }
  }
#pragma unroll
  for (int k = 0; k < NACC; ++k) acc[k].zero();
  nonfinite = 0.f;
  __syncthreads();
  if (R.flag[0]) return false;
  if (warp < NUSED) {
    double v = lane < CONSUMER_WARPS ? R.red[lane * NQ + warp] : 0.0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if (lane == 0) {
      P.partials[(size_t)warp * P.nslot + sg.slot] = v;
      __threadfence();
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    const LatConst& L = P.lat[sg.lat];
    const unsigned nslot = (unsigned)(L.slot_end - L.slot_begin);
    const unsigned prev = atomicAdd(&P.counters[sg.lat], 1u);
    R.flag[2] = sg.lat;
    if (prev == nslot - 1u) R.pend[R.flag[3]++] = sg.lat;
  }
  __syncthreads();
  return true;
}

// Lattice-wide sums of the first NUSED quantities into red[32 * NQ + k]:
// warp k sums the lattice's slots of quantity k in a fixed order
// (warp_slot_sum), so the result does not depend on timing.  All threads;
// ends with a barrier.
template <int NUSED>
__device__ void ring_slot_sums(const Ring& R, const PassArgs& P, const LatConst& L, int warp,
                               int lane) {
  if (warp < NUSED) {
    const double s = warp_slot_sum(P.partials + (size_t)warp * P.nslot, L.slot_begin, L.slot_end, lane);
    if (lane == 0) R.red[32 * NQ + warp] = s;
  }
  __syncthreads();
}

// Between two passes of one launch (warp 0, all lanes): the previous pass's
// writes are all done before any of its planes is read; the first planes of
// the pass are issued; then the updated scalars are awaited.
template <typename T, int NA, bool MOWN = false>
__device__ void ring_pass_start(const Ring& R, const PassArgs& P, int pass, int ptot, int parity, int lane) {
  int go = 0;
  if (lane == 0) {
    if (pass > 0 && !R.flag[0] && !wait_counter(&P.gsync[0], gridDim.x * (unsigned)pass, P.wait_limit_ns))
      R.flag[0] = 1;
    go = !R.flag[0];
  }
  go = __shfl_sync(0xffffffffu, go, 0);
  if (pass > 0) fence_proxy_async_global();
  if (go)
    for (int g = 0; g < R.S && g < ptot; ++g)
      ring_issue_warp<T, NA, MOWN>(R, g, (pass * ptot + g) % R.S, parity, lane);
  if (lane == 0 && pass > 0 && !R.flag[0] &&
      !wait_counter(&P.gsync[1], (unsigned)P.nlat * (unsigned)pass, P.wait_limit_ns))
    R.flag[0] = 1;
}

// After a timed-out wait (thread 0): wait, bounded, for copies still in
// flight so that none lands in shared memory after exit, and record it.
__device__ inline void ring_drain(const Ring& R, const PassArgs& P) {
  for (int s = 0; s < R.S; ++s)
    for (int par = 0; par < 2; ++par) mbar_wait_bounded(&R.full[s], (uint32_t)par, 1000000ull);
  P.sc[R.flag[2]].status = CL_ETIMEOUT;
}

}  // namespace clg
