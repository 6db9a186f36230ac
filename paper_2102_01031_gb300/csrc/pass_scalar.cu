// pass_scalar.cu -- fused drift + kick pass for real scalar singlets
// (CosmoLattice manual, Sec. 3.5.2, Hamiltonian form):
//
//   drift (deferred from the previous pass):  phi += cd * pi,   cd = h abar^{alpha-3}
//   kick:   pi += c_k [ a^{1+alpha} Lap phi - a^{3+alpha} V_{,phi} ]
//   Lap phi = sum_i [phi(n+i) - 2 phi(n) + phi(n-i)] / dx^2       (eqs. neutrald, forwardbackwardd)
//   sums:   sum pi^2 before / after the kick, sum_i (grad^+_i phi)^2 (as -sum phi Lap phi
//           in the Friedmann passes), sum V (+ means in measurement passes)
//
// One pass per integrator stage: each field and momentum array is read once
// from HBM and written once.  A CTA owns runs of (y-tile, z-plane) tasks
// ("segments"): BY full x-rows marched along z.  Its segments form one
// continuous sequence of planes (each segment adds a halo plane at both
// ends); every plane tile (plus one halo row on each side in y) of every
// array streams into a ring of shared-memory stages by 1-D bulk async copies
// (TMA), completion counted on the stage's mbarrier.  The 16 warps never meet
// at a block barrier while marching: each waits for the stage it needs,
// applies the drift in registers as it reads (z-neighbours stay in registers,
// y-neighbours come from the stage, x-neighbours from warp shuffles), kicks,
// stores, and releases the stage; the last warp to release a stage (shared
// memory count) issues the copies of the plane S places further in the
// sequence, so the ring runs on across segment boundaries.  Sums are formed
// per plane in the storage precision, added once per plane to compensated
// (FP32) or plain (FP64) accumulators and flushed once per run into the run's
// slot; the last slot of a lattice to be written reduces all of them in a
// fixed order and runs the Friedmann update (tail.cuh).
#include "common.cuh"
#include "tail.cuh"

namespace clg {

// Program potentials (eq. PotNat): NF = 1: phi^4/4; NF = 2: phi^4/4 + (q/2) phi^2 chi^2.
template <int NF> struct ScalarPot;
template <> struct ScalarPot<1> {
  static constexpr int NPOT = 1;
  template <typename T>
  __device__ __forceinline__ static T total(const T (&f)[1], T hq) {
    const T f2 = f[0] * f[0];
    return T(0.25) * f2 * f2;
  }
  template <typename T>
  __device__ __forceinline__ static void eval(const T (&f)[1], T q, T (&d)[1], T (&t)[1]) {
    const T f2 = f[0] * f[0];
    d[0] = f2 * f[0];
    t[0] = T(0.25) * f2 * f2;
  }
};
template <> struct ScalarPot<2> {
  static constexpr int NPOT = 2;
  // phi^4/4 + (q/2) phi^2 chi^2 = p2 (p2/4 + (q/2) c2), hq = q/2
  template <typename T>
  __device__ __forceinline__ static T total(const T (&f)[2], T hq) {
    const T p2 = f[0] * f[0], c2 = f[1] * f[1];
    return p2 * fmaT(T(0.25), p2, hq * c2);
  }
  template <typename T>
  __device__ __forceinline__ static void eval(const T (&f)[2], T q, T (&d)[2], T (&t)[2]) {
    const T p2 = f[0] * f[0], c2 = f[1] * f[1];
    if constexpr (sizeof(T) == 8)
      d[0] = f[0] * fmaT(q, c2, p2);  // phi (phi^2 + q chi^2): one operation fewer on the FP64 pipe
    else
      d[0] = p2 * f[0] + q * f[0] * c2;
    d[1] = q * p2 * f[1];
    t[0] = T(0.25) * p2 * p2;
    t[1] = T(0.5) * q * p2 * c2;
  }
};

template <typename T, int VX>
__device__ __forceinline__ void ld_vec(T (&v)[VX], const T* p) {
  *reinterpret_cast<typename V16<T>::type*>(v) = *reinterpret_cast<const typename V16<T>::type*>(p);
}
template <typename T, int VX>
__device__ __forceinline__ void st_vec(T* p, const T (&v)[VX]) {
  *reinterpret_cast<typename V16<T>::type*>(p) = *reinterpret_cast<const typename V16<T>::type*>(v);
}

// z of plane j of a segment (j = 0 and nz + 1 are its halo planes)
__device__ __forceinline__ int seg_plane_z(const Seg& sg, int N, int j) {
  const int z = sg.dir > 0 ? sg.z0 - 1 + j : sg.z0 + sg.nz - j;
  return z < 0 ? z + N : (z >= N ? z - N : z);
}

// RED: 0 = no sums, 1 = sums for the Friedmann kick, 2 = full measurement.
// P.npass > 1: several passes in one cooperative launch; between two passes
// every CTA signals that its writes are done, the CTAs that close a lattice's
// sums run its Friedmann update, and every CTA prefetches the first planes of
// the next pass as soon as all writes are done, before it waits for the
// updated scalars.
template <typename T, int NF, int RED>
__global__ void __launch_bounds__(THREADS, 1) dk_pass_scalar(const PassArgs P) {
  constexpr int VX = V16<T>::n;
  constexpr int NA = 2 * NF;
  constexpr int NPOT = ScalarPot<NF>::NPOT;
  // RED = 1 sums: pi^2 after the kick, phi Lap phi (= -(grad^+ phi)^2 summed), V.  The pre-kick sum of
  // pi^2 is the previous kick's post-kick sum (a drift leaves pi unchanged),
  // carried in the lattice scalars.
  constexpr int NACC = RED == 0 ? 1 : (RED == 1 ? 3 : 6 * NF + NPOT);
  // slots a pass reduces: the Friedmann sums, or every measured sum plus the
  // non-finite count (slot NQ - 1)
  constexpr int NUSED = RED == 0 ? 0 : (RED == 1 ? 3 : NQ);
  // arrivals per partial-sum slot on the lattice's count (one per quantity; one when there are none)
  constexpr int NARRIVE = NUSED > 0 ? NUSED : 1;

  extern __shared__ __align__(128) unsigned char smem[];
  const int S = P.stages;
  unsigned char* tail = smem + (size_t)S * P.stage_bytes_max;
  uint64_t* full = reinterpret_cast<uint64_t*>(tail + SM_FULL);
  unsigned* released = reinterpret_cast<unsigned*>(tail + SM_RELEASED);  // warps done with a stage
  int* off = reinterpret_cast<int*>(tail + SM_OFF);                      // plane offsets of segments
  double* red = reinterpret_cast<double*>(tail + SM_RED);                // [33][NQ]
  volatile int* flag = reinterpret_cast<volatile int*>(tail + SM_FLAG);  // timeout, last, lattice, #pending
  int* pend = reinterpret_cast<int*>(tail + SM_FLAG + 16);               // lattices whose tail is due
  IssueInfo* info = reinterpret_cast<IssueInfo*>(tail + SM_INFO);
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int sb = P.cta_seg[blockIdx.x], ns = P.cta_seg[blockIdx.x + 1] - sb;
  const bool multi = P.npass > 1;

  if (tid == 0) {
    for (int s = 0; s < S; ++s) {
      mbar_init(&full[s], 1);
      released[s] = 0u;
    }
    fence_mbar_init();
    flag[0] = 0;
    flag[1] = 0;
    flag[2] = ns > 0 ? P.segs[sb].lat : 0;
    flag[3] = 0;
    off[0] = 0;
    for (int i = 0; i < ns; ++i) {
      const Seg& sg = P.segs[sb + i];
      const LatConst& L = P.lat[sg.lat];
      off[i + 1] = off[i] + sg.nz + 2;
      IssueInfo& in = info[i];
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
  __syncthreads();
  const int ptot = off[ns];
  int parity = P.parity;
  // planes of earlier passes of this launch: plane g of the current pass is
  // plane gbase + g of the CTA's whole sequence and sits in stage (gbase+g) mod S
  int gbase = 0;
  // passes reading buffer 1 march the CTA's sequence backwards (plane g is
  // plane ptot-1-g of the forward sequence: segments in reverse order, each
  // marched the other way), so that a pass starts on the planes the previous
  // pass wrote last, while they are still in L2
  bool rev = false;

  // bulk copies of plane g of this pass into stage s, issued by a whole warp:
  // lane a + NA k copies run k of array a (a tile's rows form up to three
  // runs where they wrap around the periodic y boundary).  Stage memory is only
  // ever read through the generic proxy, and its reuse is ordered by the
  // release count, so no proxy fence precedes the copies.  Warp-uniform calls.
  auto issue_warp = [&](int g, int s) {
    const int gf = rev ? ptot - 1 - g : g;  // position in the forward sequence
    int i = 0;
    while (gf >= off[i + 1]) ++i;
    const IssueInfo& in = info[i];
    const int N = in.N, rows = in.rows, arr_elems = rows * N;
    const int j = gf - off[i];
    int zp = in.dir > 0 ? in.z0 - 1 + j : in.z0 + in.nz - j;
    zp = zp < 0 ? zp + N : (zp >= N ? zp - N : zp);
    // rows ylo-1 .. ylo+rows-2 of the plane, periodic in y: r1 rows from y1, then
    // r2 rows from row 0, then (a tile as tall as the lattice wraps twice) r3 from row 0
    const int y0 = in.ylo - 1;
    const int y1 = y0 < 0 ? y0 + N : y0;
    const int r1 = min(rows, N - y1), r2 = min(rows - r1, N), r3 = rows - r1 - r2;
    if (lane == 0) mbar_arrive_expect_tx(&full[s], (uint32_t)((size_t)NA * arr_elems * sizeof(T)));
    __syncwarp();
    if (lane < 3 * NA) {
      const int run = lane / NA, a = lane - run * NA;
      const int nr = run == 0 ? r1 : (run == 1 ? r2 : r3);
      if (nr > 0) {
        const int d = run == 0 ? 0 : (run == 1 ? r1 : r1 + r2), ys = run == 0 ? y1 : 0;
        T* st = reinterpret_cast<T*>(smem + (size_t)s * P.stage_bytes_max) + (size_t)a * arr_elems;
        const T* src = reinterpret_cast<const T*>(in.src[parity][a]) + (long long)zp * N * N;
        bulk_g2s(st + (size_t)d * N, src + (long long)ys * N, (uint32_t)(nr * N * sizeof(T)), &full[s]);
      }
    }
  };
  // a warp is done with plane g (in stage s); the last of the 16 refills s with
  // plane g + S (which belongs in the same stage)
  auto release = [&](int g, int s) {
    __syncwarp();
    int refill = 0;
    if (lane == 0) {
      __threadfence_block();
      const unsigned prev = atomicAdd(&released[s], 1u);
      if (prev == CONSUMER_WARPS - 1u) {
        released[s] = 0u;
        refill = g + S < ptot && !flag[0];
      }
    }
    if (__shfl_sync(0xffffffffu, refill, 0)) issue_warp(g + S, s);
    __syncwarp();
  };
  auto wait_full = [&](int s, uint32_t par) {
    if (flag[0]) return;
    if (!mbar_wait_bounded(&full[s], par, P.wait_limit_ns)) flag[0] = 1;
  };
  auto stage_ptr = [&](int s) -> const T* {
    return reinterpret_cast<const T*>(smem + (size_t)s * P.stage_bytes_max);
  };

  // Friedmann updates of the lattices pend[base .. base + nb) (nb <= 32) once
  // all their slots are written: the warps share the (lattice, quantity)
  // sums, each over the lattice's slots in a fixed order (warp_slot_sum), so
  // the result does not depend on timing; then lane l of the last warp updates
  // a, b and the next pass's coefficients of lattice pend[base + l], all
  // lattices at once.  That thread reads the lattice's scalars and constants
  // into registers and forms the sum-independent factors while the slots are
  // summed (FP64 has a long dependent latency, and this runs between passes).
  auto run_tails = [&](int base, int nb, const PassStep& st, double* lg) {
    const bool tt = warp == CONSUMER_WARPS - 1 && lane < nb;
    int lat = 0;
    LatConst L;
    ScalarState W;
    double ck = 0.0, cg = 0.0;
    FriedPre F = {};
    bool self = false;
    if (tt) {
      lat = pend[base + lane];
      L = P.lat[lat];
      load_state_cg(W, &P.sc[lat]);
      const double a = W.a, ia2 = 1.0 / (a * a);
      ck = 0.5 * L.inv_V * (ia2 * ia2 * ia2);
      cg = 0.5 * L.inv_V * L.inv_dx2 * ia2;
      self = RED > 0 && L.expansion == CL_EXP_SELF;
      if (self) F = friedmann_pre(L, a, st.wout, st.win);
    }
    for (int it = warp; it < nb * NUSED; it += CONSUMER_WARPS) {
      constexpr int NQU = NUSED > 0 ? NUSED : 1;
      const int l = it / NQU, q = it - l * NQU;
      const LatConst& L = P.lat[pend[base + l]];
      const double s = warp_slot_sum(P.partials + (size_t)q * P.nslot, L.slot_begin, L.slot_end, lane);
      if (lane == 0) red[l * NQ + q] = s;
    }
    __syncthreads();
    if (tt) {
      PassArgs Q = P;
      Q.ck = st.ck;
      Q.wout = st.wout;
      Q.win = st.win;
      Q.dnext = st.dnext;
      const double* sum = red + lane * NQ;
      PassSums E = {0, 0, 0, 0, 0, 0, 0};
      if (RED > 0) {
        double spre = 0, spost = 0, gg = 0, vs = 0;
        if (RED == 1) {
          // slot 1 holds sum phi Lap phi = -sum (grad^+ phi)^2
          spre = W.pi2; spost = sum[0]; gg = -sum[1]; vs = sum[2];
        } else {
          for (int f = 0; f < NF; ++f) {
            spre += sum[6 * f]; spost += sum[6 * f + 1]; gg += sum[6 * f + 2];
          }
          for (int t = 0; t < NPOT; ++t) vs += sum[6 * NF + t];
        }
        E.EKpre = spre * ck;
        W.pi2 = spost;
        E.EKpost = spost * ck;
        E.EG = gg * cg;
        E.EV = vs * L.inv_V;
      }
      if (self) W.b = friedmann_kicks_scalar(F, E, W.b);
      if (lg && lat == 0)
        lg[5] = RED > 0 && L.expansion == CL_EXP_SELF ? kernel_a_da(Q, L, W.a, E) : 0.0;
      if (RED == 2) {
        cl_energies_t& o = P.sc[lat].obs;
        for (int k = 0; k < 4; ++k) {
          o.EK[k] = o.EG[k] = o.EV[k] = 0.0;
          o.mean_phi[k] = o.mean_phi2[k] = o.mean_pi[k] = o.mean_pi2[k] = 0.0;
        }
        o.EKA = o.EGA = 0.0;
        for (int f = 0; f < NF; ++f) {
          o.EK[f] = sum[6 * f + 1] * ck;
          o.EG[f] = sum[6 * f + 2] * cg;
          o.mean_phi[f] = sum[6 * f + 3] * L.inv_V;
          o.mean_phi2[f] = sum[6 * f + 4] * L.inv_V;
          o.mean_pi[f] = sum[6 * f + 5] * L.inv_V;
          o.mean_pi2[f] = sum[6 * f + 1] * L.inv_V;
        }
        for (int t = 0; t < NPOT; ++t) o.EV[t] = sum[6 * NF + t] * L.inv_V;
        o.nonfinite = (int64_t)sum[NQ - 1];
        finish_obs(Q, L, W, o);
      }
      advance_drift(Q, L, W);
      store_state(&P.sc[lat], W);
      P.counters[lat] = 0u;
      __threadfence();
      if (multi) atomicAdd(&P.gsync[1], 1u);
    }
    __syncthreads();
  };

  // stage and full-barrier phase of the current plane, advanced without divisions
  int s_cur = 0;
  uint32_t p_cur = 0u;
  auto advance = [&](int& s, uint32_t& p) {
    if (++s == S) {
      s = 0;
      p ^= 1u;
    }
  };

  Acc<T> acc[NACC];
  float nonfinite = 0.f;
  int fbuf = 0;
#pragma unroll
  for (int k = 0; k < NACC; ++k) acc[k].zero();

  for (int pass = 0; pass < P.npass; ++pass) {
    parity = P.parity ^ (pass & 1);
    rev = parity != 0;
    gbase = pass * ptot;
    if (warp == 0) {
      int go = 0;
      if (lane == 0) {
        // the previous pass's writes are all done before any of its planes is read
        if (pass > 0 && !flag[0] && !wait_counter(&P.gsync[0], gridDim.x * (unsigned)pass, P.wait_limit_ns))
          flag[0] = 1;
        go = !flag[0];
      }
      go = __shfl_sync(0xffffffffu, go, 0);
      if (pass > 0) fence_proxy_async_global();
      if (go)
        for (int g = 0; g < S && g < ptot; ++g) issue_warp(g, (gbase + g) % S);
      if (lane == 0 && pass > 0 && !flag[0] &&
          !wait_counter(&P.gsync[1], (unsigned)P.nlat * (unsigned)pass, P.wait_limit_ns))
        flag[0] = 1;
    }
    __syncthreads();
    if (flag[0]) goto timeout;
    if (P.log && blockIdx.x == 0 && tid == 0) {  // coefficients of this pass, for an adjoint sweep
      const LatScalars* S0 = &P.sc[0];
      const double ckp = P.steps ? P.steps[pass].ck : P.ck;
      double* lg = P.log + ADJ_LOG_W * (P.log_base + pass);
      lg[0] = __ldcg(&S0->cd);
      lg[1] = ckp;
      lg[2] = ckp * __ldcg(&S0->apow1) * P.lat[0].inv_dx2;
      lg[3] = ckp * __ldcg(&S0->apow3);
      lg[4] = __ldcg(&S0->a);
    }

    for (int ii = 0; ii < ns; ++ii) {
      const int i = rev ? ns - 1 - ii : ii;
      Seg sg = P.segs[sb + i];
      // the last segment of a run on a lattice, in this pass's order
      const bool run_end = rev ? (i == 0 || P.segs[sb + i - 1].lat != sg.lat) : sg.flush != 0;
      if (rev) sg.dir = -sg.dir;
      const LatConst& L = P.lat[sg.lat];
      const int N = L.N, BY = L.BY, TX = N / VX;
      const int tx = tid % TX, ty = tid / TX;
      const bool active = ty < BY;  // active threads are 0 .. TX*BY-1
      const int x0 = tx * VX;
      const int y = sg.ytile * BY + ty;
      const int arr_elems = (BY + 2) * N;
      const long long NN = (long long)N * N;
      const int g0 = rev ? ptot - off[i + 1] : off[i];
      // coefficients of the segment: FP64 products formed by one lane (the
      // FP64 pipe is narrow) and broadcast in the storage precision
      T cf[3];
      if (lane == 0) {
        const LatScalars* SC = &P.sc[sg.lat];
        const double ckp = P.steps ? __ldg(&P.steps[pass].ck) : P.ck;
        cf[0] = (T)__ldcg(&SC->cd);
        cf[1] = (T)(ckp * __ldcg(&SC->apow1) * L.inv_dx2);
        cf[2] = (T)(ckp * __ldcg(&SC->apow3));
      }
#pragma unroll
      for (int k = 0; k < 3; ++k) cf[k] = __shfl_sync(0xffffffffu, cf[k], 0);
      const T cd = cf[0], A1 = cf[1], A3 = cf[2];
      const bool drifting = cd != T(0);
      const T q = (T)L.q, hq = (T)(0.5 * L.q);
      T* dst[NA];
#pragma unroll
      for (int a = 0; a < NA; ++a) dst[a] = reinterpret_cast<T*>(L.buf[parity ^ 1][a]);
      const int own = (ty + 1) * N + x0;
      const int exl = (ty + 1) * N + (x0 == 0 ? N - 1 : x0 - 1), exr = (ty + 1) * N + (x0 + VX == N ? 0 : x0 + VX);

      // own values of a stage, drifted: phi + cd * pi
      auto read_own = [&](const T* st, T (&ph)[NF][VX]) {
#pragma unroll
        for (int f = 0; f < NF; ++f) {
          ld_vec<T, VX>(ph[f], st + (size_t)(2 * f) * arr_elems + own);
          if (drifting) {
            T pm[VX];
            ld_vec<T, VX>(pm, st + (size_t)(2 * f + 1) * arr_elems + own);
#pragma unroll
            for (int v = 0; v < VX; ++v) ph[f][v] = fmaT(cd, pm[v], ph[f][v]);
          }
        }
      };

      // FP64 (bound by its arithmetic, not by memory): a site's drifted fields are
      // formed once and written back into its stage, where the next plane reads
      // them as y- and x-neighbours; all threads drift the tile's two halo rows in
      // place; then a proxy fence (bulk copies refill the stage later) and one CTA
      // barrier per plane.  `drifting` is the same in every thread of the CTA.
      constexpr bool SHARE = sizeof(T) == 8;
      const bool share = SHARE && drifting;
      auto share_own = [&](int s, const T (&ph)[NF][VX]) {  // active threads
        T* st = reinterpret_cast<T*>(smem + (size_t)s * P.stage_bytes_max);
#pragma unroll
        for (int f = 0; f < NF; ++f) st_vec<T, VX>(st + (size_t)(2 * f) * arr_elems + own, ph[f]);
      };
      auto share_halo = [&](int s) {  // every thread of the CTA
        if (!flag[0]) {
          T* st = reinterpret_cast<T*>(smem + (size_t)s * P.stage_bytes_max);
          for (int k = tid; k < 2 * N; k += THREADS) {
            const int e = k < N ? k : (BY + 1) * N + (k - N);
#pragma unroll
            for (int f = 0; f < NF; ++f) {
              T* ph = st + (size_t)(2 * f) * arr_elems;
              ph[e] = fmaT(cd, st[(size_t)(2 * f + 1) * arr_elems + e], ph[e]);
            }
          }
          fence_proxy_async_smem();
        }
        __syncthreads();
      };

      // drifted fields of three consecutive planes; the roles below / current /
      // above rotate through b0, b1, b2 (the march is unrolled by three, so the
      // rotation costs no register moves)
      T b0[NF][VX], b1[NF][VX], b2[NF][VX];
      // planes 0 and 1 of the segment
      wait_full(s_cur, p_cur);
      if (active && !flag[0]) read_own(stage_ptr(s_cur), b0);
      release(g0, s_cur);
      advance(s_cur, p_cur);
      wait_full(s_cur, p_cur);
      if (active && !flag[0]) {
        read_own(stage_ptr(s_cur), b1);
        if (share) share_own(s_cur, b1);
      }
      if (share) share_halo(s_cur);
      int s_nxt = s_cur;
      uint32_t p_nxt = p_cur;
      advance(s_nxt, p_nxt);

      // plane j of the segment (stage s_cur), its neighbours below and above
      // (the above plane is read from stage s_nxt into `above`)
      auto plane = [&](int j, const T (&below)[NF][VX], const T (&cur)[NF][VX], T (&above)[NF][VX]) {
        wait_full(s_nxt, p_nxt);
        if (active && !flag[0]) {
          const T* sa = stage_ptr(s_nxt);
          const T* sc = stage_ptr(s_cur);
          read_own(sa, above);
          if (share && j < sg.nz) share_own(s_nxt, above);
          T lap[NF][VX], g2[VX];
#pragma unroll
          for (int v = 0; v < VX; ++v) g2[v] = T(0);
#pragma unroll
          for (int f = 0; f < NF; ++f) {
            const T* ph = sc + (size_t)(2 * f) * arr_elems;
            const T* pm = sc + (size_t)(2 * f + 1) * arr_elems;
            T yl[VX], yh[VX];
            ld_vec<T, VX>(yl, ph + ty * N + x0);
            ld_vec<T, VX>(yh, ph + (ty + 2) * N + x0);
            if (drifting && !SHARE) {
              T ml[VX], mh[VX];
              ld_vec<T, VX>(ml, pm + ty * N + x0);
              ld_vec<T, VX>(mh, pm + (ty + 2) * N + x0);
#pragma unroll
              for (int v = 0; v < VX; ++v) {
                yl[v] = fmaT(cd, ml[v], yl[v]);
                yh[v] = fmaT(cd, mh[v], yh[v]);
              }
            }
            // x-neighbours beyond this thread's sites, read from the stage and
            // drifted like the owner's copy (no shuffle, no divergent edge branch)
            const T left = drifting && !SHARE ? fmaT(cd, pm[exl], ph[exl]) : ph[exl];
            const T right = drifting && !SHARE ? fmaT(cd, pm[exr], ph[exr]) : ph[exr];
            T gf = T(0);
#pragma unroll
            for (int v = 0; v < VX; ++v) {
              const T c = cur[f][v];
              const T xl = v == 0 ? left : cur[f][v - 1];
              const T xr = v == VX - 1 ? right : cur[f][v + 1];
              const T zl = below[f][v], zh = above[f][v];
              if constexpr (sizeof(T) == 8) {
                // FP64: the six neighbours summed, then -6 c in one FMA (the fewest
                // operations on the narrow FP64 pipe); FP32 keeps each direction's
                // small difference from its own pair sum
                lap[f][v] = fmaT(T(-6), c, ((xl + xr) + (yl[v] + yh[v])) + (zl + zh));
              } else {
                lap[f][v] = ((xl + xr) - T(2) * c) + ((yl[v] + yh[v]) - T(2) * c) +
                            ((zl + zh) - T(2) * c);
              }
              if (RED == 2) {  // forward differences (eq. EK_EG_EV with grad^+)
                const T zp = sg.dir > 0 ? zh : zl;
                const T gx = xr - c, gy = yh[v] - c, gz = zp - c;
                gf += gx * gx + gy * gy + gz * gz;
              } else if (RED == 1) {
                // sum_n (grad^+ phi)^2 = -sum_n phi Lap phi (summation by parts on the
                // periodic lattice): one FMA on the Laplacian the kick needs anyway
                g2[v] = fmaT(c, lap[f][v], g2[v]);
              }
            }
            if (RED == 2) acc[6 * f + 2].add(gf);
          }
          T pn[NF][VX], pic[NF][VX];  // momenta of the current plane, from its stage
#pragma unroll
          for (int f = 0; f < NF; ++f) ld_vec<T, VX>(pic[f], sc + (size_t)(2 * f + 1) * arr_elems + own);
          T spost = T(0), vs = T(0), gsum = T(0);
#pragma unroll
          for (int v = 0; v < VX; ++v) {
            T fv[NF], dv[NF], tv[NPOT];
#pragma unroll
            for (int f = 0; f < NF; ++f) fv[f] = cur[f][v];
            ScalarPot<NF>::eval(fv, q, dv, tv);
#pragma unroll
            for (int f = 0; f < NF; ++f) {
              // FP32 adds the small increment last (one rounding at the momentum's
              // size); FP64 takes two FMAs
              if constexpr (sizeof(T) == 8)
                pn[f][v] = fmaT(-A3, dv[f], fmaT(A1, lap[f][v], pic[f][v]));
              else
                pn[f][v] = pic[f][v] + (A1 * lap[f][v] - A3 * dv[f]);
            }
            if (RED == 1) {
#pragma unroll
              for (int f = 0; f < NF; ++f) spost = fmaT(pn[f][v], pn[f][v], spost);
              vs += ScalarPot<NF>::total(fv, hq);
              gsum += g2[v];
            } else if (RED == 2) {
#pragma unroll
              for (int f = 0; f < NF; ++f) {
                acc[6 * f + 0].add(pic[f][v] * pic[f][v]);
                acc[6 * f + 1].add(pn[f][v] * pn[f][v]);
                acc[6 * f + 3].add(fv[f]);
                acc[6 * f + 4].add(fv[f] * fv[f]);
                acc[6 * f + 5].add(pn[f][v]);
                if (!isfinite(pn[f][v])) nonfinite += 1.f;
              }
#pragma unroll
              for (int t = 0; t < NPOT; ++t) acc[6 * NF + t].add(tv[t]);
            }
          }
          if (RED == 1) {
            acc[0].add(spost);
            acc[1].add(gsum);
            acc[2].add(vs);
          }
          if (P.write) {
            const long long gi = (long long)seg_plane_z(sg, N, j) * NN + (long long)y * N + x0;
#pragma unroll
            for (int f = 0; f < NF; ++f) {
              st_vec<T, VX>(dst[2 * f] + gi, cur[f]);
              st_vec<T, VX>(dst[2 * f + 1] + gi, pn[f]);
            }
          }
        }
        if (share && j < sg.nz) share_halo(s_nxt);
        release(g0 + j, s_cur);
        s_cur = s_nxt;
        p_cur = p_nxt;
        advance(s_nxt, p_nxt);
      };
      for (int j = 1; j <= sg.nz; j += 3) {
        plane(j, b0, b1, b2);
        if (j + 1 > sg.nz) break;
        plane(j + 1, b1, b2, b0);
        if (j + 2 > sg.nz) break;
        plane(j + 2, b2, b0, b1);
      }
      release(g0 + sg.nz + 1, s_cur);
      advance(s_cur, p_cur);

      if (!run_end) continue;

      // ---- end of this CTA's run on the lattice: flush the sums into its slot ----
      // (two halves of red[] alternate: a warp can reach the next flush while
      // others still read this one, but not the one after, which waits for all)
      double* rb = red + fbuf * CONSUMER_WARPS * NQ;
      fbuf ^= 1;
      if (RED > 0) {
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
          if (lane == 0) rb[warp * NQ + k] = v;
        }
      }
#pragma unroll
      for (int k = 0; k < NACC; ++k) acc[k].zero();
      nonfinite = 0.f;
      __syncthreads();
      if (flag[0]) goto timeout;
      // warp k: fixed shuffle tree over the 16 warp partials of quantity k, the
      // slot's value, and one arrival on the lattice's count (no further block
      // barrier: the next segment starts at once); the arrival that completes
      // the count queues the lattice's tail
      if (warp < NARRIVE) {
        double v = 0.0;
        if (NUSED > 0) {
          v = lane < CONSUMER_WARPS ? rb[lane * NQ + warp] : 0.0;
#pragma unroll
          for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
        }
        if (lane == 0) {
          if (NUSED > 0) P.partials[(size_t)warp * P.nslot + sg.slot] = v;
          __threadfence();
          const unsigned nslot = (unsigned)(L.slot_end - L.slot_begin);
          const unsigned prev = atomicAdd(&P.counters[sg.lat], 1u);
          if (prev == NARRIVE * nslot - 1u) pend[atomicAdd(const_cast<int*>(&flag[3]), 1)] = sg.lat;
        }
      }
      if (tid == 0) flag[2] = sg.lat;
    }

    // ---- end of the pass ----
    __syncthreads();  // every warp's writes and arrivals of the pass are done
    if (multi && tid == 0) {  // this CTA's writes are done
      __threadfence();
      fence_proxy_async_global();
      atomicAdd(&P.gsync[0], 1u);
    }
    {
      const int npend = flag[3];
      const PassStep pst = P.steps ? P.steps[pass] : PassStep{P.ck, P.wout, P.win, P.dnext};
      for (int base = 0; base < npend; base += 32) {
        __threadfence();
        run_tails(base, min(32, npend - base), pst, P.log ? P.log + ADJ_LOG_W * (P.log_base + pass) : nullptr);
      }
      __syncthreads();
      if (tid == 0) flag[3] = 0;
    }
  }
  return;

timeout:
  // A bounded wait gave up: record it, wait (bounded) for copies still in
  // flight so that none lands in shared memory after exit, and leave.
  if (tid == 0) {
    for (int s = 0; s < S; ++s)
      for (int par = 0; par < 2; ++par) mbar_wait_bounded(&full[s], (uint32_t)par, 1000000ull);
    P.sc[flag[2]].status = CL_ETIMEOUT;
  }
  __syncthreads();
}

// Explicit instantiations, looked up by the host launcher.
template __global__ void dk_pass_scalar<float, 1, 0>(const PassArgs);
template __global__ void dk_pass_scalar<float, 1, 1>(const PassArgs);
template __global__ void dk_pass_scalar<float, 1, 2>(const PassArgs);
template __global__ void dk_pass_scalar<float, 2, 0>(const PassArgs);
template __global__ void dk_pass_scalar<float, 2, 1>(const PassArgs);
template __global__ void dk_pass_scalar<float, 2, 2>(const PassArgs);
template __global__ void dk_pass_scalar<double, 1, 0>(const PassArgs);
template __global__ void dk_pass_scalar<double, 1, 1>(const PassArgs);
template __global__ void dk_pass_scalar<double, 1, 2>(const PassArgs);
template __global__ void dk_pass_scalar<double, 2, 0>(const PassArgs);
template __global__ void dk_pass_scalar<double, 2, 1>(const PassArgs);
template __global__ void dk_pass_scalar<double, 2, 2>(const PassArgs);

typedef void (*PassKernel)(const PassArgs);

PassKernel scalar_pass_kernel(int fp32, int nf, int red) {
  static const PassKernel tab[2][2][3] = {
      {{dk_pass_scalar<double, 1, 0>, dk_pass_scalar<double, 1, 1>, dk_pass_scalar<double, 1, 2>},
       {dk_pass_scalar<double, 2, 0>, dk_pass_scalar<double, 2, 1>, dk_pass_scalar<double, 2, 2>}},
      {{dk_pass_scalar<float, 1, 0>, dk_pass_scalar<float, 1, 1>, dk_pass_scalar<float, 1, 2>},
       {dk_pass_scalar<float, 2, 0>, dk_pass_scalar<float, 2, 1>, dk_pass_scalar<float, 2, 2>}}};
  if (nf < 1 || nf > 2 || red < 0 || red > 2) return nullptr;
  return tab[fp32 ? 1 : 0][nf - 1][red];
}

}  // namespace clg
