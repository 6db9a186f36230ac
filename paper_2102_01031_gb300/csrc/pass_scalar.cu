// pass_scalar.cu -- fused drift + kick pass for real scalar singlets
// (CosmoLattice manual, Sec. 3.5.2, Hamiltonian form):
//
//   drift (deferred from the previous pass):  phi += cd * pi,   cd = h abar^{alpha-3}
//   kick:   pi += c_k [ a^{1+alpha} Lap phi - a^{3+alpha} V_{,phi} ]
//   Lap phi = sum_i [phi(n+i) - 2 phi(n) + phi(n-i)] / dx^2       (eq. neutrald/forwardbackwardd)
//   sums:   sum pi^2 before / after the kick, sum_i (grad^+_i phi)^2, sum V, means
//
// One pass per integrator stage: each field and momentum array is read once
// from HBM and written once.  A CTA owns a tile of BY full x-rows and marches
// along z over a run of planes ("segment"); every plane tile (with one halo
// row on each side in y) of every array arrives in shared memory by 1-D bulk
// async copies (TMA) into a ring of stages, completion tracked by mbarriers.
// The drift is applied in shared memory, z-neighbours live in registers, y
// neighbours come from the stage, x neighbours from warp shuffles.  Partial
// sums go to one slot per segment; the last segment of a lattice to finish
// reduces them in a fixed order and runs the Friedmann update (tail.cuh).
#include "common.cuh"
#include "tail.cuh"

namespace clg {

// Program potentials (eq. PotNat): NF = 1: phi^4/4; NF = 2: phi^4/4 + (q/2) phi^2 chi^2.
template <int NF> struct ScalarPot;
template <> struct ScalarPot<1> {
  static constexpr int NPOT = 1;
  template <typename T>
  __device__ __forceinline__ static void eval(const T (&f)[1], T q, T (&d)[1], T (&t)[1]) {
    const T f2 = f[0] * f[0];
    d[0] = f2 * f[0];
    t[0] = T(0.25) * f2 * f2;
  }
};
template <> struct ScalarPot<2> {
  static constexpr int NPOT = 2;
  template <typename T>
  __device__ __forceinline__ static void eval(const T (&f)[2], T q, T (&d)[2], T (&t)[2]) {
    const T p2 = f[0] * f[0], c2 = f[1] * f[1];
    d[0] = p2 * f[0] + q * f[0] * c2;
    d[1] = q * p2 * f[1];
    t[0] = T(0.25) * p2 * p2;
    t[1] = T(0.5) * q * p2 * c2;
  }
};

// RED: 0 = no sums, 1 = sums for the Friedmann kick, 2 = full measurement.
template <typename T, int NF, int RED>
__global__ void __launch_bounds__(THREADS, 1) dk_pass_scalar(const PassArgs P) {
  constexpr int VX = V16<T>::n;
  constexpr int NA = 2 * NF;
  constexpr int NPOT = ScalarPot<NF>::NPOT;
  constexpr int NACC = RED == 0 ? 1 : (RED == 1 ? 4 : 6 * NF + NPOT);
  typedef typename V16<T>::type VT;

  extern __shared__ __align__(128) unsigned char smem[];
  const int S = P.stages;
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem + (size_t)S * P.stage_bytes_max);
  double* red = reinterpret_cast<double*>(bar + 8);  // [33][NQ]
  volatile int* flag = reinterpret_cast<volatile int*>(red + 33 * NQ);
  const int tid = threadIdx.x, lane = tid & 31;

  if (tid == 0) {
    for (int s = 0; s < S; ++s) mbar_init(&bar[s], 1);
    fence_mbar_init();
    flag[0] = 0;
    flag[1] = 0;
  }
  __syncthreads();

  unsigned long long jg = 0;  // planes consumed by this CTA so far: stage/phase bookkeeping
  const int seg_end = P.cta_seg[blockIdx.x + 1];
  for (int si = P.cta_seg[blockIdx.x]; si < seg_end; ++si) {
    const Seg sg = P.segs[si];
    const LatConst& L = P.lat[sg.lat];
    if (tid == 0) flag[2] = sg.lat;
    const int N = L.N, BY = L.BY, TX = N / VX;
    const int tx = tid % TX, ty = tid / TX;
    const bool active = ty < BY;
    const unsigned amask = __ballot_sync(0xffffffffu, active);  // active threads are 0 .. TX*BY-1
    const int x0 = tx * VX;
    const int ylo = sg.ytile * BY, y = ylo + ty;
    const LatScalars& SC = P.sc[sg.lat];
    const double dx = L.dx;
    const T cd = (T)SC.cd;
    const T A1 = (T)(P.ck * SC.apow1 / (dx * dx));
    const T A3 = (T)(P.ck * SC.apow3);
    const T q = (T)L.q;
    const int rows = BY + 2;
    const int arr_elems = rows * N;
    const int nplanes = sg.nz + 2;
    const long long NN = (long long)N * N;
    const T* src[NA];
    T* dst[NA];
#pragma unroll
    for (int a = 0; a < NA; ++a) {
      src[a] = reinterpret_cast<const T*>(L.buf[P.parity][a]);
      dst[a] = reinterpret_cast<T*>(L.buf[P.parity ^ 1][a]);
    }
    auto plane_z = [&](int j) -> int {
      int z = sg.dir > 0 ? sg.z0 - 1 + j : sg.z0 + sg.nz - j;
      z %= N;
      return z < 0 ? z + N : z;
    };
    auto stage = [&](int j) -> T* {
      return reinterpret_cast<T*>(smem + (size_t)((jg + j) % S) * P.stage_bytes_max);
    };
    auto issue = [&](int j) {  // thread 0 only
      T* st = stage(j);
      uint64_t* b = &bar[(jg + j) % S];
      const long long zoff = (long long)plane_z(j) * NN;
      mbar_arrive_expect_tx(b, (uint32_t)((size_t)NA * arr_elems * sizeof(T)));
      int r = 0;
      while (r < rows) {
        int g = ylo - 1 + r;
        g = g < 0 ? g + N : (g >= N ? g - N : g);
        int run = 1;
        while (r + run < rows && g + run < N) ++run;
#pragma unroll
        for (int a = 0; a < NA; ++a)
          bulk_g2s(st + (size_t)a * arr_elems + (size_t)r * N, src[a] + zoff + (long long)g * N,
                   (uint32_t)(run * N * sizeof(T)), b);
        r += run;
      }
    };
    auto wait = [&](int j) {
      uint64_t* b = &bar[(jg + j) % S];
      const uint32_t par = (uint32_t)(((jg + j) / S) & 1ull);
      if (!mbar_wait_bounded(b, par, P.wait_limit_ns)) flag[0] = 1;
    };
    auto drift = [&](int j) {  // phi += cd * pi over the whole stage, in shared memory
      if (cd == T(0)) return;
      T* st = stage(j);
#pragma unroll
      for (int f = 0; f < NF; ++f) {
        T* ph = st + (size_t)(2 * f) * arr_elems;
        const T* pm = st + (size_t)(2 * f + 1) * arr_elems;
        for (int e = tid * VX; e < arr_elems; e += blockDim.x * VX) {
          T p[VX], m[VX];
          *reinterpret_cast<VT*>(p) = *reinterpret_cast<const VT*>(ph + e);
          *reinterpret_cast<VT*>(m) = *reinterpret_cast<const VT*>(pm + e);
#pragma unroll
          for (int v = 0; v < VX; ++v) p[v] = fma(cd, m[v], p[v]);
          *reinterpret_cast<VT*>(ph + e) = *reinterpret_cast<VT*>(p);
        }
      }
    };

    // prologue
    if (tid == 0) {
      fence_proxy_async_smem();
      const int npre = nplanes < S ? nplanes : S;
      for (int j = 0; j < npre; ++j) issue(j);
    }
    wait(0);
    wait(1);
    drift(0);
    drift(1);
    __syncthreads();
    if (flag[0]) goto timeout;

    {
      T below[NF][VX], cur[NF][VX], above[NF][VX], pic[NF][VX], pia[NF][VX];
      Acc<T> acc[NACC];
      float nonfinite = 0.f;
#pragma unroll
      for (int k = 0; k < NACC; ++k) acc[k].zero();
      if (active) {
        const T* s0 = stage(0);
        const T* s1 = stage(1);
        const int own = (ty + 1) * N + x0;
#pragma unroll
        for (int f = 0; f < NF; ++f) {
          *reinterpret_cast<VT*>(below[f]) =
              *reinterpret_cast<const VT*>(s0 + (size_t)(2 * f) * arr_elems + own);
          *reinterpret_cast<VT*>(cur[f]) =
              *reinterpret_cast<const VT*>(s1 + (size_t)(2 * f) * arr_elems + own);
          *reinterpret_cast<VT*>(pic[f]) =
              *reinterpret_cast<const VT*>(s1 + (size_t)(2 * f + 1) * arr_elems + own);
        }
      }

      for (int j = 1; j <= sg.nz; ++j) {
        wait(j + 1);
        drift(j + 1);
        __syncthreads();
        if (flag[0]) goto timeout;
        if (tid == 0 && j - 1 + S < nplanes) {
          fence_proxy_async_smem();
          issue(j - 1 + S);
        }
        if (active) {
          const T* sa = stage(j + 1);
          const T* sc = stage(j);
          const int own = (ty + 1) * N + x0;
#pragma unroll
          for (int f = 0; f < NF; ++f) {
            *reinterpret_cast<VT*>(above[f]) =
                *reinterpret_cast<const VT*>(sa + (size_t)(2 * f) * arr_elems + own);
            *reinterpret_cast<VT*>(pia[f]) =
                *reinterpret_cast<const VT*>(sa + (size_t)(2 * f + 1) * arr_elems + own);
          }
          T lap[NF][VX], g2[VX];
#pragma unroll
          for (int v = 0; v < VX; ++v) g2[v] = T(0);
#pragma unroll
          for (int f = 0; f < NF; ++f) {
            const T* ph = sc + (size_t)(2 * f) * arr_elems;
            T yl[VX], yh[VX];
            *reinterpret_cast<VT*>(yl) = *reinterpret_cast<const VT*>(ph + ty * N + x0);
            *reinterpret_cast<VT*>(yh) = *reinterpret_cast<const VT*>(ph + (ty + 2) * N + x0);
            T left = __shfl_up_sync(amask, cur[f][VX - 1], 1);
            T right = __shfl_down_sync(amask, cur[f][0], 1);
            if (tx == 0 || lane == 0) left = ph[(ty + 1) * N + (x0 == 0 ? N - 1 : x0 - 1)];
            if (tx == TX - 1 || lane == 31)
              right = ph[(ty + 1) * N + (x0 + VX == N ? 0 : x0 + VX)];
#pragma unroll
            for (int v = 0; v < VX; ++v) {
              const T c = cur[f][v];
              const T xl = v == 0 ? left : cur[f][v - 1];
              const T xr = v == VX - 1 ? right : cur[f][v + 1];
              const T zl = below[f][v], zh = above[f][v];
              lap[f][v] = ((xl + xr) - T(2) * c) + ((yl[v] + yh[v]) - T(2) * c) +
                          ((zl + zh) - T(2) * c);
              if (RED > 0) {
                const T zp = sg.dir > 0 ? zh : zl;
                const T gx = xr - c, gy = yh[v] - c, gz = zp - c;
                const T gg = gx * gx + gy * gy + gz * gz;
                if (RED == 2) acc[6 * f + 2].add(gg);
                else g2[v] += gg;
              }
            }
          }
          T pn[NF][VX];
#pragma unroll
          for (int v = 0; v < VX; ++v) {
            T fv[NF], dv[NF], tv[NPOT];
#pragma unroll
            for (int f = 0; f < NF; ++f) fv[f] = cur[f][v];
            ScalarPot<NF>::eval(fv, q, dv, tv);
#pragma unroll
            for (int f = 0; f < NF; ++f) pn[f][v] = pic[f][v] + (A1 * lap[f][v] - A3 * dv[f]);
            if (RED == 1) {
              T spre = T(0), spost = T(0), vs = T(0);
#pragma unroll
              for (int f = 0; f < NF; ++f) {
                spre += pic[f][v] * pic[f][v];
                spost += pn[f][v] * pn[f][v];
                if (!isfinite(pn[f][v])) nonfinite += 1.f;
              }
#pragma unroll
              for (int t = 0; t < NPOT; ++t) vs += tv[t];
              acc[0].add(spre);
              acc[1].add(spost);
              acc[2].add(g2[v]);
              acc[3].add(vs);
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
          if (P.write) {
            const long long gi = (long long)plane_z(j) * NN + (long long)y * N + x0;
#pragma unroll
            for (int f = 0; f < NF; ++f) {
              *reinterpret_cast<VT*>(dst[2 * f] + gi) = *reinterpret_cast<VT*>(cur[f]);
              *reinterpret_cast<VT*>(dst[2 * f + 1] + gi) = *reinterpret_cast<VT*>(pn[f]);
            }
          }
#pragma unroll
          for (int f = 0; f < NF; ++f)
#pragma unroll
            for (int v = 0; v < VX; ++v) {
              below[f][v] = cur[f][v];
              cur[f][v] = above[f][v];
              pic[f][v] = pia[f][v];
            }
        }
      }
      jg += (unsigned long long)nplanes;

      // segment partial sums -> slot si; last segment of the lattice runs the tail
      double vals[NQ];
#pragma unroll
      for (int k = 0; k < NQ; ++k) vals[k] = 0.0;
      if (RED > 0) {
#pragma unroll
        for (int k = 0; k < NACC; ++k) vals[k] = acc[k].value();
        vals[NQ - 1] = (double)nonfinite;
      }
      block_reduce_nq(vals, red);
      if (tid < NQ) {
        P.partials[(size_t)si * NQ + tid] = red[32 * NQ + tid];
        __threadfence();
      }
      __syncthreads();
      if (tid == 0) {
        const unsigned nseg = (unsigned)(L.seg_end - L.seg_begin);
        const unsigned prev = atomicAdd(&P.counters[sg.lat], 1u);
        flag[1] = (prev == nseg - 1u) ? 1 : 0;
      }
      __syncthreads();
      if (flag[1]) {
        __threadfence();
        if (tid < NQ) {
          double s = 0.0;
          for (int k = L.seg_begin; k < L.seg_end; ++k) s += __ldcg(&P.partials[(size_t)k * NQ + tid]);
          red[32 * NQ + tid] = s;
        }
        __syncthreads();
        if (tid == 0) {
          LatScalars& W = P.sc[sg.lat];
          const double* sum = red + 32 * NQ;
          const double a = W.a, V = (double)L.V;
          const double a2 = a * a, a6 = a2 * a2 * a2;
          PassSums E = {0, 0, 0, 0, 0, 0, 0};
          if (RED > 0) {
            double spre = 0, spost = 0, gg = 0, vs = 0;
            if (RED == 1) {
              spre = sum[0]; spost = sum[1]; gg = sum[2]; vs = sum[3];
            } else {
              for (int f = 0; f < NF; ++f) {
                spre += sum[6 * f]; spost += sum[6 * f + 1]; gg += sum[6 * f + 2];
              }
              for (int t = 0; t < NPOT; ++t) vs += sum[6 * NF + t];
            }
            E.EKpre = spre / (2.0 * a6 * V);
            E.EKpost = spost / (2.0 * a6 * V);
            E.EG = gg / (2.0 * a2 * dx * dx * V);
            E.EV = vs / V;
          }
          advance_scalars(P, L, W, E, RED > 0);
          if (RED == 2) {
            cl_energies_t& o = W.obs;
            for (int k = 0; k < 4; ++k) {
              o.EK[k] = o.EG[k] = o.EV[k] = 0.0;
              o.mean_phi[k] = o.mean_phi2[k] = o.mean_pi[k] = o.mean_pi2[k] = 0.0;
            }
            o.EKA = o.EGA = 0.0;
            for (int f = 0; f < NF; ++f) {
              o.EK[f] = sum[6 * f + 1] / (2.0 * a6 * V);
              o.EG[f] = sum[6 * f + 2] / (2.0 * a2 * dx * dx * V);
              o.mean_phi[f] = sum[6 * f + 3] / V;
              o.mean_phi2[f] = sum[6 * f + 4] / V;
              o.mean_pi[f] = sum[6 * f + 5] / V;
              o.mean_pi2[f] = sum[6 * f + 1] / V;
            }
            for (int t = 0; t < NPOT; ++t) o.EV[t] = sum[6 * NF + t] / V;
            o.nonfinite = (int64_t)sum[NQ - 1];
            finish_obs(P, L, W);
          }
          advance_drift(P, L, W);
          P.counters[sg.lat] = 0u;
        }
      }
      __syncthreads();
    }
  }
  return;

timeout:
  // A bounded wait gave up: record it, wait (bounded) for this CTA's copies
  // in flight so that no bulk copy targets freed shared memory, and leave.
  if (tid == 0) {
    for (int s = 0; s < S; ++s)
      for (int par = 0; par < 2; ++par) mbar_wait_bounded(&bar[s], (uint32_t)par, 1000000ull);
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
