// pass_adjoint.cu -- one reversed DK pass fused with its adjoint, for the
// gradient of a final observable (scalar models).
//
// Forward pass (Sec. 3.5.2, Hamiltonian form; see pass_scalar.cu):
//     drift  a_k = a_{k-1} + w b,  phi' = phi + cd pi,  cd = w abar^{alpha-3}
//     kick   pi' = pi + F(phi'),   F_f = A1 Lap phi_f - A3 dV/dphi_f
// with A1 = c_k a_k^{1+alpha}/dx^2, A3 = c_k a_k^{3+alpha}, and, with
// self-consistent expansion, the Friedmann kicks b += w_out K_a(pi) before
// and b += w_in K_a(pi') after the field kick.  From the pass's output
// (phi', pi') and the adjoint (lam_phi', lam_pi', lam_a, lam_b) = dJ/d(phi', pi', a, b)
// this kernel computes, site by site,
//     pi  = pi' - F(phi'),   phi = phi' - cd pi                  (the state before the pass)
//     l'  = lam_pi' + lam_b w_in dK_a/dpi' = lam_pi' + b_post pi'
//     mu_f = lam_phi'_f + A1 Lap l'_f - A3 sum_g V_{,fg}(phi') l'_g
//            + lam_b (w_in + w_out) dK_a/dphi_f = ... + b_phi Lap phi'_f + b_V dV/dphi_f
//     l    = l' + lam_b w_out dK_a/dpi = l' + b_pre pi
//     lam_phi = mu,   lam_pi = l + cd mu                           (dJ/d(phi, pi))
// and the lattice sums
//     Q0 = sum_f l'_f (-A3) d(dV/dphi_f)/dq + b_V dV/dq           (dJ/dq)
//     Q1 = sum_f l'_f Lap phi'_f,  Q2 = sum_f l'_f dV/dphi_f,  Q3 = sum_f mu_f pi_f
// from which the pass's tail updates the scale-factor adjoints:
//     lam_a(k) = lam_a + lam_b dKa + [(1+alpha) A1 Q1 - (3+alpha) A3 Q2]/a_k
//     lam_a   <- lam_a(k) + Q3 cab,   lam_b <- lam_b + w lam_a(k) + (w/2) Q3 cab
// (cab = w (alpha-3) abar^{alpha-4}; dKa = the a-derivative of the two
// Friedmann kicks, recorded by the forward run).  On a fixed background the
// b_* terms, Q1..Q3 and the scalar adjoints are absent (kernel variant SELF =
// false).  The Laplacian is symmetric, so the transposed kick applies it to
// l'.  Each array crosses HBM once each way: the pass reads the state and the
// adjoint (4 NF arrays) and writes both, twice the bytes of a forward pass.
//
// Coefficients of reversed pass r at P.adj + ADJ_COEF_W r:
//   0 cd, 1 c_k, 2 A1, 3 A3, then (self-consistent expansion only; b_* = lam_b g_*)
//   4 g_post, 5 g_pre, 6 g_phi, 7 g_V, 8 1/a_k, 9 dKa, 10 cab, 11 w.
//
// Same plane ring as the forward passes (ring.cuh): the stage holds
// phi'_f, pi'_f (arrays 2f, 2f+1) and lam_phi'_f, lam_pi'_f (2NF + 2f, 2NF + 2f + 1).
#include "common.cuh"
#include "ring.cuh"
#include "tail.cuh"

namespace clg {

namespace {

// Potential (eq. PotNat) of the scalar models: dV/dphi, the Hessian, and
// d(dV/dphi)/dq at one site; vq = dV/dq.
template <int NF> struct AdjPot;
template <> struct AdjPot<1> {
  template <typename T>
  __device__ __forceinline__ static void eval(const T (&f)[1], T q, T (&d)[1], T (&H)[1][1], T (&dq)[1]) {
    const T f2 = f[0] * f[0];
    d[0] = f2 * f[0];
    H[0][0] = T(3) * f2;
    dq[0] = T(0);
  }
  template <typename T>
  __device__ __forceinline__ static T vq(const T (&f)[1]) {
    return T(0);
  }
};
template <> struct AdjPot<2> {
  template <typename T>
  __device__ __forceinline__ static void eval(const T (&f)[2], T q, T (&d)[2], T (&H)[2][2], T (&dq)[2]) {
    const T p2 = f[0] * f[0], c2 = f[1] * f[1], pc = f[0] * f[1];
    d[0] = p2 * f[0] + q * f[0] * c2;
    d[1] = q * p2 * f[1];
    H[0][0] = T(3) * p2 + q * c2;
    H[0][1] = H[1][0] = T(2) * q * pc;
    H[1][1] = q * p2;
    dq[0] = f[0] * c2;
    dq[1] = p2 * f[1];
  }
  template <typename T>
  __device__ __forceinline__ static T vq(const T (&f)[2]) {
    return T(0.5) * (f[0] * f[0]) * (f[1] * f[1]);
  }
};

template <typename T, int VX>
__device__ __forceinline__ void ld_v(T (&v)[VX], const T* p) {
  *reinterpret_cast<typename V16<T>::type*>(v) = *reinterpret_cast<const typename V16<T>::type*>(p);
}
template <typename T, int VX>
__device__ __forceinline__ void st_v(T* p, const T (&v)[VX]) {
  *reinterpret_cast<typename V16<T>::type*>(p) = *reinterpret_cast<const typename V16<T>::type*>(v);
}

}  // namespace

template <typename T, int NF, bool SELF>
__global__ void __launch_bounds__(THREADS, 1) adj_pass_scalar(const PassArgs P) {
  constexpr int VX = V16<T>::n;
  constexpr int NA = 4 * NF;
  constexpr int LF = 2 * NF;  // first adjoint array
  constexpr int NACC = SELF ? 4 : 1;

  extern __shared__ __align__(128) unsigned char smem[];
  const Ring R = ring_view(smem, P);
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int sb = P.cta_seg[blockIdx.x], ns = P.cta_seg[blockIdx.x + 1] - sb;
  const bool multi = P.npass > 1;
  if (tid == 0) ring_setup<NA>(R, P, sb, ns);
  __syncthreads();
  const int ptot = R.off[ns];
  const int S = R.S;

  int s_cur = 0;
  uint32_t p_cur = 0u;
  Acc<T> acc[NACC];
  float nonfinite = 0.f;
#pragma unroll
  for (int k = 0; k < NACC; ++k) acc[k].zero();

  for (int pass = 0; pass < P.npass; ++pass) {
    const int parity = P.parity ^ (pass & 1);
    const double* cfp = P.adj + ADJ_COEF_W * pass;
    if (warp == 0) ring_pass_start<T, NA>(R, P, pass, ptot, parity, lane);
    __syncthreads();
    if (R.flag[0]) goto timeout;

    for (int i = 0; i < ns; ++i) {
      const Seg sg = P.segs[sb + i];
      const LatConst& L = P.lat[sg.lat];
      const int N = L.N, BY = L.BY, TX = N / VX;
      const int tx = tid % TX, ty = tid / TX;
      const bool active = ty < BY;
      const int x0 = tx * VX;
      const int y = sg.ytile * BY + ty;
      const int ae = (BY + 2) * N;
      const long long NN = (long long)N * N;
      const int g0 = R.off[i];
      const T cd = (T)__ldg(cfp), A1 = (T)__ldg(cfp + 2), A3 = (T)__ldg(cfp + 3);
      const T q = (T)L.q;
      // lam_b-scaled Friedmann-kick coefficients (lam_b is set by the previous reversed pass)
      T bpost = T(0), bpre = T(0), bphi = T(0), bV = T(0);
      if (SELF) {
        const double lb = __ldcg(&P.sc[sg.lat].adjb);
        bpost = (T)(lb * __ldg(cfp + 4));
        bpre = (T)(lb * __ldg(cfp + 5));
        bphi = (T)(lb * __ldg(cfp + 6));
        bV = (T)(lb * __ldg(cfp + 7));
      }
      const int xl = x0 == 0 ? N - 1 : x0 - 1, xr = x0 + VX == N ? 0 : x0 + VX;
      const int own = (ty + 1) * N + x0;

      // phi' and l' = lam_pi' + b_post pi' (the Laplacian inputs) at the centre of planes j-1, j, j+1
      T bF[NF][VX], cF[NF][VX], aF[NF][VX], bL[NF][VX], cL[NF][VX], aL[NF][VX];
      auto centre = [&](const T* st, T (&f)[NF][VX], T (&l)[NF][VX]) {
#pragma unroll
        for (int k = 0; k < NF; ++k) {
          ld_v<T, VX>(f[k], st + (2 * k) * ae + own);
          ld_v<T, VX>(l[k], st + (LF + 2 * k + 1) * ae + own);
          if (SELF) {
            T pv[VX];
            ld_v<T, VX>(pv, st + (2 * k + 1) * ae + own);
#pragma unroll
            for (int v = 0; v < VX; ++v) l[k][v] = fmaT(bpost, pv[v], l[k][v]);
          }
        }
      };
      ring_wait(R, s_cur, p_cur, P.wait_limit_ns);
      if (active && !R.flag[0]) centre(ring_stage<T>(R, s_cur), bF, bL);
      ring_release<T, NA>(R, g0, s_cur, parity, ptot, lane);
      ring_advance(S, s_cur, p_cur);
      ring_wait(R, s_cur, p_cur, P.wait_limit_ns);
      if (active && !R.flag[0]) centre(ring_stage<T>(R, s_cur), cF, cL);
      int s_nxt = s_cur;
      uint32_t p_nxt = p_cur;
      ring_advance(S, s_nxt, p_nxt);

      for (int j = 1; j <= sg.nz; ++j) {
        ring_wait(R, s_nxt, p_nxt, P.wait_limit_ns);
        if (active && !R.flag[0]) {
          const T* sa = ring_stage<T>(R, s_nxt);
          const T* sc = ring_stage<T>(R, s_cur);
          centre(sa, aF, aL);
          // Laplacians of phi' and l'
          T lapF[NF][VX], lapL[NF][VX];
#pragma unroll
          for (int k = 0; k < NF; ++k) {
#pragma unroll
            for (int m = 0; m < 2; ++m) {
              const int arr = m == 0 ? 2 * k : LF + 2 * k + 1;
              const T* base = sc + arr * ae;
              T (&c)[VX] = m == 0 ? cF[k] : cL[k];
              T (&b)[VX] = m == 0 ? bF[k] : bL[k];
              T (&a)[VX] = m == 0 ? aF[k] : aL[k];
              T (&out)[VX] = m == 0 ? lapF[k] : lapL[k];
              T yl[VX], yh[VX];
              ld_v<T, VX>(yl, base + ty * N + x0);
              ld_v<T, VX>(yh, base + (ty + 2) * N + x0);
              // x-neighbours beyond the thread's sites, straight from the stage
              T left = base[(ty + 1) * N + xl];
              T right = base[(ty + 1) * N + xr];
              if (SELF && m == 1) {  // l' = lam_pi' + b_post pi' at the in-plane neighbours
                const T* pb = sc + (2 * k + 1) * ae;
                T pl[VX], ph[VX];
                ld_v<T, VX>(pl, pb + ty * N + x0);
                ld_v<T, VX>(ph, pb + (ty + 2) * N + x0);
#pragma unroll
                for (int v = 0; v < VX; ++v) {
                  yl[v] = fmaT(bpost, pl[v], yl[v]);
                  yh[v] = fmaT(bpost, ph[v], yh[v]);
                }
                left = fmaT(bpost, pb[(ty + 1) * N + xl], left);
                right = fmaT(bpost, pb[(ty + 1) * N + xr], right);
              }
#pragma unroll
              for (int v = 0; v < VX; ++v) {
                const T cv = c[v];
                const T xm = v == 0 ? left : c[v - 1];
                const T xp = v == VX - 1 ? right : c[v + 1];
                out[v] = ((xm + xp) - T(2) * cv) + ((yl[v] + yh[v]) - T(2) * cv) + ((b[v] + a[v]) - T(2) * cv);
              }
            }
          }
          T npi[NF][VX], nphi[NF][VX], nlf[NF][VX], nlp[NF][VX];
          T dqs = T(0), vqs = T(0), s1 = T(0), s2 = T(0), s3 = T(0);
#pragma unroll
          for (int v = 0; v < VX; ++v) {
            T f[NF], d[NF], H[NF][NF], g[NF];
#pragma unroll
            for (int k = 0; k < NF; ++k) f[k] = cF[k][v];
            AdjPot<NF>::eval(f, q, d, H, g);
            if (SELF) vqs += AdjPot<NF>::vq(f);
#pragma unroll
            for (int k = 0; k < NF; ++k) {
              const T pi1 = sc[(2 * k + 1) * ae + own + v];
              const T lf1 = sc[(LF + 2 * k) * ae + own + v];
              T hl = T(0);
#pragma unroll
              for (int m = 0; m < NF; ++m) hl = fmaT(H[k][m], cL[m][v], hl);
              const T pi0 = pi1 - (A1 * lapF[k][v] - A3 * d[k]);
              npi[k][v] = pi0;
              nphi[k][v] = fmaT(-cd, pi0, f[k]);
              T mu = lf1 + (A1 * lapL[k][v] - A3 * hl);
              T lpre = cL[k][v];
              if (SELF) {
                mu = fmaT(bphi, lapF[k][v], fmaT(bV, d[k], mu));
                lpre = fmaT(bpre, pi0, lpre);
                s1 = fmaT(cL[k][v], lapF[k][v], s1);
                s2 = fmaT(cL[k][v], d[k], s2);
                s3 = fmaT(mu, pi0, s3);
              }
              nlf[k][v] = mu;
              nlp[k][v] = fmaT(cd, mu, lpre);
              dqs = fmaT(cL[k][v], g[k], dqs);
            }
          }
          acc[0].add(SELF ? fmaT(-A3, dqs, bV * vqs) : -A3 * dqs);
          if constexpr (SELF) {
            acc[1].add(s1);
            acc[2].add(s2);
            acc[3].add(s3);
          }
          const long long gi =
              (long long)(sg.dir > 0 ? sg.z0 - 1 + j : sg.z0 + sg.nz - j) * NN + (long long)y * N + x0;
#pragma unroll
          for (int k = 0; k < NF; ++k) {
            st_v<T, VX>(reinterpret_cast<T*>(L.buf[parity ^ 1][2 * k]) + gi, nphi[k]);
            st_v<T, VX>(reinterpret_cast<T*>(L.buf[parity ^ 1][2 * k + 1]) + gi, npi[k]);
            st_v<T, VX>(reinterpret_cast<T*>(L.buf[parity ^ 1][LF + 2 * k]) + gi, nlf[k]);
            st_v<T, VX>(reinterpret_cast<T*>(L.buf[parity ^ 1][LF + 2 * k + 1]) + gi, nlp[k]);
          }
#pragma unroll
          for (int k = 0; k < NF; ++k)
#pragma unroll
            for (int v = 0; v < VX; ++v) {
              bF[k][v] = cF[k][v];
              cF[k][v] = aF[k][v];
              bL[k][v] = cL[k][v];
              cL[k][v] = aL[k][v];
            }
        }
        ring_release<T, NA>(R, g0 + j, s_cur, parity, ptot, lane);
        s_cur = s_nxt;
        p_cur = p_nxt;
        ring_advance(S, s_nxt, p_nxt);
      }
      ring_release<T, NA>(R, g0 + sg.nz + 1, s_cur, parity, ptot, lane);
      ring_advance(S, s_cur, p_cur);

      if (!sg.flush) continue;
      if (!ring_flush<NACC, NACC>(R, P, sg, acc, nonfinite, warp, lane)) goto timeout;
    }

    // ---- end of the pass: all writes done; the lattice's dJ/dq share and scale-factor adjoints ----
    if (multi && tid == 0) {
      __threadfence();
      fence_proxy_async_global();
      atomicAdd(&P.gsync[0], 1u);
    }
    {
      const int npend = R.flag[3];
      for (int k = 0; k < npend; ++k) {
        __threadfence();
        const int lat = R.pend[k];
        const LatConst& L = P.lat[lat];
        ring_slot_sums<NACC>(R, P, L, warp, lane);
        if (tid == 0) {
          const double* Q = R.red + 32 * NQ;
          LatScalars& Sc = P.sc[lat];
          Sc.adjq = __ldcg(&Sc.adjq) + Q[0];
          if (SELF) {
            const double al = L.alpha, A1d = cfp[2], A3d = cfp[3];
            const double la = __ldcg(&Sc.adja), lb = __ldcg(&Sc.adjb);
            const double lak =
                la + lb * cfp[9] + ((1.0 + al) * A1d * Q[1] - (3.0 + al) * A3d * Q[2]) * cfp[8];
            const double cq = Q[3] * cfp[10], w = cfp[11];
            Sc.adja = lak + cq;
            Sc.adjb = lb + w * lak + 0.5 * w * cq;
          }
          P.counters[lat] = 0u;
          __threadfence();
          if (multi) atomicAdd(&P.gsync[1], 1u);
        }
        __syncthreads();
      }
      __syncthreads();
      if (tid == 0) R.flag[3] = 0;
    }
  }
  return;

timeout:
  if (tid == 0) ring_drain(R, P);
  __syncthreads();
}

template __global__ void adj_pass_scalar<float, 1, false>(const PassArgs);
template __global__ void adj_pass_scalar<float, 2, false>(const PassArgs);
template __global__ void adj_pass_scalar<double, 1, false>(const PassArgs);
template __global__ void adj_pass_scalar<double, 2, false>(const PassArgs);
template __global__ void adj_pass_scalar<float, 1, true>(const PassArgs);
template __global__ void adj_pass_scalar<float, 2, true>(const PassArgs);
template __global__ void adj_pass_scalar<double, 1, true>(const PassArgs);
template __global__ void adj_pass_scalar<double, 2, true>(const PassArgs);

typedef void (*PassKernel)(const PassArgs);

PassKernel adjoint_pass_kernel(int fp32, int nf, int self) {
  static const PassKernel tab[2][2][2] = {
      {{adj_pass_scalar<double, 1, false>, adj_pass_scalar<double, 2, false>},
       {adj_pass_scalar<float, 1, false>, adj_pass_scalar<float, 2, false>}},
      {{adj_pass_scalar<double, 1, true>, adj_pass_scalar<double, 2, true>},
       {adj_pass_scalar<float, 1, true>, adj_pass_scalar<float, 2, true>}}};
  if (nf < 1 || nf > 2) return nullptr;
  return tab[self ? 1 : 0][fp32 ? 1 : 0][nf - 1];
}

}  // namespace clg
