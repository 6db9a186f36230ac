// pass_u1.cu -- fused drift + kick pass of the U(1) Abelian-Higgs model
// (CosmoLattice manual Sec. 4.3, Hamiltonian form in temporal gauge; the
// lattice operators of the U(1) toolkit, Sec. 4.2):
//
//   drift (deferred from the previous pass):
//       phi_c += cd pi_c,  A_i += cdA pi_A,i       cd = h abar^{alpha-3}, cdA = h abar^{alpha-1}
//   kick:
//       pi_c   += c_k [ a^{1+alpha} (D^2 phi)_c - a^{3+alpha} 2 lam (|phi|^2 - v^2) phi_c ]
//       pi_A,i += c_k [ a^{1+alpha} (f_s/omega_s)^2 J_i + a^{alpha-1} C_i ]
//
// with phi = (phi_0 + i phi_1)/sqrt2 stored as its two real components, links
// V_i(n) = exp(-i theta_i(n)), theta_i = gQ dx A_i(n), and
//   D^2 phi = sum_i [V_i(n) phi(n+i) - 2 phi(n) + V_i^*(n-i) phi(n-i)] / dx^2
//   J_i     = (2 gQ/dx) Im[phi^*(n) V_i(n) phi(n+i)]
//   C_i     = -(1/(gQ dx^3)) sum_{j != i} [sin theta_ij(n) - sin theta_ij(n-j)]
//   theta_ij(n) = gQ dx [A_i(n) + A_j(n+i) - A_i(n+j) - A_j(n)]      (plaquette angle)
// Sums: |phi|-momenta^2 and link momenta^2 after the kick, sum_i |V_i phi(n+i) - phi(n)|^2,
// sum_{i<j} (1 - cos theta_ij) (as 2 sin^2(theta_ij/2)), the potential, and means.
//
// Same plane ring as the scalar pass (ring.cuh), with all ten arrays in a
// stage.  Segments march up in z only: the link phase of A_z(n-z) and the
// plaquette sines theta_xz(n-z), theta_yz(n-z) are those of the plane below,
// carried in registers, so a plane needs its own stage and the one above.
// Each thread owns VX consecutive sites of one x-row; x-neighbours come from
// registers and warp shuffles, y-neighbours from the stage's halo rows.
#include "common.cuh"
#include "ring.cuh"
#include "tail.cuh"
#include "kd_drift.cuh"

namespace clg {

namespace {

enum : int { F0 = 0, P0 = 1, F1 = 2, P1 = 3, AX = 4, PAX = 5, AY = 6, PAY = 7, AZ = 8, PAZ = 9 };

template <typename T> struct U1Vec;
template <> struct U1Vec<float> { typedef float2 type; static constexpr int n = 2; };
template <> struct U1Vec<double> { typedef double type; static constexpr int n = 1; };
static_assert(U1Vec<float>::n == u1_vx(4) && U1Vec<double>::n == u1_vx(8), "host and device tile widths");

template <typename T>
__device__ __forceinline__ void ldv(T (&v)[U1Vec<T>::n], const T* p) {
  *reinterpret_cast<typename U1Vec<T>::type*>(v) = *reinterpret_cast<const typename U1Vec<T>::type*>(p);
}
template <typename T>
__device__ __forceinline__ void stv(T* p, const T (&v)[U1Vec<T>::n]) {
  *reinterpret_cast<typename U1Vec<T>::type*>(p) = *reinterpret_cast<const typename U1Vec<T>::type*>(v);
}


// Plaquette angle from its four link fields, one evaluation order everywhere
// so that a plaquette shared by several sites has one value.
template <typename T>
__device__ __forceinline__ T plaq(T gd, T ai_n, T aj_npi, T ai_npj, T aj_n) {
  return gd * ((ai_n + aj_npi) - (ai_npj + aj_n));
}

}  // namespace

// RED: 0 = no sums, 1 = sums for the Friedmann kick, 2 = full measurement.
// KD: the pass's own drift follows its kick at each site (kick, then drift by
// the pass's dnext), instead of being deferred to the next pass's reads.  The
// order of operations on every value is the same; it needs the drift
// coefficient before the pass's sums are known, so it is taken when a(eta)
// does not depend on them (no expansion, or a fixed power law), and saves
// every neighbour read its momentum load and drift.
// NC: 0 = lattice size and tile height from the lattice constants; > 0 = the
// kernel is built for N = NC with full tiles of THREADS threads (every stage
// offset a compile-time constant).
template <typename T, int RED, bool KD, int NC>
__global__ void __launch_bounds__(THREADS, 1) dk_pass_u1(const PassArgs P) {
  constexpr int VX = U1Vec<T>::n;
  constexpr int NAR = 10;  // arrays in a ring stage
  // RED 1: pi_phi^2, pi_A^2, |D+ phi|^2, magnetic, V.
  // RED 2: pi_0^2, pi_1^2, pi_A^2, |D+ phi|^2, magnetic, V, <phi_c>, <phi_c^2>, <pi_c>.
  constexpr int NACC = RED == 0 ? 1 : (RED == 1 ? 5 : 12);
  constexpr int NUSED = RED == 0 ? 0 : (RED == 1 ? 5 : NQ);

  extern __shared__ __align__(128) unsigned char smem[];
  const Ring R = ring_view(smem, P);
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int sb = P.cta_seg[blockIdx.x], ns = P.cta_seg[blockIdx.x + 1] - sb;
  const bool multi = P.npass > 1;
  if (tid == 0) ring_setup<NAR>(R, P, sb, ns);
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
    if (warp == 0) ring_pass_start<T, NAR>(R, P, pass, ptot, parity, lane);
    __syncthreads();
    if (R.flag[0]) goto timeout;

    for (int i = 0; i < ns; ++i) {
      const Seg sg = P.segs[sb + i];
      const LatConst& L = P.lat[sg.lat];
      const int N = NC ? NC : L.N, BY = NC ? THREADS / (NC / VX) : L.BY, TX = N / VX;
      const int tx = tid % TX, ty = tid / TX;
      const bool active = ty < BY;  // threads 0 .. TX*BY-1
      const int x0 = tx * VX;
      const int y = sg.ytile * BY + ty;
      const int ae = (BY + 2) * N;  // elements of one array in a stage
      const long long NN = (long long)N * N;
      const int g0 = R.off[i];
      // coefficients of the segment: FP64 products formed by one lane (the
      // FP64 pipe is narrow) and broadcast in the storage precision
      T cf[10];
      if (lane == 0) {
        const LatScalars* SC = &P.sc[sg.lat];
        const double ckp = P.steps ? __ldg(&P.steps[pass].ck) : P.ck;
        const double ap1 = __ldcg(&SC->apow1);
        if constexpr (KD) {
          // no deferred drift to apply on read; this pass's drift, after its kick
          double kd, kdA;
          kd_drift_coefficients(L, SC, P.steps ? __ldg(&P.steps[pass].dnext) : P.dnext, kd, kdA);
          cf[0] = cf[1] = T(0);
          cf[8] = (T)kd;
          cf[9] = (T)kdA;
        } else {
          cf[0] = (T)__ldcg(&SC->cd);
          cf[1] = (T)__ldcg(&SC->cdA);
          cf[8] = cf[9] = T(0);
        }
        cf[2] = (T)(ckp * ap1 * L.inv_dx2);
        cf[3] = (T)(ckp * __ldcg(&SC->apow3));
        cf[4] = (T)(ckp * ap1 * L.u1_cJ);   // (2 gQ/dx) Im[...] = (gQ/dx)(phi_0 u_1 - phi_1 u_0)
        cf[5] = (T)(-ckp * __ldcg(&SC->apowm1) * L.u1_cC);
        cf[6] = (T)L.u1_gd;
        cf[7] = (T)(L.v * L.v);
      }
#pragma unroll
      for (int k = 0; k < 10; ++k) cf[k] = __shfl_sync(0xffffffffu, cf[k], 0);
      const T cd = cf[0], cdA = cf[1], A1 = cf[2], A3 = cf[3], AJ = cf[4], AC = cf[5], gd = cf[6], v2 = cf[7];
      const T kd = cf[8], kdA = cf[9];  // KD: the drift after the kick
      const bool drifting = !KD && (cd != T(0) || cdA != T(0));
      const T lam = (T)L.lam;
      const int xl = x0 == 0 ? N - 1 : x0 - 1, xr = x0 + VX == N ? 0 : x0 + VX;
      // output buffer: array a of a lattice buffer starts a * V elements after array 0
      T* const dbase = reinterpret_cast<T*>(L.buf[parity ^ 1][0]);
      const long long Vs = L.V;

      // drifted vector of field array a (its momentum is a + 1) on stage row `row`
      auto rdv = [&](const T* st, int a, int row, T coef, T (&o)[VX]) {
        ldv<T>(o, st + a * ae + row * N + x0);
        if (drifting) {
          T m[VX];
          ldv<T>(m, st + (a + 1) * ae + row * N + x0);
#pragma unroll
          for (int v = 0; v < VX; ++v) o[v] = fmaT(coef, m[v], o[v]);
        }
      };
      auto rds = [&](const T* st, int a, int row, int x, T coef) -> T {
        const T f = st[a * ae + row * N + x];
        return drifting ? fmaT(coef, st[(a + 1) * ae + row * N + x], f) : f;
      };
      // value at x0 - 1 (x0 + VX) of a row, read from the stage and drifted like
      // the owning thread's own copy (no shuffles: every lane reads its own
      // neighbour, with no divergent edge branch)
      auto left = [&](const T* st, int a, int row, T coef) -> T { return rds(st, a, row, xl, coef); };
      auto right = [&](const T* st, int a, int row, T coef) -> T { return rds(st, a, row, xr, coef); };

      // carried from the plane below: phi, the z-link phase, theta_xz and theta_yz sines
      T bF[2][VX], bCz[VX], bSz[VX], bSxz[VX], bSyz[VX];
      // current plane, drifted
      T cF[2][VX], cA[3][VX];

      // ---- planes 0 and 1 of the segment ----
      T axm[VX], aym[VX], azm[VX], azm_xp[VX], azm_yp[VX];
      ring_wait(R, s_cur, p_cur, P.wait_limit_ns);
      if (active && !R.flag[0]) {
        const T* st = ring_stage<T>(R, s_cur);
        rdv(st, F0, ty + 1, cd, bF[0]);
        rdv(st, F1, ty + 1, cd, bF[1]);
        rdv(st, AX, ty + 1, cdA, axm);
        rdv(st, AY, ty + 1, cdA, aym);
        rdv(st, AZ, ty + 1, cdA, azm);
        rdv(st, AZ, ty + 2, cdA, azm_yp);
        const T r = right(st, AZ, ty + 1, cdA);
#pragma unroll
        for (int v = 0; v < VX; ++v) {
          azm_xp[v] = v + 1 < VX ? azm[v + 1] : r;
          sincos_t(gd * azm[v], bSz[v], bCz[v]);
        }
      }
      ring_release<T, NAR>(R, g0, s_cur, parity, ptot, lane);
      ring_advance(S, s_cur, p_cur);
      ring_wait(R, s_cur, p_cur, P.wait_limit_ns);
      if (active && !R.flag[0]) {
        const T* st = ring_stage<T>(R, s_cur);
        rdv(st, F0, ty + 1, cd, cF[0]);
        rdv(st, F1, ty + 1, cd, cF[1]);
        rdv(st, AX, ty + 1, cdA, cA[0]);
        rdv(st, AY, ty + 1, cdA, cA[1]);
        rdv(st, AZ, ty + 1, cdA, cA[2]);
#pragma unroll
        for (int v = 0; v < VX; ++v) {
          bSxz[v] = sin_t(plaq(gd, axm[v], azm_xp[v], cA[0][v], azm[v]));
          bSyz[v] = sin_t(plaq(gd, aym[v], azm_yp[v], cA[1][v], azm[v]));
        }
      }
      int s_nxt = s_cur;
      uint32_t p_nxt = p_cur;
      ring_advance(S, s_nxt, p_nxt);

      for (int j = 1; j <= sg.nz; ++j) {  // plane j in stage s_cur, plane j + 1 in s_nxt
        ring_wait(R, s_nxt, p_nxt, P.wait_limit_ns);
        if (active && !R.flag[0]) {
          const T* sa = ring_stage<T>(R, s_nxt);
          const T* sc = ring_stage<T>(R, s_cur);
          const int own = (ty + 1) * N + x0;
          // segments march up and never wrap: plane j is z0 + j - 1
          T* const out = dbase + (long long)(sg.z0 + j - 1) * NN + (long long)y * N + x0;
          T aF[2][VX], aA[3][VX];  // plane above, drifted
          rdv(sa, F0, ty + 1, cd, aF[0]);
          rdv(sa, F1, ty + 1, cd, aF[1]);
          // link phases of this plane's sites, and of the x- and y-links into them
          T cxv[VX], sxv[VX], cyv[VX], syv[VX], czv[VX], szv[VX], ay_ym[VX];
#pragma unroll
          for (int v = 0; v < VX; ++v) {
            sincos_t(gd * cA[0][v], sxv[v], cxv[v]);
            sincos_t(gd * cA[1][v], syv[v], cyv[v]);
            sincos_t(gd * cA[2][v], szv[v], czv[v]);
          }
          rdv(sc, AY, ty, cdA, ay_ym);
          const T ax_l = left(sc, AX, ty + 1, cdA);
          T s_g = T(0), s_v = T(0), s_pi = T(0);
          T Jx[VX], Jy[VX], Jz[VX];
          // ---- charged scalar: covariant Laplacian, currents, potential, kick ----
          {
            T fym[2][VX], fyp[2][VX];
            rdv(sc, F0, ty, cd, fym[0]);
            rdv(sc, F1, ty, cd, fym[1]);
            rdv(sc, F0, ty + 2, cd, fyp[0]);
            rdv(sc, F1, ty + 2, cd, fyp[1]);
            const T f0_l = left(sc, F0, ty + 1, cd);
            const T f1_l = left(sc, F1, ty + 1, cd);
            const T f0_r = right(sc, F0, ty + 1, cd);
            const T f1_r = right(sc, F1, ty + 1, cd);
            T sxl, cxl;
            sincos_t(gd * ax_l, sxl, cxl);
            T p0[VX], p1[VX], pn0[VX], pn1[VX];
            ldv<T>(p0, sc + P0 * ae + own);
            ldv<T>(p1, sc + P1 * ae + own);
#pragma unroll
            for (int v = 0; v < VX; ++v) {
              const T f0 = cF[0][v], f1 = cF[1][v];
              const T f0xp = v + 1 < VX ? cF[0][v + 1] : f0_r, f1xp = v + 1 < VX ? cF[1][v + 1] : f1_r;
              const T f0xm = v > 0 ? cF[0][v - 1] : f0_l, f1xm = v > 0 ? cF[1][v - 1] : f1_l;
              // V_i(n) phi(n+i) and V_i^*(n-i) phi(n-i), with V = c - i s
              const T cxm = v > 0 ? cxv[v - 1] : cxl, sxm = v > 0 ? sxv[v - 1] : sxl;
              T sym, cym;
              sincos_t(gd * ay_ym[v], sym, cym);
              const T ux0 = cxv[v] * f0xp + sxv[v] * f1xp, ux1 = cxv[v] * f1xp - sxv[v] * f0xp;
              const T uy0 = cyv[v] * fyp[0][v] + syv[v] * fyp[1][v];
              const T uy1 = cyv[v] * fyp[1][v] - syv[v] * fyp[0][v];
              const T uz0 = czv[v] * aF[0][v] + szv[v] * aF[1][v], uz1 = czv[v] * aF[1][v] - szv[v] * aF[0][v];
              const T wx0 = cxm * f0xm - sxm * f1xm, wx1 = cxm * f1xm + sxm * f0xm;
              const T wy0 = cym * fym[0][v] - sym * fym[1][v], wy1 = cym * fym[1][v] + sym * fym[0][v];
              const T wz0 = bCz[v] * bF[0][v] - bSz[v] * bF[1][v], wz1 = bCz[v] * bF[1][v] + bSz[v] * bF[0][v];
              const T D0 = ((ux0 + wx0) - T(2) * f0) + ((uy0 + wy0) - T(2) * f0) + ((uz0 + wz0) - T(2) * f0);
              const T D1 = ((ux1 + wx1) - T(2) * f1) + ((uy1 + wy1) - T(2) * f1) + ((uz1 + wz1) - T(2) * f1);
              Jx[v] = f0 * ux1 - f1 * ux0;
              Jy[v] = f0 * uy1 - f1 * uy0;
              Jz[v] = f0 * uz1 - f1 * uz0;
              // potential lam (|phi|^2 - v^2)^2 and its force 2 lam (|phi|^2 - v^2) phi_c
              const T dd = T(0.5) * (f0 * f0 + f1 * f1) - v2;
              const T gp = T(2) * lam * dd;
              pn0[v] = p0[v] + (A1 * D0 - A3 * gp * f0);
              pn1[v] = p1[v] + (A1 * D1 - A3 * gp * f1);
              if constexpr (RED > 0) {
                const T g0 = ux0 - f0, g1 = ux1 - f1, g2 = uy0 - f0, g3 = uy1 - f1, g4 = uz0 - f0, g5 = uz1 - f1;
                s_g += g0 * g0 + g1 * g1 + g2 * g2 + g3 * g3 + g4 * g4 + g5 * g5;
                s_v += lam * dd * dd;
                if constexpr (RED == 1) {
                  s_pi += pn0[v] * pn0[v] + pn1[v] * pn1[v];
                } else {
                  acc[0].add(pn0[v] * pn0[v]);
                  acc[1].add(pn1[v] * pn1[v]);
                  acc[6].add(f0);
                  acc[7].add(f1);
                  acc[8].add(f0 * f0);
                  acc[9].add(f1 * f1);
                  acc[10].add(pn0[v]);
                  acc[11].add(pn1[v]);
                  if (!isfinite(pn0[v]) || !isfinite(pn1[v])) nonfinite += 1.f;
                }
              }
            }
            if (P.write) {
              if constexpr (KD) {
                T d0[VX], d1[VX];
#pragma unroll
                for (int v = 0; v < VX; ++v) {
                  d0[v] = fmaT(kd, pn0[v], cF[0][v]);
                  d1[v] = fmaT(kd, pn1[v], cF[1][v]);
                }
                stv<T>(out + F0 * Vs, d0);
                stv<T>(out + F1 * Vs, d1);
              } else {
                stv<T>(out + F0 * Vs, cF[0]);
                stv<T>(out + F1 * Vs, cF[1]);
              }
              stv<T>(out + P0 * Vs, pn0);
              stv<T>(out + P1 * Vs, pn1);
            }
          }
          // ---- links: currents, compact curl from plaquettes, kick ----
          T pxz[VX], pyz[VX];
          T s_piA = T(0), s_m = T(0);
          {
            T ay_ymzp[VX], ax_yp[VX], ax_ym[VX], az_yp[VX], az_ym[VX];
            rdv(sa, AX, ty + 1, cdA, aA[0]);
            rdv(sa, AY, ty + 1, cdA, aA[1]);
            rdv(sa, AZ, ty + 1, cdA, aA[2]);
            rdv(sa, AY, ty, cdA, ay_ymzp);
            rdv(sc, AX, ty + 2, cdA, ax_yp);
            rdv(sc, AX, ty, cdA, ax_ym);
            rdv(sc, AZ, ty + 2, cdA, az_yp);
            rdv(sc, AZ, ty, cdA, az_ym);
            const T axzp_l = left(sa, AX, ty + 1, cdA);
            const T ay_l = left(sc, AY, ty + 1, cdA);
            const T az_l = left(sc, AZ, ty + 1, cdA);
            const T axyp_l = left(sc, AX, ty + 2, cdA);
            const T ay_r = right(sc, AY, ty + 1, cdA);
            const T az_r = right(sc, AZ, ty + 1, cdA);
            const T ayym_r = right(sc, AY, ty, cdA);
            T pax[VX], pay[VX], paz[VX], pnx[VX], pny[VX], pnz[VX], pxy[VX];
            ldv<T>(pax, sc + PAX * ae + own);
            ldv<T>(pay, sc + PAY * ae + own);
            ldv<T>(paz, sc + PAZ * ae + own);
#pragma unroll
            for (int v = 0; v < VX; ++v) {
              const T ax = cA[0][v], ay = cA[1][v], az = cA[2][v];
              const T axxm = v > 0 ? cA[0][v - 1] : ax_l;
              const T ayxp = v + 1 < VX ? cA[1][v + 1] : ay_r, ayxm = v > 0 ? cA[1][v - 1] : ay_l;
              const T azxp = v + 1 < VX ? cA[2][v + 1] : az_r, azxm = v > 0 ? cA[2][v - 1] : az_l;
              const T axxmyp = v > 0 ? ax_yp[v - 1] : axyp_l;
              const T ayxpym = v + 1 < VX ? ay_ym[v + 1] : ayym_r;
              const T axxmzp = v > 0 ? aA[0][v - 1] : axzp_l;
              // plaquette sines at n and at its lower neighbours (n-z: carried)
              const T txy = plaq(gd, ax, ayxp, ax_yp[v], ay);
              const T txz = plaq(gd, ax, azxp, aA[0][v], az);
              const T tyz = plaq(gd, ay, az_yp[v], aA[1][v], az);
              pxy[v] = sin_t(txy);
              pxz[v] = sin_t(txz);
              pyz[v] = sin_t(tyz);
              const T sxy_xm = v > 0 ? pxy[v - 1] : sin_t(plaq(gd, axxm, ay, axxmyp, ayxm));
              const T sxz_xm = v > 0 ? pxz[v - 1] : sin_t(plaq(gd, axxm, az, axxmzp, azxm));
              const T sxy_ym = sin_t(plaq(gd, ax_ym[v], ayxpym, ax, ay_ym[v]));
              const T syz_ym = sin_t(plaq(gd, ay_ym[v], az, ay_ymzp[v], az_ym[v]));
              const T Cx = (pxy[v] - sxy_ym) + (pxz[v] - bSxz[v]);
              const T Cy = (sxy_xm - pxy[v]) + (pyz[v] - bSyz[v]);
              const T Cz = (sxz_xm - pxz[v]) + (syz_ym - pyz[v]);
              pnx[v] = pax[v] + (AJ * Jx[v] + AC * Cx);
              pny[v] = pay[v] + (AJ * Jy[v] + AC * Cy);
              pnz[v] = paz[v] + (AJ * Jz[v] + AC * Cz);
              if constexpr (RED > 0) {
                const T hx = sin_t(T(0.5) * txy), hy = sin_t(T(0.5) * txz), hz = sin_t(T(0.5) * tyz);
                s_m += T(2) * (hx * hx + hy * hy + hz * hz);
                s_piA += pnx[v] * pnx[v] + pny[v] * pny[v] + pnz[v] * pnz[v];
                if constexpr (RED == 2)
                  if (!isfinite(pnx[v]) || !isfinite(pny[v]) || !isfinite(pnz[v])) nonfinite += 1.f;
              }
            }
            if (P.write) {
              if constexpr (KD) {
                T dx_[VX], dy_[VX], dz_[VX];
#pragma unroll
                for (int v = 0; v < VX; ++v) {
                  dx_[v] = fmaT(kdA, pnx[v], cA[0][v]);
                  dy_[v] = fmaT(kdA, pny[v], cA[1][v]);
                  dz_[v] = fmaT(kdA, pnz[v], cA[2][v]);
                }
                stv<T>(out + AX * Vs, dx_);
                stv<T>(out + AY * Vs, dy_);
                stv<T>(out + AZ * Vs, dz_);
              } else {
                stv<T>(out + AX * Vs, cA[0]);
                stv<T>(out + AY * Vs, cA[1]);
                stv<T>(out + AZ * Vs, cA[2]);
              }
              stv<T>(out + PAX * Vs, pnx);
              stv<T>(out + PAY * Vs, pny);
              stv<T>(out + PAZ * Vs, pnz);
            }
          }
          if constexpr (RED == 1) {
            acc[0].add(s_pi);
            acc[1].add(s_piA);
            acc[2].add(s_g);
            acc[3].add(s_m);
            acc[4].add(s_v);
          } else if constexpr (RED == 2) {
            acc[2].add(s_piA);
            acc[3].add(s_g);
            acc[4].add(s_m);
            acc[5].add(s_v);
          }
#pragma unroll
          for (int v = 0; v < VX; ++v) {
            bF[0][v] = cF[0][v];
            bF[1][v] = cF[1][v];
            cF[0][v] = aF[0][v];
            cF[1][v] = aF[1][v];
            cA[0][v] = aA[0][v];
            cA[1][v] = aA[1][v];
            cA[2][v] = aA[2][v];
            bCz[v] = czv[v];
            bSz[v] = szv[v];
            bSxz[v] = pxz[v];
            bSyz[v] = pyz[v];
          }
        }
        ring_release<T, NAR>(R, g0 + j, s_cur, parity, ptot, lane);
        s_cur = s_nxt;
        p_cur = p_nxt;
        ring_advance(S, s_nxt, p_nxt);
      }
      ring_release<T, NAR>(R, g0 + sg.nz + 1, s_cur, parity, ptot, lane);
      ring_advance(S, s_cur, p_cur);

      if (!sg.flush) continue;
      if (!ring_flush<NACC, NUSED>(R, P, sg, acc, nonfinite, warp, lane)) goto timeout;
    }

    // ---- end of the pass ----
    if (multi && tid == 0) {  // this CTA's writes are done
      __threadfence();
      fence_proxy_async_global();
      atomicAdd(&P.gsync[0], 1u);
    }
    {
      const int npend = R.flag[3];
      const PassStep pst = P.steps ? P.steps[pass] : PassStep{P.ck, P.wout, P.win, P.dnext};
      for (int k = 0; k < npend; ++k) {
        __threadfence();
        const int lat = R.pend[k];
        const LatConst& L = P.lat[lat];
        ring_slot_sums<NUSED>(R, P, L, warp, lane);
        if (tid == 0) {
          PassArgs Q = P;
          Q.ck = pst.ck;
          Q.wout = pst.wout;
          Q.win = pst.win;
          Q.dnext = pst.dnext;
          ScalarState W;
          load_state_cg(W, &P.sc[lat]);
          const double* sum = R.red + 32 * NQ;
          const double a = W.a, a2 = a * a, a4 = a2 * a2, a6 = a4 * a2;
          const double gdx2 = L.gQ * L.dx * L.dx;
          const double kphi = 0.5 * L.inv_V / a6;                       // E_K per sum of pi_c^2
          const double gphi = 0.5 * L.inv_V * L.inv_dx2 / a2;           // E_G per sum |D+ phi|^2
          const double kA = 0.5 * L.inv_V / (L.fo2 * a4);               // E_K^A per sum pi_A^2
          const double mA = L.inv_V / (L.fo2 * a4 * gdx2 * gdx2);       // E_G^A per sum (1 - cos)
          PassSums E = {0, 0, 0, 0, 0, 0, 0};
          double spost = 0.0;
          if (RED > 0) {
            constexpr int o = RED == 1 ? 0 : 1;
            spost = RED == 1 ? sum[0] : sum[0] + sum[1];
            const double spA = sum[1 + o], gg = sum[2 + o], mag = sum[3 + o], vs = sum[4 + o];
            E.EKpre = W.pi2 * kphi;
            E.EKpost = spost * kphi;
            E.EKApre = W.pi2A * kA;
            E.EKA = spA * kA;
            E.EG = gg * gphi;
            E.EGA = mag * mA;
            E.EV = vs * L.inv_V;
            W.pi2 = spost;
            W.pi2A = spA;
          }
          advance_scalars(Q, L, W, E, RED > 0);
          if (RED == 2) {
            cl_energies_t& ob = P.sc[lat].obs;
            for (int k2 = 0; k2 < 4; ++k2) {
              ob.EK[k2] = ob.EG[k2] = ob.EV[k2] = 0.0;
              ob.mean_phi[k2] = ob.mean_phi2[k2] = ob.mean_pi[k2] = ob.mean_pi2[k2] = 0.0;
            }
            ob.EK[0] = E.EKpost;
            ob.EG[0] = E.EG;
            ob.EV[0] = E.EV;
            ob.EKA = E.EKA;
            ob.EGA = E.EGA;
            for (int c = 0; c < 2; ++c) {
              ob.mean_phi[c] = sum[6 + c] * L.inv_V;
              ob.mean_phi2[c] = sum[8 + c] * L.inv_V;
              ob.mean_pi[c] = sum[10 + c] * L.inv_V;
              ob.mean_pi2[c] = sum[c] * L.inv_V;
            }
            ob.nonfinite = (int64_t)sum[NQ - 1];
            finish_obs(Q, L, W, ob);
          }
          advance_drift(Q, L, W);
          store_state(&P.sc[lat], W);
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

template __global__ void dk_pass_u1<float, 0, false, 0>(const PassArgs);
template __global__ void dk_pass_u1<float, 1, false, 0>(const PassArgs);
template __global__ void dk_pass_u1<float, 2, false, 0>(const PassArgs);
template __global__ void dk_pass_u1<double, 0, false, 0>(const PassArgs);
template __global__ void dk_pass_u1<double, 1, false, 0>(const PassArgs);
template __global__ void dk_pass_u1<double, 2, false, 0>(const PassArgs);
template __global__ void dk_pass_u1<float, 0, true, 0>(const PassArgs);
template __global__ void dk_pass_u1<float, 2, true, 0>(const PassArgs);
template __global__ void dk_pass_u1<double, 0, true, 0>(const PassArgs);
template __global__ void dk_pass_u1<double, 2, true, 0>(const PassArgs);
template __global__ void dk_pass_u1<float, 0, true, 256>(const PassArgs);
template __global__ void dk_pass_u1<float, 2, true, 256>(const PassArgs);

typedef void (*PassKernel)(const PassArgs);

// kd: kick-then-drift passes (only without self-consistent expansion, where the
// Friedmann sums of RED 1 are not needed).  n256: one FP32 lattice of N = 256 with full
// tiles (the tile height THREADS / (N / 2)), built with its sizes as constants.
PassKernel u1_pass_kernel(int fp32, int red, int kd, int n256) {
  static const PassKernel tab[2][3] = {
      {dk_pass_u1<double, 0, false, 0>, dk_pass_u1<double, 1, false, 0>, dk_pass_u1<double, 2, false, 0>},
      {dk_pass_u1<float, 0, false, 0>, dk_pass_u1<float, 1, false, 0>, dk_pass_u1<float, 2, false, 0>}};
  static const PassKernel tab_kd[2][3] = {
      {dk_pass_u1<double, 0, true, 0>, nullptr, dk_pass_u1<double, 2, true, 0>},
      {dk_pass_u1<float, 0, true, 0>, nullptr, dk_pass_u1<float, 2, true, 0>}};
  static const PassKernel tab_kd256[3] = {dk_pass_u1<float, 0, true, 256>, nullptr,
                                          dk_pass_u1<float, 2, true, 256>};
  if (red < 0 || red > 2) return nullptr;
  if (kd && n256 && fp32) return tab_kd256[red];
  return kd ? tab_kd[fp32 ? 1 : 0][red] : tab[fp32 ? 1 : 0][red];
}

}  // namespace clg
