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
// A plane ring (ring.cuh) with all ten arrays in a stage (the momenta without
// halo rows where the pass kicks, then drifts).  Segments march up in z only:
// the link phase of A_z(n-z) and the plaquette sines theta_xz(n-z),
// theta_yz(n-z) are those of the plane below, carried in registers, so a plane
// needs its own stage and the one above.  Each thread owns VX consecutive sites
// of one x-row, worked as one value (an FP32 pair in the packed two-lane form);
// x-neighbours come from registers and the stage, y-neighbours from the stage's
// halo rows.  The sines and cosines a plane needs are evaluated together, after
// one range check.
#include "common.cuh"
#include "ring.cuh"
#include "tail.cuh"
#include "kd_drift.cuh"
#include "trig2.cuh"

namespace clg {

namespace {

enum : int { F0 = 0, P0 = 1, F1 = 2, P1 = 3, AX = 4, PAX = 5, AY = 6, PAY = 7, AZ = 8, PAZ = 9 };

template <typename T> struct U1Vec;
template <> struct U1Vec<float> { typedef float2 type; static constexpr int n = 2; };
template <> struct U1Vec<double> { typedef double type; static constexpr int n = 1; };
static_assert(U1Vec<float>::n == u1_vx(4) && U1Vec<double>::n == u1_vx(8), "host and device tile widths");

// A thread's VX sites of one x-row as one value: an FP32 pair is worked in the
// packed two-lane form (one instruction for both sites), an FP64 site alone.
// Every operation is rounded on its own (no contraction), so a value formed by
// two threads (a link phase or a plaquette sine shared by neighbours) is the same.
__device__ __forceinline__ float2 vset(float a) { return make_float2(a, a); }
__device__ __forceinline__ double vset(double a) { return a; }
__device__ __forceinline__ float2 vadd(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ double vadd(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ float2 vmul(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ double vmul(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ float2 vfma(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ double vfma(double a, double b, double c) { return fma(a, b, c); }
// a - b, exactly rounded (b times -1 is exact)
__device__ __forceinline__ float2 vsub(float2 a, float2 b) { return __ffma2_rn(b, vset(-1.f), a); }
__device__ __forceinline__ double vsub(double a, double b) { return __dsub_rn(a, b); }
// the row's values one site up (down) in x, given the next thread's first
// (the previous thread's last) value
__device__ __forceinline__ float2 vxp(float2 v, float r) { return make_float2(v.y, r); }
__device__ __forceinline__ double vxp(double, double r) { return r; }
__device__ __forceinline__ float2 vxm(float2 v, float l) { return make_float2(l, v.x); }
__device__ __forceinline__ double vxm(double, double l) { return l; }
__device__ __forceinline__ float vget(float2 v, int i) { return i ? v.y : v.x; }
__device__ __forceinline__ double vget(double v, int) { return v; }
__device__ __forceinline__ void vsincos(float2 x, float2& s, float2& c) { sincos2_t(x, s, c); }
__device__ __forceinline__ void vsincos(double x, double& s, double& c) { sincos_t(x, s, c); }
__device__ __forceinline__ float2 vsin(float2 x) { return sin2_t(x); }
__device__ __forceinline__ double vsin(double x) { return sin_t(x); }
// Sines and cosines of the angle vectors xc[] and of one single angle xs, and
// sines of the angle vectors xn[]: one range check for all of them, then every
// polynomial in one block (independent chains the scheduler interleaves).
// Where any angle is beyond pi/4 each lane of each angle takes the scalar path,
// which gives an in-range angle the same value.
template <int NCS, int NSN>
__device__ __forceinline__ void trig_block(const float2 (&xc)[NCS], float2 (&s)[NCS], float2 (&c)[NCS], float xs,
                                           float& ss, float& cs, const float2 (&xn)[NSN], float2 (&sn)[NSN]) {
  float m = fabsf(xs);
#pragma unroll
  for (int k = 0; k < NCS; ++k) m = fmaxf(m, fmaxf(fabsf(xc[k].x), fabsf(xc[k].y)));
#pragma unroll
  for (int k = 0; k < NSN; ++k) m = fmaxf(m, fmaxf(fabsf(xn[k].x), fabsf(xn[k].y)));
  if (m <= TRIG_PI4) {
#pragma unroll
    for (int k = 0; k < NCS; ++k) {
      const float2 x2 = __fmul2_rn(xc[k], xc[k]);
      s[k] = __fmul2_rn(xc[k], sin_taylor2(x2));
      c[k] = cos_taylor2(x2);
    }
#pragma unroll
    for (int k = 0; k < NSN; ++k) sn[k] = __fmul2_rn(xn[k], sin_taylor2(__fmul2_rn(xn[k], xn[k])));
    const float x2 = __fmul_rn(xs, xs);
    ss = __fmul_rn(xs, sin_taylor(x2));
    cs = cos_taylor(x2);
  } else {
#pragma unroll
    for (int k = 0; k < NCS; ++k) {
      sincos_rn(xc[k].x, s[k].x, c[k].x);
      sincos_rn(xc[k].y, s[k].y, c[k].y);
    }
#pragma unroll
    for (int k = 0; k < NSN; ++k) sn[k] = make_float2(sin_rn(xn[k].x), sin_rn(xn[k].y));
    sincos_rn(xs, ss, cs);
  }
}
template <int NCS, int NSN>
__device__ __forceinline__ void trig_block(const double (&xc)[NCS], double (&s)[NCS], double (&c)[NCS], double xs,
                                           double& ss, double& cs, const double (&xn)[NSN], double (&sn)[NSN]) {
#pragma unroll
  for (int k = 0; k < NCS; ++k) sincos_t(xc[k], s[k], c[k]);
#pragma unroll
  for (int k = 0; k < NSN; ++k) sn[k] = sin_t(xn[k]);
  sincos_t(xs, ss, cs);
}

// Plaquette angle from its four link fields, one evaluation order everywhere
// so that a plaquette shared by several sites has one value.
template <typename V>
__device__ __forceinline__ V plaq(V gd, V ai_n, V aj_npi, V ai_npj, V aj_n) {
  return vmul(gd, vsub(vadd(ai_n, aj_npi), vadd(ai_npj, aj_n)));
}

}  // namespace

// RED: 0 = no sums, 1 = sums for the Friedmann kick, 2 = full measurement.
// KD: the pass's own drift follows its kick at each site (kick, then drift by
// the pass's dnext), instead of being deferred to the next pass's reads.  The
// order of operations on every value is the same; it needs the drift
// coefficient before the pass's sums are known, so it is taken when a(eta)
// does not depend on them (no expansion, or a fixed power law), and saves
// every neighbour read its momentum load and drift; the momenta are then read
// at the own sites only, so the stages hold them without halo rows (four
// stages fit instead of three).
// NC: 0 = lattice size and tile height from the lattice constants; > 0 = the
// kernel is built for N = NC with full tiles of THREADS threads (every stage
// offset a compile-time constant).
template <typename T, int RED, bool KD, int NC>
__global__ void __launch_bounds__(THREADS, 1) dk_pass_u1(const PassArgs P) {
  constexpr int VX = U1Vec<T>::n;
  typedef typename U1Vec<T>::type V;
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
    if (warp == 0) ring_pass_start<T, NAR, KD>(R, P, pass, ptot, parity, lane);
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
      // stage offset of array a: KD keeps (field, momentum) pairs of BY + 2 and BY rows
      auto aoff = [&](int a) { return KD ? (a >> 1) * (2 * BY + 2) * N + (a & 1) * ae : a * ae; };
      const int mrow = KD ? -N : 0;  // KD: a momentum's stage rows start at the tile's first row
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
      const V gdv = vset(gd);
      const int xl = x0 == 0 ? N - 1 : x0 - 1, xr = x0 + VX == N ? 0 : x0 + VX;
      // output buffer: array a of a lattice buffer starts a * V elements after array 0
      T* const dbase = reinterpret_cast<T*>(L.buf[parity ^ 1][0]);
      const long long Vs = L.V;

      // the thread's sites of field array a (its momentum is a + 1) on stage row `row`, drifted
      auto rdv = [&](const T* st, int a, int row, T coef) -> V {
        const V o = *reinterpret_cast<const V*>(st + aoff(a) + row * N + x0);
        return drifting ? vfma(vset(coef), *reinterpret_cast<const V*>(st + aoff(a + 1) + row * N + x0), o) : o;
      };
      auto rds = [&](const T* st, int a, int row, int x, T coef) -> T {
        const T f = st[aoff(a) + row * N + x];
        return drifting ? fmaT(coef, st[aoff(a + 1) + row * N + x], f) : f;
      };
      // value at x0 - 1 (x0 + VX) of a row, read from the stage and drifted like
      // the owning thread's own copy (no shuffles: every lane reads its own
      // neighbour, with no divergent edge branch)
      auto left = [&](const T* st, int a, int row, T coef) -> T { return rds(st, a, row, xl, coef); };
      auto right = [&](const T* st, int a, int row, T coef) -> T { return rds(st, a, row, xr, coef); };
      auto stv = [&](T* p, V v) { *reinterpret_cast<V*>(p) = v; };

      // carried from the plane below: phi, the z-link phase, theta_xz and theta_yz sines
      V bF0, bF1, bCz, bSz, bSxz, bSyz;
      // current plane, drifted
      V cF0, cF1, cA0, cA1, cA2;

      // ---- planes 0 and 1 of the segment ----
      V axm, aym, azm, azm_xp, azm_yp;
      ring_wait(R, s_cur, p_cur, P.wait_limit_ns);
      if (active && !R.flag[0]) {
        const T* st = ring_stage<T>(R, s_cur);
        bF0 = rdv(st, F0, ty + 1, cd);
        bF1 = rdv(st, F1, ty + 1, cd);
        axm = rdv(st, AX, ty + 1, cdA);
        aym = rdv(st, AY, ty + 1, cdA);
        azm = rdv(st, AZ, ty + 1, cdA);
        azm_yp = rdv(st, AZ, ty + 2, cdA);
        azm_xp = vxp(azm, right(st, AZ, ty + 1, cdA));
        vsincos(vmul(gdv, azm), bSz, bCz);
      }
      ring_release<T, NAR, KD>(R, g0, s_cur, parity, ptot, lane);
      ring_advance(S, s_cur, p_cur);
      ring_wait(R, s_cur, p_cur, P.wait_limit_ns);
      if (active && !R.flag[0]) {
        const T* st = ring_stage<T>(R, s_cur);
        cF0 = rdv(st, F0, ty + 1, cd);
        cF1 = rdv(st, F1, ty + 1, cd);
        cA0 = rdv(st, AX, ty + 1, cdA);
        cA1 = rdv(st, AY, ty + 1, cdA);
        cA2 = rdv(st, AZ, ty + 1, cdA);
        bSxz = vsin(plaq(gdv, axm, azm_xp, cA0, azm));
        bSyz = vsin(plaq(gdv, aym, azm_yp, cA1, azm));
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
          const V aF0 = rdv(sa, F0, ty + 1, cd), aF1 = rdv(sa, F1, ty + 1, cd);  // plane above, drifted
          const V aA0 = rdv(sa, AX, ty + 1, cdA), aA1 = rdv(sa, AY, ty + 1, cdA);
          const V ay_ym = rdv(sc, AY, ty, cdA), ay_ymzp = rdv(sa, AY, ty, cdA);
          const V ax_yp = rdv(sc, AX, ty + 2, cdA), ax_ym = rdv(sc, AX, ty, cdA);
          const V az_yp = rdv(sc, AZ, ty + 2, cdA), az_ym = rdv(sc, AZ, ty, cdA);
          const T ax_l = left(sc, AX, ty + 1, cdA), axzp_l = left(sa, AX, ty + 1, cdA);
          const T ay_l = left(sc, AY, ty + 1, cdA), az_l = left(sc, AZ, ty + 1, cdA);
          const T axyp_l = left(sc, AX, ty + 2, cdA);
          const V ayxp = vxp(cA1, right(sc, AY, ty + 1, cdA));
          const V azxp = vxp(cA2, right(sc, AZ, ty + 1, cdA));
          const V ayxpym = vxp(ay_ym, right(sc, AY, ty, cdA));
          // link phases of this plane's sites and of the y-links into them (cosine
          // and sine), of the x-link into the first site; plaquette sines at n, at
          // n-y, and at n-x of the first site (n-z: carried)
          const V txy = plaq(gdv, cA0, ayxp, ax_yp, cA1);
          const V txz = plaq(gdv, cA0, azxp, aA0, cA2);
          const V tyz = plaq(gdv, cA1, az_yp, aA1, cA2);
          constexpr int NE = VX == 2 ? 1 : 2;  // the first site's two n-x plaquettes: one FP32 pair, two FP64 values
          V xc[4], sc4[4], cc4[4], xn[5 + NE], sn[5 + NE];
          xc[0] = vmul(gdv, cA0);
          xc[1] = vmul(gdv, cA1);
          xc[2] = vmul(gdv, cA2);
          xc[3] = vmul(gdv, ay_ym);
          xn[0] = txy;
          xn[1] = txz;
          xn[2] = tyz;
          xn[3] = plaq(gdv, ax_ym, ayxpym, cA0, ay_ym);
          xn[4] = plaq(gdv, ay_ym, cA2, ay_ymzp, az_ym);
          {
            const T ay0 = vget(cA1, 0), az0 = vget(cA2, 0);
            const T e_xy = gd * ((ax_l + ay0) - (axyp_l + ay_l)), e_xz = gd * ((ax_l + az0) - (axzp_l + az_l));
            if constexpr (VX == 2) {
              xn[5] = V{e_xy, e_xz};
            } else {
              xn[5] = V{e_xy};
              xn[4 + NE] = V{e_xz};
            }
          }
          T sxl, cxl;
          trig_block(xc, sc4, cc4, gd * ax_l, sxl, cxl, xn, sn);
          const V sx = sc4[0], cx = cc4[0], sy = sc4[1], cy = cc4[1], sz = sc4[2], cz = cc4[2];
          const V sym = sc4[3], cym = cc4[3];
          const V pxy = sn[0], pxz = sn[1], pyz = sn[2], sxy_ym = sn[3], syz_ym = sn[4];
          const V sxy_xm = vxm(pxy, vget(sn[5], 0)), sxz_xm = vxm(pxz, vget(sn[4 + NE], VX - 1));
          T s_g = T(0), s_v = T(0), s_pi = T(0);
          V Jx, Jy, Jz;
          // ---- charged scalar: covariant Laplacian, currents, potential, kick ----
          {
            const V fym0 = rdv(sc, F0, ty, cd), fym1 = rdv(sc, F1, ty, cd);
            const V fyp0 = rdv(sc, F0, ty + 2, cd), fyp1 = rdv(sc, F1, ty + 2, cd);
            const V f0xp = vxp(cF0, right(sc, F0, ty + 1, cd)), f1xp = vxp(cF1, right(sc, F1, ty + 1, cd));
            const V f0xm = vxm(cF0, left(sc, F0, ty + 1, cd)), f1xm = vxm(cF1, left(sc, F1, ty + 1, cd));
            const V cxm = vxm(cx, cxl), sxm = vxm(sx, sxl);
            const V p0 = *reinterpret_cast<const V*>(sc + aoff(P0) + own + mrow);
            const V p1 = *reinterpret_cast<const V*>(sc + aoff(P1) + own + mrow);
            const V f0 = cF0, f1 = cF1;
            // V_i(n) phi(n+i) = u and V_i^*(n-i) phi(n-i) = w, with V = c - i s
            const V ux0 = vfma(cx, f0xp, vmul(sx, f1xp)), ux1 = vsub(vmul(cx, f1xp), vmul(sx, f0xp));
            const V uy0 = vfma(cy, fyp0, vmul(sy, fyp1)), uy1 = vsub(vmul(cy, fyp1), vmul(sy, fyp0));
            const V uz0 = vfma(cz, aF0, vmul(sz, aF1)), uz1 = vsub(vmul(cz, aF1), vmul(sz, aF0));
            const V wx0 = vsub(vmul(cxm, f0xm), vmul(sxm, f1xm)), wx1 = vfma(cxm, f1xm, vmul(sxm, f0xm));
            const V wy0 = vsub(vmul(cym, fym0), vmul(sym, fym1)), wy1 = vfma(cym, fym1, vmul(sym, fym0));
            const V wz0 = vsub(vmul(bCz, bF0), vmul(bSz, bF1)), wz1 = vfma(bCz, bF1, vmul(bSz, bF0));
            const V m2 = vset(T(-2));
            const V D0 = vadd(vadd(vfma(m2, f0, vadd(ux0, wx0)), vfma(m2, f0, vadd(uy0, wy0))), vfma(m2, f0, vadd(uz0, wz0)));
            const V D1 = vadd(vadd(vfma(m2, f1, vadd(ux1, wx1)), vfma(m2, f1, vadd(uy1, wy1))), vfma(m2, f1, vadd(uz1, wz1)));
            Jx = vsub(vmul(f0, ux1), vmul(f1, ux0));
            Jy = vsub(vmul(f0, uy1), vmul(f1, uy0));
            Jz = vsub(vmul(f0, uz1), vmul(f1, uz0));
            // potential lam (|phi|^2 - v^2)^2 and its force 2 lam (|phi|^2 - v^2) phi_c
            const V dd = vfma(vset(T(0.5)), vfma(f0, f0, vmul(f1, f1)), vset(-v2));
            const V ngp = vmul(vset(-A3 * T(2) * lam), dd);  // -A3 2 lam (|phi|^2 - v^2)
            const V pn0 = vadd(p0, vfma(ngp, f0, vmul(vset(A1), D0)));
            const V pn1 = vadd(p1, vfma(ngp, f1, vmul(vset(A1), D1)));
            if constexpr (RED > 0) {
              const V g0 = vsub(ux0, f0), g1 = vsub(ux1, f1), g2 = vsub(uy0, f0), g3 = vsub(uy1, f1);
              const V g4 = vsub(uz0, f0), g5 = vsub(uz1, f1);
#pragma unroll
              for (int v = 0; v < VX; ++v) {
                const T e0 = vget(g0, v), e1 = vget(g1, v), e2 = vget(g2, v), e3 = vget(g3, v), e4 = vget(g4, v),
                        e5 = vget(g5, v);
                const T q0 = vget(pn0, v), q1 = vget(pn1, v), h0 = vget(f0, v), h1 = vget(f1, v), d = vget(dd, v);
                s_g += e0 * e0 + e1 * e1 + e2 * e2 + e3 * e3 + e4 * e4 + e5 * e5;
                s_v += lam * d * d;
                if constexpr (RED == 1) {
                  s_pi += q0 * q0 + q1 * q1;
                } else {
                  acc[0].add(q0 * q0);
                  acc[1].add(q1 * q1);
                  acc[6].add(h0);
                  acc[7].add(h1);
                  acc[8].add(h0 * h0);
                  acc[9].add(h1 * h1);
                  acc[10].add(q0);
                  acc[11].add(q1);
                  if (!isfinite(q0) || !isfinite(q1)) nonfinite += 1.f;
                }
              }
            }
            if (P.write) {
              if constexpr (KD) {
                stv(out + F0 * Vs, vfma(vset(kd), pn0, f0));
                stv(out + F1 * Vs, vfma(vset(kd), pn1, f1));
              } else {
                stv(out + F0 * Vs, f0);
                stv(out + F1 * Vs, f1);
              }
              stv(out + P0 * Vs, pn0);
              stv(out + P1 * Vs, pn1);
            }
          }
          // ---- links: currents, compact curl from plaquettes, kick ----
          T s_piA = T(0), s_m = T(0);
          {
            const V pax = *reinterpret_cast<const V*>(sc + aoff(PAX) + own + mrow);
            const V pay = *reinterpret_cast<const V*>(sc + aoff(PAY) + own + mrow);
            const V paz = *reinterpret_cast<const V*>(sc + aoff(PAZ) + own + mrow);
            const V Cx = vadd(vsub(pxy, sxy_ym), vsub(pxz, bSxz));
            const V Cy = vadd(vsub(sxy_xm, pxy), vsub(pyz, bSyz));
            const V Cz = vadd(vsub(sxz_xm, pxz), vsub(syz_ym, pyz));
            const V AJv = vset(AJ), ACv = vset(AC);
            const V pnx = vadd(pax, vfma(AJv, Jx, vmul(ACv, Cx)));
            const V pny = vadd(pay, vfma(AJv, Jy, vmul(ACv, Cy)));
            const V pnz = vadd(paz, vfma(AJv, Jz, vmul(ACv, Cz)));
            if constexpr (RED > 0) {
              const V hxy = vsin(vmul(vset(T(0.5)), txy)), hxz = vsin(vmul(vset(T(0.5)), txz));
              const V hyz = vsin(vmul(vset(T(0.5)), tyz));
#pragma unroll
              for (int v = 0; v < VX; ++v) {
                const T hx = vget(hxy, v), hy = vget(hxz, v), hz = vget(hyz, v);
                const T qx = vget(pnx, v), qy = vget(pny, v), qz = vget(pnz, v);
                s_m += T(2) * (hx * hx + hy * hy + hz * hz);
                s_piA += qx * qx + qy * qy + qz * qz;
                if constexpr (RED == 2)
                  if (!isfinite(qx) || !isfinite(qy) || !isfinite(qz)) nonfinite += 1.f;
              }
            }
            if (P.write) {
              if constexpr (KD) {
                stv(out + AX * Vs, vfma(vset(kdA), pnx, cA0));
                stv(out + AY * Vs, vfma(vset(kdA), pny, cA1));
                stv(out + AZ * Vs, vfma(vset(kdA), pnz, cA2));
              } else {
                stv(out + AX * Vs, cA0);
                stv(out + AY * Vs, cA1);
                stv(out + AZ * Vs, cA2);
              }
              stv(out + PAX * Vs, pnx);
              stv(out + PAY * Vs, pny);
              stv(out + PAZ * Vs, pnz);
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
          bF0 = cF0;
          bF1 = cF1;
          cF0 = aF0;
          cF1 = aF1;
          cA0 = aA0;
          cA1 = aA1;
          cA2 = rdv(sa, AZ, ty + 1, cdA);
          bCz = cz;
          bSz = sz;
          bSxz = pxz;
          bSyz = pyz;
        }
        ring_release<T, NAR, KD>(R, g0 + j, s_cur, parity, ptot, lane);
        s_cur = s_nxt;
        p_cur = p_nxt;
        ring_advance(S, s_nxt, p_nxt);
      }
      ring_release<T, NAR, KD>(R, g0 + sg.nz + 1, s_cur, parity, ptot, lane);
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
