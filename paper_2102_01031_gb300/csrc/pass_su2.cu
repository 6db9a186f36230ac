// pass_su2.cu -- fused drift + kick pass of the SU(2) x U(1) doublet model
// (the gauge content of the CosmoLattice manual's lphi4SU2U1 example: Sec. 4.1
// action, Sec. 4.3 Hamiltonian form in temporal gauge, links, plaquettes and
// covariant derivatives of the U(1) and SU(N) toolkits of Sec. 4.2).
//
// State (35 arrays of one slab, array a at a * V elements):
//   0..3   phi_c, Phi = (phi_0 + i phi_1, phi_2 + i phi_3)/sqrt2 (psi = sqrt2 Phi below)
//   4..7   pi_c
//   8..10  A_i (U(1) link fields, V_i = exp(-i gQ dx A_i)),   11..13 pi_A,i
//   14 + 4 i + k   SU(2) link U_i = u0 - i (u1 s1 + u2 s2 + u3 s3) (s_a Pauli)
//   26 + 3 i + (a - 1)   pi_B,i^a
//
//   drift (deferred from the previous pass):
//       phi_c += cd pi_c,   A_i += cdA pi_A,i,
//       U_i <- exp(-i (gQB dx cdA) pi_B,i^a s_a/2) U_i
//   kick (W_i = V_i U_i, the doublet's hopping link):
//       pi_c     += c_k [ a^{1+alpha} (D^2 psi)_c - a^{3+alpha} 2 lam (|Phi|^2 - v^2) phi_c ]
//       pi_A,i   += c_k [ a^{1+alpha} (f_s/omega_s)^2 (gQ/dx) Im(psi^dag W_i psi(n+i)) + a^{alpha-1} C_i ]
//       pi_B,i^a += c_k [ a^{1+alpha} (f_s/omega_s)^2 (gQB/(2dx)) Im(psi^dag s_a W_i psi(n+i))
//                         - a^{alpha-1} (2/(gQB dx^3)) m_a(U_i S_i) ]
//   with D^2 psi = sum_i [W_i psi(n+i) - 2 psi + W_i^dag(n-i) psi(n-i)]/dx^2, C_i the compact
//   U(1) curl of the U(1) model, S_i the sum of the four staples of U_i(n) and m_a the
//   vector part of a quaternion (Im Tr[s_a M] = -2 m_a).  These are the kernels of one
//   lattice Hamiltonian (kinetic terms, covariant hopping, compact U(1) plaquettes,
//   SU(2) plaquette traces), so that both lattice Gauss laws hold exactly.
//
// Kernel layout.  A work item is a TX x TY tile of x-y sites over a chunk of
// z-planes; the resident CTAs (two per SM) take items in a round-robin that
// keeps neighbouring tiles on the same planes at the same time.  Each plane of
// the tile plus a one-site halo (corners included) is loaded from HBM (all 35
// loads of a site in flight at once), drifted in registers and kept, drifted,
// in a three-plane shared-memory ring (links as one 16-byte quaternion per
// site and direction, the doublet as one quaternion, the three U(1) link
// fields); the drifted fields of the CTA's own sites are written out right
// away.  The kick of plane z then reads every neighbour, staple and plaquette
// it needs from the ring (the stencil reaches n +- x, n +- y, n +- z and the
// diagonal neighbours n + i - j), and re-reads its own momenta, prefetched
// into L1 while the next plane loads.  The two CTAs of an SM overlap one's
// loads with the other's arithmetic.  The last CTA to finish sums the per-CTA
// partial sums in a fixed order and advances the scale factor (tail.cuh).
#include "su2_common.cuh"

namespace clg {

// Bytes of one ring slot: per halo site 3 links + doublet (quaternions) and 3 U(1)
// fields, and for lphi4SU2U1 also the singlet and vphi's two components.
__host__ __device__ constexpr size_t su2_slot_bytes(int TX, int TY, int esz, bool full = false) {
  return ((full ? 22 : 19) * (size_t)(TX + 2) * (TY + 2) * esz + 127) / 128 * 128;
}

// RED: 0 = no sums, 1 = sums for the Friedmann kicks, 2 = full measurement.
// FULL: the lphi4SU2U1 model (Sec. 4.5): also a singlet phi_s and a U(1)-charged
// scalar vphi (charge Qc in units of the doublet's, hopping with exp(-i Qc gQ dx A_i)),
// coupled through V = lam (|Phi|^2 - v^2)^2 + qG |Phi|^2 phi_s^2 + 2 qH |Phi|^2 |vphi|^2:
//   pi_s   += c_k [a^{1+alpha} Lap phi_s - a^{3+alpha} 2 qG |Phi|^2 phi_s]
//   pi_vc  += c_k [a^{1+alpha} (D^2 vphi)_c - a^{3+alpha} 2 qH |Phi|^2 vphi_c]
//   pi_c   (doublet) gains - a^{3+alpha} (qG phi_s^2 + 2 qH |vphi|^2) phi_c
//   pi_A,i gains a^{1+alpha} (f_s/omega_s)^2 Qc (gQ/dx) (vphi_0 u_1 - vphi_1 u_0), u = its hop.
template <typename T, int RED, int TX, bool FULL>
__global__ void __launch_bounds__(256, (RED == 2 || sizeof(T) == 8) ? 1 : 2) dk_pass_su2(const PassArgs P) {
  constexpr int NACC = RED == 0 ? 1 : (RED == 1 ? 6 : (FULL ? 29 : 23));
  constexpr int NLD = FULL ? SNARR_FULL : SNARR;  // arrays loaded per halo site
  extern __shared__ __align__(128) unsigned char smem[];
  __shared__ double red_s[SU2_NQ][9];
  __shared__ unsigned last_s;
  const LatConst& L = P.lat[0];
  const int N = L.N;
  constexpr int TY = SU2_TY, nth = TX * TY;
  const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * TX + tx;
  const int lane = tid & 31, warp = tid >> 5;
  constexpr int HX = TX + 2, HS = HX * (TY + 2);
  const int ntx = N / TX, nty = N / TY;
  const long long NN = (long long)N * N, V = L.V;
  const int parity = P.parity;
  const T* const src = reinterpret_cast<const T*>(L.buf[parity][0]);
  T* const dst = reinterpret_cast<T*>(L.buf[parity ^ 1][0]);
  constexpr size_t slot_b = su2_slot_bytes(TX, TY, sizeof(T), FULL);

  // coefficients: FP64 products by one lane, broadcast in the storage precision
  T cf[17];
  if (lane == 0) {
    const LatScalars* SC = P.sc;
    const double ck = P.ck, ap1 = __ldcg(&SC->apow1), apm1 = __ldcg(&SC->apowm1);
    const double cdA = __ldcg(&SC->cdA), dx = L.dx;
    cf[0] = (T)__ldcg(&SC->cd);
    cf[1] = (T)cdA;
    cf[2] = (T)(0.5 * L.gQB * dx * cdA);                        // half the SU(2) drift angle per momentum
    cf[3] = (T)(ck * ap1 * L.inv_dx2);                           // doublet Laplacian
    cf[4] = (T)(ck * __ldcg(&SC->apow3));                        // potential force
    cf[5] = (T)(ck * ap1 * L.fo2 * L.gQ / dx);                   // U(1) current
    cf[6] = (T)(L.gQ != 0.0 ? -ck * apm1 / (L.gQ * dx * dx * dx) : 0.0);  // U(1) curl
    cf[7] = (T)(ck * ap1 * L.fo2 * L.gQB / (2.0 * dx));          // SU(2) current
    cf[8] = (T)(-2.0 * ck * apm1 / (L.gQB * dx * dx * dx));      // SU(2) plaquette force
    cf[9] = (T)(L.gQ * dx);
    cf[10] = (T)(L.v * L.v);
    cf[11] = (T)L.lam;
    cf[12] = (T)(2.0 * L.lam);
    cf[13] = (T)L.qG;
    cf[14] = (T)L.qH;
    cf[15] = (T)(L.Qc * L.gQ * dx);                              // vphi's link phase per A_i
    cf[16] = (T)(ck * ap1 * L.fo2 * L.Qc * L.gQ / dx);            // vphi's U(1) current
  }
#pragma unroll
  for (int k = 0; k < 17; ++k) cf[k] = __shfl_sync(0xffffffffu, cf[k], 0);
  const T cd = cf[0], cdA = cf[1], hB = cf[2], A1 = cf[3], A3 = cf[4], AJA = cf[5], ACA = cf[6], AJB = cf[7],
          AMB = cf[8], gd = cf[9], v2 = cf[10], lam = cf[11], lam2 = cf[12], qG = cf[13], qH = cf[14],
          gdc = cf[15], AJC = cf[16];
  const bool drifting = cd != T(0) || cdA != T(0);

  Acc<T> acc[NACC];
#pragma unroll
  for (int k = 0; k < NACC; ++k) acc[k].zero();
  float nonfinite = 0.f;

  // ring slot s: links [3][HS], doublet [HS], U(1) fields [3][HS]
  auto sU = [&](int s, int i) { return reinterpret_cast<Q4<T>*>(smem + s * slot_b) + i * HS; };
  auto sF = [&](int s) { return reinterpret_cast<Q4<T>*>(smem + s * slot_b) + 3 * HS; };
  auto sA = [&](int s, int i) { return reinterpret_cast<T*>(smem + s * slot_b) + 16 * HS + i * HS; };
  // FULL: the singlet (k = 0) and vphi's components (k = 1, 2)
  auto sX = [&](int s, int k) { return reinterpret_cast<T*>(smem + s * slot_b) + 19 * HS + k * HS; };

  // the 35 raw values of halo site k of plane zp, all loads issued before any use
  // (the source buffer is read-only during the pass)
  auto fetch = [&](int k, int x0, int y0, int zp, T (&r)[NLD]) {
    const int hx = k % HX, hy = k / HX;
    int gx = x0 + hx - 1, gy = y0 + hy - 1;
    gx = gx < 0 ? gx + N : (gx >= N ? gx - N : gx);
    gy = gy < 0 ? gy + N : (gy >= N ? gy - N : gy);
    const T* p = src + ((long long)zp * NN + (long long)gy * N + gx);
#pragma unroll
    for (int a = 0; a < NLD; ++a) {
      r[a] = __ldg(p);
      p += V;
    }
  };
  // drift halo site k into ring slot s; own sites written out when `own`
  auto put = [&](int s, int k, int x0, int y0, int zp, bool own, const T (&r)[NLD]) {
    Q4<T> f, u[3];
    T a[3];
    f.w = r[SF];
    f.x = r[SF + 1];
    f.y = r[SF + 2];
    f.z = r[SF + 3];
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      a[i] = r[SA + i];
      u[i].w = r[SU + 4 * i];
      u[i].x = r[SU + 4 * i + 1];
      u[i].y = r[SU + 4 * i + 2];
      u[i].z = r[SU + 4 * i + 3];
    }
    if (drifting) {
      f.w = fmaT(cd, r[SP], f.w);
      f.x = fmaT(cd, r[SP + 1], f.x);
      f.y = fmaT(cd, r[SP + 2], f.y);
      f.z = fmaT(cd, r[SP + 3], f.z);
#pragma unroll
      for (int i = 0; i < 3; ++i) {
        a[i] = fmaT(cdA, r[SPA + i], a[i]);
        // E = exp(-i hB pi.s) = (cos x, sin(x)/x hB pi), x = hB |pi|
        const T p1 = hB * r[SPB + 3 * i], p2 = hB * r[SPB + 3 * i + 1], p3 = hB * r[SPB + 3 * i + 2];
        T c, sc;
        cos_sinc(p1 * p1 + p2 * p2 + p3 * p3, c, sc);
        Q4<T> e;
        e.w = c;
        e.x = sc * p1;
        e.y = sc * p2;
        e.z = sc * p3;
        u[i] = qmul(e, u[i]);
        renorm(u[i]);
      }
    }
    sF(s)[k] = f;
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      sU(s, i)[k] = u[i];
      sA(s, i)[k] = a[i];
    }
    T xs[3] = {T(0), T(0), T(0)};  // FULL: phi_s, vphi_0, vphi_1, drifted
    if constexpr (FULL) {
      xs[0] = drifting ? fmaT(cd, r[SPS], r[SS]) : r[SS];
      xs[1] = drifting ? fmaT(cd, r[SPC], r[SC]) : r[SC];
      xs[2] = drifting ? fmaT(cd, r[SPC + 1], r[SC + 1]) : r[SC + 1];
#pragma unroll
      for (int m = 0; m < 3; ++m) sX(s, m)[k] = xs[m];
    }
    const int hx = k % HX, hy = k / HX;
    if (own && P.write && hx >= 1 && hx <= TX && hy >= 1 && hy <= TY) {
      T* o = dst + ((long long)zp * NN + (long long)(y0 + hy - 1) * N + (x0 + hx - 1));
      const T vals[19] = {f.w, f.x, f.y, f.z, a[0], a[1], a[2], u[0].w, u[0].x, u[0].y, u[0].z,
                          u[1].w, u[1].x, u[1].y, u[1].z, u[2].w, u[2].x, u[2].y, u[2].z};
#pragma unroll
      for (int m = 0; m < 19; ++m) {  // arrays 0..3, 8..10, 14..25
        const int arr = m < 4 ? SF + m : (m < 7 ? SA + (m - 4) : SU + (m - 7));
        o[arr * V] = vals[m];
      }
      if constexpr (FULL) {
        o[SS * V] = xs[0];
        o[SC * V] = xs[1];
        o[(SC + 1) * V] = xs[2];
      }
    }
  };
  // plane zp of tile (x0, y0) into slot s, drifted
  auto load_plane = [&](int s, int x0, int y0, int zp, bool own) {
    for (int k = tid; k < HS; k += nth) {
      T r0[NLD];
      fetch(k, x0, y0, zp, r0);
      put(s, k, x0, y0, zp, own, r0);
    }
  };

  // work items: (tile, z-chunk), tile = by * ntx + bx, numbered chunk-major; CTA b takes
  // items b, b + gridDim.x, ...  A round of items covers about one chunk of every tile,
  // so neighbouring tiles march the same planes at about the same time and the halo
  // rows and columns a CTA reads come from L2 rather than DRAM.
  const int ntiles = ntx * nty, nzc = L.su2_nzc, nitems = ntiles * nzc;
  for (int item = blockIdx.x; item < nitems; item += gridDim.x) {
    const int tile = item % ntiles, chunk = item / ntiles;
    const int z0 = (int)((long long)chunk * N / nzc);
    const int nz = (int)((long long)(chunk + 1) * N / nzc) - z0;
    const int x0 = (tile % ntx) * TX, y0 = (tile / ntx) * TY;
    __syncthreads();  // the previous item's reads of the ring are done
    load_plane(0, x0, y0, (z0 - 1 + N) % N, false);
    load_plane(1, x0, y0, z0, true);
    const int hx = tx + 1, hy = ty + 1, own = hy * HX + hx;
    const long long gown = (long long)(y0 + ty) * N + x0 + tx;
    for (int j = 0; j < nz; ++j) {
      const int z = z0 + j;
      const int sm = j % 3, sc = (j + 1) % 3, sp = (j + 2) % 3;
      const long long g = (long long)z * NN + gown;
      {  // the kick's own momenta move into L1 while the next plane loads
        const T* pp = src + g;
        prefetch_l1(pp + SP * V);
        prefetch_l1(pp + (SP + 1) * V);
        prefetch_l1(pp + (SP + 2) * V);
        prefetch_l1(pp + (SP + 3) * V);
#pragma unroll
        for (int m = 0; m < 3; ++m) prefetch_l1(pp + (SPA + m) * V);
#pragma unroll
        for (int m = 0; m < 9; ++m) prefetch_l1(pp + (SPB + m) * V);
        if constexpr (FULL) {
          prefetch_l1(pp + SPS * V);
          prefetch_l1(pp + SPC * V);
          prefetch_l1(pp + (SPC + 1) * V);
        }
      }
      load_plane(sp, x0, y0, (z + 1) % N, j + 1 < nz);
      __syncthreads();
      // neighbours in the ring: (dx, dy) in the plane, slot for dz
      auto at = [&](int ddx, int ddy) { return own + ddy * HX + ddx; };
      const Q4<T> psi = sF(sc)[own];
      Q4<T> D;
      D.w = T(-6) * psi.w;
      D.x = T(-6) * psi.x;
      D.y = T(-6) * psi.y;
      D.z = T(-6) * psi.z;
      T s_g = T(0), s_pA = T(0), s_pB = T(0), s_mA = T(0), s_mB = T(0);
      T pnA[3], pnB[3][3];
      // FULL: the singlet's Laplacian and gradient sum, vphi's covariant Laplacian and gradient sum
      T xs0 = T(0), xc0 = T(0), xc1 = T(0), Ls = T(0), Dv0 = T(0), Dv1 = T(0), s_gs = T(0), s_gc = T(0);
      if constexpr (FULL) {
        xs0 = sX(sc, 0)[own];
        xc0 = sX(sc, 1)[own];
        xc1 = sX(sc, 2)[own];
        Ls = T(-6) * xs0;
        Dv0 = T(-6) * xc0;
        Dv1 = T(-6) * xc1;
      }
      // U(1) plaquette sines: xy, xz, yz at n, then the lower ones
      const T ax = sA(sc, 0)[own], ay = sA(sc, 1)[own], az = sA(sc, 2)[own];
      T sxy = T(0), sxz = T(0), syz = T(0), Cx = T(0), Cy = T(0), Cz = T(0);
      if (ACA != T(0) || RED > 0) {
        const T txy = gd * ((ax + sA(sc, 1)[at(1, 0)]) - (sA(sc, 0)[at(0, 1)] + ay));
        const T txz = gd * ((ax + sA(sc, 2)[at(1, 0)]) - (sA(sp, 0)[own] + az));
        const T tyz = gd * ((ay + sA(sc, 2)[at(0, 1)]) - (sA(sp, 1)[own] + az));
        sxy = sin_t(txy);
        sxz = sin_t(txz);
        syz = sin_t(tyz);
        const T sxy_ym = sin_t(gd * ((sA(sc, 0)[at(0, -1)] + sA(sc, 1)[at(1, -1)]) - (ax + sA(sc, 1)[at(0, -1)])));
        const T sxy_xm = sin_t(gd * ((sA(sc, 0)[at(-1, 0)] + ay) - (sA(sc, 0)[at(-1, 1)] + sA(sc, 1)[at(-1, 0)])));
        const T sxz_zm = sin_t(gd * ((sA(sm, 0)[own] + sA(sm, 2)[at(1, 0)]) - (ax + sA(sm, 2)[own])));
        const T sxz_xm = sin_t(gd * ((sA(sc, 0)[at(-1, 0)] + az) - (sA(sp, 0)[at(-1, 0)] + sA(sc, 2)[at(-1, 0)])));
        const T syz_zm = sin_t(gd * ((sA(sm, 1)[own] + sA(sm, 2)[at(0, 1)]) - (ay + sA(sm, 2)[own])));
        const T syz_ym = sin_t(gd * ((sA(sc, 1)[at(0, -1)] + az) - (sA(sp, 1)[at(0, -1)] + sA(sc, 2)[at(0, -1)])));
        Cx = (sxy - sxy_ym) + (sxz - sxz_zm);
        Cy = (sxy_xm - sxy) + (syz - syz_zm);
        Cz = (sxz_xm - sxz) + (syz_ym - syz);
        if constexpr (RED > 0) {
          const T hx2 = sin_t(T(0.5) * txy), hy2 = sin_t(T(0.5) * txz), hz2 = sin_t(T(0.5) * tyz);
          s_mA = T(2) * (hx2 * hx2 + hy2 * hy2 + hz2 * hz2);
        }
      }
      const T Cc[3] = {Cx, Cy, Cz};
#pragma unroll
      for (int i = 0; i < 3; ++i) {
        // ---- doublet hops along i, currents ----
        const Q4<T> Ui = sU(sc, i)[own];
        const int fx = i == 0 ? 1 : 0, fy = i == 1 ? 1 : 0;
        const Q4<T> fn = i == 2 ? sF(sp)[own] : sF(sc)[at(fx, fy)];
        Q4<T> chi = umul(Ui, fn);
        T c, s;
        sincos_t(gd * sA(sc, i)[own], s, c);
        phase(chi, c, s);
        const int bs = i == 2 ? sm : sc;
        const int bk = i == 2 ? own : at(-fx, -fy);
        Q4<T> back = udmul(sU(bs, i)[bk], sF(bs)[bk]);
        sincos_t(gd * sA(bs, i)[bk], s, c);
        phase(back, c, -s);
        D.w += chi.w + back.w;
        D.x += chi.x + back.x;
        D.y += chi.y + back.y;
        D.z += chi.z + back.z;
        // psi = (p, q) = (w + i x, y + i z), chi = (c1, c2)
        const T ImA = (psi.w * chi.x - psi.x * chi.w) + (psi.y * chi.z - psi.z * chi.y);     // Im psi^dag chi
        const T Im1 = (psi.w * chi.z - psi.x * chi.y) + (psi.y * chi.x - psi.z * chi.w);     // Im psi^dag s1 chi
        const T Im2 = (psi.y * chi.w + psi.z * chi.x) - (psi.w * chi.y + psi.x * chi.z);     // Im psi^dag s2 chi
        const T Im3 = (psi.w * chi.x - psi.x * chi.w) - (psi.y * chi.z - psi.z * chi.y);     // Im psi^dag s3 chi
        if constexpr (RED > 0) {
          const T e0 = chi.w - psi.w, e1 = chi.x - psi.x, e2 = chi.y - psi.y, e3 = chi.z - psi.z;
          s_g += (e0 * e0 + e1 * e1) + (e2 * e2 + e3 * e3);
        }
        // ---- SU(2) staples of U_i(n) ----
        Q4<T> S;
        S.w = S.x = S.y = S.z = T(0);
#pragma unroll
        for (int jj = 1; jj <= 2; ++jj) {
          const int j = (i + jj) % 3;
          const int gx = j == 0 ? 1 : 0, gy = j == 1 ? 1 : 0;
          // U_j(n+i), U_i(n+j), U_j(n)
          const Q4<T> ujni = i == 2 ? sU(sp, j)[own] : sU(sc, j)[at(fx, fy)];
          const Q4<T> uinj = j == 2 ? sU(sp, i)[own] : sU(sc, i)[at(gx, gy)];
          const Q4<T> ujn = sU(sc, j)[own];
          const Q4<T> up = qmul(qmul(ujni, qconj(uinj)), qconj(ujn));
          // U_j(n+i-j), U_i(n-j), U_j(n-j)
          Q4<T> ujnimj, uinmj, ujnmj;
          if (j == 2) {
            ujnimj = i == 2 ? sU(sc, j)[own] : sU(sm, j)[at(fx, fy)];
            uinmj = sU(sm, i)[own];
            ujnmj = sU(sm, j)[own];
          } else if (i == 2) {
            ujnimj = sU(sp, j)[at(-gx, -gy)];
            uinmj = sU(sc, i)[at(-gx, -gy)];
            ujnmj = sU(sc, j)[at(-gx, -gy)];
          } else {
            ujnimj = sU(sc, j)[at(fx - gx, fy - gy)];
            uinmj = sU(sc, i)[at(-gx, -gy)];
            ujnmj = sU(sc, j)[at(-gx, -gy)];
          }
          const Q4<T> lo = qmul(qmul(qconj(ujnimj), qconj(uinmj)), ujnmj);
          qadd(S, up);
          qadd(S, lo);
          if constexpr (RED > 0) {
            if (j > i) s_mB += one_minus_w(qmul(Ui, up));
          }
        }
        const Q4<T> M = qmul(Ui, S);
        // ---- link kicks ----
        const T pA = __ldg(src + (SPA + i) * V + g);
        pnA[i] = pA + (AJA * ImA + ACA * Cc[i]);
        if constexpr (FULL) {
          // singlet neighbours along i
          const T sfw = i == 2 ? sX(sp, 0)[own] : sX(sc, 0)[at(fx, fy)];
          const T sbw = sX(bs, 0)[bk];
          Ls += sfw + sbw;
          // vphi: forward hop Vc_i(n) vphi(n+i), backward hop Vc_i^*(n-i) vphi(n-i), Vc = exp(-i Qc gQ dx A)
          const T y0 = i == 2 ? sX(sp, 1)[own] : sX(sc, 1)[at(fx, fy)];
          const T y1 = i == 2 ? sX(sp, 2)[own] : sX(sc, 2)[at(fx, fy)];
          T cc, sc2;
          sincos_t(gdc * sA(sc, i)[own], sc2, cc);
          const T u0 = cc * y0 + sc2 * y1, u1 = cc * y1 - sc2 * y0;
          const T b0 = sX(bs, 1)[bk], b1 = sX(bs, 2)[bk];
          sincos_t(gdc * sA(bs, i)[bk], sc2, cc);
          const T w0 = cc * b0 - sc2 * b1, w1 = cc * b1 + sc2 * b0;
          Dv0 += u0 + w0;
          Dv1 += u1 + w1;
          pnA[i] += AJC * (xc0 * u1 - xc1 * u0);
          if constexpr (RED > 0) {
            const T gs = sfw - xs0, g0 = u0 - xc0, g1 = u1 - xc1;
            s_gs += gs * gs;
            s_gc += g0 * g0 + g1 * g1;
          }
        }
        const T Ims[3] = {Im1, Im2, Im3};
        const T Ms[3] = {M.x, M.y, M.z};
#pragma unroll
        for (int a = 0; a < 3; ++a) {
          const T pB = __ldg(src + (SPB + 3 * i + a) * V + g);
          pnB[i][a] = pB + (AJB * Ims[a] + AMB * Ms[a]);
        }
        if constexpr (RED > 0) {
          s_pA += pnA[i] * pnA[i];
          s_pB += pnB[i][0] * pnB[i][0] + pnB[i][1] * pnB[i][1] + pnB[i][2] * pnB[i][2];
        }
      }
      // ---- doublet kick ----
      const T r2 = T(0.5) * ((psi.w * psi.w + psi.x * psi.x) + (psi.y * psi.y + psi.z * psi.z));
      const T dd = r2 - v2;
      T gp = lam2 * dd;
      T c2v = T(0);  // FULL: |vphi|^2
      if constexpr (FULL) {
        c2v = T(0.5) * (xc0 * xc0 + xc1 * xc1);
        gp += qG * xs0 * xs0 + T(2) * qH * c2v;
      }
      T pn[4];
      const T Dc[4] = {D.w, D.x, D.y, D.z};
      const T fc[4] = {psi.w, psi.x, psi.y, psi.z};
#pragma unroll
      for (int c2 = 0; c2 < 4; ++c2) pn[c2] = __ldg(src + (SP + c2) * V + g) + (A1 * Dc[c2] - A3 * gp * fc[c2]);
      // FULL: kicks of the singlet and of vphi
      T pns = T(0), pnc0 = T(0), pnc1 = T(0);
      if constexpr (FULL) {
        pns = __ldg(src + SPS * V + g) + (A1 * Ls - A3 * (T(2) * qG * r2) * xs0);
        pnc0 = __ldg(src + SPC * V + g) + (A1 * Dv0 - A3 * (T(2) * qH * r2) * xc0);
        pnc1 = __ldg(src + (SPC + 1) * V + g) + (A1 * Dv1 - A3 * (T(2) * qH * r2) * xc1);
        if (P.write) {
          dst[SPS * V + g] = pns;
          dst[SPC * V + g] = pnc0;
          dst[(SPC + 1) * V + g] = pnc1;
        }
      }
      if (P.write) {
#pragma unroll
        for (int c2 = 0; c2 < 4; ++c2) dst[(SP + c2) * V + g] = pn[c2];
#pragma unroll
        for (int i = 0; i < 3; ++i) {
          dst[(SPA + i) * V + g] = pnA[i];
#pragma unroll
          for (int a = 0; a < 3; ++a) dst[(SPB + 3 * i + a) * V + g] = pnB[i][a];
        }
      }
      if constexpr (RED == 1) {
        acc[0].add((pn[0] * pn[0] + pn[1] * pn[1]) + (pn[2] * pn[2] + pn[3] * pn[3]));
        acc[1].add(s_pA + s_pB);
        acc[2].add(s_g);
        acc[3].add(s_mA);
        acc[4].add(s_mB);
        acc[5].add(lam * dd * dd);
        if constexpr (FULL) {  // the Friedmann kick takes the totals
          acc[0].add(pns * pns + (pnc0 * pnc0 + pnc1 * pnc1));
          acc[2].add(s_gs + s_gc);
          acc[5].add(qG * r2 * xs0 * xs0 + T(2) * qH * r2 * c2v);
        }
      } else if constexpr (RED == 2) {
#pragma unroll
        for (int c2 = 0; c2 < 4; ++c2) {
          acc[c2].add(pn[c2] * pn[c2]);
          acc[10 + c2].add(fc[c2]);
          acc[14 + c2].add(fc[c2] * fc[c2]);
          acc[18 + c2].add(pn[c2]);
          if (!isfinite(pn[c2])) nonfinite += 1.f;
        }
        acc[4].add(s_pA);
        acc[5].add(s_pB);
        acc[6].add(s_g);
        acc[7].add(s_mA);
        acc[8].add(s_mB);
        acc[9].add(lam * dd * dd);
        if (!isfinite(s_pA) || !isfinite(s_pB)) nonfinite += 1.f;
        if constexpr (FULL) {  // per species: singlet, vphi
          acc[23].add(pns * pns);
          acc[24].add(pnc0 * pnc0 + pnc1 * pnc1);
          acc[25].add(s_gs);
          acc[26].add(s_gc);
          acc[27].add(qG * r2 * xs0 * xs0);
          acc[28].add(T(2) * qH * r2 * c2v);
          if (!isfinite(pns) || !isfinite(pnc0) || !isfinite(pnc1)) nonfinite += 1.f;
        }
      }
      __syncthreads();  // slot sm is overwritten by the next load
    }
  }

  su2_pass_end<T, RED, FULL>(P, L, acc, nonfinite, red_s, last_s, tid, lane, warp, nth);
}

typedef void (*PassKernel)(const PassArgs);

PassKernel su2_pass_kernel(int fp32, int red, int TX, int full) {
  static const PassKernel tab[2][2][3] = {
      {{dk_pass_su2<double, 0, 16, false>, dk_pass_su2<double, 1, 16, false>, dk_pass_su2<double, 2, 16, false>},
       {dk_pass_su2<float, 0, 16, false>, dk_pass_su2<float, 1, 16, false>, dk_pass_su2<float, 2, 16, false>}},
      {{dk_pass_su2<double, 0, 32, false>, dk_pass_su2<double, 1, 32, false>, dk_pass_su2<double, 2, 32, false>},
       {dk_pass_su2<float, 0, 32, false>, dk_pass_su2<float, 1, 32, false>, dk_pass_su2<float, 2, 32, false>}}};
  static const PassKernel tab_full[2][2][3] = {
      {{dk_pass_su2<double, 0, 16, true>, dk_pass_su2<double, 1, 16, true>, dk_pass_su2<double, 2, 16, true>},
       {dk_pass_su2<float, 0, 16, true>, dk_pass_su2<float, 1, 16, true>, dk_pass_su2<float, 2, 16, true>}},
      {{dk_pass_su2<double, 0, 32, true>, dk_pass_su2<double, 1, 32, true>, dk_pass_su2<double, 2, 32, true>},
       {dk_pass_su2<float, 0, 32, true>, dk_pass_su2<float, 1, 32, true>, dk_pass_su2<float, 2, 32, true>}}};
  if (red < 0 || red > 2 || (TX != 16 && TX != 32)) return nullptr;
  return (full ? tab_full : tab)[TX == 32 ? 1 : 0][fp32 ? 1 : 0][red];
}

size_t su2_smem_bytes(int TX, int TY, int esz, int full) { return 3 * su2_slot_bytes(TX, TY, esz, full != 0); }

// ---------------------------------------------------------------------------
// Initial state and the Gauss-law monitor of the doublet model.
// ---------------------------------------------------------------------------

// links at the identity (eqs. Inflc1-2): u0 = 1, the rest zero (caller zeroed the slab)
template <typename T>
__global__ void su2_identity_links_kernel(T* base, long long V) {
  for (long long n = (long long)blockIdx.x * blockDim.x + threadIdx.x; n < V;
       n += (long long)gridDim.x * blockDim.x)
#pragma unroll
    for (int i = 0; i < 3; ++i) base[(SU + 4 * i) * V + n] = T(1);
}

template <typename T>
__device__ __forceinline__ Q4<double> dq(const T* b, int a, long long V, long long n) {
  Q4<double> r;
  r.w = (double)b[a * V + n];
  r.x = (double)b[(a + 1) * V + n];
  r.y = (double)b[(a + 2) * V + n];
  r.z = (double)b[(a + 3) * V + n];
  return r;
}

// Charge density of generator g (0: U(1); 1..3: SU(2) colour g) at site n:
//   U(1):  (f_s/omega_s)^2 gQ Im[psi^dag pi_psi]
//   SU(2): (f_s/omega_s)^2 (gQB/2) Im[psi^dag s_g pi_psi]
template <typename T>
__device__ double su2_rho(const LatConst& L, const T* b, int g, long long n) {
  const long long V = L.V;
  const Q4<double> f = dq(b, SF, V, n), p = dq(b, SP, V, n);
  double im;
  if (g == 0) im = (f.w * p.x - f.x * p.w) + (f.y * p.z - f.z * p.y);
  else if (g == 1) im = (f.w * p.z - f.x * p.y) + (f.y * p.x - f.z * p.w);
  else if (g == 2) im = (f.y * p.w + f.z * p.x) - (f.w * p.y + f.x * p.z);
  else im = (f.w * p.x - f.x * p.w) - (f.y * p.z - f.z * p.y);
  if (g == 0 && L.model == CL_MODEL_LPHI4_SU2U1)  // vphi's charge density, charge Qc in units of the doublet's
    im += L.Qc * ((double)b[SC * V + n] * (double)b[(SPC + 1) * V + n] -
                  (double)b[(SC + 1) * V + n] * (double)b[SPC * V + n]);
  return L.fo2 * (g == 0 ? L.gQ : 0.5 * L.gQB) * im;
}

template <typename T>
__global__ void su2_rho_kernel(const LatConst* Lc, int parity, int g, double2* rho) {
  const LatConst& L = *Lc;
  const T* b = reinterpret_cast<const T*>(L.buf[parity][0]);
  for (long long n = (long long)blockIdx.x * blockDim.x + threadIdx.x; n < L.V;
       n += (long long)gridDim.x * blockDim.x)
    rho[n] = make_double2(su2_rho<T>(L, b, g, n), 0.0);
}

// |L - R|, |L + R| summed over the four laws, and max |L - R|, per block.
template <typename T>
__global__ void su2_gauss_monitor_kernel(const LatConst* Lc, int parity, double* part) {
  __shared__ double sh[3][32];
  const LatConst& L = *Lc;
  const T* b = reinterpret_cast<const T*>(L.buf[parity][0]);
  const int N = L.N;
  const long long NN = (long long)N * N, V = L.V;
  double sd = 0.0, ss = 0.0, mx = 0.0;
  for (long long n = (long long)blockIdx.x * blockDim.x + threadIdx.x; n < V;
       n += (long long)gridDim.x * blockDim.x) {
    const int x = (int)(n % N), y = (int)((n / N) % N), z = (int)(n / NN);
    const long long nm[3] = {x ? n - 1 : n + N - 1, y ? n - N : n + NN - N, z ? n - NN : n + V - NN};
    double lhs[4] = {0.0, 0.0, 0.0, 0.0};
    for (int i = 0; i < 3; ++i) {
      const long long m = nm[i];
      lhs[0] += (double)b[(SPA + i) * V + n] - (double)b[(SPA + i) * V + m];
      // (U^dag P U)^a, P = p.s/2 at n - i: rotation of p by the link
      const Q4<double> u = dq(b, SU + 4 * i, V, m);
      Q4<double> pq;
      pq.w = 0.0;
      pq.x = (double)b[(SPB + 3 * i) * V + m];
      pq.y = (double)b[(SPB + 3 * i + 1) * V + m];
      pq.z = (double)b[(SPB + 3 * i + 2) * V + m];
      const Q4<double> r = qmul(qmul(qconj(u), pq), u);
      lhs[1] += (double)b[(SPB + 3 * i) * V + n] - r.x;
      lhs[2] += (double)b[(SPB + 3 * i + 1) * V + n] - r.y;
      lhs[3] += (double)b[(SPB + 3 * i + 2) * V + n] - r.z;
    }
    for (int g2 = 0; g2 < 4; ++g2) {
      const double l = lhs[g2] / L.dx, r = su2_rho<T>(L, b, g2, n);
      const double d = fabs(l - r);
      sd += d;
      ss += fabs(l + r);
      mx = fmax(mx, d);
    }
  }
  for (int o = 16; o > 0; o >>= 1) {
    sd += __shfl_down_sync(0xffffffffu, sd, o);
    ss += __shfl_down_sync(0xffffffffu, ss, o);
    mx = fmax(mx, __shfl_down_sync(0xffffffffu, mx, o));
  }
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (lane == 0) {
    sh[0][w] = sd;
    sh[1][w] = ss;
    sh[2][w] = mx;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double a = 0.0, c = 0.0, m = 0.0;
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) {
      a += sh[0][i];
      c += sh[1][i];
      m = fmax(m, sh[2][i]);
    }
    part[3 * blockIdx.x] = a;
    part[3 * blockIdx.x + 1] = c;
    part[3 * blockIdx.x + 2] = m;
  }
}

__global__ void su2_gauss_final_kernel(const double* part, int nblk, long long V, double* out) {
  if (threadIdx.x | blockIdx.x) return;
  double a = 0.0, b = 0.0, m = 0.0;
  for (int i = 0; i < nblk; ++i) {
    a += part[3 * i];
    b += part[3 * i + 1];
    m = fmax(m, part[3 * i + 2]);
  }
  out[0] = b > 0.0 ? a / b : 0.0;
  out[1] = a / (double)V;
  out[2] = b / (double)V;
  out[3] = m;
}

cudaError_t launch_su2_identity_links(int fp32, void* base, long long V, cudaStream_t st) {
  const int tb = 256;
  const int g = (int)((V + tb - 1) / tb < 65536 ? (V + tb - 1) / tb : 65536);
  if (fp32) su2_identity_links_kernel<float><<<g, tb, 0, st>>>((float*)base, V);
  else su2_identity_links_kernel<double><<<g, tb, 0, st>>>((double*)base, V);
  return cudaGetLastError();
}

cudaError_t launch_su2_rho(int fp32, const LatConst* L, int parity, int g, double2* rho, long long V,
                           cudaStream_t st) {
  const int tb = 256;
  const int gr = (int)((V + tb - 1) / tb < 65536 ? (V + tb - 1) / tb : 65536);
  if (fp32) su2_rho_kernel<float><<<gr, tb, 0, st>>>(L, parity, g, rho);
  else su2_rho_kernel<double><<<gr, tb, 0, st>>>(L, parity, g, rho);
  return cudaGetLastError();
}

cudaError_t launch_su2_gauss_monitor(int fp32, const LatConst* L, int parity, double* part, int nblk,
                                     long long V, cudaStream_t st) {
  if (fp32) su2_gauss_monitor_kernel<float><<<nblk, 256, 0, st>>>(L, parity, part);
  else su2_gauss_monitor_kernel<double><<<nblk, 256, 0, st>>>(L, parity, part);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  su2_gauss_final_kernel<<<1, 32, 0, st>>>(part, nblk, V, part + 3 * nblk);
  return cudaGetLastError();
}

}  // namespace clg
