// ic_fft.cu -- initial conditions, 3-D FFT and binned power spectra, all on
// the GPU (outside the timed evolution loop).
//
// Initial conditions (CosmoLattice manual Sec. 3.5.1, eqs. fpr_influct,
// fpr_influct2, QuantumFlucts2; Sec. 4.4.1 eqs. InConstr:1-2 for the charged
// field): in Fourier space each mode gets two left/right moving waves with
// Rayleigh amplitudes (<|d|^2> = P) and uniform phases,
//   P = (omega_s/f_s)^2 (N/dx)^3 / (2 a^2 omega_k),  omega_k = sqrt(k^2 + a^2 m^2),
// drawn from the counter-based generator Philox4x32-10 (Salmon et al., SC'11)
// keyed by the seed, with counter (Fourier index, field, draw, 0).  Only the
// member of each (n, -n) pair with the smaller index is drawn; its partner is
// the complex conjugate so that the field is real.
#include <stdint.h>

#include "common.cuh"

namespace clg {


// ---------------------------------------------------------------------------
// Philox4x32-10: 10 rounds of (two 32x32 -> 64 bit products, xor with the
// other words and the round key), key advanced by the Weyl constants.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void philox4x32_10(uint32_t c[4], uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    if (r) {
      k0 += 0x9E3779B9u;
      k1 += 0xBB67AE85u;
    }
    const uint32_t lo0 = 0xD2511F53u * c[0], hi0 = __umulhi(0xD2511F53u, c[0]);
    const uint32_t lo1 = 0xCD9E8D57u * c[2], hi1 = __umulhi(0xCD9E8D57u, c[2]);
    const uint32_t n0 = hi1 ^ c[1] ^ k0, n2 = hi0 ^ c[3] ^ k1;
    c[0] = n0;
    c[1] = lo1;
    c[2] = n2;
    c[3] = lo0;
  }
}

// (0, 1] with 53 bits: top 27 bits of the first word, top 26 of the second.
__device__ __forceinline__ double unit_open0(uint32_t hi, uint32_t lo) {
  const unsigned long long m = ((unsigned long long)(hi >> 5) << 26) | (unsigned long long)(lo >> 6);
  return ((double)m + 1.0) * 0x1.0p-53;
}

__device__ __forceinline__ void draw_pair(unsigned long long seed, unsigned idx, int f, int j,
                                          double& u0, double& u1) {
  uint32_t c[4] = {idx, (uint32_t)f, (uint32_t)j, 0u};
  philox4x32_10(c, (uint32_t)(seed & 0xffffffffull), (uint32_t)(seed >> 32));
  u0 = unit_open0(c[0], c[1]);
  u1 = unit_open0(c[2], c[3]);
}

// Potential of each model at homogeneous values, and d^2V/dphi_f^2 (the
// initial effective masses of eq. QuantumFlucts2).
__device__ double pot_hom(const ICArgs& A) {
  const double* f = A.phi0;
  if (A.model == CL_MODEL_LPHI4) return 0.25 * f[0] * f[0] * f[0] * f[0];
  if (A.model == CL_MODEL_LPHI4_CHI)
    return 0.25 * f[0] * f[0] * f[0] * f[0] + 0.5 * A.q * f[0] * f[0] * f[1] * f[1];
  double r2 = 0.0;  // |phi|^2 (|Phi|^2 for the doublet) = half the sum of squares of the components
  for (int k = 0; k < A.nf; ++k) r2 += 0.5 * f[k] * f[k];
  const double m2 = r2 - A.v * A.v;
  return A.lam * m2 * m2;
}

__device__ double mass2_hom(const ICArgs& A, int k) {
  const double* f = A.phi0;
  if (A.model == CL_MODEL_LPHI4) return 3.0 * f[0] * f[0];
  if (A.model == CL_MODEL_LPHI4_CHI)
    return k == 0 ? 3.0 * f[0] * f[0] + A.q * f[1] * f[1] : A.q * f[0] * f[0];
  double r2 = 0.0;
  for (int c = 0; c < A.nf; ++c) r2 += 0.5 * f[c] * f[c];
  // lphi4SU2U1 (eq. PotGauge): the singlet (k = 4) and vphi (k = 5, 6) start at
  // zero, so only their own masses 2 qG |Phi|^2 and 2 qH |Phi|^2 are new
  if (A.model == CL_MODEL_LPHI4_SU2U1 && k == 4) return 2.0 * A.qG * r2;
  if (A.model == CL_MODEL_LPHI4_SU2U1 && k > 4) return 2.0 * A.qH * r2;
  return 2.0 * A.lam * (r2 - A.v * A.v) + 2.0 * A.lam * f[k] * f[k];
}

// Scale factor and b = a' at t0 (ScalarFactorInitializer: homogeneous values).
__global__ void init_scalars_kernel(const LatConst* Lc, LatScalars* Sc, const ICArgs A) {
  if (threadIdx.x | blockIdx.x) return;
  const LatConst& L = *Lc;
  LatScalars& S = *Sc;
  const double al = L.alpha;
  S.a = S.a0 = 1.0;
  S.eta = S.eta0 = 0.0;
  S.cd = S.cdA = 0.0;
  S.apow1 = S.apow3 = S.apowm1 = 1.0;
  S.status = 0;
  S.rho0 = 0.0;
  S.pi2 = 0.0;
  S.pi2A = 0.0;
  S.adjq = 0.0;
  double kin = 0.0;
  for (int k = 0; k < A.nf; ++k) kin += 0.5 * A.dphi0[k] * A.dphi0[k];
  const double rho = kin / pow(S.a, 2.0 * al) + pot_hom(A);
  const double r = pow(S.a, 2.0 * al + 2.0) / 3.0 * L.fm2 * rho;
  const double bh = r > 0.0 ? sqrt(r) : 0.0;
  if (L.expansion == CL_EXP_SELF) {
    S.Hfix = 0.0;
    S.b = bh;
  } else if (L.expansion == CL_EXP_FIXED) {
    S.Hfix = A.H0 > 0.0 ? A.H0 : bh / S.a;
    S.b = S.a * S.Hfix;
  } else {
    S.Hfix = 0.0;
    S.b = 0.0;
  }
  S.H_ic = S.b / S.a;
}

// Fourier modes of the fluctuation of component f (F) and of its derivative (G).
// Buffers are zeroed by the caller; only drawn modes are written.
// Draws of component f at Fourier site idx (its canonical member: idx <=
// partner, *pid_out receives the partner): amplitudes r1, r2, phases t1, t2
// in units of pi, and omega_k.  False for sites that stay zero.
__device__ bool mode_draw(const LatConst& L, const ICArgs& A, double a, long long idx, int f,
                          long long* pid_out, double& r1, double& r2, double& t1, double& t2,
                          double& omf) {
  const int N = L.N;
  if (idx == 0) return false;
  const int x = (int)(idx % N), y = (int)((idx / N) % N), z = (int)(idx / ((long long)N * N));
  const int px = x ? N - x : 0, py = y ? N - y : 0, pz = z ? N - z : 0;
  const long long pid = px + (long long)N * (py + (long long)N * pz);
  *pid_out = pid;
  if (pid < idx) return false;
  const bool gauge = A.model == CL_MODEL_U1_HIGGS || A.model == CL_MODEL_SU2U1_HIGGS ||
                     A.model == CL_MODEL_LPHI4_SU2U1;
  if (pid == idx && gauge) return false;  // keeps the charge density's zero mode at 0
  // components: the model's nf, and for lphi4SU2U1 also the singlet (4) and vphi (5, 6)
  const int nc = A.model == CL_MODEL_LPHI4_SU2U1 ? 7 : A.nf;
  // charged groups draw their phases under eqs. InConstr:1-2 with their first component as reference
  const bool charged = gauge && f != 4;
  const int fref = f < 4 ? 0 : 5;
  const int nx = x <= N / 2 ? x : x - N, ny = y <= N / 2 ? y : y - N, nz = z <= N / 2 ? z : z - N;
  const double k = A.kIR * sqrt((double)(nx * nx + ny * ny + nz * nz));
  if (A.kcut >= 0.0 && k > A.kcut) return false;
  if (A.amp2 <= 0.0) return false;
  // every component must have a real frequency for the mode to be populated
  double om[7] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
  for (int c = 0; c < nc; ++c) {
    const double w2 = k * k + a * a * mass2_hom(A, c);
    if (w2 <= 0.0) return false;
    om[c] = sqrt(w2);
  }
  omf = om[f];
  const double vol = (double)N / L.dx;
  const double P = A.amp2 * vol * vol * vol / (2.0 * a * a * om[f]);
  if (!charged) {
    double u0, u1, v0, v1;
    draw_pair(A.seed, (unsigned)idx, f, 0, u0, u1);
    draw_pair(A.seed, (unsigned)idx, f, 1, v0, v1);
    r1 = sqrt(-P * log(u0));
    r2 = sqrt(-P * log(u1));
    t1 = 2.0 * v0;  // phases in units of pi
    t2 = 2.0 * v1;
  } else {
    // eqs. InConstr:1-2: equal amplitudes per component, theta_n2 = theta_02 + theta_n1 - theta_01
    double u0, u1, v0, v1;
    draw_pair(A.seed, (unsigned)idx, f, 0, u0, u1);
    r1 = r2 = sqrt(-P * log(u0));
    draw_pair(A.seed, (unsigned)idx, fref, 1, v0, v1);  // theta_01, theta_02 of the group
    if (f == fref) {
      t1 = 2.0 * v0;
      t2 = 2.0 * v1;
    } else {
      double w0, w1;
      draw_pair(A.seed, (unsigned)idx, f, 1, w0, w1);  // theta_f1
      t1 = 2.0 * w0;
      t2 = 2.0 * v1 + 2.0 * w0 - 2.0 * v0;
    }
  }
  return true;
}

__global__ void ic_modes_kernel(double2* F, double2* G, const LatConst* Lc, const LatScalars* Sc,
                                const ICArgs A, int f) {
  const LatConst& L = *Lc;
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= L.V) return;
  const double a = Sc->a, al = L.alpha;
  long long pid = 0;
  double r1, r2, t1, t2, om;
  if (!mode_draw(L, A, a, idx, f, &pid, r1, r2, t1, t2, om)) return;
  const bool selfc = pid == idx;
  double s1, c1, s2, c2;
  sincospi(t1, &s1, &c1);
  sincospi(t2, &s2, &c2);
  const double isq2 = 0.70710678118654752440;
  const double z1r = r1 * c1, z1i = r1 * s1, z2r = r2 * c2, z2i = r2 * s2;
  double fr = (z1r + z2r) * isq2, fi = (z1i + z2i) * isq2;
  // derivative: a^{alpha-1} i omega (z1 - z2)/sqrt2 - H dphi, H = b/a
  const double pre = pow(a, al - 1.0) * om * isq2;
  const double H = Sc->b / a;
  double gr = -pre * (z1i - z2i) - H * fr;
  double gi = pre * (z1r - z2r) - H * fi;
  if (selfc) {
    fi = 0.0;
    gi = 0.0;
  }
  F[idx] = make_double2(fr, fi);
  G[idx] = make_double2(gr, gi);
  F[pid] = make_double2(fr, -fi);
  G[pid] = make_double2(gr, -gi);
}

// Gradient of an objective with respect to the drawn amplitudes |z1|, |z2| of
// component f, from the gradient lam with respect to the initial state:
// Lf = sum_x lam_phi(x) e^{+ik.x}, Lp = sum_x lam_pi(x) e^{+ik.x} (unnormalised
// transforms), and with e_j = e^{i pi t_j}/sqrt2,
//   dJ/d|z_j| = (s/V) Re[ e_j Lf + a^{3-alpha} (+-a^{alpha-1} i omega - H_ic) e_j Lp ],
// s = 2 for a mode and its conjugate partner, 1 for a self-conjugate site;
// zero at non-canonical sites and at modes that were not drawn.
__global__ void ic_amp_grad_kernel(const double2* Lf, const double2* Lp, double* out1, double* out2,
                                   const LatConst* Lc, const LatScalars* Sc, const ICArgs A, int f) {
  const LatConst& L = *Lc;
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= L.V) return;
  out1[idx] = 0.0;
  out2[idx] = 0.0;
  const double a = Sc->a0, al = L.alpha;
  long long pid = 0;
  double r1, r2, t1, t2, om;
  if (!mode_draw(L, A, a, idx, f, &pid, r1, r2, t1, t2, om)) return;
  const double s = (pid == idx ? 1.0 : 2.0) / (double)L.V;
  const double isq2 = 0.70710678118654752440;
  const double a3 = pow(a, 3.0 - al), am1 = pow(a, al - 1.0), H = Sc->H_ic;
  const double2 F = Lf[idx], G = Lp[idx];
  for (int j = 0; j < 2; ++j) {
    double sn, cs;
    sincospi(j == 0 ? t1 : t2, &sn, &cs);
    const double er = cs * isq2, ei = sn * isq2;
    const double sg = j == 0 ? 1.0 : -1.0;
    // c = a^{3-alpha} (sg a^{alpha-1} i omega - H) e
    const double wr = -a3 * H, wi = a3 * sg * am1 * om;
    const double cr = wr * er - wi * ei, ci = wr * ei + wi * er;
    const double v = s * ((er * F.x - ei * F.y) + (cr * G.x - ci * G.y));
    (j == 0 ? out1 : out2)[idx] = v;
  }
}

// phi = phi0 + Re(F)/V, pi = a^{3-alpha} (phi0' + Re(G)/V), stored in T.
template <typename T>
__global__ void ic_assemble_kernel(T* phi, T* pi, const double2* F, const double2* G,
                                   const LatConst* Lc, const LatScalars* Sc, double phi0,
                                   double dphi0) {
  const long long V = Lc->V;
  const double invV = 1.0 / (double)V;
  const double a3 = pow(Sc->a, 3.0 - Lc->alpha);
  for (long long n = (long long)blockIdx.x * blockDim.x + threadIdx.x; n < V;
       n += (long long)gridDim.x * blockDim.x) {
    phi[n] = (T)(phi0 + F[n].x * invV);
    pi[n] = (T)(a3 * (dphi0 + G[n].x * invV));
  }
}
template __global__ void ic_assemble_kernel<float>(float*, float*, const double2*, const double2*,
                                                   const LatConst*, const LatScalars*, double, double);
template __global__ void ic_assemble_kernel<double>(double*, double*, const double2*, const double2*,
                                                    const LatConst*, const LatScalars*, double,
                                                    double);

// ---------------------------------------------------------------------------
// 3-D FFT: batched 1-D transforms along one axis, `batch` lines per CTA
// (consecutive in the fastest other index, so that the strided axes read whole
// cache lines), self-sorting Stockham passes of radix 4, 2 and 3 in shared
// memory.  Stage with radix R after sub-length Ns: for j < N/R, k = j mod Ns,
//   v_r = x[j + r N/R] w^{k r},  w = exp(sign 2 pi i/(Ns R)),
//   y[(j/Ns) Ns R + k + q Ns] = sum_r v_r exp(sign 2 pi i r q / R).
// The twiddles come from a table of the N-th roots of unity (w^{k r} is root
// (k r mod Ns R) N/(Ns R)), made once per transform by fft_twiddle_kernel.
// ---------------------------------------------------------------------------

__device__ __forceinline__ double2 cmul(double2 a, double2 b) {
  return make_double2(fma(a.x, b.x, -a.y * b.y), fma(a.x, b.y, a.y * b.x));
}

__global__ void fft_twiddle_kernel(double2* tw, int N) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= N) return;
  double sn, cs;
  sincospi(2.0 * (double)e / (double)N, &sn, &cs);
  tw[e] = make_double2(cs, sn);
}

// The Stockham stages on B lines held in shared memory (line pitch Pt), the
// roots of unity in w; returns the buffer (a or b) that holds the result.
__device__ double2* stockham_lines(double2* a, double2* b, const double2* w, const FftPlan& plan, int B, int Pt) {
  const int N = plan.N, nt = blockDim.x, tid = threadIdx.x;
  int Ns = 1;
  for (int s = 0; s < plan.nrad; ++s) {
    const int R = plan.rad[s];
    const int NR = N / R;
    const int L = Ns * R;
    const int ts = N / L;  // table stride of this stage's roots
    for (int t = tid; t < B * NR; t += nt) {
      const int j = t % NR, line = t / NR;
      const double2* ai = a + line * Pt;
      const int k = j % Ns;
      double2 v[4];
      for (int r = 0; r < R; ++r) {
        double2 x = ai[j + r * NR];
        if (k != 0 && r != 0) x = cmul(x, w[((k * r) % L) * ts]);
        v[r] = x;
      }
      double2 o[4];
      if (R == 2) {
        o[0] = make_double2(v[0].x + v[1].x, v[0].y + v[1].y);
        o[1] = make_double2(v[0].x - v[1].x, v[0].y - v[1].y);
      } else if (R == 4) {
        // j = sign * i
        const double2 t0 = make_double2(v[0].x + v[2].x, v[0].y + v[2].y);
        const double2 t1 = make_double2(v[0].x - v[2].x, v[0].y - v[2].y);
        const double2 t2 = make_double2(v[1].x + v[3].x, v[1].y + v[3].y);
        const double2 d = make_double2(v[1].x - v[3].x, v[1].y - v[3].y);
        const double2 t3 = make_double2(-plan.sign * d.y, plan.sign * d.x);  // j*(v1 - v3)
        o[0] = make_double2(t0.x + t2.x, t0.y + t2.y);
        o[1] = make_double2(t1.x + t3.x, t1.y + t3.y);
        o[2] = make_double2(t0.x - t2.x, t0.y - t2.y);
        o[3] = make_double2(t1.x - t3.x, t1.y - t3.y);
      } else {  // R == 3, w = (-1/2, sign sqrt3/2)
        const double h = 0.86602540378443864676 * plan.sign;
        const double2 s3 = make_double2(v[1].x + v[2].x, v[1].y + v[2].y);
        const double2 d = make_double2(v[1].x - v[2].x, v[1].y - v[2].y);
        const double2 m = make_double2(v[0].x - 0.5 * s3.x, v[0].y - 0.5 * s3.y);
        o[0] = make_double2(v[0].x + s3.x, v[0].y + s3.y);
        o[1] = make_double2(m.x - h * d.y, m.y + h * d.x);
        o[2] = make_double2(m.x + h * d.y, m.y - h * d.x);
      }
      double2* bo = b + line * Pt + (j / Ns) * L + k;
      for (int q2 = 0; q2 < R; ++q2) bo[q2 * Ns] = o[q2];
    }
    __syncthreads();
    double2* t = a;
    a = b;
    b = t;
    Ns = L;
  }
  return a;
}

__device__ __forceinline__ void load_roots(double2* w, const FftPlan& plan) {
  for (int e = threadIdx.x; e < plan.N; e += blockDim.x) {
    const double2 t = plan.tw[e];
    w[e] = make_double2(t.x, plan.sign * t.y);
  }
}

// Element (line u, position j) of an array of x extent P = plan.pitch:
// axis 0: j + P (u + N w) (rows, P = N); axis 1: u + P (j + N w); axis 2: u + P (w + N j).
// A CTA takes `batch` lines with consecutive u (and one w); lines with u >= nu are
// not loaded or stored (the last group of a half spectrum's N/2 + 1 columns).
__global__ void fft_lines_kernel(double2* data, const FftPlan plan) {
  extern __shared__ double2 fbuf[];
  const int N = plan.N, B = plan.batch, Pt = N + 1;  // padded line pitch: no bank conflicts across lines
  const int nt = blockDim.x, tid = threadIdx.x;
  double2* a = fbuf;
  double2* b = fbuf + B * Pt;
  double2* w = fbuf + 2 * B * Pt;
  const int P = plan.pitch, nu = plan.nu;
  const int ng = (nu + B - 1) / B;
  const long long u0 = (long long)(blockIdx.x % ng) * B, ww = blockIdx.x / ng;
  const long long PN = (long long)P * N;
  load_roots(w, plan);
  if (plan.axis == 0) {
    const double2* src = data + PN * ww + (long long)N * u0;  // B whole rows, contiguous
    for (int t = tid; t < B * N; t += nt) a[(t / N) * Pt + t % N] = src[t];
  } else {
    const long long base = plan.axis == 1 ? PN * ww + u0 : (long long)P * ww + u0;
    const long long js = plan.axis == 1 ? P : PN;
    for (int t = tid; t < B * N; t += nt) {
      const int l = t % B;
      a[l * Pt + t / B] = u0 + l < nu ? data[base + (t / B) * js + l] : make_double2(0.0, 0.0);
    }
  }
  __syncthreads();
  a = stockham_lines(a, b, w, plan, B, Pt);
  if (plan.axis == 0) {
    double2* dst = data + PN * ww + (long long)N * u0;
    for (int t = tid; t < B * N; t += nt) dst[t] = a[(t / N) * Pt + t % N];
  } else {
    const long long base = plan.axis == 1 ? PN * ww + u0 : (long long)P * ww + u0;
    const long long js = plan.axis == 1 ? P : PN;
    for (int t = tid; t < B * N; t += nt) {
      const int l = t % B;
      if (u0 + l < nu) data[base + (t / B) * js + l] = a[l * Pt + t / B];
    }
  }
}

// Real-to-complex transform along x of a real N^3 field f into the half
// spectrum H (x extent N/2 + 1, element kx + (N/2 + 1)(y + N z)): rows 2p and
// 2p + 1 (the same z, y even and odd) are transformed together as the complex
// row f_2p + i f_2p+1, Z = X_a + i X_b, and separated by the Hermitian symmetry
// of real transforms: X_a(k) = (Z(k) + Z^*(N-k))/2, X_b(k) = (Z(k) - Z^*(N-k))/(2i),
// for k = 0 .. N/2.  A CTA takes `batch` row pairs.
template <typename T>
__global__ void rfft_rows_kernel(const T* f, double2* H, const FftPlan plan) {
  extern __shared__ double2 fbuf[];
  const int N = plan.N, B = plan.batch, Pt = N + 1, NH = N / 2 + 1;
  const int nt = blockDim.x, tid = threadIdx.x;
  double2* a = fbuf;
  double2* b = fbuf + B * Pt;
  double2* w = fbuf + 2 * B * Pt;
  const long long p0 = (long long)blockIdx.x * B;  // first row pair of the CTA
  load_roots(w, plan);
  const T* src = f + 2 * p0 * N;  // 2B whole rows, contiguous
  for (int t = tid; t < 2 * B * N; t += nt) {
    const int row = t / N, j = t % N;
    double* slot = reinterpret_cast<double*>(&a[(row >> 1) * Pt + j]);
    slot[row & 1] = (double)src[t];
  }
  __syncthreads();
  a = stockham_lines(a, b, w, plan, B, Pt);
  for (int t = tid; t < B * NH; t += nt) {
    const int l = t / NH, k = t % NH;
    const double2 Z = a[l * Pt + k], Y = a[l * Pt + (k == 0 ? 0 : N - k)];  // Y = Z(N - k)
    const double2 Xa = make_double2(0.5 * (Z.x + Y.x), 0.5 * (Z.y - Y.y));
    const double2 Xb = make_double2(0.5 * (Z.y + Y.y), 0.5 * (Y.x - Z.x));
    const long long ra = 2 * (p0 + l);
    H[ra * NH + k] = Xa;
    H[(ra + 1) * NH + k] = Xb;
  }
}

// Shell sums of a half spectrum H (as rfft_rows_kernel writes it, all three
// axes transformed): each kept mode stands for itself and, for 0 < kx < N/2,
// for its conjugate partner (-kx, -ky, -kz) with the same |F|^2 and |n|, so it
// counts twice.  Runs of equal bins along kx are summed before the atomics.
__global__ void bin_half_kernel(const double2* H, int N, double dk, int nb, double* part) {
  extern __shared__ double sb[];
  double* sp = sb;
  double* sn = sb + nb;
  double* sc = sb + 2 * nb;
  for (int i = threadIdx.x; i < 3 * nb; i += blockDim.x) sb[i] = 0.0;
  __syncthreads();
  constexpr int CH = 8;
  const int NH = N / 2 + 1, nchr = (NH + CH - 1) / CH;
  const long long nch = (long long)N * N * nchr;
  for (long long ch = (long long)blockIdx.x * blockDim.x + threadIdx.x; ch < nch;
       ch += (long long)gridDim.x * blockDim.x) {
    const long long row = ch / nchr;
    const int x0 = (int)(ch % nchr) * CH;
    const int y = (int)(row % N), z = (int)(row / N);
    const int ny = y <= N / 2 ? y : y - N, nz = z <= N / 2 ? z : z - N;
    const int c2 = ny * ny + nz * nz;
    int cur = -1;
    double rp = 0.0, rn = 0.0, rc = 0.0;
    const int x1 = x0 + CH < NH ? x0 + CH : NH;
    for (int kx = x0; kx < x1; ++kx) {
      const int m2 = kx * kx + c2;
      if (m2 == 0) continue;  // the zero mode is in no bin
      const double nn = sqrt((double)m2);
      int bb = (int)floor(nn / dk);
      if (bb >= nb) bb = nb - 1;
      if (bb != cur) {
        if (cur >= 0) {
          atomicAdd(&sp[cur], rp);
          atomicAdd(&sn[cur], rn);
          atomicAdd(&sc[cur], rc);
        }
        cur = bb;
        rp = rn = rc = 0.0;
      }
      const double wgt = (kx == 0 || kx == N / 2) ? 1.0 : 2.0;
      const double2 v = H[row * NH + kx];
      rp += wgt * (v.x * v.x + v.y * v.y);
      rn += wgt * nn;
      rc += wgt;
    }
    if (cur >= 0) {
      atomicAdd(&sp[cur], rp);
      atomicAdd(&sn[cur], rn);
      atomicAdd(&sc[cur], rc);
    }
  }
  __syncthreads();
  for (int i = threadIdx.x; i < 3 * nb; i += blockDim.x) part[(size_t)blockIdx.x * 3 * nb + i] = sb[i];
}

template <typename T>
__global__ void to_complex_kernel(const T* f, double2* out, long long V) {
  for (long long n = (long long)blockIdx.x * blockDim.x + threadIdx.x; n < V;
       n += (long long)gridDim.x * blockDim.x)
    out[n] = make_double2((double)f[n], 0.0);
}
template __global__ void to_complex_kernel<float>(const float*, double2*, long long);
template __global__ void to_complex_kernel<double>(const double*, double2*, long long);

// One component of the U(1) magnetic field, B = sin(theta_jl)/(gQ dx^2) with the
// plaquette angle theta_jl(n) = gQ dx [A_j(n) + A_l(n+j) - A_j(n+l) - A_l(n)]
// (directions j, l: 0 = x, 1 = y, 2 = z), in FP64, imaginary part 0.
template <typename T>
__global__ void u1_plaquette_field_kernel(const T* Aj, const T* Al, int j, int l, int N, double gd,
                                          double inv_gdx2, double2* out) {
  const long long V = (long long)N * N * N;
  for (long long n = (long long)blockIdx.x * blockDim.x + threadIdx.x; n < V;
       n += (long long)gridDim.x * blockDim.x) {
    const int c[3] = {(int)(n % N), (int)((n / N) % N), (int)(n / ((long long)N * N))};
    auto shifted = [&](int d) -> long long {
      int cc[3] = {c[0], c[1], c[2]};
      cc[d] = cc[d] + 1 == N ? 0 : cc[d] + 1;
      return cc[0] + (long long)N * (cc[1] + (long long)N * cc[2]);
    };
    const double th = gd * (((double)Aj[n] + (double)Al[shifted(j)]) - ((double)Aj[shifted(l)] + (double)Al[n]));
    out[n] = make_double2(sin(th) * inv_gdx2, 0.0);
  }
}

// Colour component a (1..3) of the SU(2) field strength of plaquette (j, l) at
// every site, G_jl^a = Tr[(i s_a/2)(U_jl - U_jl^dag)]/(gQB dx^2) = 2 p_a/(gQB dx^2),
// with p the vector part of the plaquette U_j(n) U_l(n+j) U_j^dag(n+l) U_l^dag(n)
// in the links' quaternion form U = u0 - i u.s (FP64 from the stored values).
struct Quat {
  double w, x, y, z;
};
__device__ inline Quat qprod(const Quat& a, const Quat& b) {
  return Quat{a.w * b.w - a.x * b.x - a.y * b.y - a.z * b.z, a.w * b.x + b.w * a.x + (a.y * b.z - a.z * b.y),
              a.w * b.y + b.w * a.y + (a.z * b.x - a.x * b.z), a.w * b.z + b.w * a.z + (a.x * b.y - a.y * b.x)};
}
template <typename T>
__global__ void su2_plaquette_field_kernel(const T* Uj, const T* Ul, int j, int l, int a, int N, double inv,
                                           double2* out) {
  const long long V = (long long)N * N * N;
  for (long long n = (long long)blockIdx.x * blockDim.x + threadIdx.x; n < V;
       n += (long long)gridDim.x * blockDim.x) {
    const int c[3] = {(int)(n % N), (int)((n / N) % N), (int)(n / ((long long)N * N))};
    auto shifted = [&](int d) -> long long {
      int cc[3] = {c[0], c[1], c[2]};
      cc[d] = cc[d] + 1 == N ? 0 : cc[d] + 1;
      return cc[0] + (long long)N * (cc[1] + (long long)N * cc[2]);
    };
    // component k of a link array block: (u0, u1, u2, u3) at k V
    auto link = [&](const T* U, long long m, bool conj) {
      const double s = conj ? -1.0 : 1.0;
      return Quat{(double)U[m], s * (double)U[V + m], s * (double)U[2 * V + m], s * (double)U[3 * V + m]};
    };
    const Quat P = qprod(qprod(qprod(link(Uj, n, false), link(Ul, shifted(j), false)), link(Uj, shifted(l), true)),
                         link(Ul, n, true));
    const double pa = a == 1 ? P.x : (a == 2 ? P.y : P.z);
    out[n] = make_double2(2.0 * pa * inv, 0.0);
  }
}

// out = cx x + cy y (FP64), imaginary part 0.
template <typename T>
__global__ void combine_to_complex_kernel(const T* x, double cx, const T* y, double cy, double2* out, long long V) {
  for (long long n = (long long)blockIdx.x * blockDim.x + threadIdx.x; n < V;
       n += (long long)gridDim.x * blockDim.x)
    out[n] = make_double2(cx * (double)x[n] + cy * (double)y[n], 0.0);
}

// Shell binning of |F(n)|^2, bins b = floor(|n|/dk) over n != 0.  Each block
// accumulates in shared memory and writes its own partial row (3 x nb).  A
// thread takes 8 consecutive sites of one x-row (N is a multiple of 8) and
// sums a run of sites in one bin in registers before its shared-memory atomics
// (along a row |n| changes slowly, so runs are usually longer than one).
__global__ void bin_partial_kernel(const double2* F, int N, double dk, int nb, double* part) {
  extern __shared__ double sb[];
  double* sp = sb;
  double* sn = sb + nb;
  double* sc = sb + 2 * nb;
  for (int i = threadIdx.x; i < 3 * nb; i += blockDim.x) sb[i] = 0.0;
  __syncthreads();
  constexpr int CH = 8;
  const long long NN = (long long)N * N, nch = NN * N / CH;
  for (long long ch = (long long)blockIdx.x * blockDim.x + threadIdx.x; ch < nch;
       ch += (long long)gridDim.x * blockDim.x) {
    const long long i0 = ch * CH;
    const int x0 = (int)(i0 % N), y = (int)((i0 / N) % N), z = (int)(i0 / NN);
    const int ny = y <= N / 2 ? y : y - N, nz = z <= N / 2 ? z : z - N;
    const int c2 = ny * ny + nz * nz;
    int cur = -1;
    double rp = 0.0, rn = 0.0, rc = 0.0;
#pragma unroll
    for (int k = 0; k < CH; ++k) {
      const int x = x0 + k;
      const int nx = x <= N / 2 ? x : x - N;
      const int m2 = nx * nx + c2;
      if (m2 == 0) continue;  // the zero mode is in no bin
      const double nn = sqrt((double)m2);
      int b = (int)floor(nn / dk);
      if (b >= nb) b = nb - 1;
      if (b != cur) {
        if (cur >= 0) {
          atomicAdd(&sp[cur], rp);
          atomicAdd(&sn[cur], rn);
          atomicAdd(&sc[cur], rc);
        }
        cur = b;
        rp = rn = rc = 0.0;
      }
      const double2 v = F[i0 + k];
      rp += v.x * v.x + v.y * v.y;
      rn += nn;
      rc += 1.0;
    }
    if (cur >= 0) {
      atomicAdd(&sp[cur], rp);
      atomicAdd(&sn[cur], rn);
      atomicAdd(&sc[cur], rc);
    }
  }
  __syncthreads();
  for (int i = threadIdx.x; i < 3 * nb; i += blockDim.x) part[(size_t)blockIdx.x * 3 * nb + i] = sb[i];
}

// Shell geometry of a lattice size and bin width, cached by the caller: the bin
// of every |n|^2 up to 3 (N/2)^2 (-1 for the zero mode), and per bin the mode
// count and the sum of |n| over all N^3 - 1 modes (partial rows per block,
// summed by geo_final_kernel in a fixed order).
__global__ void geo_table_kernel(int* bin_of, int m2max, double dk, int nb) {
  for (int m2 = blockIdx.x * blockDim.x + threadIdx.x; m2 <= m2max; m2 += gridDim.x * blockDim.x) {
    int b = -1;
    if (m2 > 0) {
      b = (int)floor(sqrt((double)m2) / dk);
      if (b >= nb) b = nb - 1;
    }
    bin_of[m2] = b;
  }
}

__global__ void geo_partial_kernel(const int* bin_of, int N, int nb, double* part) {
  extern __shared__ double sb[];
  double* sn = sb;
  double* sc = sb + nb;
  for (int i = threadIdx.x; i < 2 * nb; i += blockDim.x) sb[i] = 0.0;
  __syncthreads();
  const long long NN = (long long)N * N;
  for (long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x; r < NN; r += (long long)gridDim.x * blockDim.x) {
    const int y = (int)(r % N), z = (int)(r / N);
    const int ny = y <= N / 2 ? y : y - N, nz = z <= N / 2 ? z : z - N;
    for (int x = 0; x < N; ++x) {  // one whole row per thread (this runs once per lattice size and bin width)
      const int nx = x <= N / 2 ? x : x - N;
      const int m2 = nx * nx + ny * ny + nz * nz;
      const int b = bin_of[m2];
      if (b < 0) continue;
      atomicAdd(&sn[b], sqrt((double)m2));
      atomicAdd(&sc[b], 1.0);
    }
  }
  __syncthreads();
  for (int i = threadIdx.x; i < 2 * nb; i += blockDim.x) part[(size_t)blockIdx.x * 2 * nb + i] = sb[i];
}

__global__ void geo_final_kernel(const double* part, int nblk, int nb, double* geo) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= nb) return;
  double sn = 0.0, sc = 0.0;
  for (int i = 0; i < nblk; ++i) {
    sn += part[(size_t)i * 2 * nb + b];
    sc += part[(size_t)i * 2 * nb + nb + b];
  }
  geo[b] = sn;
  geo[nb + b] = sc;
}

// Shell sums of |F|^2 of a half spectrum with the cached bins: each kept mode
// counts twice for 0 < kx < N/2 (its conjugate partner), runs of equal bins
// along kx are summed before the atomic.  Partial rows of nb per block.
__global__ void bin_power_half_kernel(const double2* H, const int* bin_of, int N, int nb, double* part) {
  extern __shared__ double sb[];
  for (int i = threadIdx.x; i < nb; i += blockDim.x) sb[i] = 0.0;
  __syncthreads();
  constexpr int CH = 8;
  const int NH = N / 2 + 1, nchr = (NH + CH - 1) / CH;
  const long long nch = (long long)N * N * nchr;
  for (long long ch = (long long)blockIdx.x * blockDim.x + threadIdx.x; ch < nch;
       ch += (long long)gridDim.x * blockDim.x) {
    const long long row = ch / nchr;
    const int x0 = (int)(ch % nchr) * CH;
    const int y = (int)(row % N), z = (int)(row / N);
    const int ny = y <= N / 2 ? y : y - N, nz = z <= N / 2 ? z : z - N;
    const int c2 = ny * ny + nz * nz;
    const int x1 = x0 + CH < NH ? x0 + CH : NH;
    int cur = -1;
    double rp = 0.0;
    for (int kx = x0; kx < x1; ++kx) {
      const int b = bin_of[kx * kx + c2];
      if (b < 0) continue;
      if (b != cur) {
        if (cur >= 0) atomicAdd(&sb[cur], rp);
        cur = b;
        rp = 0.0;
      }
      const double2 v = H[row * NH + kx];
      rp += ((kx == 0 || kx == N / 2) ? 1.0 : 2.0) * (v.x * v.x + v.y * v.y);
    }
    if (cur >= 0) atomicAdd(&sb[cur], rp);
  }
  __syncthreads();
  for (int i = threadIdx.x; i < nb; i += blockDim.x) part[(size_t)blockIdx.x * nb + i] = sb[i];
}

// eq. discretePS per bin from the power rows and the cached geometry (as bin_final_kernel).
__global__ void bin_final_geo_kernel(const double* part, int nblk, int nb, const double* geo, double kIR, double dx,
                                     int N, double* k, double* delta, double* mult) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= nb) return;
  double sp = 0.0;
  for (int i = 0; i < nblk; ++i) sp += part[(size_t)i * nb + b];
  const double sn = geo[b], sc = geo[nb + b];
  if (sc == 0.0) {
    k[b] = 0.0;
    delta[b] = 0.0;
    mult[b] = 0.0;
    return;
  }
  const double nbar = sn / sc;
  const double kb = kIR * nbar;
  const double fac = pow(dx / (double)N, 3.0);
  const double pi = 3.14159265358979323846;
  k[b] = kb;
  delta[b] = kb * kb * kb / (2.0 * pi * pi) * fac * sp / (4.0 * pi * nbar * nbar);
  mult[b] = sc;
}

// Sum the block rows in a fixed order and form eq. discretePS per bin (raw:
// the shell sum of |F|^2 instead of delta_b).
__global__ void bin_final_kernel(const double* part, int nblk, int nb, double kIR, double dx, int N,
                                 double* k, double* delta, double* mult, int raw) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= nb) return;
  double sp = 0.0, sn = 0.0, sc = 0.0;
  for (int i = 0; i < nblk; ++i) {
    const double* r = part + (size_t)i * 3 * nb;
    sp += r[b];
    sn += r[nb + b];
    sc += r[2 * nb + b];
  }
  if (sc == 0.0) {
    k[b] = 0.0;
    delta[b] = 0.0;
    mult[b] = 0.0;
    return;
  }
  const double nbar = sn / sc;
  const double kb = kIR * nbar;
  const double fac = pow(dx / (double)N, 3.0);
  const double pi = 3.14159265358979323846;
  k[b] = kb;
  delta[b] = raw ? sp : kb * kb * kb / (2.0 * pi * pi) * fac * sp / (4.0 * pi * nbar * nbar);
  mult[b] = sc;
}

// FP64 <-> storage conversion for state transfer.
template <typename T>
__global__ void convert_to_double_kernel(const T* in, double* out, long long V) {
  for (long long n = (long long)blockIdx.x * blockDim.x + threadIdx.x; n < V;
       n += (long long)gridDim.x * blockDim.x)
    out[n] = (double)in[n];
}
template <typename T>
__global__ void convert_from_double_kernel(const double* in, T* out, long long V) {
  for (long long n = (long long)blockIdx.x * blockDim.x + threadIdx.x; n < V;
       n += (long long)gridDim.x * blockDim.x)
    out[n] = (T)in[n];
}
template __global__ void convert_to_double_kernel<float>(const float*, double*, long long);
template __global__ void convert_to_double_kernel<double>(const double*, double*, long long);
template __global__ void convert_from_double_kernel<float>(const double*, float*, long long);
template __global__ void convert_from_double_kernel<double>(const double*, double*, long long);

// ---------------------------------------------------------------------------
// Host-side launchers (the kernels above are launched only through these).
// ---------------------------------------------------------------------------
namespace {
int grid_for(long long n, int tb) { long long b = (n + tb - 1) / tb; return (int)(b < 65536 ? b : 65536); }
}

cudaError_t launch_init_scalars(const LatConst* L, LatScalars* S, const ICArgs& A, cudaStream_t st) {
  init_scalars_kernel<<<1, 32, 0, st>>>(L, S, A);
  return cudaGetLastError();
}

cudaError_t launch_ic_modes(double2* F, double2* G, const LatConst* L, const LatScalars* S,
                            const ICArgs& A, int f, long long V, cudaStream_t st) {
  const int tb = 256;
  ic_modes_kernel<<<(unsigned)((V + tb - 1) / tb), tb, 0, st>>>(F, G, L, S, A, f);
  return cudaGetLastError();
}

cudaError_t launch_ic_assemble(int fp32, void* phi, void* pi, const double2* F, const double2* G,
                               const LatConst* L, const LatScalars* S, double phi0, double dphi0,
                               long long V, cudaStream_t st) {
  const int tb = 256;
  if (fp32)
    ic_assemble_kernel<float><<<grid_for(V, tb), tb, 0, st>>>((float*)phi, (float*)pi, F, G, L, S, phi0, dphi0);
  else
    ic_assemble_kernel<double><<<grid_for(V, tb), tb, 0, st>>>((double*)phi, (double*)pi, F, G, L, S, phi0, dphi0);
  return cudaGetLastError();
}

// Lines per CTA: the largest divisor of N with batch * N <= 2048 (at most 72 KB
// of shared memory per CTA).
int fft_batch(int N) {
  int b = 1;
  for (int d = 1; d <= N && d * N <= 2048; ++d)
    if (N % d == 0) b = d;
  return b;
}

size_t fft_smem_bytes(int N) { return (2 * (size_t)fft_batch(N) * (N + 1) + N) * sizeof(double2); }

cudaError_t launch_fft_twiddles(double2* tw, int N, cudaStream_t st) {
  fft_twiddle_kernel<<<(N + 127) / 128, 128, 0, st>>>(tw, N);
  return cudaGetLastError();
}

cudaError_t launch_fft_axis(double2* data, const FftPlan& pl, cudaStream_t st) {
  cudaError_t e = cudaFuncSetAttribute((const void*)fft_lines_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)fft_smem_bytes(pl.N));
  if (e != cudaSuccess) return e;
  const int work = pl.batch * pl.N / 4;
  const int threads = work < 64 ? 64 : (work > 512 ? 512 : (work + 31) / 32 * 32);
  const long long ng = pl.axis == 0 ? pl.N / pl.batch : (pl.nu + pl.batch - 1) / pl.batch;
  const unsigned grid = (unsigned)(ng * pl.N);
  fft_lines_kernel<<<grid, threads, fft_smem_bytes(pl.N), st>>>(data, pl);
  return cudaGetLastError();
}

// Binned spectrum of a real field through the half spectrum: x-axis transform of
// row pairs, y and z transforms of the N/2 + 1 columns kept, shell sums with the
// conjugate partners counted, then eq. discretePS per bin (as launch_bins).
// H holds (N/2 + 1) N^2 complex values; pl is the forward plan of N (tw set).
// The shell geometry of (N, dk) into bin_of (3 (N/2)^2 + 1 ints) and geo (2 nb
// doubles: the sum of |n| and the count per bin); part holds 2 nb nblk doubles.
cudaError_t launch_shell_geometry(int N, double dk, int nb, int nblk, int* bin_of, double* geo, double* part,
                                  cudaStream_t st) {
  const int m2max = 3 * (N / 2) * (N / 2);
  geo_table_kernel<<<(m2max + 256) / 256, 256, 0, st>>>(bin_of, m2max, dk, nb);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  geo_partial_kernel<<<nblk, 128, 2 * nb * sizeof(double), st>>>(bin_of, N, nb, part);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  geo_final_kernel<<<(nb + 127) / 128, 128, 0, st>>>(part, nblk, nb, geo);
  return cudaGetLastError();
}

cudaError_t launch_real_spectrum(int fp32, const void* f, double2* H, const FftPlan& pl, double dk, int nb,
                                 int nblk, double* part, double kIR, double dx, double* out, cudaStream_t st,
                                 const int* bin_of, const double* geo) {
  const int N = pl.N;
  cudaError_t e;
  const void* kern = fp32 ? (const void*)rfft_rows_kernel<float> : (const void*)rfft_rows_kernel<double>;
  e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)fft_smem_bytes(N));
  if (e != cudaSuccess) return e;
  const int work = pl.batch * N / 4;
  const int threads = work < 64 ? 64 : (work > 512 ? 512 : (work + 31) / 32 * 32);
  const unsigned grid = (unsigned)((long long)N * N / 2 / pl.batch);
  if (fp32) rfft_rows_kernel<float><<<grid, threads, fft_smem_bytes(N), st>>>((const float*)f, H, pl);
  else rfft_rows_kernel<double><<<grid, threads, fft_smem_bytes(N), st>>>((const double*)f, H, pl);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  FftPlan ph = pl;
  ph.pitch = ph.nu = N / 2 + 1;
  for (int axis = 1; axis < 3; ++axis) {
    ph.axis = axis;
    e = launch_fft_axis(H, ph, st);
    if (e != cudaSuccess) return e;
  }
  if (bin_of && geo) {  // the cached shell geometry: only the power is summed
    bin_power_half_kernel<<<nblk, 256, nb * sizeof(double), st>>>(H, bin_of, N, nb, part);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    bin_final_geo_kernel<<<(nb + 127) / 128, 128, 0, st>>>(part, nblk, nb, geo, kIR, dx, N, out, out + nb,
                                                            out + 2 * nb);
    return cudaGetLastError();
  }
  bin_half_kernel<<<nblk, 256, 3 * nb * sizeof(double), st>>>(H, N, dk, nb, part);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  bin_final_kernel<<<(nb + 127) / 128, 128, 0, st>>>(part, nblk, nb, kIR, dx, N, out, out + nb, out + 2 * nb, 0);
  return cudaGetLastError();
}

cudaError_t launch_to_complex(int fp32, const void* f, double2* out, long long V, cudaStream_t st) {
  const int tb = 256;
  if (fp32) to_complex_kernel<float><<<grid_for(V, tb), tb, 0, st>>>((const float*)f, out, V);
  else to_complex_kernel<double><<<grid_for(V, tb), tb, 0, st>>>((const double*)f, out, V);
  return cudaGetLastError();
}

// Ensemble mean of binned spectra: rows [nl][3 nb] (k, delta, mult) of
// lattices that share N and kIR; k and mult are those of the first.
__global__ void spec_mean_kernel(const double* rows, int nl, int nb, double* out) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= nb) return;
  double s = 0.0;
  for (int l = 0; l < nl; ++l) s += rows[(size_t)l * 3 * nb + nb + b];
  out[b] = rows[b];
  out[nb + b] = s / (double)nl;
  out[2 * nb + b] = rows[2 * nb + b];
}

cudaError_t launch_spec_mean(const double* rows, int nl, int nb, double* out, cudaStream_t st) {
  spec_mean_kernel<<<(nb + 127) / 128, 128, 0, st>>>(rows, nl, nb, out);
  return cudaGetLastError();
}

cudaError_t launch_ic_amp_grad(const double2* Lf, const double2* Lp, double* out1, double* out2,
                               const LatConst* L, const LatScalars* S, const ICArgs& A, int f,
                               long long V, cudaStream_t st) {
  ic_amp_grad_kernel<<<(unsigned)((V + 255) / 256), 256, 0, st>>>(Lf, Lp, out1, out2, L, S, A, f);
  return cudaGetLastError();
}

cudaError_t launch_bins(const double2* F, int N, double dk, int nb, int nblk, double* part,
                        double kIR, double dx, double* out, cudaStream_t st, int raw) {
  bin_partial_kernel<<<nblk, 256, 3 * nb * sizeof(double), st>>>(F, N, dk, nb, part);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  bin_final_kernel<<<(nb + 127) / 128, 128, 0, st>>>(part, nblk, nb, kIR, dx, N, out, out + nb, out + 2 * nb,
                                                     raw);
  return cudaGetLastError();
}

cudaError_t launch_u1_plaquette_field(int fp32, const void* Aj, const void* Al, int j, int l, int N, double gd,
                                      double inv_gdx2, double2* out, cudaStream_t st) {
  const long long V = (long long)N * N * N;
  const int tb = 256;
  if (fp32)
    u1_plaquette_field_kernel<float><<<grid_for(V, tb), tb, 0, st>>>((const float*)Aj, (const float*)Al, j, l, N,
                                                                      gd, inv_gdx2, out);
  else
    u1_plaquette_field_kernel<double><<<grid_for(V, tb), tb, 0, st>>>((const double*)Aj, (const double*)Al, j, l,
                                                                       N, gd, inv_gdx2, out);
  return cudaGetLastError();
}

cudaError_t launch_su2_plaquette_field(int fp32, const void* Uj, const void* Ul, int j, int l, int a, int N,
                                       double inv_bdx2, double2* out, cudaStream_t st) {
  const long long V = (long long)N * N * N;
  const int tb = 256;
  if (fp32)
    su2_plaquette_field_kernel<float><<<grid_for(V, tb), tb, 0, st>>>((const float*)Uj, (const float*)Ul, j, l, a, N,
                                                                       inv_bdx2, out);
  else
    su2_plaquette_field_kernel<double><<<grid_for(V, tb), tb, 0, st>>>((const double*)Uj, (const double*)Ul, j, l, a,
                                                                        N, inv_bdx2, out);
  return cudaGetLastError();
}

cudaError_t launch_combine_to_complex(int fp32, const void* x, double cx, const void* y, double cy, double2* out,
                                      long long V, cudaStream_t st) {
  const int tb = 256;
  if (fp32)
    combine_to_complex_kernel<float><<<grid_for(V, tb), tb, 0, st>>>((const float*)x, cx, (const float*)y, cy, out, V);
  else
    combine_to_complex_kernel<double><<<grid_for(V, tb), tb, 0, st>>>((const double*)x, cx, (const double*)y, cy,
                                                                       out, V);
  return cudaGetLastError();
}

// Modulus of a charged field and its time derivative (FP64 from the stored
// values): r = sqrt(sum_c phi_c^2/2), r' = sum_c phi_c phi_c'/(2 r) with
// phi_c' = apm pi_c (0 where r = 0).  mode 0: r; 1: r'; 2: r' + H r.
struct NormArgs {
  const void* f[4];
  const void* p[4];
  int nc, mode;
  double apm, H;
};
template <typename T>
__global__ void norm_field_kernel(const NormArgs A, double2* out, long long V) {
  for (long long n = (long long)blockIdx.x * blockDim.x + threadIdx.x; n < V;
       n += (long long)gridDim.x * blockDim.x) {
    double r2 = 0.0, rr = 0.0;
    for (int c = 0; c < A.nc; ++c) {
      const double f = (double)reinterpret_cast<const T*>(A.f[c])[n];
      const double q = (double)reinterpret_cast<const T*>(A.p[c])[n];
      r2 += 0.5 * f * f;
      rr += 0.5 * f * (A.apm * q);
    }
    const double r = sqrt(r2), rp = r > 0.0 ? rr / r : 0.0;
    const double v = A.mode == 0 ? r : (A.mode == 1 ? rp : rp + A.H * r);
    out[n] = make_double2(v, 0.0);
  }
}

cudaError_t launch_norm_field(int fp32, const void* const* f, const void* const* p, int nc, double apm, double H,
                              int mode, double2* out, long long V, cudaStream_t st) {
  NormArgs A;
  for (int c = 0; c < 4; ++c) {
    A.f[c] = c < nc ? f[c] : nullptr;
    A.p[c] = c < nc ? p[c] : nullptr;
  }
  A.nc = nc;
  A.mode = mode;
  A.apm = apm;
  A.H = H;
  const int tb = 256;
  if (fp32) norm_field_kernel<float><<<grid_for(V, tb), tb, 0, st>>>(A, out, V);
  else norm_field_kernel<double><<<grid_for(V, tb), tb, 0, st>>>(A, out, V);
  return cudaGetLastError();
}

// Per-block partial sums of w0 f0^2 + w1 f1^2 + w2 f2^2 over the lattice (volume
// averages a spectrum needs that the measurement does not keep).  A fixed grid and
// a fixed order of every sum, so the result does not depend on timing; the host
// adds the blocks' partials in order.
template <typename T>
__global__ void sum_sq_kernel(const T* f0, const T* f1, const T* f2, double w0, double w1, double w2, long long V,
                              double* part) {
  __shared__ double ws[32];
  double s = 0.0;
  for (long long n = (long long)blockIdx.x * blockDim.x + threadIdx.x; n < V;
       n += (long long)gridDim.x * blockDim.x) {
    const double a = (double)f0[n], b = (double)f1[n], c = (double)f2[n];
    s += w0 * a * a + w1 * b * b + w2 * c * c;
  }
  for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x < 32) {
    s = threadIdx.x < (blockDim.x >> 5) ? ws[threadIdx.x] : 0.0;
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if (threadIdx.x == 0) part[blockIdx.x] = s;
  }
}

cudaError_t launch_sum_sq(int fp32, const void* f0, const void* f1, const void* f2, double w0, double w1,
                          double w2, long long V, int nblk, double* part, cudaStream_t st) {
  const int tb = 256;
  if (fp32)
    sum_sq_kernel<float><<<nblk, tb, 0, st>>>(reinterpret_cast<const float*>(f0), reinterpret_cast<const float*>(f1),
                                              reinterpret_cast<const float*>(f2), w0, w1, w2, V, part);
  else
    sum_sq_kernel<double><<<nblk, tb, 0, st>>>(reinterpret_cast<const double*>(f0),
                                               reinterpret_cast<const double*>(f1),
                                               reinterpret_cast<const double*>(f2), w0, w1, w2, V, part);
  return cudaGetLastError();
}

cudaError_t launch_convert(int fp32, int to_double, const void* in, void* out, long long V, cudaStream_t st) {
  const int tb = 256;
  if (to_double) {
    if (fp32) convert_to_double_kernel<float><<<grid_for(V, tb), tb, 0, st>>>((const float*)in, (double*)out, V);
    else convert_to_double_kernel<double><<<grid_for(V, tb), tb, 0, st>>>((const double*)in, (double*)out, V);
  } else {
    if (fp32) convert_from_double_kernel<float><<<grid_for(V, tb), tb, 0, st>>>((const double*)in, (float*)out, V);
    else convert_from_double_kernel<double><<<grid_for(V, tb), tb, 0, st>>>((const double*)in, (double*)out, V);
  }
  return cudaGetLastError();
}


// The generator as the initial conditions use it, for a bit-exact check
// against the oracle: for element i, either the raw Philox4x32-10 of
// (ctr[4i..4i+3], key[2i..2i+1]) (mode 0) or the draw pair of the initial
// conditions at Fourier index ctr[4i], component ctr[4i+1], draw ctr[4i+2]
// with the seed key[2i] + 2^32 key[2i+1] (mode 1, draw_pair itself).  out
// receives the four words (mode 0) and u the two 53-bit deviates in (0, 1].
__global__ void philox_probe_kernel(const uint32_t* ctr, const uint32_t* key, int n, int mode, uint32_t* out,
                                    double* u) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  if (mode == 0) {
    uint32_t c[4] = {ctr[4 * i], ctr[4 * i + 1], ctr[4 * i + 2], ctr[4 * i + 3]};
    philox4x32_10(c, key[2 * i], key[2 * i + 1]);
    for (int k = 0; k < 4; ++k) out[4 * i + k] = c[k];
    u[2 * i] = unit_open0(c[0], c[1]);
    u[2 * i + 1] = unit_open0(c[2], c[3]);
  } else {
    const unsigned long long seed = (unsigned long long)key[2 * i] | ((unsigned long long)key[2 * i + 1] << 32);
    double u0, u1;
    draw_pair(seed, ctr[4 * i], (int)ctr[4 * i + 1], (int)ctr[4 * i + 2], u0, u1);
    for (int k = 0; k < 4; ++k) out[4 * i + k] = 0u;
    u[2 * i] = u0;
    u[2 * i + 1] = u1;
  }
}

}  // namespace clg

extern "C" cl_status cl_philox_draws(void* stream, int mode, int n, const uint32_t* ctr, const uint32_t* key,
                                     uint32_t* out, double* u) {
  if (n < 0 || n > (1 << 24) || (mode != 0 && mode != 1) || (n > 0 && (!ctr || !key || !out || !u)))
    return CL_EINVAL;
  if (n == 0) return CL_OK;
  cudaStream_t st = (cudaStream_t)stream;
  const size_t bc = (size_t)n * 4 * sizeof(uint32_t), bk = (size_t)n * 2 * sizeof(uint32_t),
               bu = (size_t)n * 2 * sizeof(double);
  char* d = nullptr;
  if (cudaMalloc(&d, 2 * bc + bk + bu) != cudaSuccess) return CL_ENOMEM;
  uint32_t* dc = (uint32_t*)d;
  uint32_t* dout = (uint32_t*)(d + bc);
  uint32_t* dk = (uint32_t*)(d + 2 * bc);
  double* du = (double*)(d + 2 * bc + bk);
  cl_status s = CL_OK;
  if (cudaMemcpyAsync(dc, ctr, bc, cudaMemcpyHostToDevice, st) != cudaSuccess ||
      cudaMemcpyAsync(dk, key, bk, cudaMemcpyHostToDevice, st) != cudaSuccess)
    s = CL_ECUDA;
  if (s == CL_OK) {
    clg::philox_probe_kernel<<<(n + 255) / 256, 256, 0, st>>>(dc, dk, n, mode, dout, du);
    if (cudaGetLastError() != cudaSuccess) s = CL_ECUDA;
  }
  if (s == CL_OK && (cudaMemcpyAsync(out, dout, bc, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
                     cudaMemcpyAsync(u, du, bu, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
                     cudaStreamSynchronize(st) != cudaSuccess))
    s = CL_ECUDA;
  cudaFree(d);
  return s;
}
