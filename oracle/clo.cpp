// clo.cpp -- FP64 CPU oracle for the lattice kick-drift method of the
// CosmoLattice manual (arXiv:2102.01031).
//
// TEST INFRASTRUCTURE ONLY: plain, slow, unfused and single threaded, written
// so that each step can be checked by eye against the paper.  Only tests/,
// __graft_entry__.smoke() and bench.py (cpu_baseline leg, reference arm) may
// load it.  It shares no code with the CUDA library.
//
// Where the paper is silent or garbled, the reading taken is stated at the
// place it is used (tag "reading:").  Parity pins for every function live in
// tests/test_oracle_*.py.
#include "clo.h"

#include <cmath>
#include <complex>
#include <cstdlib>
#include <cstring>
#include <vector>

namespace {

typedef std::complex<double> cplx;
const double PI = 3.14159265358979323846;

// ---------------------------------------------------------------------------
// Counter-based generator: Philox4x32-10 (Salmon, Moraes, Dror, Shaw,
// "Parallel random numbers: as easy as 1, 2, 3", SC'11).  Round function:
// two 32x32->64 multiplies, key added by xor, Weyl key schedule.
// ---------------------------------------------------------------------------
void philox(const uint32_t ctr_in[4], const uint32_t key_in[2], uint32_t out[4]) {
  const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
  const uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
  uint32_t c0 = ctr_in[0], c1 = ctr_in[1], c2 = ctr_in[2], c3 = ctr_in[3];
  uint32_t k0 = key_in[0], k1 = key_in[1];
  for (int round = 0; round < 10; ++round) {
    if (round > 0) { k0 += W0; k1 += W1; }
    uint64_t p0 = (uint64_t)M0 * (uint64_t)c0;
    uint64_t p1 = (uint64_t)M1 * (uint64_t)c2;
    uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    uint32_t n0 = hi1 ^ c1 ^ k0;
    uint32_t n1 = lo1;
    uint32_t n2 = hi0 ^ c3 ^ k1;
    uint32_t n3 = lo0;
    c0 = n0; c1 = n1; c2 = n2; c3 = n3;
  }
  out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

// Uniform deviate in (0, 1] with 53 random bits: 27 bits of `hi`, 26 of `lo`.
double u01(uint32_t hi, uint32_t lo) {
  uint64_t m = ((uint64_t)(hi >> 5) << 26) | (uint64_t)(lo >> 6);
  return ((double)m + 1.0) * (1.0 / 9007199254740992.0);
}

// ---------------------------------------------------------------------------
// FFT: recursive decimation in time by the smallest prime factor.  For
// n = p*m, X[k1 + m*k2] = sum_q w_n^{q k1} w_p^{q k2} Y_q[k1], where Y_q is the
// length-m DFT of x[q + p*j].  w_n = exp(sign*2*pi*i/n).
// ---------------------------------------------------------------------------
cplx root(long e, long n, int sign) {
  e %= n;
  if (e < 0) e += n;
  double t = 2.0 * PI * (double)e / (double)n;
  return cplx(std::cos(t), sign * std::sin(t));
}

void fft_rec(const cplx* x, long n, long stride, cplx* out, int sign) {
  if (n == 1) { out[0] = x[0]; return; }
  long p = 2;
  while (n % p) ++p;
  long m = n / p;
  std::vector<cplx> Y(n);
  for (long q = 0; q < p; ++q) fft_rec(x + q * stride, m, stride * p, &Y[q * m], sign);
  for (long k1 = 0; k1 < m; ++k1)
    for (long k2 = 0; k2 < p; ++k2) {
      cplx s = 0.0;
      for (long q = 0; q < p; ++q)
        s += root(q * k1, n, sign) * root(q * k2, p, sign) * Y[q * m + k1];
      out[k1 + m * k2] = s;
    }
}

// 3-D transform as 1-D transforms along x, then y, then z (unnormalised).
void fft3d(std::vector<cplx>& a, int N, int sign) {
  std::vector<cplx> line(N), res(N);
  long NN = (long)N * N;
  for (int axis = 0; axis < 3; ++axis) {
    long stride = axis == 0 ? 1 : (axis == 1 ? N : NN);
    for (long u = 0; u < N; ++u)
      for (long w = 0; w < N; ++w) {
        long base;
        if (axis == 0) base = N * (u + (long)N * w);
        else if (axis == 1) base = u + NN * w;
        else base = u + (long)N * w;
        for (long j = 0; j < N; ++j) line[j] = a[base + j * stride];
        fft_rec(line.data(), N, 1, res.data(), sign);
        for (long j = 0; j < N; ++j) a[base + j * stride] = res[j];
      }
  }
}

// ---------------------------------------------------------------------------
// Integrator schedules.  VV2 (Stoermer-Verlet) is the base symmetric step.
// VV4 = Yoshida (1990) triple jump; VV6, VV8, VV10 = the same triple-jump
// construction applied again (order 2k -> 2k+2 with z = 1/(2 - 2^{1/(2k+1)})).
// reading: the manual names VV4..VV10 but prints no coefficients; any
// symmetric composition of the right order is a member of "the family".
// reading: LF is the same kick/drift stream as VV2 (kicks merged across
// steps, momenta synchronised by a half kick before measuring).
// ---------------------------------------------------------------------------
void schedule(int order, double h, std::vector<double>& d) {
  if (order <= 2) { d.push_back(h); return; }
  double e = 1.0 / (double)(order - 1);
  double z1 = 1.0 / (2.0 - std::pow(2.0, e));
  double z0 = 1.0 - 2.0 * z1;
  schedule(order - 2, z1 * h, d);
  schedule(order - 2, z0 * h, d);
  schedule(order - 2, z1 * h, d);
}

}  // namespace

// ---------------------------------------------------------------------------
// Context
// ---------------------------------------------------------------------------
struct clo_ctx {
  int model, N, nf;   // nf: real scalar components evolved by a scalar kick
  long V;             // N^3
  double kIR, dx, alpha;
  clo_params p;
  double a, b, eta, a0, eta0, rho0;
  double Hfix;        // fixed background: initial a'/a
  uint64_t seed;      // seed of the initial conditions
  double H_ic;        // a'/a used by the initial conditions
  std::vector<double> phi[4], pi[4];
  std::vector<double> A[3], piA[3];
  std::vector<double> U[3][4], piB[3][3];  // SU(2) links (u0..u3) and momenta (doublet model)
  std::vector<double> sph, spi;            // lphi4SU2U1: the singlet and its momentum
  std::vector<double> cph[2], cpi[2];      // lphi4SU2U1: the U(1)-charged scalar's components
  bool gauge() const { return model >= CLO_MODEL_U1_HIGGS; }
  bool su2() const { return model == CLO_MODEL_SU2U1_HIGGS || model == CLO_MODEL_LPHI4_SU2U1; }
  bool full() const { return model == CLO_MODEL_LPHI4_SU2U1; }
  long at(long x, long y, long z) const {
    x %= N; if (x < 0) x += N;
    y %= N; if (y < 0) y += N;
    z %= N; if (z < 0) z += N;
    return x + (long)N * (y + (long)N * z);
  }
  void coords(long n, long& x, long& y, long& z) const {
    x = n % N; y = (n / N) % N; z = n / ((long)N * N);
  }
  long shift(long n, int dir, int s) const {
    long x, y, z;
    coords(n, x, y, z);
    if (dir == 0) x += s; else if (dir == 1) y += s; else z += s;
    return at(x, y, z);
  }
};

namespace {

int n_pot_terms(int model) {
  return model == CLO_MODEL_LPHI4_CHI ? 2 : (model == CLO_MODEL_LPHI4_SU2U1 ? 3 : 1);
}

// Program potential V~ term by term.  lphi4: phi^4/4 (eq. PotNat with chi = 0);
// lphi4 + chi: phi^4/4 + (q/2) phi^2 chi^2 (eq. PotNat, q = g^2/lambda);
// U(1) Abelian-Higgs: lam (|phi|^2 - v^2)^2 with |phi|^2 = (phi_0^2+phi_1^2)/2;
// SU(2) x U(1) doublet: the same with |Phi|^2 = (phi_0^2+...+phi_3^2)/2.
double half_norm2(const clo_ctx* c, const double* f) {
  double s = 0.0;
  for (int k = 0; k < c->nf; ++k) s += f[k] * f[k];
  return 0.5 * s;
}
void pot_terms(const clo_ctx* c, const double* f, double* t) {
  if (c->model == CLO_MODEL_LPHI4) {
    t[0] = 0.25 * f[0] * f[0] * f[0] * f[0];
  } else if (c->model == CLO_MODEL_LPHI4_CHI) {
    t[0] = 0.25 * f[0] * f[0] * f[0] * f[0];
    t[1] = 0.5 * c->p.q * f[0] * f[0] * f[1] * f[1];
  } else {
    double d = half_norm2(c, f) - c->p.v * c->p.v;
    t[0] = c->p.lam * d * d;
  }
}

// Force terms: dV/dphi_f for singlets; for the complex field the component
// form of (1/2) V_{,|phi|} phi/|phi| = dV/dphi^*, i.e. 2 lam (|phi|^2 - v^2) phi_c
// (reading: written polynomially, no division by |phi|; sign as in eq.
// higgsU1-eom, the "+" printed in eq. kernelcomplexscalar is taken as a typo).
void pot_deriv(const clo_ctx* c, const double* f, double* d) {
  if (c->model == CLO_MODEL_LPHI4) {
    d[0] = f[0] * f[0] * f[0];
  } else if (c->model == CLO_MODEL_LPHI4_CHI) {
    d[0] = f[0] * f[0] * f[0] + c->p.q * f[0] * f[1] * f[1];
    d[1] = c->p.q * f[0] * f[0] * f[1];
  } else {
    double g = 2.0 * c->p.lam * (half_norm2(c, f) - c->p.v * c->p.v);
    for (int k = 0; k < c->nf; ++k) d[k] = g * f[k];
  }
}

// lphi4SU2U1 (Sec. 4.5, eq. PotGauge in program units, with the doublet's
// quartic written lam (|Phi|^2 - v^2)^2 as in the doublet model; the manual's
// example is lam = 1, v = 0):
//   V = lam (|Phi|^2 - v^2)^2 + q_G |Phi|^2 phi_s^2 + 2 q_H |Phi|^2 |vphi|^2,
// site values f[0..3] = doublet components, f[4] = phi_s, f[5], f[6] = vphi_c;
// |Phi|^2 = sum_k f_k^2/2 (k < 4), |vphi|^2 = (f_5^2 + f_6^2)/2.
void full_pot(const clo_ctx* c, const double* f, double* t) {
  double P2 = 0.0;
  for (int k = 0; k < 4; ++k) P2 += 0.5 * f[k] * f[k];
  const double C2 = 0.5 * (f[5] * f[5] + f[6] * f[6]);
  const double d = P2 - c->p.v * c->p.v;
  t[0] = c->p.lam * d * d;
  t[1] = c->p.qG * P2 * f[4] * f[4];
  t[2] = 2.0 * c->p.qH * P2 * C2;
}
// dV/df_k of each real component (the doublet's and vphi's components carry
// the canonical kinetic term of a real field, as in the doublet model).
void full_force(const clo_ctx* c, const double* f, double* d) {
  double P2 = 0.0;
  for (int k = 0; k < 4; ++k) P2 += 0.5 * f[k] * f[k];
  const double C2 = 0.5 * (f[5] * f[5] + f[6] * f[6]);
  const double g = 2.0 * c->p.lam * (P2 - c->p.v * c->p.v) + c->p.qG * f[4] * f[4] + 2.0 * c->p.qH * C2;
  for (int k = 0; k < 4; ++k) d[k] = g * f[k];
  d[4] = 2.0 * c->p.qG * P2 * f[4];
  d[5] = 2.0 * c->p.qH * P2 * f[5];
  d[6] = 2.0 * c->p.qH * P2 * f[6];
}
// d^2V/df_k^2 (the initial effective masses of eq. QuantumFlucts2).
double full_mass2(const clo_ctx* c, const double* f, int k) {
  double P2 = 0.0;
  for (int m = 0; m < 4; ++m) P2 += 0.5 * f[m] * f[m];
  const double C2 = 0.5 * (f[5] * f[5] + f[6] * f[6]);
  if (k < 4)
    return 2.0 * c->p.lam * (P2 - c->p.v * c->p.v) + 2.0 * c->p.lam * f[k] * f[k] + c->p.qG * f[4] * f[4] +
           2.0 * c->p.qH * C2;
  if (k == 4) return 2.0 * c->p.qG * P2;
  return 2.0 * c->p.qH * P2;
}
// The seven site values of the full model at site n.
void full_site(const clo_ctx* c, long n, double* f) {
  for (int k = 0; k < 4; ++k) f[k] = c->phi[k][n];
  f[4] = c->sph[n];
  f[5] = c->cph[0][n];
  f[6] = c->cph[1][n];
}

// Real scalar components that get initial fluctuations: the full model adds
// the singlet (component 4) and the charged scalar's two (5, 6) to the doublet's.
int ncomp(const clo_ctx* c) { return c->full() ? 7 : c->nf; }

// Effective mass squared d^2V/dphi_f^2 at the homogeneous values (eq. QuantumFlucts2).
double mass2(const clo_ctx* c, const double* f, int k) {
  if (c->model == CLO_MODEL_LPHI4) return 3.0 * f[0] * f[0];
  if (c->model == CLO_MODEL_LPHI4_CHI)
    return k == 0 ? 3.0 * f[0] * f[0] + c->p.q * f[1] * f[1] : c->p.q * f[0] * f[0];
  return 2.0 * c->p.lam * (half_norm2(c, f) - c->p.v * c->p.v) + 2.0 * c->p.lam * f[k] * f[k];
}

// U(1) link phases theta = gQ dx A_i; link V_i = exp(-i theta) (U(1) toolkit).
// Plaquette angle theta_ij(n) = gQ dx [A_i(n) + A_j(n+i) - A_i(n+j) - A_j(n)],
// so that V_ij = V_i V_j(+i) V_i^*(+j) V_j^* = exp(-i theta_ij).
// reading: the toolkit prints V_mu V_{mu,+mu} V*_{mu,+nu} V*_nu; the
// SU(N) toolkit's ordering U_mu U_{nu,+mu} U^dag_{mu,+nu} U^dag_nu is used.
double plaq(const clo_ctx* c, long n, int i, int j) {
  double s = c->A[i][n] + c->A[j][c->shift(n, i, +1)] - c->A[i][c->shift(n, j, +1)] - c->A[j][n];
  return c->p.gQ * c->dx * s;
}

// V_i(n) phi(n+i) in components of phi = (phi0 + i phi1)/sqrt2 (same scaling).
void link_fwd(const clo_ctx* c, long n, int i, double& w0, double& w1) {
  long m = c->shift(n, i, +1);
  double th = c->p.gQ * c->dx * c->A[i][n];
  double co = std::cos(th), si = std::sin(th);
  double x = c->phi[0][m], y = c->phi[1][m];
  w0 = co * x + si * y;   // (co - i si)(x + i y)
  w1 = co * y - si * x;
}
// V_i^*(n-i) phi(n-i)
void link_bwd(const clo_ctx* c, long n, int i, double& w0, double& w1) {
  long m = c->shift(n, i, -1);
  double th = c->p.gQ * c->dx * c->A[i][m];
  double co = std::cos(th), si = std::sin(th);
  double x = c->phi[0][m], y = c->phi[1][m];
  w0 = co * x - si * y;   // (co + i si)(x + i y)
  w1 = co * y + si * x;
}

// ---------------------------------------------------------------------------
// Kernels of the momenta (Sec. 3.5.2, Hamiltonian form; Sec. 4.3 for U(1)).
// ---------------------------------------------------------------------------

// K_phi = -a^{3+alpha} V_{,phi} + a^{1+alpha} Lap phi, Lap = sum_i grad^-_i grad^+_i.
void kernel_scalars(const clo_ctx* c, std::vector<double>* K) {
  double a1 = std::pow(c->a, 1.0 + c->alpha), a3 = std::pow(c->a, 3.0 + c->alpha);
  double idx2 = 1.0 / (c->dx * c->dx);
  for (long n = 0; n < c->V; ++n) {
    double f[2] = {0, 0}, d[2] = {0, 0};
    for (int k = 0; k < c->nf; ++k) f[k] = c->phi[k][n];
    pot_deriv(c, f, d);
    for (int k = 0; k < c->nf; ++k) {
      double s = 0.0;
      for (int i = 0; i < 3; ++i)
        s += c->phi[k][c->shift(n, i, +1)] + c->phi[k][c->shift(n, i, -1)] - 2.0 * c->phi[k][n];
      K[k][n] = a1 * s * idx2 - a3 * d[k];
    }
  }
}

// U(1): K_phi = a^{1+alpha} D^2 phi - a^{3+alpha} dV/dphi^*, with the lattice
// covariant Laplacian D^2 phi = sum_i [V_i phi(n+i) - 2 phi + V_i^*(n-i) phi(n-i)]/dx^2;
// K_{A_i} = a^{1+alpha} (f*/omega*)^2 J_i + a^{alpha-1} (lattice d_j F_ji), with
// J_i = (2 gQ/dx) Im[phi^*(n) V_i(n) phi(n+i)] and the compact curl
// -(1/(gQ dx^3)) sum_{j != i} [sin theta_ij(n) - sin theta_ij(n-j)].
// reading: the factor (f*/omega*)^2 on J (eq. U1eom) is kept although the
// kernel line of Sec. 4.3 omits it; both terms follow from one lattice
// Hamiltonian so that the lattice Gauss law is conserved exactly.
void kernel_u1(const clo_ctx* c, std::vector<double>* Kphi, std::vector<double>* KA) {
  double a1 = std::pow(c->a, 1.0 + c->alpha), a3 = std::pow(c->a, 3.0 + c->alpha);
  double am1 = std::pow(c->a, c->alpha - 1.0);
  double idx2 = 1.0 / (c->dx * c->dx);
  double fo2 = c->p.fstar_over_omegastar * c->p.fstar_over_omegastar;
  double gQ = c->p.gQ, dx = c->dx;
  for (long n = 0; n < c->V; ++n) {
    double f[2] = {c->phi[0][n], c->phi[1][n]}, d[2];
    pot_deriv(c, f, d);
    double D0 = 0.0, D1 = 0.0;
    for (int i = 0; i < 3; ++i) {
      double u0, u1, w0, w1;
      link_fwd(c, n, i, u0, u1);
      link_bwd(c, n, i, w0, w1);
      D0 += u0 + w0 - 2.0 * f[0];
      D1 += u1 + w1 - 2.0 * f[1];
    }
    Kphi[0][n] = a1 * D0 * idx2 - a3 * d[0];
    Kphi[1][n] = a1 * D1 * idx2 - a3 * d[1];
    for (int i = 0; i < 3; ++i) {
      double u0, u1;
      link_fwd(c, n, i, u0, u1);
      // Im[phi^* w] with both in the sqrt2-scaled components: (f0 w1 - f1 w0)/2
      double J = (2.0 * gQ / dx) * 0.5 * (f[0] * u1 - f[1] * u0);
      double curl = 0.0;
      for (int j = 0; j < 3; ++j) {
        if (j == i) continue;
        curl += std::sin(plaq(c, n, i, j)) - std::sin(plaq(c, c->shift(n, j, -1), i, j));
      }
      curl *= -1.0 / (gQ * dx * dx * dx);
      KA[i][n] = a1 * fo2 * J + am1 * curl;
    }
  }
}

// ---------------------------------------------------------------------------
// SU(2) x U(1) doublet model: the gauge content of the manual's lphi4SU2U1
// example (Sec. 4.1-4.3, SU(N) toolkit of Sec. 4.2) -- a doublet Phi charged
// under a U(1) field A_i (coupling gQ = g_A Q_A) and an SU(2) field B_i^a
// (coupling gQB = g_B Q_B) -- with V = lam (|Phi|^2 - v^2)^2.
// Phi = (phi0 + i phi1, phi2 + i phi3)/sqrt2; psi = sqrt2 Phi below is the
// complex 2-vector of the stored real components.
// SU(2) links U_i(n) = exp(-i gQB dx B_i^a T_a), T_a = sigma_a/2, stored as
// four reals with U = u0 I - i (u1 sigma1 + u2 sigma2 + u3 sigma3), and
// multiplied here as explicit 2x2 complex matrices.  U(1) links are
// V_i = exp(-i gQ dx A_i) as in the U(1) model; the doublet hops with W_i = V_i U_i.
// reading: the manual leaves the lattice equations of the non-Abelian sector
// to its companion paper.  They are derived here, as for U(1), from one
// lattice Hamiltonian made of the toolkit's pieces (covariant hopping terms,
// compact U(1) plaquettes, the SU(2) plaquette trace), so that both lattice
// Gauss laws hold exactly.  At a = 1:
//   H = sum_n [ pi_c^2/2 + (1/(2 dx^2)) sum_i |W_i psi(n+i) - psi(n)|^2 + V ]
//     + (omega*/f*)^2 sum_n [ pi_A^2/2 + pi_B^2/2 + sum_{i<j} (1 - cos theta_ij)/(gQ dx^2)^2
//                             + sum_{i<j} 2 (2 - Tr U_ij)/(gQB dx^2)^2 ],
// the last term being (1/2) sum_a (G_ij^a)^2 to leading order (toolkit
// expansion of Tr U_ij).  The momentum pi_B,i^a(n) moves U_i(n) by left
// multiplication with exp(-i gQB dx delta T_a); its kernel is minus
// (f*/omega*)^2 times the derivative of H along that direction.  The powers
// of a of the kernels are those of Sec. 4.3.
// ---------------------------------------------------------------------------
struct M2 {
  cplx m[2][2];
};
struct D2 {
  cplx v[2];
};

M2 m_zero() {
  M2 r;
  r.m[0][0] = r.m[0][1] = r.m[1][0] = r.m[1][1] = cplx(0.0, 0.0);
  return r;
}
M2 mat_of(const double u[4]) {
  const cplx I(0.0, 1.0);
  M2 r;
  r.m[0][0] = u[0] - I * u[3];
  r.m[0][1] = -I * u[1] - u[2];
  r.m[1][0] = -I * u[1] + u[2];
  r.m[1][1] = u[0] + I * u[3];
  return r;
}
// (u0, u1, u2, u3) of an SU(2) matrix (each read symmetrically from the two
// entries that hold it)
void quat_of(const M2& M, double u[4]) {
  u[0] = 0.5 * (M.m[0][0].real() + M.m[1][1].real());
  u[3] = 0.5 * (M.m[1][1].imag() - M.m[0][0].imag());
  u[1] = -0.5 * (M.m[0][1].imag() + M.m[1][0].imag());
  u[2] = 0.5 * (M.m[1][0].real() - M.m[0][1].real());
}
M2 mul(const M2& A, const M2& B) {
  M2 r = m_zero();
  for (int i = 0; i < 2; ++i)
    for (int j = 0; j < 2; ++j)
      for (int k = 0; k < 2; ++k) r.m[i][j] += A.m[i][k] * B.m[k][j];
  return r;
}
M2 dag(const M2& A) {
  M2 r;
  for (int i = 0; i < 2; ++i)
    for (int j = 0; j < 2; ++j) r.m[i][j] = std::conj(A.m[j][i]);
  return r;
}
M2 add(const M2& A, const M2& B) {
  M2 r;
  for (int i = 0; i < 2; ++i)
    for (int j = 0; j < 2; ++j) r.m[i][j] = A.m[i][j] + B.m[i][j];
  return r;
}
cplx trace(const M2& A) { return A.m[0][0] + A.m[1][1]; }
// Pauli matrix sigma_a, a = 1, 2, 3
M2 pauli(int a) {
  const cplx I(0.0, 1.0);
  M2 r = m_zero();
  if (a == 1) { r.m[0][1] = 1.0; r.m[1][0] = 1.0; }
  if (a == 2) { r.m[0][1] = -I; r.m[1][0] = I; }
  if (a == 3) { r.m[0][0] = 1.0; r.m[1][1] = -1.0; }
  return r;
}
D2 mv(const M2& A, const D2& x) {
  D2 r;
  for (int i = 0; i < 2; ++i) r.v[i] = A.m[i][0] * x.v[0] + A.m[i][1] * x.v[1];
  return r;
}
cplx dot(const D2& x, const D2& y) { return std::conj(x.v[0]) * y.v[0] + std::conj(x.v[1]) * y.v[1]; }

// exp(-i theta.sigma/2) = cos(|theta|/2) I - i sin(|theta|/2) (theta/|theta|).sigma
void su2_exp(const double th[3], double u[4]) {
  const double t = std::sqrt(th[0] * th[0] + th[1] * th[1] + th[2] * th[2]);
  u[0] = std::cos(0.5 * t);
  const double s = t > 0.0 ? std::sin(0.5 * t) / t : 0.5;
  for (int a = 0; a < 3; ++a) u[a + 1] = s * th[a];
}

M2 su2_link(const clo_ctx* c, long n, int i) {
  double u[4];
  for (int k = 0; k < 4; ++k) u[k] = c->U[i][k][n];
  return mat_of(u);
}
D2 doublet(const clo_ctx* c, long n) {
  D2 r;
  r.v[0] = cplx(c->phi[0][n], c->phi[1][n]);
  r.v[1] = cplx(c->phi[2][n], c->phi[3][n]);
  return r;
}
D2 doublet_mom(const clo_ctx* c, long n) {
  D2 r;
  r.v[0] = cplx(c->pi[0][n], c->pi[1][n]);
  r.v[1] = cplx(c->pi[2][n], c->pi[3][n]);
  return r;
}
// W_i(n) psi(n+i) and W_i^dag(n-i) psi(n-i)
D2 hop_fwd(const clo_ctx* c, long n, int i) {
  const double th = c->p.gQ * c->dx * c->A[i][n];
  D2 r = mv(su2_link(c, n, i), doublet(c, c->shift(n, i, +1)));
  const cplx ph = std::polar(1.0, -th);
  r.v[0] *= ph;
  r.v[1] *= ph;
  return r;
}
D2 hop_bwd(const clo_ctx* c, long n, int i) {
  const long m = c->shift(n, i, -1);
  const double th = c->p.gQ * c->dx * c->A[i][m];
  D2 r = mv(dag(su2_link(c, m, i)), doublet(c, m));
  const cplx ph = std::polar(1.0, th);
  r.v[0] *= ph;
  r.v[1] *= ph;
  return r;
}
// SU(2) plaquette U_ij(n) = U_i(n) U_j(n+i) U_i^dag(n+j) U_j^dag(n)  (SU(N) toolkit)
M2 su2_plaq(const clo_ctx* c, long n, int i, int j) {
  M2 r = mul(su2_link(c, n, i), su2_link(c, c->shift(n, i, +1), j));
  r = mul(r, dag(su2_link(c, c->shift(n, j, +1), i)));
  return mul(r, dag(su2_link(c, n, j)));
}
// Staples of U_i(n): sum over j != i of U_j(n+i) U_i^dag(n+j) U_j^dag(n)
// (plaquette U_ij(n)) and U_j^dag(n+i-j) U_i^dag(n-j) U_j(n-j) (the plaquette
// at n-j, traversed from U_i(n)), so that Re Tr[U_i(n) S] is the sum of
// Re Tr over the four plaquettes holding U_i(n).
M2 su2_staples(const clo_ctx* c, long n, int i) {
  M2 S = m_zero();
  const long ni = c->shift(n, i, +1);
  for (int j = 0; j < 3; ++j) {
    if (j == i) continue;
    const long nj = c->shift(n, j, +1), nmj = c->shift(n, j, -1), nimj = c->shift(ni, j, -1);
    M2 up = mul(mul(su2_link(c, ni, j), dag(su2_link(c, nj, i))), dag(su2_link(c, n, j)));
    M2 lo = mul(mul(dag(su2_link(c, nimj, j)), dag(su2_link(c, nmj, i))), su2_link(c, nmj, j));
    S = add(S, add(up, lo));
  }
  return S;
}

// Kernels of the doublet model (Sec. 4.3 with the Hamiltonian above):
//   K_c     = a^{1+alpha} (D^2 psi)_c - a^{3+alpha} 2 lam (|Phi|^2 - v^2) phi_c,
//             D^2 psi = sum_i [W_i psi(n+i) - 2 psi + W_i^dag(n-i) psi(n-i)]/dx^2
//   K_{A_i} = a^{1+alpha} (f*/omega*)^2 (gQ/dx) Im[psi^dag W_i psi(n+i)] + a^{alpha-1} (compact curl, as U(1))
//   K_{B_i}^a = a^{1+alpha} (f*/omega*)^2 (gQB/(2 dx)) Im[psi^dag sigma_a W_i psi(n+i)]
//             + a^{alpha-1} (1/(gQB dx^3)) Im Tr[sigma_a U_i(n) S_i(n)].
// reading: the printed doublet kernel writes D_A^2; the covariant Laplacian of
// both gauge groups is used (eq. kernelsSU21 is otherwise the U(1) form).
// gQ = 0 switches the U(1) field off: no current, no curl, E_G^A = 0.
void kernel_su2(const clo_ctx* c, std::vector<double>* Kphi, std::vector<double>* KA,
                std::vector<double> (*KB)[3]) {
  const double a1 = std::pow(c->a, 1.0 + c->alpha), a3 = std::pow(c->a, 3.0 + c->alpha);
  const double am1 = std::pow(c->a, c->alpha - 1.0);
  const double idx2 = 1.0 / (c->dx * c->dx);
  const double fo2 = c->p.fstar_over_omegastar * c->p.fstar_over_omegastar;
  const double gQ = c->p.gQ, gB = c->p.gQB, dx = c->dx;
  for (long n = 0; n < c->V; ++n) {
    double f[7], d[7];
    if (c->full()) {
      full_site(c, n, f);
      full_force(c, f, d);
    } else {
      for (int k = 0; k < 4; ++k) f[k] = c->phi[k][n];
      pot_deriv(c, f, d);
    }
    const D2 psi = doublet(c, n);
    D2 D;
    D.v[0] = D.v[1] = cplx(0.0, 0.0);
    for (int i = 0; i < 3; ++i) {
      const D2 u = hop_fwd(c, n, i), w = hop_bwd(c, n, i);
      for (int r = 0; r < 2; ++r) D.v[r] += u.v[r] + w.v[r] - 2.0 * psi.v[r];
    }
    const double Dc[4] = {D.v[0].real(), D.v[0].imag(), D.v[1].real(), D.v[1].imag()};
    for (int k = 0; k < 4; ++k) Kphi[k][n] = a1 * Dc[k] * idx2 - a3 * d[k];
    for (int i = 0; i < 3; ++i) {
      const D2 u = hop_fwd(c, n, i);
      const double JA = (gQ / dx) * dot(psi, u).imag();
      double curl = 0.0;
      for (int j = 0; j < 3 && gQ != 0.0; ++j) {
        if (j == i) continue;
        curl += std::sin(plaq(c, n, i, j)) - std::sin(plaq(c, c->shift(n, j, -1), i, j));
      }
      if (gQ != 0.0) curl *= -1.0 / (gQ * dx * dx * dx);
      KA[i][n] = a1 * fo2 * JA + am1 * curl;
      const M2 M = mul(su2_link(c, n, i), su2_staples(c, n, i));
      for (int a = 1; a <= 3; ++a) {
        const double Ja = (gB / (2.0 * dx)) * dot(psi, mv(pauli(a), u)).imag();
        const double mag = trace(mul(pauli(a), M)).imag() / (gB * dx * dx * dx);
        KB[i][a - 1][n] = a1 * fo2 * Ja + am1 * mag;
      }
    }
  }
}

// lphi4SU2U1: kernels of the singlet and of the U(1)-charged scalar, and the
// charged scalar's share of the U(1) current (Sec. 4.3 Hamiltonian form):
//   K_s     = a^{1+alpha} Lap phi_s - a^{3+alpha} dV/dphi_s,
//   K_vphi  = a^{1+alpha} (D^2 vphi)_c/dx^2 - a^{3+alpha} dV/dvphi_c,
//             D^2 vphi = sum_i [Vc_i vphi(n+i) - 2 vphi + Vc_i^*(n-i) vphi(n-i)],
//             Vc_i = exp(-i Qc gQ dx A_i) (the charge Qc gQ = g_A Q_A^(vphi)),
//   K_{A_i} += a^{1+alpha} (f*/omega*)^2 Qc (gQ/dx) (vphi_0 u_1 - vphi_1 u_0),
//             u = Vc_i vphi(n+i) in components, as the U(1) model's current.
// reading: the doublet's charge is the unit of U(1) charge (gQ = g_A Q_A^(Phi)
// also scales the plaquette, as in the doublet model), and Qc is the charged
// scalar's charge in that unit.
void vphi_fwd(const clo_ctx* c, long n, int i, double& w0, double& w1) {
  const long m = c->shift(n, i, +1);
  const double th = c->p.Qc * c->p.gQ * c->dx * c->A[i][n];
  const double co = std::cos(th), si = std::sin(th);
  const double x = c->cph[0][m], y = c->cph[1][m];
  w0 = co * x + si * y;
  w1 = co * y - si * x;
}
void vphi_bwd(const clo_ctx* c, long n, int i, double& w0, double& w1) {
  const long m = c->shift(n, i, -1);
  const double th = c->p.Qc * c->p.gQ * c->dx * c->A[i][m];
  const double co = std::cos(th), si = std::sin(th);
  const double x = c->cph[0][m], y = c->cph[1][m];
  w0 = co * x - si * y;
  w1 = co * y + si * x;
}
void kernel_full_extra(const clo_ctx* c, std::vector<double>& Ks, std::vector<double>* Kc,
                       std::vector<double>* KA) {
  const double a1 = std::pow(c->a, 1.0 + c->alpha), a3 = std::pow(c->a, 3.0 + c->alpha);
  const double idx2 = 1.0 / (c->dx * c->dx);
  const double fo2 = c->p.fstar_over_omegastar * c->p.fstar_over_omegastar;
  const double gQc = c->p.Qc * c->p.gQ, dx = c->dx;
  for (long n = 0; n < c->V; ++n) {
    double f[7], d[7];
    full_site(c, n, f);
    full_force(c, f, d);
    double Ls = 0.0, D0 = 0.0, D1 = 0.0;
    for (int i = 0; i < 3; ++i) {
      Ls += c->sph[c->shift(n, i, +1)] + c->sph[c->shift(n, i, -1)] - 2.0 * f[4];
      double u0, u1, w0, w1;
      vphi_fwd(c, n, i, u0, u1);
      vphi_bwd(c, n, i, w0, w1);
      D0 += u0 + w0 - 2.0 * f[5];
      D1 += u1 + w1 - 2.0 * f[6];
      KA[i][n] += a1 * fo2 * (gQc / dx) * (f[5] * u1 - f[6] * u0);
    }
    Ks[n] = a1 * Ls * idx2 - a3 * d[4];
    Kc[0][n] = a1 * D0 * idx2 - a3 * d[5];
    Kc[1][n] = a1 * D1 * idx2 - a3 * d[6];
  }
}

// U_i(n) <- exp(-i gQB dx w_B pi_B,i^a T_a) U_i(n)   (w_B = step abar^{alpha-1})
void drift_su2_links(clo_ctx* c, double wB) {
  const double e = c->p.gQB * c->dx * wB;
  for (int i = 0; i < 3; ++i)
    for (long n = 0; n < c->V; ++n) {
      double th[3], g[4], u[4];
      for (int a = 0; a < 3; ++a) th[a] = e * c->piB[i][a][n];
      su2_exp(th, g);
      quat_of(mul(mat_of(g), su2_link(c, n, i)), u);
      for (int k = 0; k < 4; ++k) c->U[i][k][n] = u[k];
    }
}

// Gauss-law residuals of the doublet model at site n (derived from the
// invariance of H under a gauge transformation at n, SU(N) toolkit):
//   U(1):   sum_i grad^-_i pi_A,i - (f*/omega*)^2 gQ Im[psi^dag pi_psi]
//   SU(2):  sum_i [pi_B,i^a(n) - (U_i^dag(n-i) pi_B,i(n-i) U_i(n-i))^a]/dx
//           - (f*/omega*)^2 (gQB/2) Im[psi^dag sigma_a pi_psi]
// with pi_B = pi_B^b sigma_b/2 and X^a = Tr[sigma_a X].  lhs, rhs: the two sides.
void gauss_su2_site(const clo_ctx* c, long n, int g, double& lhs, double& rhs) {
  const double fo2 = c->p.fstar_over_omegastar * c->p.fstar_over_omegastar;
  const D2 psi = doublet(c, n), mom = doublet_mom(c, n);
  lhs = 0.0;
  if (g == 0) {
    for (int i = 0; i < 3; ++i) lhs += (c->piA[i][n] - c->piA[i][c->shift(n, i, -1)]) / c->dx;
    rhs = fo2 * c->p.gQ * dot(psi, mom).imag();
    if (c->full())  // the charged scalar's charge density, U(1) model form with charge Qc
      rhs += fo2 * c->p.Qc * c->p.gQ * (c->cph[0][n] * c->cpi[1][n] - c->cph[1][n] * c->cpi[0][n]);
    return;
  }
  for (int i = 0; i < 3; ++i) {
    const long m = c->shift(n, i, -1);
    M2 P = m_zero();
    for (int b = 1; b <= 3; ++b) {
      M2 s = pauli(b);
      for (int r = 0; r < 2; ++r)
        for (int q = 0; q < 2; ++q) P.m[r][q] += 0.5 * c->piB[i][b - 1][m] * s.m[r][q];
    }
    const M2 Um = su2_link(c, m, i);
    const double tr = trace(mul(pauli(g), mul(dag(Um), mul(P, Um)))).real();
    lhs += (c->piB[i][g - 1][n] - tr) / c->dx;
  }
  rhs = fo2 * 0.5 * c->p.gQB * dot(psi, mv(pauli(g), mom)).imag();
}

// ---------------------------------------------------------------------------
// Volume averages (eq. EK_EG_EV; eq. energy-contrib for U(1)).
// reading: the gradient energy uses forward differences grad^+, so that
// sum_n (grad^+ phi)^2 = -sum_n phi Lap phi matches the kick's Laplacian.
// ---------------------------------------------------------------------------
struct Avg {
  double EK[4], EG[4], EV[4], EKA, EGA, EKB, EGB;
  double mphi[4], mphi2[4], mpi[4], mpi2[4];
};

void averages(const clo_ctx* c, Avg& r) {
  std::memset(&r, 0, sizeof(r));
  double sp2[4] = {0, 0, 0, 0}, sg[2] = {0, 0}, sv[4] = {0, 0, 0, 0};
  double spA = 0.0, smag = 0.0, spB = 0.0, smagB = 0.0;
  double spS = 0.0, spC = 0.0, sgS = 0.0, sgC = 0.0;  // lphi4SU2U1: singlet and charged scalar
  for (long n = 0; n < c->V; ++n) {
    double f[7] = {0, 0, 0, 0, 0, 0, 0}, t[4] = {0, 0, 0, 0};
    for (int k = 0; k < c->nf; ++k) {
      f[k] = c->phi[k][n];
      double pv = c->pi[k][n];
      sp2[k] += pv * pv;
      r.mphi[k] += f[k];
      r.mphi2[k] += f[k] * f[k];
      r.mpi[k] += pv;
      r.mpi2[k] += pv * pv;
    }
    if (c->full()) {
      full_site(c, n, f);
      full_pot(c, f, t);
      spS += c->spi[n] * c->spi[n];
      spC += c->cpi[0][n] * c->cpi[0][n] + c->cpi[1][n] * c->cpi[1][n];
      for (int i = 0; i < 3; ++i) {
        const double g = c->sph[c->shift(n, i, +1)] - f[4];
        sgS += g * g;
        double u0, u1;
        vphi_fwd(c, n, i, u0, u1);
        sgC += (u0 - f[5]) * (u0 - f[5]) + (u1 - f[6]) * (u1 - f[6]);
      }
    } else {
      pot_terms(c, f, t);
    }
    for (int m = 0; m < n_pot_terms(c->model); ++m) sv[m] += t[m];
    if (!c->gauge()) {
      for (int k = 0; k < c->nf; ++k)
        for (int i = 0; i < 3; ++i) {
          double g = c->phi[k][c->shift(n, i, +1)] - c->phi[k][n];
          sg[k] += g * g;
        }
    } else if (!c->su2()) {
      for (int i = 0; i < 3; ++i) {
        double u0, u1;
        link_fwd(c, n, i, u0, u1);
        sg[0] += (u0 - f[0]) * (u0 - f[0]) + (u1 - f[1]) * (u1 - f[1]);
        spA += c->piA[i][n] * c->piA[i][n];
        for (int j = i + 1; j < 3; ++j) smag += 1.0 - std::cos(plaq(c, n, i, j));
      }
    } else {
      const D2 psi = doublet(c, n);
      for (int i = 0; i < 3; ++i) {
        const D2 u = hop_fwd(c, n, i);
        for (int r = 0; r < 2; ++r) sg[0] += std::norm(u.v[r] - psi.v[r]);
        spA += c->piA[i][n] * c->piA[i][n];
        for (int a = 0; a < 3; ++a) spB += c->piB[i][a][n] * c->piB[i][a][n];
        for (int j = i + 1; j < 3; ++j) {
          smag += 1.0 - std::cos(plaq(c, n, i, j));
          smagB += 2.0 - trace(su2_plaq(c, n, i, j)).real();
        }
      }
    }
  }
  double V = (double)c->V, a = c->a;
  double a2 = a * a, a4 = a2 * a2, a6 = a4 * a2;
  if (!c->gauge()) {
    for (int k = 0; k < c->nf; ++k) {
      r.EK[k] = sp2[k] / (2.0 * a6 * V);
      r.EG[k] = sg[k] / (2.0 * a2 * c->dx * c->dx * V);
    }
  } else {
    r.EK[0] = (sp2[0] + sp2[1] + sp2[2] + sp2[3]) / (2.0 * a6 * V);
    r.EG[0] = sg[0] / (2.0 * a2 * c->dx * c->dx * V);
    if (c->full()) {  // E_K, E_G of the singlet [1] and of the charged scalar [2]
      r.EK[1] = spS / (2.0 * a6 * V);
      r.EK[2] = spC / (2.0 * a6 * V);
      r.EG[1] = sgS / (2.0 * a2 * c->dx * c->dx * V);
      r.EG[2] = sgC / (2.0 * a2 * c->dx * c->dx * V);
    }
    double of2 = 1.0 / (c->p.fstar_over_omegastar * c->p.fstar_over_omegastar);
    double gdx2 = c->p.gQ * c->dx * c->dx;
    r.EKA = of2 * spA / (2.0 * a4 * V);
    r.EGA = gdx2 != 0.0 ? of2 * smag / (a4 * gdx2 * gdx2 * V) : 0.0;
    if (c->su2()) {
      // E_K^B, E_G^B: (omega*/f*)^2/a^4 times <pi_B^2/2> and <sum_{i<j} 2 (2 - Tr U_ij)>/(gQB dx^2)^2
      double bdx2 = c->p.gQB * c->dx * c->dx;
      r.EKB = of2 * spB / (2.0 * a4 * V);
      r.EGB = of2 * 2.0 * smagB / (a4 * bdx2 * bdx2 * V);
    }
  }
  for (int m = 0; m < n_pot_terms(c->model); ++m) r.EV[m] = sv[m] / V;
  for (int k = 0; k < c->nf; ++k) {
    r.mphi[k] /= V; r.mphi2[k] /= V; r.mpi[k] /= V; r.mpi2[k] /= V;
  }
}

double sum4(const double* x) { return x[0] + x[1] + x[2] + x[3]; }

// b' = K_a = a^{2alpha+1}/3 (f*/m_p)^2 [(alpha-2)E_K + alpha E_G
//            + (alpha-1)(E_K^A + E_G^A + E_K^B + E_G^B) + (alpha+1) E_V]   (Sec. 4.3)
double kernel_a(const clo_ctx* c, const Avg& r) {
  double al = c->alpha, fm = c->p.fstar_over_mp;
  double br = (al - 2.0) * sum4(r.EK) + al * sum4(r.EG) +
              (al - 1.0) * (r.EKA + r.EGA + r.EKB + r.EGB) + (al + 1.0) * sum4(r.EV);
  return std::pow(c->a, 2.0 * al + 1.0) / 3.0 * fm * fm * br;
}

// Fixed power-law background, eq. ScaleFactorPowerLaw (a_* = a0 at eta_*).
double a_fixed(const clo_ctx* c, double eta) {
  double p = 2.0 / (3.0 * (1.0 + c->p.omega_eos) - 2.0 * c->alpha);
  return c->a0 * std::pow(1.0 + c->Hfix * (eta - c->eta0) / p, p);
}
double H_fixed(const clo_ctx* c, double eta) {
  double p = 2.0 / (3.0 * (1.0 + c->p.omega_eos) - 2.0 * c->alpha);
  return c->Hfix / (1.0 + c->Hfix * (eta - c->eta0) / p);
}

// ---------------------------------------------------------------------------
// The three moves of the velocity-Verlet step (Sec. 3.5.2).
// reading (the manual defers the discrete scheme to its companion paper):
//   kick-in (h/2):  pi += h/2 K[a, phi];   b += h/2 K_a(a, E_K(pi_new), E_G, E_V)
//   drift (h):      a1 = a + h b;  phi += h abar^{alpha-3} pi,  abar = (a+a1)/2
//                   (U(1) links: A += h abar^{alpha-1} pi_A);   a = a1
//   kick-out (h/2): b += h/2 K_a(a, E_K(pi), E_G, E_V);  pi += h/2 K[a, phi]
// kick-out is the reverse of kick-in and the drift is symmetric, so the
// step is time reversible and second order.
// ---------------------------------------------------------------------------
void kick_fields(clo_ctx* c, double w) {
  if (!c->gauge()) {
    std::vector<double> K[2];
    for (int k = 0; k < c->nf; ++k) K[k].assign(c->V, 0.0);
    kernel_scalars(c, K);
    for (int k = 0; k < c->nf; ++k)
      for (long n = 0; n < c->V; ++n) c->pi[k][n] += w * K[k][n];
  } else if (!c->su2()) {
    std::vector<double> Kp[2], KA[3];
    for (int k = 0; k < 2; ++k) Kp[k].assign(c->V, 0.0);
    for (int i = 0; i < 3; ++i) KA[i].assign(c->V, 0.0);
    kernel_u1(c, Kp, KA);
    for (int k = 0; k < 2; ++k)
      for (long n = 0; n < c->V; ++n) c->pi[k][n] += w * Kp[k][n];
    for (int i = 0; i < 3; ++i)
      for (long n = 0; n < c->V; ++n) c->piA[i][n] += w * KA[i][n];
  } else {
    std::vector<double> Kp[4], KA[3], KB[3][3];
    for (int k = 0; k < 4; ++k) Kp[k].assign(c->V, 0.0);
    for (int i = 0; i < 3; ++i) {
      KA[i].assign(c->V, 0.0);
      for (int a = 0; a < 3; ++a) KB[i][a].assign(c->V, 0.0);
    }
    kernel_su2(c, Kp, KA, KB);
    if (c->full()) {
      std::vector<double> Ks(c->V, 0.0), Kc[2];
      for (int k = 0; k < 2; ++k) Kc[k].assign(c->V, 0.0);
      kernel_full_extra(c, Ks, Kc, KA);
      for (long n = 0; n < c->V; ++n) c->spi[n] += w * Ks[n];
      for (int k = 0; k < 2; ++k)
        for (long n = 0; n < c->V; ++n) c->cpi[k][n] += w * Kc[k][n];
    }
    for (int k = 0; k < 4; ++k)
      for (long n = 0; n < c->V; ++n) c->pi[k][n] += w * Kp[k][n];
    for (int i = 0; i < 3; ++i) {
      for (long n = 0; n < c->V; ++n) c->piA[i][n] += w * KA[i][n];
      for (int a = 0; a < 3; ++a)
        for (long n = 0; n < c->V; ++n) c->piB[i][a][n] += w * KB[i][a][n];
    }
  }
}

void kick_scale(clo_ctx* c, double w) {
  if (c->p.expansion != CLO_EXP_SELF) return;
  Avg r;
  averages(c, r);
  c->b += w * kernel_a(c, r);
}

void drift(clo_ctx* c, double w) {
  double a1, abar;
  if (c->p.expansion == CLO_EXP_SELF) {
    a1 = c->a + w * c->b;
  } else if (c->p.expansion == CLO_EXP_FIXED) {
    a1 = a_fixed(c, c->eta + w);
  } else {
    a1 = c->a;
  }
  abar = 0.5 * (c->a + a1);
  double cphi = w * std::pow(abar, c->alpha - 3.0);
  for (int k = 0; k < c->nf; ++k)
    for (long n = 0; n < c->V; ++n) c->phi[k][n] += cphi * c->pi[k][n];
  if (c->full()) {
    for (long n = 0; n < c->V; ++n) c->sph[n] += cphi * c->spi[n];
    for (int k = 0; k < 2; ++k)
      for (long n = 0; n < c->V; ++n) c->cph[k][n] += cphi * c->cpi[k][n];
  }
  if (c->gauge()) {
    double cA = w * std::pow(abar, c->alpha - 1.0);
    for (int i = 0; i < 3; ++i)
      for (long n = 0; n < c->V; ++n) c->A[i][n] += cA * c->piA[i][n];
    if (c->su2()) drift_su2_links(c, cA);
  }
  c->a = a1;
  c->eta += w;
  if (c->p.expansion == CLO_EXP_FIXED) c->b = a1 * H_fixed(c, c->eta);
}

void vv2(clo_ctx* c, double h) {
  kick_fields(c, 0.5 * h);
  kick_scale(c, 0.5 * h);
  drift(c, h);
  kick_scale(c, 0.5 * h);
  kick_fields(c, 0.5 * h);
}

double rho_of(const Avg& r) {
  return sum4(r.EK) + sum4(r.EG) + sum4(r.EV) + r.EKA + r.EGA + r.EKB + r.EGB;
}

// ---------------------------------------------------------------------------
// Initial conditions (Sec. 3.5.1 eqs. fpr_influct, fpr_influct2,
// QuantumFlucts2; Sec. 4.4.1 for the charged field and the gauge momenta).
// reading of the generator (the manual fixes the distributions, not the
// generator): for field component f and Fourier site with linear index idx
// (x fastest, wave numbers n~_i in (-N/2, N/2]), with key (seed lo, seed hi),
//   r = Philox(idx, f, 0, 0): u1 = u01(r0,r1), u2 = u01(r2,r3)  (amplitudes)
//   s = Philox(idx, f, 1, 0): v1 = u01(s0,s1), v2 = u01(s2,s3)  (phases)
//   |d_j| = sqrt(-P ln u_j) (Rayleigh, <|d|^2> = P), theta_j = 2 pi v_j,
//   P = fluct_amp2 (N/dx)^3 / (2 a^2 omega_k), omega_k = sqrt(k^2 + a^2 m^2), k = kIR |n~|.
// Only the member of each (n~, -n~) pair with the smaller linear index is
// drawn; the other is set to its complex conjugate so that the field is real;
// self-conjugate sites keep the real part; n~ = 0, k > kcut and omega_k^2 <= 0
// are set to zero.
// ---------------------------------------------------------------------------
long partner_index(const clo_ctx* c, long idx) {
  long x, y, z;
  c->coords(idx, x, y, z);
  return c->at(-x, -y, -z);
}
double mode_k(const clo_ctx* c, long idx) {
  long x, y, z;
  c->coords(idx, x, y, z);
  long n[3] = {x, y, z};
  double s = 0.0;
  for (int i = 0; i < 3; ++i) {
    long w = n[i] <= c->N / 2 ? n[i] : n[i] - c->N;
    s += (double)(w * w);
  }
  return c->kIR * std::sqrt(s);
}

void draw4(uint64_t seed, long idx, int f, int j, double u[2]) {
  uint32_t ctr[4] = {(uint32_t)idx, (uint32_t)f, (uint32_t)j, 0u};
  uint32_t key[2] = {(uint32_t)(seed & 0xffffffffu), (uint32_t)(seed >> 32)};
  uint32_t r[4];
  philox(ctr, key, r);
  u[0] = u01(r[0], r[1]);
  u[1] = u01(r[2], r[3]);
}

// Draws of the canonical site idx (idx <= partner): the two complex
// amplitudes z1, z2 of each field (|z| Rayleigh, phase uniform) and the
// frequency omega_k.  Returns false for sites that stay zero.
bool mode_draws(const clo_ctx* c, uint64_t seed, long idx, cplx* z1, cplx* z2, double* om) {
  double a = c->a, amp2 = c->p.fluct_amp2;
  double vol = std::pow((double)c->N / c->dx, 3.0);
  if (idx == 0) return false;
  long pid = partner_index(c, idx);
  bool selfc = pid == idx;
  if (selfc && c->gauge()) return false;  // reading: keeps the charge density's zero mode exactly 0
  double k = mode_k(c, idx);
  if (c->p.kcut >= 0.0 && k > c->p.kcut) return false;
  if (amp2 <= 0.0) return false;
  const int nc = ncomp(c);
  double h7[7] = {0, 0, 0, 0, 0, 0, 0};  // homogeneous values (the full model's extra fields start at 0)
  for (int f = 0; f < c->nf; ++f) h7[f] = c->p.phi0[f];
  for (int f = 0; f < nc; ++f) {
    double w2 = k * k + a * a * (c->full() ? full_mass2(c, h7, f) : mass2(c, c->p.phi0, f));
    if (w2 <= 0.0) return false;
    om[f] = std::sqrt(w2);
  }
  if (!c->gauge()) {
    for (int f = 0; f < c->nf; ++f) {
      double P = amp2 * vol / (2.0 * a * a * om[f]);
      double u[2], v[2];
      draw4(seed, idx, f, 0, u);
      draw4(seed, idx, f, 1, v);
      z1[f] = std::polar(std::sqrt(-P * std::log(u[0])), 2.0 * PI * v[0]);
      z2[f] = std::polar(std::sqrt(-P * std::log(u[1])), 2.0 * PI * v[1]);
    }
    return true;
  }
  // eqs. InConstr:1-2 for the components n of each charged field (components
  // f0 .. f0 + m - 1, f0 its reference): |d_{n1}| = |d_{n2}|,
  // theta_{n2} = theta_{f0,2} + theta_{n1} - theta_{f0,1}
  auto charged = [&](int f0, int m) {
    double u0[2], v0[2];
    draw4(seed, idx, f0, 0, u0);
    draw4(seed, idx, f0, 1, v0);
    double t01 = 2.0 * PI * v0[0], t02 = 2.0 * PI * v0[1];
    for (int f = f0; f < f0 + m; ++f) {
      double P = amp2 * vol / (2.0 * a * a * om[f]);
      double u[2], v[2];
      if (f == f0) {
        u[0] = u0[0]; u[1] = u0[1]; v[0] = v0[0]; v[1] = v0[1];
      } else {
        draw4(seed, idx, f, 0, u);
        draw4(seed, idx, f, 1, v);
      }
      double r = std::sqrt(-P * std::log(u[0]));
      double t1 = f == f0 ? t01 : 2.0 * PI * v[0];
      double t2 = f == f0 ? t02 : t02 + t1 - t01;
      z1[f] = std::polar(r, t1);
      z2[f] = std::polar(r, t2);
    }
  };
  charged(0, c->nf);
  if (c->full()) {
    // the singlet (component 4): independent amplitudes and phases as a scalar singlet
    double P = amp2 * vol / (2.0 * a * a * om[4]);
    double u[2], v[2];
    draw4(seed, idx, 4, 0, u);
    draw4(seed, idx, 4, 1, v);
    z1[4] = std::polar(std::sqrt(-P * std::log(u[0])), 2.0 * PI * v[0]);
    z2[4] = std::polar(std::sqrt(-P * std::log(u[1])), 2.0 * PI * v[1]);
    charged(5, 2);  // the U(1)-charged scalar
  }
  return true;
}

// Fourier values of the fluctuation (F[f]) and of its time derivative (G[f])
// at the canonical site idx (idx <= partner).  Returns false for sites that
// stay zero.
bool mode_values(const clo_ctx* c, uint64_t seed, double H, long idx, cplx* F, cplx* G) {
  const double isq2 = 1.0 / std::sqrt(2.0);
  cplx z1[8], z2[8];
  double om[8];
  if (!mode_draws(c, seed, idx, z1, z2, om)) return false;
  bool selfc = partner_index(c, idx) == idx;
  for (int f = 0; f < ncomp(c); ++f) {
    cplx df = (z1[f] + z2[f]) * isq2;
    cplx dv = std::pow(c->a, c->alpha - 1.0) * cplx(0.0, om[f]) * (z1[f] - z2[f]) * isq2 - H * df;
    if (selfc) { df = cplx(df.real(), 0.0); dv = cplx(dv.real(), 0.0); }
    F[f] = df;
    G[f] = dv;
  }
  return true;
}

// Fourier modes of the field fluctuation (F) and of its time derivative (G).
void fluct_modes(const clo_ctx* c, uint64_t seed, double H, std::vector<cplx>* F,
                 std::vector<cplx>* G) {
  for (int k = 0; k < ncomp(c); ++k) {
    F[k].assign(c->V, cplx(0, 0));
    G[k].assign(c->V, cplx(0, 0));
  }
  for (long idx = 1; idx < c->V; ++idx) {
    long pid = partner_index(c, idx);
    if (pid < idx) continue;
    cplx f[8], g[8];
    if (!mode_values(c, seed, H, idx, f, g)) continue;
    for (int k = 0; k < ncomp(c); ++k) {
      F[k][idx] = f[k]; G[k][idx] = g[k];
      F[k][pid] = std::conj(f[k]); G[k][pid] = std::conj(g[k]);
    }
  }
}

// Gauss-law momenta for the U(1) links (eq. GaugeCurrentFluc, on the lattice).
// reading: the lattice backward-difference symbol kappa_i = (1 - e^{-2 pi i n_i/N})/dx
// replaces the continuum k_i, so that sum_i grad^-_i pi_A,i equals the charge
// density to roundoff:  pi_A,i(k) = kappa_i^* rho(k)/|kappa|^2, rho(0) -> 0.
// The doublet model (links start at the identity, so both laws are linear
// there) takes the same inversion for the U(1) density and for each SU(2)
// colour's density.
// pi_A,i at Fourier site idx from the transformed density rhok.
cplx gauss_mode(const clo_ctx* c, const std::vector<cplx>& rhok, long idx, int i) {
  if (idx == 0) return cplx(0.0, 0.0);
  long x, y, z;
  c->coords(idx, x, y, z);
  long nn[3] = {x, y, z};
  double kk = 0.0;
  cplx ki;
  for (int j = 0; j < 3; ++j) {
    double t = 2.0 * PI * (double)nn[j] / (double)c->N;
    cplx kap = (1.0 - cplx(std::cos(t), -std::sin(t))) / c->dx;
    kk += std::norm(kap);
    if (j == i) ki = kap;
  }
  return std::conj(ki) * rhok[idx] / kk;
}

void invert_gauss(const clo_ctx* c, std::vector<cplx> rho, std::vector<double>* out) {
  bool zero = true;  // a zero density inverts to zero exactly: skip the transforms
  for (long n = 0; n < c->V && zero; ++n) zero = rho[n] == cplx(0.0, 0.0);
  if (zero) {
    for (int i = 0; i < 3; ++i) out[i].assign(c->V, 0.0);
    return;
  }
  fft3d(rho, c->N, -1);
  for (int i = 0; i < 3; ++i) {
    std::vector<cplx> E(c->V);
    for (long idx = 1; idx < c->V; ++idx) E[idx] = gauss_mode(c, rho, idx, i);
    fft3d(E, c->N, +1);
    for (long n = 0; n < c->V; ++n) out[i][n] = E[n].real() / (double)c->V;
  }
}

// Charge density of the U(1) Gauss law from the charged field and its momentum.
void u1_charge_density(const clo_ctx* c, std::vector<cplx>& rho) {
  double fo2 = c->p.fstar_over_omegastar * c->p.fstar_over_omegastar;
  rho.assign(c->V, cplx(0.0, 0.0));
  for (long n = 0; n < c->V; ++n)
    rho[n] = fo2 * c->p.gQ * (c->phi[0][n] * c->pi[1][n] - c->phi[1][n] * c->pi[0][n]);
}

void gauss_momenta(clo_ctx* c) {
  std::vector<cplx> rho(c->V);
  double lhs, rhs;
  if (!c->su2()) {
    u1_charge_density(c, rho);
    invert_gauss(c, rho, c->piA);
    return;
  }
  for (int g = 0; g < 4; ++g) {
    for (long n = 0; n < c->V; ++n) {
      gauss_su2_site(c, n, g, lhs, rhs);  // the density does not depend on the link momenta
      rho[n] = rhs;
    }
    if (g == 0) {
      invert_gauss(c, rho, c->piA);
    } else {
      std::vector<double> E[3];
      for (int i = 0; i < 3; ++i) E[i].assign(c->V, 0.0);
      invert_gauss(c, rho, E);
      for (int i = 0; i < 3; ++i) c->piB[i][g - 1] = E[i];
    }
  }
}

double homogeneous_rho(const clo_ctx* c) {
  double f[7] = {0, 0, 0, 0, 0, 0, 0}, t[4] = {0, 0, 0, 0};
  double kin = 0.0;
  for (int k = 0; k < c->nf; ++k) {
    f[k] = c->p.phi0[k];
    kin += 0.5 * c->p.dphi0[k] * c->p.dphi0[k];
  }
  if (c->full()) full_pot(c, f, t);  // singlet and charged scalar start at 0
  else pot_terms(c, f, t);
  return kin / std::pow(c->a, 2.0 * c->alpha) + sum4(t);
}

double b_from_hubble(const clo_ctx* c, double rho) {
  double fm = c->p.fstar_over_mp;
  double r = std::pow(c->a, 2.0 * c->alpha + 2.0) / 3.0 * fm * fm * rho;
  return r > 0.0 ? std::sqrt(r) : 0.0;
}

}  // namespace

// ===========================================================================
// C interface
// ===========================================================================
extern "C" {

void clo_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
  philox(ctr, key, out);
}
double clo_u01(uint32_t hi, uint32_t lo) { return u01(hi, lo); }

int clo_fft3d(double* re, double* im, int N, int sign) {
  if (N < 1 || (sign != 1 && sign != -1)) return -1;
  long V = (long)N * N * N;
  std::vector<cplx> a(V);
  for (long n = 0; n < V; ++n) a[n] = cplx(re[n], im[n]);
  fft3d(a, N, sign);
  for (long n = 0; n < V; ++n) { re[n] = a[n].real(); im[n] = a[n].imag(); }
  return 0;
}

// Definition of the 3-D DFT written out, O(N^6); for tiny N only.
int clo_dft3d_naive(const double* re, const double* im, double* ore, double* oim, int N,
                    int sign) {
  if (N < 1 || N > 16) return -1;
  long V = (long)N * N * N;
  for (long k = 0; k < V; ++k) {
    long kx = k % N, ky = (k / N) % N, kz = k / ((long)N * N);
    cplx s = 0.0;
    for (long n = 0; n < V; ++n) {
      long x = n % N, y = (n / N) % N, z = n / ((long)N * N);
      long e = (kx * x + ky * y + kz * z) % N;
      s += cplx(re[n], im[n]) * root(e, N, sign);
    }
    ore[k] = s.real(); oim[k] = s.imag();
  }
  return 0;
}

int clo_schedule(int integrator, double h, double* drifts, int cap) {
  std::vector<double> d;
  int order = integrator == CLO_LF ? 2 : integrator;
  if (order != 2 && order != 4 && order != 6 && order != 8 && order != 10) return -1;
  schedule(order, h, d);
  if ((int)d.size() > cap) return -2;
  for (size_t i = 0; i < d.size(); ++i) drifts[i] = d[i];
  return (int)d.size();
}

int clo_init(clo_ctx** out, int model, int N, double kIR, double alpha, uint64_t seed,
             const clo_params* p) {
  if (!out || !p) return -1;
  if (model < CLO_MODEL_LPHI4 || model > CLO_MODEL_LPHI4_SU2U1) return -1;
  if (N < 2 || kIR <= 0.0) return -1;
  if (model >= CLO_MODEL_SU2U1_HIGGS && !(p->gQB != 0.0)) return -1;
  clo_ctx* c = new clo_ctx();
  c->model = model;
  c->N = N;
  c->V = (long)N * N * N;
  c->nf = model == CLO_MODEL_LPHI4 ? 1 : (model >= CLO_MODEL_SU2U1_HIGGS ? 4 : 2);
  c->kIR = kIR;
  c->dx = 2.0 * PI / ((double)N * kIR);
  c->alpha = alpha;
  c->p = *p;
  c->a = c->a0 = 1.0;
  c->eta = c->eta0 = 0.0;
  for (int k = 0; k < c->nf; ++k) {
    c->phi[k].assign(c->V, 0.0);
    c->pi[k].assign(c->V, 0.0);
  }
  if (c->gauge())
    for (int i = 0; i < 3; ++i) {
      c->A[i].assign(c->V, 0.0);
      c->piA[i].assign(c->V, 0.0);
    }
  if (c->su2())  // eqs. Inflc1-4: links at the identity, momenta from the Gauss law
    for (int i = 0; i < 3; ++i) {
      for (int k = 0; k < 4; ++k) c->U[i][k].assign(c->V, k == 0 ? 1.0 : 0.0);
      for (int a = 0; a < 3; ++a) c->piB[i][a].assign(c->V, 0.0);
    }
  if (c->full()) {  // reading: the singlet and the charged scalar start with zero homogeneous values
    c->sph.assign(c->V, 0.0);
    c->spi.assign(c->V, 0.0);
    for (int k = 0; k < 2; ++k) {
      c->cph[k].assign(c->V, 0.0);
      c->cpi[k].assign(c->V, 0.0);
    }
  }
  // initial a' (Sec. 5.2 ScaleFactorInitializer: from homogeneous values)
  double rho_h = homogeneous_rho(c);
  if (p->expansion == CLO_EXP_SELF) {
    c->b = b_from_hubble(c, rho_h);
  } else if (p->expansion == CLO_EXP_FIXED) {
    c->Hfix = p->H0 > 0.0 ? p->H0 : b_from_hubble(c, rho_h) / c->a;
    c->b = c->a * c->Hfix;
  } else {
    c->b = 0.0;
  }
  double H = c->b / c->a;
  c->seed = seed;
  c->H_ic = H;
  double a3ma = std::pow(c->a, 3.0 - alpha);
  if (p->fluct_amp2 > 0.0) {
    std::vector<cplx> F[8], G[8];
    fluct_modes(c, seed, H, F, G);
    for (int k = 0; k < c->nf; ++k) {
      fft3d(F[k], N, +1);
      fft3d(G[k], N, +1);
      for (long n = 0; n < c->V; ++n) {
        c->phi[k][n] = p->phi0[k] + F[k][n].real() / (double)c->V;
        c->pi[k][n] = a3ma * (p->dphi0[k] + G[k][n].real() / (double)c->V);
      }
    }
    for (int k = 4; k < ncomp(c); ++k) {  // full model: singlet (4), charged scalar (5, 6)
      fft3d(F[k], N, +1);
      fft3d(G[k], N, +1);
      std::vector<double>& fk = k == 4 ? c->sph : c->cph[k - 5];
      std::vector<double>& pk = k == 4 ? c->spi : c->cpi[k - 5];
      for (long n = 0; n < c->V; ++n) {
        fk[n] = F[k][n].real() / (double)c->V;
        pk[n] = a3ma * (G[k][n].real() / (double)c->V);
      }
    }
  } else {  // no fluctuations: every Fourier mode but the homogeneous one is zero
    for (int k = 0; k < c->nf; ++k)
      for (long n = 0; n < c->V; ++n) {
        c->phi[k][n] = p->phi0[k];
        c->pi[k][n] = a3ma * p->dphi0[k];
      }
  }
  if (c->gauge()) gauss_momenta(c);
  Avg r;
  averages(c, r);
  if (p->expansion == CLO_EXP_SELF && p->b0_mode == 1) c->b = b_from_hubble(c, rho_of(r));
  c->rho0 = rho_of(r);
  *out = c;
  return 0;
}

// Fourier values of the initial fluctuations at selected sites, without
// building the lattice: out[(i*nf + f)*4 + {0,1,2,3}] = Re F, Im F, Re G, Im G
// of field f at site idx[i] (same conventions as clo_init).
int clo_ic_sample(int model, int N, double kIR, double alpha, uint64_t seed, const clo_params* p,
                  int n, const int64_t* idx, double* out) {
  if (!p || !idx || !out || model < CLO_MODEL_LPHI4 || model > CLO_MODEL_LPHI4_SU2U1) return -1;
  clo_ctx c;
  c.model = model;
  c.N = N;
  c.V = (long)N * N * N;
  c.nf = model == CLO_MODEL_LPHI4 ? 1 : (model >= CLO_MODEL_SU2U1_HIGGS ? 4 : 2);
  c.kIR = kIR;
  c.dx = 2.0 * PI / ((double)N * kIR);
  c.alpha = alpha;
  c.p = *p;
  c.a = c.a0 = 1.0;
  c.eta = c.eta0 = 0.0;
  double rho_h = homogeneous_rho(&c);
  if (p->expansion == CLO_EXP_SELF) c.b = b_from_hubble(&c, rho_h);
  else if (p->expansion == CLO_EXP_FIXED) c.b = c.a * (p->H0 > 0.0 ? p->H0 : b_from_hubble(&c, rho_h) / c.a);
  else c.b = 0.0;
  for (int i = 0; i < n; ++i) {
    long id = (long)idx[i];
    if (id < 0 || id >= c.V) return -1;
    long pid = partner_index(&c, id);
    cplx f[8], g[8];
    bool conj = pid < id;
    if (!mode_values(&c, seed, c.b / c.a, conj ? pid : id, f, g)) {
      for (int k = 0; k < 8; ++k) f[k] = g[k] = cplx(0, 0);
    }
    const int nc = ncomp(&c);
    for (int k = 0; k < nc; ++k) {
      cplx F = conj ? std::conj(f[k]) : f[k], G = conj ? std::conj(g[k]) : g[k];
      double* o = out + ((size_t)i * nc + k) * 4;
      o[0] = F.real(); o[1] = F.imag(); o[2] = G.real(); o[3] = G.imag();
    }
  }
  return 0;
}

int clo_free(clo_ctx* c) {
  delete c;
  return 0;
}

int clo_step_h(clo_ctx* c, int n, double h) {
  if (!c || n < 0) return -1;
  std::vector<double> d;
  int order = c->p.integrator == CLO_LF ? 2 : c->p.integrator;
  if (order != 2 && order != 4 && order != 6 && order != 8 && order != 10) return -1;
  schedule(order, h, d);
  for (int s = 0; s < n; ++s)
    for (size_t j = 0; j < d.size(); ++j) vv2(c, d[j]);
  return 0;
}

int clo_step(clo_ctx* c, int n) { return c ? clo_step_h(c, n, c->p.dt) : -1; }

int clo_energies(clo_ctx* c, clo_energies_t* o) {
  if (!c || !o) return -1;
  Avg r;
  averages(c, r);
  std::memset(o, 0, sizeof(*o));
  o->eta = c->eta; o->a = c->a; o->b = c->b;
  for (int k = 0; k < 4; ++k) {
    o->EK[k] = r.EK[k]; o->EG[k] = r.EG[k]; o->EV[k] = r.EV[k];
    o->mean_phi[k] = r.mphi[k]; o->mean_phi2[k] = r.mphi2[k];
    o->mean_pi[k] = r.mpi[k]; o->mean_pi2[k] = r.mpi2[k];
  }
  o->EKA = r.EKA; o->EGA = r.EGA;
  o->EKB = r.EKB; o->EGB = r.EGB;
  o->rho = rho_of(r);
  // Hubble constraint eq. NewFriedmannEQsI and its monitor (Sec. 3.3.2 outputs)
  double fm = c->p.fstar_over_mp;
  o->hubble_lhs = c->b * c->b;
  o->hubble_rhs = std::pow(c->a, 2.0 * c->alpha + 2.0) / 3.0 * fm * fm * o->rho;
  double den = o->hubble_lhs + o->hubble_rhs;
  o->hubble_viol = den > 0.0 ? (o->hubble_lhs - o->hubble_rhs) / den : 0.0;
  o->energy_cons = c->rho0 != 0.0 ? 1.0 - o->rho / c->rho0 : 0.0;
  return 0;
}

static std::vector<double>* field_ptr(const clo_ctx* c, int field, int what) {
  clo_ctx* m = const_cast<clo_ctx*>(c);
  if (what != 0 && what != 1) return nullptr;
  if (field >= 0 && field < c->nf) return what == 0 ? &m->phi[field] : &m->pi[field];
  if (c->gauge() && field >= c->nf && field < c->nf + 3)
    return what == 0 ? &m->A[field - c->nf] : &m->piA[field - c->nf];
  if (c->full() && field == 7) return what == 0 ? &m->sph : &m->spi;
  if (c->full() && (field == 8 || field == 9)) return what == 0 ? &m->cph[field - 8] : &m->cpi[field - 8];
  return nullptr;
}

int clo_get_state(const clo_ctx* c, int field, int what, double* out) {
  if (!c || !out) return -1;
  std::vector<double>* v = field_ptr(c, field, what);
  if (!v) return -1;
  std::memcpy(out, v->data(), sizeof(double) * c->V);
  return 0;
}

int clo_set_state(clo_ctx* c, int field, int what, const double* in) {
  if (!c || !in) return -1;
  std::vector<double>* v = field_ptr(c, field, what);
  if (!v) return -1;
  std::memcpy(v->data(), in, sizeof(double) * c->V);
  return 0;
}

int clo_get_scalars(const clo_ctx* c, double* eta, double* a, double* b) {
  if (!c) return -1;
  if (eta) *eta = c->eta;
  if (a) *a = c->a;
  if (b) *b = c->b;
  return 0;
}

int clo_set_scalars(clo_ctx* c, double eta, double a, double b) {
  if (!c) return -1;
  c->eta = eta; c->a = a; c->b = b;
  return 0;
}

int clo_nfields(const clo_ctx* c) { return c ? (c->full() ? 10 : (c->gauge() ? c->nf + 3 : c->nf)) : -1; }

static std::vector<double>* array_ptr(const clo_ctx* c, int a) {
  clo_ctx* m = const_cast<clo_ctx*>(c);
  if (!c->su2() || a < 0 || a >= (c->full() ? 41 : 35)) return nullptr;
  if (a >= 35) {  // full model: 35 phi_s, 36 pi_s, 37, 38 vphi_c, 39, 40 pi_vphi,c
    if (a == 35) return &m->sph;
    if (a == 36) return &m->spi;
    return a < 39 ? &m->cph[a - 37] : &m->cpi[a - 39];
  }
  if (a < 4) return &m->phi[a];
  if (a < 8) return &m->pi[a - 4];
  if (a < 11) return &m->A[a - 8];
  if (a < 14) return &m->piA[a - 11];
  if (a < 26) return &m->U[(a - 14) / 4][(a - 14) % 4];
  return &m->piB[(a - 26) / 3][(a - 26) % 3];
}

int clo_get_array(const clo_ctx* c, int a, double* out) {
  if (!c || !out) return -1;
  std::vector<double>* v = array_ptr(c, a);
  if (!v) return -1;
  std::memcpy(out, v->data(), sizeof(double) * c->V);
  return 0;
}

int clo_set_array(clo_ctx* c, int a, const double* in) {
  if (!c || !in) return -1;
  std::vector<double>* v = array_ptr(c, a);
  if (!v) return -1;
  std::memcpy(v->data(), in, sizeof(double) * c->V);
  return 0;
}

int clo_gauss_residual(const clo_ctx* c, int g, double* out) {
  if (!c || !out || !c->gauge() || g < 0 || g > (c->su2() ? 3 : 0)) return -1;
  const double fo2 = c->p.fstar_over_omegastar * c->p.fstar_over_omegastar;
  for (long n = 0; n < c->V; ++n) {
    double L = 0.0, R = 0.0;
    if (c->su2()) {
      gauss_su2_site(c, n, g, L, R);
    } else {
      for (int i = 0; i < 3; ++i) L += (c->piA[i][n] - c->piA[i][c->shift(n, i, -1)]) / c->dx;
      R = fo2 * c->p.gQ * (c->phi[0][n] * c->pi[1][n] - c->phi[1][n] * c->pi[0][n]);
    }
    out[n] = L - R;
  }
  return 0;
}

void clo_su2_exp(const double theta[3], double u[4]) { su2_exp(theta, u); }

// Gauss-law monitor (Sec. 4.5 output "average_gauss"): LHS = sum_i grad^-_i pi_A,i,
// RHS = (f*/omega*)^2 2 gQ Im[phi^* pi_phi]; rel = <|L-R|>/<|L+R|>.  Doublet
// model: the sums run over the U(1) law and the three SU(2) colours.
int clo_gauss_constraint(const clo_ctx* c, double* rel, double* lhs_abs, double* rhs_abs,
                         double* max_abs) {
  if (!c || !c->gauge()) return -1;
  double fo2 = c->p.fstar_over_omegastar * c->p.fstar_over_omegastar;
  double sd = 0.0, ss = 0.0, mx = 0.0;
  for (long n = 0; n < c->V; ++n) {
    const int ng = c->su2() ? 4 : 1;
    for (int g = 0; g < ng; ++g) {
      double L = 0.0, R = 0.0;
      if (c->su2()) {
        gauss_su2_site(c, n, g, L, R);
      } else {
        for (int i = 0; i < 3; ++i) L += (c->piA[i][n] - c->piA[i][c->shift(n, i, -1)]) / c->dx;
        R = fo2 * c->p.gQ * (c->phi[0][n] * c->pi[1][n] - c->phi[1][n] * c->pi[0][n]);
      }
      sd += std::fabs(L - R);
      ss += std::fabs(L + R);
      if (std::fabs(L - R) > mx) mx = std::fabs(L - R);
    }
  }
  double V = (double)c->V;
  if (lhs_abs) *lhs_abs = sd / V;
  if (rhs_abs) *rhs_abs = ss / V;
  if (rel) *rel = ss > 0.0 ? sd / ss : 0.0;
  if (max_abs) *max_abs = mx;
  return 0;
}

// Binned power spectrum, eqs. discretePS and discretePSII.
// Bins b = floor(|n~|/dk_bin) over n~ != 0; n~_b = mean |n~| in the bin;
// k_b = kIR n~_b; Delta_b = k_b^3/(2 pi^2) (dx/N)^3 sum_b |f(n~)|^2 / (4 pi n~_b^2).
int clo_spectrum(const clo_ctx* c, int field, int what, double dk_bin, double* k,
                 double* delta, int64_t* mult, int cap, int* nbins) {
  if (!c || dk_bin <= 0.0) return -1;
  std::vector<double>* v = field_ptr(c, field, what);
  if (!v) return -1;
  int nb = (int)std::floor(std::sqrt(3.0) * (c->N / 2) / dk_bin) + 1;
  if (nbins) *nbins = nb;
  if (nb > cap) return -2;
  std::vector<cplx> a(c->V);
  for (long n = 0; n < c->V; ++n) a[n] = cplx((*v)[n], 0.0);
  fft3d(a, c->N, -1);
  std::vector<double> sp(nb, 0.0), sn(nb, 0.0);
  std::vector<int64_t> cnt(nb, 0);
  for (long idx = 1; idx < c->V; ++idx) {
    double nn = mode_k(c, idx) / c->kIR;
    int b = (int)std::floor(nn / dk_bin);
    if (b >= nb) b = nb - 1;
    sp[b] += std::norm(a[idx]);
    sn[b] += nn;
    cnt[b] += 1;
  }
  double fac = std::pow(c->dx / (double)c->N, 3.0);
  for (int b = 0; b < nb; ++b) {
    if (cnt[b] == 0) { k[b] = 0.0; delta[b] = 0.0; mult[b] = 0; continue; }
    double nbar = sn[b] / (double)cnt[b];
    double kb = c->kIR * nbar;
    k[b] = kb;
    delta[b] = kb * kb * kb / (2.0 * PI * PI) * fac * sp[b] / (4.0 * PI * nbar * nbar);
    mult[b] = cnt[b];
  }
  return 0;
}

// Spectra of the electric and magnetic fields of the U(1) model (the gauge
// spectra of the outputs of Sec. 5.3; defined from eq. ElectricMagneticDefs):
//   E_i = F_0i = a^{alpha-1} pi_A,i      (pi_A = a^{1-alpha} F_0i, program units)
//   B_i = (1/2) eps_ijk F_jk,   F_jk = sin theta_jk/(gQ dx^2)
// with the compact plaquette angle theta_jk = gQ dx^2 F_jk of the U(1) toolkit,
// so B_x = F_yz, B_y = -F_xz, B_z = F_xy at the plaquette's corner n.  Each
// field's spectrum is eq. discretePS with |f(k)|^2 summed over the three
// components, on clo_spectrum's shells.  which = 0: E, 1: B.
// reading: the manual names these outputs without a formula; the field
// strength from the plaquette's sine is the compact form whose small-angle
// limit is the forward-difference curl.
//
// Doublet model: which = 0, 1 are the U(1) field's E and B as above (B needs
// gQ != 0); which = 2, 3 the SU(2) field's, summed over the 9 components (a, i):
//   E_i^a = a^{alpha-1} pi_B,i^a,
//   B_i^a = (1/2) eps_ijk G_jk^a,  G_jk^a = Tr[(i sigma_a/2)(U_jk - U_jk^dag)]/(gQB dx^2)
// (the SU(N) toolkit's expression for G from the plaquette; its small-angle limit
// is the forward-difference curl of B_i^a).
// reading: the manual's spectra_norm_SU2 output names these without a formula;
// the colour components are summed like the spatial ones.
int clo_em_spectrum(const clo_ctx* c, int which, double dk_bin, double* k, double* delta, int64_t* mult,
                    int cap, int* nbins) {
  const int wmax = c && c->su2() ? 3 : 1;
  if (!c || !c->gauge() || which < 0 || which > wmax || !(dk_bin > 0.0)) return -1;
  if (which == 1 && c->p.gQ == 0.0) return -1;  // no U(1) field
  const int nb = (int)std::floor(std::sqrt(3.0) * (c->N / 2) / dk_bin) + 1;
  if (nbins) *nbins = nb;
  if (nb > cap) return -2;
  const double gdx2 = c->p.gQ * c->dx * c->dx, ae = std::pow(c->a, c->alpha - 1.0);
  const double bdx2 = c->p.gQB * c->dx * c->dx;
  std::vector<double> sp(nb, 0.0), sn(nb, 0.0);
  std::vector<int64_t> cnt(nb, 0);
  const int ncomp = which >= 2 ? 9 : 3;
  for (int comp = 0; comp < ncomp; ++comp) {
    std::vector<cplx> F(c->V);
    const int i = which >= 2 ? comp / 3 : comp, a = comp % 3 + 1;
    const int j = (i + 1) % 3, l = (i + 2) % 3;  // B_i = F_jl for (i, j, l) cyclic
    for (long n = 0; n < c->V; ++n) {
      double v;
      if (which == 0) {
        v = ae * c->piA[i][n];
      } else if (which == 1) {
        v = std::sin(plaq(c, n, j, l)) / gdx2;
      } else if (which == 2) {
        v = ae * c->piB[i][a - 1][n];
      } else {
        const M2 P = su2_plaq(c, n, j, l), Pd = dag(P);
        M2 D;
        for (int r = 0; r < 2; ++r)
          for (int q = 0; q < 2; ++q) D.m[r][q] = P.m[r][q] - Pd.m[r][q];
        v = (cplx(0.0, 0.5) * trace(mul(pauli(a), D))).real() / bdx2;
      }
      F[n] = cplx(v, 0.0);
    }
    fft3d(F, c->N, -1);
    for (long idx = 1; idx < c->V; ++idx) {
      const double nn = mode_k(c, idx) / c->kIR;
      int b = (int)std::floor(nn / dk_bin);
      if (b >= nb) b = nb - 1;
      sp[b] += std::norm(F[idx]);
      if (comp == 0) {
        sn[b] += nn;
        cnt[b] += 1;
      }
    }
  }
  const double fac = std::pow(c->dx / (double)c->N, 3.0);
  for (int b = 0; b < nb; ++b) {
    if (cnt[b] == 0) { k[b] = 0.0; delta[b] = 0.0; mult[b] = 0; continue; }
    const double nbar = sn[b] / (double)cnt[b], kb = c->kIR * nbar;
    k[b] = kb;
    delta[b] = kb * kb * kb / (2.0 * PI * PI) * fac * sp[b] / (4.0 * PI * nbar * nbar);
    mult[b] = cnt[b];
  }
  return 0;
}

// Lattice occupation number of a scalar field (eq. OccuppationNum, in the
// outputs of the scalar-field module): per bin b of clo_spectrum's shells,
//   n_b = a^2 L^3/(2 N^6) (f*/omega*)^2 [ w_b <|phi_k|^2>_b + a^{2(1-alpha)}/w_b <|phi'_k + (a'/a) phi_k|^2>_b ]
// with <.>_b the mean over the bin's modes (k != 0), phi_k the forward DFT of
// the field, phi' = a^{alpha-3} pi, L = N dx and w_b^2 = k_b^2 + a^2 <V_{,ff}>
// (k_b = kIR times the bin's mean |n|; <V_{,ff}> the volume average of the
// field's diagonal Hessian element).  fo2 = (f*/omega*)^2.
// reading: w is taken at the bin's k, as the formula writes it outside the
// shell average; bins with w_b^2 <= 0 are NaN.
int clo_occupation(const clo_ctx* c, int field, double dk_bin, double fo2, double* k, double* n,
                   int64_t* mult, int cap, int* nbins) {
  if (!c || !(dk_bin > 0.0) || !(fo2 > 0.0) || c->gauge() || field < 0 || field >= c->nf) return -1;
  const int nb = (int)std::floor(std::sqrt(3.0) * (c->N / 2) / dk_bin) + 1;
  if (nbins) *nbins = nb;
  if (nb > cap) return -2;
  const double V = (double)c->V, a = c->a, H = c->b / c->a, al = c->alpha;
  double m2 = 0.0;
  for (long s = 0; s < c->V; ++s) {
    double f[2] = {0.0, 0.0};
    for (int q = 0; q < c->nf; ++q) f[q] = c->phi[q][s];
    m2 += mass2(c, f, field);
  }
  m2 /= V;
  std::vector<cplx> P(c->V), G(c->V);
  const double apm = std::pow(a, al - 3.0);
  for (long s = 0; s < c->V; ++s) {
    P[s] = cplx(c->phi[field][s], 0.0);
    G[s] = cplx(apm * c->pi[field][s] + H * c->phi[field][s], 0.0);
  }
  fft3d(P, c->N, -1);
  fft3d(G, c->N, -1);
  std::vector<double> s1(nb, 0.0), s2(nb, 0.0), sn(nb, 0.0);
  std::vector<int64_t> cnt(nb, 0);
  for (long idx = 1; idx < c->V; ++idx) {
    const double nn = mode_k(c, idx) / c->kIR;
    int b = (int)std::floor(nn / dk_bin);
    if (b >= nb) b = nb - 1;
    s1[b] += std::norm(P[idx]);
    s2[b] += std::norm(G[idx]);
    sn[b] += nn;
    cnt[b] += 1;
  }
  const double L = c->N * c->dx, C = a * a * L * L * L / (2.0 * V * V) * fo2;
  const double a2p = std::pow(a, 2.0 * (1.0 - al));
  for (int b = 0; b < nb; ++b) {
    if (cnt[b] == 0) { k[b] = 0.0; n[b] = 0.0; mult[b] = 0; continue; }
    const double kb = c->kIR * sn[b] / (double)cnt[b];
    const double w2 = kb * kb + a * a * m2;
    k[b] = kb;
    mult[b] = cnt[b];
    if (!(w2 > 0.0)) { n[b] = std::nan(""); continue; }
    const double w = std::sqrt(w2);
    n[b] = C * (w * s1[b] / (double)cnt[b] + a2p * s2[b] / ((double)cnt[b] * w));
  }
  return 0;
}

// Spectra of the modulus of a charged field (the "norm" spectra of the gauge
// models' outputs, Sec. 4.5; the modulus is what the manual's `norm` gives):
//   r = |phi| = sqrt(sum_c phi_c^2 / 2)   (U(1) field: c = 0, 1; doublet: c = 0..3),
//   r' = sum_c phi_c phi_c' / (2 r),       phi_c' = a^{alpha-3} pi_c   (0 where r = 0),
// delta_f, delta_fp = eq. discretePS of r and r' on clo_spectrum's shells, and n =
// eq. OccuppationNum applied to the canonically normalised modulus rho = sqrt2 r (each
// real component phi_c has a canonical kinetic term, so the radial field with one is
// sqrt(sum_c phi_c^2)), with w_b^2 = k_b^2 + a^2 <d^2V/drho^2>, V = lam (r^2 - v^2)^2:
// d^2V/drho^2 = V''(r)/2 = lam (6 r^2 - 2 v^2); |rho_k|^2 = 2 |r_k|^2; fo2 = (f*/omega*)^2.
// reading: the manual lists Delta, Delta' and n of these fields without formulas;
// the modulus is gauge invariant, its components are not, and eq. OccuppationNum
// is written for a canonically normalised field.
int clo_norm_spectrum(const clo_ctx* c, double dk_bin, double fo2, double* k, double* df, double* dfp,
                      double* n, int64_t* mult, int cap, int* nbins) {
  return clo_norm_spectrum_of(c, 0, dk_bin, fo2, k, df, dfp, n, mult, cap, nbins);
}

// which = 0: the model's charged field (the U(1) scalar, or the doublet); which = 1:
// lphi4SU2U1's U(1)-charged scalar vphi.  The mass of eq. OccuppationNum is the
// volume average of the potential's curvature along the canonical modulus
// rho = sqrt2 r, d^2V/drho^2 = (1/2) d^2V/dr^2, at the other fields' values:
//   U(1) scalar, doublet: V = lam (r^2 - v^2)^2 -> lam (6 r^2 - 2 v^2);
//   lphi4SU2U1 doublet (eq. PotGauge): + q_G r^2 phi_s^2 + 2 q_H r^2 |vphi|^2
//     -> lam (6 r^2 - 2 v^2) + q_G phi_s^2 + 2 q_H |vphi|^2;
//   lphi4SU2U1 vphi, r = |vphi|: 2 q_H |Phi|^2 r^2 -> 2 q_H |Phi|^2.
int clo_norm_spectrum_of(const clo_ctx* c, int which, double dk_bin, double fo2, double* k, double* df,
                         double* dfp, double* n, int64_t* mult, int cap, int* nbins) {
  if (!c || !c->gauge() || !(dk_bin > 0.0) || !(fo2 > 0.0)) return -1;
  if (which != 0 && !(which == 1 && c->full())) return -1;
  const int nb = (int)std::floor(std::sqrt(3.0) * (c->N / 2) / dk_bin) + 1;
  if (nbins) *nbins = nb;
  if (nb > cap) return -2;
  const double V = (double)c->V, a = c->a, H = c->b / c->a, al = c->alpha;
  const double apm = std::pow(a, al - 3.0);
  const int nc = which == 1 ? 2 : c->nf;
  const std::vector<double>* fq = which == 1 ? c->cph : c->phi;
  const std::vector<double>* pq = which == 1 ? c->cpi : c->pi;
  std::vector<cplx> R(c->V), Rp(c->V), G(c->V);
  double m2 = 0.0;
  for (long s = 0; s < c->V; ++s) {
    double r2 = 0.0, rr = 0.0;
    for (int q = 0; q < nc; ++q) {
      r2 += 0.5 * fq[q][s] * fq[q][s];
      rr += 0.5 * fq[q][s] * apm * pq[q][s];
    }
    const double r = std::sqrt(r2), rp = r > 0.0 ? rr / r : 0.0;
    R[s] = cplx(r, 0.0);
    Rp[s] = cplx(rp, 0.0);
    G[s] = cplx(rp + H * r, 0.0);
    if (which == 1) {
      double d2 = 0.0;  // |Phi|^2
      for (int q = 0; q < 4; ++q) d2 += 0.5 * c->phi[q][s] * c->phi[q][s];
      m2 += 2.0 * c->p.qH * d2;
    } else {
      m2 += c->p.lam * (6.0 * r2 - 2.0 * c->p.v * c->p.v);
      if (c->full()) {
        const double v2 = 0.5 * (c->cph[0][s] * c->cph[0][s] + c->cph[1][s] * c->cph[1][s]);
        m2 += c->p.qG * c->sph[s] * c->sph[s] + 2.0 * c->p.qH * v2;
      }
    }
  }
  m2 /= V;
  fft3d(R, c->N, -1);
  fft3d(Rp, c->N, -1);
  fft3d(G, c->N, -1);
  std::vector<double> s1(nb, 0.0), s1p(nb, 0.0), s2(nb, 0.0), sn(nb, 0.0);
  std::vector<int64_t> cnt(nb, 0);
  for (long idx = 1; idx < c->V; ++idx) {
    const double nn = mode_k(c, idx) / c->kIR;
    int b = (int)std::floor(nn / dk_bin);
    if (b >= nb) b = nb - 1;
    s1[b] += std::norm(R[idx]);
    s1p[b] += std::norm(Rp[idx]);
    s2[b] += std::norm(G[idx]);
    sn[b] += nn;
    cnt[b] += 1;
  }
  const double fac = std::pow(c->dx / (double)c->N, 3.0);
  const double L = c->N * c->dx, C = a * a * L * L * L / (2.0 * V * V) * fo2;
  const double a2p = std::pow(a, 2.0 * (1.0 - al));
  for (int b = 0; b < nb; ++b) {
    if (cnt[b] == 0) { k[b] = 0.0; df[b] = dfp[b] = n[b] = 0.0; mult[b] = 0; continue; }
    const double nbar = sn[b] / (double)cnt[b], kb = c->kIR * nbar;
    k[b] = kb;
    mult[b] = cnt[b];
    const double sh = kb * kb * kb / (2.0 * PI * PI) * fac / (4.0 * PI * nbar * nbar);
    df[b] = sh * s1[b];
    dfp[b] = sh * s1p[b];
    const double w2 = kb * kb + a * a * m2;
    if (!(w2 > 0.0)) { n[b] = std::nan(""); continue; }
    const double w = std::sqrt(w2);
    n[b] = 2.0 * C * (w * s1[b] / (double)cnt[b] + a2p * s2[b] / ((double)cnt[b] * w));
  }
  return 0;
}

}  // extern "C"

// ===========================================================================
// Discrete adjoint of the field evolution (gradient of a final observable),
// written from the forward map above for the scalar models.  The VV2 step is
// a sequence of elementary moves (vv2: field kick, scale-factor kick, drift,
// scale-factor kick, field kick); the adjoint
//   (lam_phi, lam_pi, lam_a, lam_b) = dJ/d(phi, pi, a, b)
// runs them backwards, each move applying its transposed Jacobian:
//   field kick (w at a, phi):  pi_f += w K_f,  K_f = a^{1+alpha} Lap phi_f/dx^2 - a^{3+alpha} dV/dphi_f
//      lam_phi_f += w [a^{1+alpha} Lap lam_pi_f/dx^2 - a^{3+alpha} sum_g V_{,fg} lam_pi_g]
//      lam_a     += w sum_n sum_f lam_pi_f dK_f/da
//      dJ/dq     += w sum_n sum_f lam_pi_f (-a^{3+alpha}) d(dV/dphi_f)/dq
//   scale-factor kick (w at a, phi, pi):  b += w K_a(a, phi, pi)
//      lam_a += w lam_b dK_a/da,  lam_phi += w lam_b dK_a/dphi,
//      lam_pi += w lam_b dK_a/dpi, dJ/dq += w lam_b dK_a/dq
//   drift (w from a, b):  a1 = a + w b,  phi_f += c pi_f,  c = w ((a + a1)/2)^{alpha-3}
//      lam_pi_f += c lam_phi_f
//      S = sum_n sum_f lam_phi_f pi_f,  c_abar = w (alpha-3) abar^{alpha-4}
//      lam_a <- lam_a1 + S c_abar,   lam_b <- lam_b + w lam_a1 + (w/2) S c_abar
// (Lap is symmetric, so it is its own transpose.)  With expansion off or on
// the fixed power law the scale factor is a known function of time: the
// scale-factor kicks are absent, lam_a and lam_b are not needed, and the
// drift coefficient c is a number.  The forward run records what each move
// read; nothing is recomputed.
// ===========================================================================
namespace {

// One recorded move of the VV2 step.
enum { MV_DRIFT = 0, MV_KICK = 1, MV_SCALE = 2 };
struct Move {
  int kind;
  double w;                    // move weight (the step fraction)
  double a, b;                 // a at the move (drift: before it), b at a drift
  double cd;                   // drift: coefficient of pi
  std::vector<double> phi[2];  // kicks: fields at the move
  std::vector<double> pi[2];   // scale-factor kicks and drifts: momenta at the move
};

// Hessian of the potential (eq. PotNat) at one site, and d(dV/dphi_f)/dq.
void pot_hessian(const clo_ctx* c, const double* f, double H[2][2], double* dq) {
  if (c->model == CLO_MODEL_LPHI4) {
    H[0][0] = 3.0 * f[0] * f[0];
    H[0][1] = H[1][0] = H[1][1] = 0.0;
    dq[0] = dq[1] = 0.0;
  } else {
    const double q = c->p.q;
    H[0][0] = 3.0 * f[0] * f[0] + q * f[1] * f[1];
    H[0][1] = H[1][0] = 2.0 * q * f[0] * f[1];
    H[1][1] = q * f[0] * f[0];
    dq[0] = f[0] * f[1] * f[1];
    dq[1] = f[0] * f[0] * f[1];
  }
}

// dV/dq at one site (eq. PotNat): phi^2 chi^2/2 for lphi4 + chi, 0 for lphi4.
double pot_dq(const clo_ctx* c, const double* f) {
  return c->model == CLO_MODEL_LPHI4_CHI ? 0.5 * f[0] * f[0] * f[1] * f[1] : 0.0;
}

double lap_at(const clo_ctx* c, const std::vector<double>& u, long n) {
  double s = 0.0;
  for (int i = 0; i < 3; ++i) s += u[c->shift(n, i, +1)] + u[c->shift(n, i, -1)] - 2.0 * u[n];
  return s;
}

// One VV2 step of size h (the moves of vv2), recorded.
void vv2_recorded(clo_ctx* c, double h, std::vector<Move>& moves) {
  const bool self = c->p.expansion == CLO_EXP_SELF;
  auto field_kick = [&](double w) {
    Move k;
    k.kind = MV_KICK;
    k.w = w;
    k.a = c->a;
    for (int f = 0; f < c->nf; ++f) k.phi[f] = c->phi[f];
    moves.push_back(std::move(k));
    kick_fields(c, w);
  };
  auto scale_kick = [&](double w) {
    if (!self) return;
    Move k;
    k.kind = MV_SCALE;
    k.w = w;
    k.a = c->a;
    for (int f = 0; f < c->nf; ++f) {
      k.phi[f] = c->phi[f];
      k.pi[f] = c->pi[f];
    }
    moves.push_back(std::move(k));
    kick_scale(c, w);
  };
  field_kick(0.5 * h);
  scale_kick(0.5 * h);
  {
    Move d;
    d.kind = MV_DRIFT;
    d.w = h;
    d.a = c->a;
    d.b = c->b;
    double a1 = c->a;
    if (self) a1 = c->a + h * c->b;
    else if (c->p.expansion == CLO_EXP_FIXED) a1 = a_fixed(c, c->eta + h);
    d.cd = h * std::pow(0.5 * (c->a + a1), c->alpha - 3.0);
    if (self)
      for (int f = 0; f < c->nf; ++f) d.pi[f] = c->pi[f];
    moves.push_back(std::move(d));
    drift(c, h);
  }
  scale_kick(0.5 * h);
  field_kick(0.5 * h);
}

// Objective J at the current state and its seeds dJ/dphi_f, dJ/dpi_f, dJ/da
// and explicit dJ/dq.  objective 0: chi energy fraction (E_K^chi + E_G^chi)/rho
// (lphi4 + chi).  objective 1: delta_b of the binned spectrum of (field, what)
// with bin width dk (as clo_spectrum).
bool objective_seed(clo_ctx* c, int objective, int field, int what, double dk, int bin, double* J,
                    std::vector<double>* lphi, std::vector<double>* lpi, double* dJdq, double* dJda) {
  const double V = (double)c->V;
  for (int f = 0; f < c->nf; ++f) {
    lphi[f].assign(c->V, 0.0);
    lpi[f].assign(c->V, 0.0);
  }
  *dJdq = 0.0;
  *dJda = 0.0;
  if (objective == 0) {
    if (c->model != CLO_MODEL_LPHI4_CHI) return false;
    Avg r;
    averages(c, r);
    const double rho = rho_of(r), a = c->a;
    const double a2 = a * a, a6 = a2 * a2 * a2;
    *J = (r.EK[1] + r.EG[1]) / rho;
    for (long n = 0; n < c->V; ++n) {
      double f[2] = {c->phi[0][n], c->phi[1][n]}, d[2];
      pot_deriv(c, f, d);
      for (int g = 0; g < 2; ++g) {
        const double num = g == 1 ? 1.0 : 0.0;
        const double dEK = c->pi[g][n] / (a6 * V);
        const double dEG = -lap_at(c, c->phi[g], n) / (a2 * c->dx * c->dx * V);
        lpi[g][n] = (num * dEK - *J * dEK) / rho;
        lphi[g][n] = (num * dEG - *J * (dEG + d[g] / V)) / rho;
      }
    }
    double s = 0.0;
    for (long n = 0; n < c->V; ++n) s += 0.5 * c->phi[0][n] * c->phi[0][n] * c->phi[1][n] * c->phi[1][n];
    *dJdq = -*J / rho * s / V;
    // E_K ~ a^-6 and E_G ~ a^-2 at fixed (phi, pi); E_V does not depend on a
    const double dnum = -(6.0 * r.EK[1] + 2.0 * r.EG[1]) / a;
    const double drho = -(6.0 * sum4(r.EK) + 2.0 * sum4(r.EG)) / a;
    *dJda = (dnum - *J * drho) / rho;
    return true;
  }
  if (objective == 1) {
    if (field < 0 || field >= c->nf || (what != 0 && what != 1) || !(dk > 0.0)) return false;
    const std::vector<double>& u = what == 0 ? c->phi[field] : c->pi[field];
    const int nb = (int)std::floor(std::sqrt(3.0) * (c->N / 2) / dk) + 1;
    if (bin < 0 || bin >= nb) return false;
    std::vector<cplx> F(c->V);
    for (long n = 0; n < c->V; ++n) F[n] = cplx(u[n], 0.0);
    fft3d(F, c->N, -1);
    double sp = 0.0, sn = 0.0;
    long cnt = 0;
    std::vector<cplx> M(c->V, cplx(0.0, 0.0));
    for (long idx = 1; idx < c->V; ++idx) {
      const double nn = mode_k(c, idx) / c->kIR;
      int b = (int)std::floor(nn / dk);
      if (b >= nb) b = nb - 1;
      if (b != bin) continue;
      sp += std::norm(F[idx]);
      sn += nn;
      ++cnt;
      M[idx] = F[idx];
    }
    if (cnt == 0) return false;
    const double nbar = sn / (double)cnt, kb = c->kIR * nbar;
    const double Cb = kb * kb * kb / (2.0 * PI * PI) * std::pow(c->dx / (double)c->N, 3.0) /
                      (4.0 * PI * nbar * nbar);
    *J = Cb * sp;
    fft3d(M, c->N, +1);
    std::vector<double>& out = what == 0 ? lphi[field] : lpi[field];
    for (long n = 0; n < c->V; ++n) out[n] = 2.0 * Cb * M[n].real();
    return true;
  }
  return false;
}

}  // namespace

extern "C" {

int clo_adjoint(clo_ctx* c, int nsteps, int objective, int field, int what, double dk, int bin,
                double* J, double* dJdq, double* lam, double* dJdab) {
  if (!c || nsteps < 0 || !J || !dJdq || !lam) return -1;
  if (c->gauge()) return -2;  // not built: see the header
  const bool self = c->p.expansion == CLO_EXP_SELF;
  // state at the start, restored at the end
  std::vector<double> phi0[2], pi0[2];
  for (int f = 0; f < c->nf; ++f) { phi0[f] = c->phi[f]; pi0[f] = c->pi[f]; }
  const double a0 = c->a, b0 = c->b, eta0 = c->eta;
  std::vector<double> d;
  schedule(c->p.integrator == CLO_LF ? 2 : c->p.integrator, c->p.dt, d);
  std::vector<Move> moves;
  for (int s = 0; s < nsteps; ++s)
    for (double h : d) vv2_recorded(c, h, moves);
  std::vector<double> lphi[2], lpi[2];
  double la = 0.0, lb = 0.0;
  const bool ok = objective_seed(c, objective, field, what, dk, bin, J, lphi, lpi, dJdq, &la);
  if (!self) la = 0.0;
  if (ok) {
    const double V = (double)c->V, al = c->alpha, idx2 = 1.0 / (c->dx * c->dx);
    const double C = c->p.fstar_over_mp * c->p.fstar_over_mp / 3.0;
    for (size_t m = moves.size(); m-- > 0;) {
      const Move& mv = moves[m];
      if (mv.kind == MV_DRIFT) {
        double S = 0.0;
        for (int f = 0; f < c->nf; ++f)
          for (long n = 0; n < c->V; ++n) {
            if (self) S += lphi[f][n] * mv.pi[f][n];
            lpi[f][n] += mv.cd * lphi[f][n];
          }
        if (self) {
          const double abar = mv.a + 0.5 * mv.w * mv.b;
          const double cab = mv.w * (al - 3.0) * std::pow(abar, al - 4.0);
          const double la1 = la;
          la = la1 + S * cab;
          lb = lb + mv.w * la1 + 0.5 * mv.w * S * cab;
        }
        continue;
      }
      if (mv.kind == MV_KICK) {
        const double a = mv.a;
        const double a1 = std::pow(a, 1.0 + al), a3 = std::pow(a, 3.0 + al);
        const double da1 = (1.0 + al) * std::pow(a, al), da3 = (3.0 + al) * std::pow(a, 2.0 + al);
        double dq = 0.0, sa = 0.0;
        for (long n = 0; n < c->V; ++n) {
          double f[2] = {0.0, 0.0}, H[2][2], g[2], dv[2] = {0.0, 0.0};
          for (int k = 0; k < c->nf; ++k) f[k] = mv.phi[k][n];
          pot_hessian(c, f, H, g);
          pot_deriv(c, f, dv);
          for (int k = 0; k < c->nf; ++k) {
            double hl = 0.0;
            for (int j = 0; j < c->nf; ++j) hl += H[k][j] * lpi[j][n];
            lphi[k][n] += mv.w * (a1 * lap_at(c, lpi[k], n) * idx2 - a3 * hl);
            dq += lpi[k][n] * g[k];
            if (self) sa += lpi[k][n] * (da1 * lap_at(c, mv.phi[k], n) * idx2 - da3 * dv[k]);
          }
        }
        *dJdq += mv.w * (-a3) * dq;
        if (self) la += mv.w * sa;
        continue;
      }
      // scale-factor kick: K_a = C a^{2 alpha+1} [(alpha-2) E_K + alpha E_G + (alpha+1) E_V]
      // with E_K = sum pi^2/(2 a^6 V), E_G = sum (grad^+ phi)^2/(2 a^2 dx^2 V), E_V = sum V/V
      const double a = mv.a, wl = mv.w * lb;
      double EK = 0.0, EG = 0.0, EV = 0.0, Vq = 0.0;
      for (long n = 0; n < c->V; ++n) {
        double f[2] = {0.0, 0.0}, t[4] = {0.0, 0.0, 0.0, 0.0};
        for (int k = 0; k < c->nf; ++k) {
          f[k] = mv.phi[k][n];
          EK += mv.pi[k][n] * mv.pi[k][n];
          for (int i = 0; i < 3; ++i) {
            const double gr = mv.phi[k][c->shift(n, i, +1)] - mv.phi[k][n];
            EG += gr * gr;
          }
        }
        pot_terms(c, f, t);
        for (int k = 0; k < n_pot_terms(c->model); ++k) EV += t[k];
        Vq += pot_dq(c, f);
      }
      const double a2 = a * a, a6 = a2 * a2 * a2;
      EK /= 2.0 * a6 * V;
      EG /= 2.0 * a2 * c->dx * c->dx * V;
      EV /= V;
      const double p1 = C * std::pow(a, 2.0 * al + 1.0);
      // d/da at fixed (phi, pi): a^{2 alpha+1} E_K ~ a^{2 alpha-5}, a^{2 alpha+1} E_G ~ a^{2 alpha-1}
      const double dKa = C * std::pow(a, 2.0 * al) *
                         ((2.0 * al - 5.0) * (al - 2.0) * EK + (2.0 * al - 1.0) * al * EG +
                          (2.0 * al + 1.0) * (al + 1.0) * EV);
      la += wl * dKa;
      *dJdq += wl * p1 * (al + 1.0) * Vq / V;
      for (long n = 0; n < c->V; ++n) {
        double f[2] = {0.0, 0.0}, dv[2] = {0.0, 0.0};
        for (int k = 0; k < c->nf; ++k) f[k] = mv.phi[k][n];
        pot_deriv(c, f, dv);
        for (int k = 0; k < c->nf; ++k) {
          // dE_G/dphi(n) = -Lap phi(n)/(a^2 dx^2 V), dE_V/dphi = V_{,phi}/V, dE_K/dpi = pi/(a^6 V)
          const double dEG = -lap_at(c, mv.phi[k], n) * idx2 / (a2 * V);
          lphi[k][n] += wl * p1 * (al * dEG + (al + 1.0) * dv[k] / V);
          lpi[k][n] += wl * p1 * (al - 2.0) * mv.pi[k][n] / (a6 * V);
        }
      }
    }
    for (int f = 0; f < c->nf; ++f) {
      std::memcpy(lam + (size_t)(2 * f) * c->V, lphi[f].data(), sizeof(double) * c->V);
      std::memcpy(lam + (size_t)(2 * f + 1) * c->V, lpi[f].data(), sizeof(double) * c->V);
    }
    if (dJdab) {
      dJdab[0] = la;
      dJdab[1] = lb;
    }
  }
  for (int f = 0; f < c->nf; ++f) { c->phi[f] = phi0[f]; c->pi[f] = pi0[f]; }
  c->a = a0; c->b = b0; c->eta = eta0;
  return ok ? 0 : -1;
}

// Gradient with respect to the drawn mode amplitudes |z1|, |z2| (Sec. 3.5.1):
// with phi(x) = phi0 + (1/V) sum_n F(n) e^{+i k.x}, F = (z1 + z2)/sqrt2 and
// pi(x) = a^{3-alpha} [phi0' + (1/V) sum_n G(n) e^{+i k.x}],
// G = a^{alpha-1} i omega (z1 - z2)/sqrt2 - H F, a canonical mode n and its
// conjugate partner contribute (s/V) Re[dF/d|z_j| e^{i k.x}] (s = 2; s = 1 for
// self-conjugate sites), so
//   dJ/d|z_j| = (s/V) Re[ e^{i th_j}/sqrt2 L_phi(n)
//                 + a^{3-alpha} (+-a^{alpha-1} i omega - H) e^{i th_j}/sqrt2 L_pi(n) ],
// L(n) = sum_x lam(x) e^{+i k.x}.  out[(2f + j) V + n] at canonical n, 0 elsewhere.
// With self-consistent expansion the initial b must not move with the
// amplitudes (b0_mode 0: a' from the homogeneous values); b0_mode 1 is refused.
int clo_ic_amplitude_grad(const clo_ctx* c, const double* lam, double* out) {
  if (!c || !lam || !out || c->gauge()) return -1;
  if (c->p.expansion == CLO_EXP_SELF && c->p.b0_mode == 1) return -2;
  const double V = (double)c->V, isq2 = 1.0 / std::sqrt(2.0);
  const double a = c->a0, a3ma = std::pow(a, 3.0 - c->alpha), aam1 = std::pow(a, c->alpha - 1.0);
  std::memset(out, 0, sizeof(double) * 2 * c->nf * c->V);
  std::vector<cplx> L[2][2];
  for (int f = 0; f < c->nf; ++f)
    for (int w = 0; w < 2; ++w) {
      L[f][w].resize(c->V);
      for (long n = 0; n < c->V; ++n) L[f][w][n] = cplx(lam[(size_t)(2 * f + w) * c->V + n], 0.0);
      fft3d(L[f][w], c->N, +1);
    }
  clo_ctx t = *c;  // draws at the initial scale factor
  t.a = c->a0;
  for (long idx = 1; idx < c->V; ++idx) {
    const long pid = partner_index(c, idx);
    if (pid < idx) continue;
    cplx z1[2], z2[2];
    double om[2];
    if (!mode_draws(&t, c->seed, idx, z1, z2, om)) continue;
    const double s = pid == idx ? 1.0 : 2.0;
    for (int f = 0; f < c->nf; ++f)
      for (int j = 0; j < 2; ++j) {
        const cplx e = std::polar(1.0, std::arg(j == 0 ? z1[f] : z2[f])) * isq2;
        const double sg = j == 0 ? 1.0 : -1.0;
        const cplx cpi = a3ma * (sg * aam1 * cplx(0.0, om[f]) - c->H_ic) * e;
        out[(size_t)(2 * f + j) * c->V + idx] = s / V * (e * L[f][0][idx] + cpi * L[f][1][idx]).real();
      }
  }
  return 0;
}

// Doublet models: the momentum kernel K (pi' = K, the rate of one kick per unit
// step weight) of momentum array `a` (clo_get_array order: 4..7, 11..13,
// 26..34, and for the full model 36, 39, 40) at the current state.
int clo_kernel(const clo_ctx* c, int a, double* out) {
  if (!c || !out || !c->su2()) return -1;
  const bool ok = (a >= 4 && a < 8) || (a >= 11 && a < 14) || (a >= 26 && a < 35) ||
                  (c->full() && (a == 36 || a == 39 || a == 40));
  if (!ok) return -1;
  std::vector<double> Kp[4], KA[3], KB[3][3], Ks, Kc[2];
  for (int k = 0; k < 4; ++k) Kp[k].assign(c->V, 0.0);
  for (int i = 0; i < 3; ++i) {
    KA[i].assign(c->V, 0.0);
    for (int b = 0; b < 3; ++b) KB[i][b].assign(c->V, 0.0);
  }
  kernel_su2(c, Kp, KA, KB);
  if (c->full()) {
    Ks.assign(c->V, 0.0);
    for (int k = 0; k < 2; ++k) Kc[k].assign(c->V, 0.0);
    kernel_full_extra(c, Ks, Kc, KA);
  }
  const std::vector<double>* src;
  if (a < 8) src = &Kp[a - 4];
  else if (a < 14) src = &KA[a - 11];
  else if (a < 35) src = &KB[(a - 26) / 3][(a - 26) % 3];
  else if (a == 36) src = &Ks;
  else src = &Kc[a - 39];
  std::memcpy(out, src->data(), sizeof(double) * c->V);
  return 0;
}

// U(1) model: the Fourier values of the Gauss-law link momenta (the initial
// conditions' inversion, eq. GaugeCurrentFluc on the lattice) of the context's
// current charged field, at Fourier sites idx[i]: out[(3 i + dir) 2 + {0, 1}] =
// Re, Im of pi_A,dir (unnormalised forward transform, like the state's FFT).
int clo_gauss_modes(const clo_ctx* c, int n, const int64_t* idx, double* out) {
  if (!c || c->model != CLO_MODEL_U1_HIGGS || n < 0 || (n > 0 && (!idx || !out))) return -1;
  std::vector<cplx> rho;
  u1_charge_density(c, rho);
  fft3d(rho, c->N, -1);
  for (int i = 0; i < n; ++i) {
    if (idx[i] < 0 || idx[i] >= c->V) return -1;
    for (int d = 0; d < 3; ++d) {
      cplx e = gauss_mode(c, rho, (long)idx[i], d);
      out[(3 * (size_t)i + d) * 2] = e.real();
      out[(3 * (size_t)i + d) * 2 + 1] = e.imag();
    }
  }
  return 0;
}

// The oracle's draw pair of the initial conditions (draw4) for element i:
// Fourier index idx[i], component f[i], draw j[i], seed `seed`.
int clo_draw_pairs(uint64_t seed, int n, const int64_t* idx, const int* f, const int* j, double* out) {
  if (n < 0 || (n > 0 && (!idx || !f || !j || !out))) return -1;
  for (int i = 0; i < n; ++i) draw4(seed, (long)idx[i], f[i], j[i], out + 2 * (size_t)i);
  return 0;
}

// Drawn amplitudes of canonical sites: out[(i nf + f) 5 + {0..4}] = |z1|, arg z1,
// |z2|, arg z2, omega_k (zeros for sites that stay zero).
int clo_ic_draws(int model, int N, double kIR, double alpha, uint64_t seed, const clo_params* p, int n,
                 const int64_t* idx, double* out) {
  if (!p || !idx || !out || model < CLO_MODEL_LPHI4 || model > CLO_MODEL_U1_HIGGS) return -1;
  clo_ctx c;
  c.model = model;
  c.N = N;
  c.V = (long)N * N * N;
  c.nf = model == CLO_MODEL_LPHI4 ? 1 : 2;
  c.kIR = kIR;
  c.dx = 2.0 * PI / ((double)N * kIR);
  c.alpha = alpha;
  c.p = *p;
  c.a = c.a0 = 1.0;
  for (int i = 0; i < n; ++i) {
    cplx z1[2], z2[2];
    double om[2];
    const bool ok = idx[i] >= 0 && idx[i] < c.V && mode_draws(&c, seed, (long)idx[i], z1, z2, om);
    for (int f = 0; f < c.nf; ++f) {
      double* o = out + ((size_t)i * c.nf + f) * 5;
      o[0] = ok ? std::abs(z1[f]) : 0.0;
      o[1] = ok ? std::arg(z1[f]) : 0.0;
      o[2] = ok ? std::abs(z2[f]) : 0.0;
      o[3] = ok ? std::arg(z2[f]) : 0.0;
      o[4] = ok ? om[f] : 0.0;
    }
  }
  return 0;
}

}  // extern "C"
