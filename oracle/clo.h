/*
 * clo.h -- C interface of the FP64 CPU oracle for the lattice kick-drift method
 * of the CosmoLattice manual (arXiv:2102.01031).
 *
 * TEST INFRASTRUCTURE ONLY.  This oracle is a plain, slow, unfused, single
 * threaded FP64 restatement of the method, written to be checked by eye
 * against the paper.  Only tests/, __graft_entry__.smoke() and bench.py's
 * cpu_baseline / reference arm may load it.  It shares no code with the CUDA
 * library (paper_2102_01031_gb300/csrc, include/cl.h) and must never be used
 * as a fallback for it.
 *
 * Notation: f_s, omega_s are the manual's f_* and omega_*.
 * Conventions (all quantities in program variables, Sec. 3.1 eq.
 * FieldSpaceTimeNaturalVariables and Sec. 4.1 eq. GaugeProgramVar):
 *   - lattice site n = (x,y,z), linear index x + N*(y + N*z), periodic;
 *   - dx = 2*pi/(N*kIR) (Sec. 2.2 "Basic lattice definitions");
 *   - DFT: forward sum_n f(n) e^{-2 pi i n.k/N}, inverse with 1/N^3 and e^{+...}
 *     (the manual's two printed sign conventions conflict; this one is used);
 *   - scalar models: field f in [0, nf); U(1) model: f = 0,1 are the real
 *     components phi_0, phi_1 of phi = (phi_0 + i phi_1)/sqrt(2) and
 *     f = 2,3,4 are the link fields A_x, A_y, A_z (non-compact storage);
 *   - SU(2) x U(1) doublet model: f = 0..3 are the real components of
 *     Phi = (phi_0 + i phi_1, phi_2 + i phi_3)/sqrt(2), f = 4,5,6 the U(1)
 *     link fields A_i; the SU(2) links and their momenta are reached through
 *     clo_get_array / clo_set_array (array order below);
 *   - lphi4SU2U1 model (Sec. 4.5: the doublet, a singlet phi_s and a U(1)-charged
 *     scalar vphi = (vphi_0 + i vphi_1)/sqrt(2), eq. PotGauge): f = 0..6 as the
 *     doublet model, f = 7 the singlet, f = 8, 9 the components of vphi.
 *
 * Every function returns 0 on success and a negative code on error.
 */
#ifndef CLO_H
#define CLO_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum { CLO_MODEL_LPHI4 = 1, CLO_MODEL_LPHI4_CHI = 2, CLO_MODEL_U1_HIGGS = 3, CLO_MODEL_SU2U1_HIGGS = 4,
       CLO_MODEL_LPHI4_SU2U1 = 5 };
enum { CLO_LF = 0, CLO_VV2 = 2, CLO_VV4 = 4, CLO_VV6 = 6, CLO_VV8 = 8, CLO_VV10 = 10 };
enum { CLO_EXP_OFF = 0, CLO_EXP_SELF = 1, CLO_EXP_FIXED = 2 };

typedef struct {
  double dt;                    /* time step (program units) */
  double q;                     /* resonance parameter g^2/lambda (lphi4 + chi) */
  double fluct_amp2;            /* (omega_s/f_s)^2 in the vacuum amplitude, eq. QuantumFlucts2 */
  double fstar_over_mp;         /* f_s/m_p in the Friedmann equations */
  double phi0[4];               /* homogeneous initial field values */
  double dphi0[4];              /* homogeneous initial derivatives phi' */
  double lam, v;                /* gauge models: V = lam (|phi|^2 - v^2)^2 */
  double gQ;                    /* U(1) gauge coupling times charge (g_A Q_A) */
  double fstar_over_omegastar;  /* f_s/omega_s (gauge models) */
  double kcut;                  /* initial-spectrum cutoff; < 0 means none */
  double omega_eos;             /* fixed background: equation of state w */
  double H0;                    /* fixed background: initial a'/a; <= 0 -> from Hubble law */
  int integrator;               /* CLO_LF, CLO_VV2 ... CLO_VV10 */
  int expansion;                /* CLO_EXP_OFF / SELF / FIXED */
  int b0_mode;                  /* 0: a' from homogeneous values; 1: from lattice averages */
  int pad_;
  double gQB;                   /* SU(2) gauge coupling times charge (g_B Q_B), doublet model */
  double qG, qH;                /* lphi4SU2U1: q_G = g^2/lambda, q_H = h^2/lambda of eq. PotGauge */
  double Qc;                    /* lphi4SU2U1: U(1) charge of the charged scalar in units of the doublet's */
} clo_params;

typedef struct {
  double eta, a, b;             /* time, scale factor, b = a' */
  double EK[4], EG[4];          /* kinetic / gradient energy per scalar species */
  double EV[4];                 /* potential energy per potential term */
  double EKA, EGA;              /* U(1) electric and magnetic energies */
  double rho;                   /* total energy density (program units) */
  double hubble_lhs, hubble_rhs, hubble_viol; /* a'^2, RHS of eq. NewFriedmannEQsI, (L-R)/(L+R) */
  double energy_cons;           /* 1 - rho/rho(t0) */
  double mean_phi[4], mean_phi2[4], mean_pi[4], mean_pi2[4];
  double EKB, EGB;              /* SU(2) electric and magnetic energies (doublet model) */
} clo_energies_t;

typedef struct clo_ctx clo_ctx;

int clo_init(clo_ctx** out, int model, int N, double kIR, double alpha,
             uint64_t seed, const clo_params* p);
int clo_free(clo_ctx* c);
int clo_step(clo_ctx* c, int n);
int clo_step_h(clo_ctx* c, int n, double h);      /* n steps with an explicit step size */
int clo_energies(clo_ctx* c, clo_energies_t* out);
int clo_get_state(const clo_ctx* c, int field, int what, double* out);
int clo_set_state(clo_ctx* c, int field, int what, const double* in);
int clo_get_scalars(const clo_ctx* c, double* eta, double* a, double* b);
int clo_set_scalars(clo_ctx* c, double eta, double a, double b);
int clo_nfields(const clo_ctx* c);
int clo_gauss_constraint(const clo_ctx* c, double* rel, double* lhs_abs, double* rhs_abs,
                         double* max_abs);
int clo_spectrum(const clo_ctx* c, int field, int what, double dk_bin, double* k,
                 double* delta, int64_t* mult, int cap, int* nbins);
/* Gauge models: binned spectrum of the U(1) electric (which = 0: E_i = a^{alpha-1} pi_A,i)
 * or magnetic (which = 1: B_i = eps_ijk sin(theta_jk)/(2 gQ dx^2)) field; doublet model
 * also the SU(2) electric (2: E_i^a = a^{alpha-1} pi_B,i^a) or magnetic (3: B_i^a from
 * G_jk^a = Tr[(i s_a/2)(U_jk - U_jk^dag)]/(gQB dx^2)) field; |.|^2 summed over
 * components, normalised as clo_spectrum.  -1 for scalar models (and which = 1 with gQ = 0). */
int clo_em_spectrum(const clo_ctx* c, int which, double dk_bin, double* k, double* delta, int64_t* mult,
                    int cap, int* nbins);
/* Lattice occupation number n_b of scalar field `field` per spectrum bin
 * (eq. OccuppationNum); fo2 = (f_s/omega_s)^2, the square of the field and frequency
 * scales of the program units.  k and mult as clo_spectrum;
 * NaN where omega_b^2 <= 0.  -1 for U(1) or bad arguments, -2 if cap < nbins. */
int clo_occupation(const clo_ctx* c, int field, double dk_bin, double fo2, double* k, double* n,
                   int64_t* mult, int cap, int* nbins);
/* SU(2) x U(1) doublet model: whole arrays in the order
 *   0..3 phi_c, 4..7 pi_c, 8..10 A_i, 11..13 pi_A,i,
 *   14 + 4 i + k: component u_k of the SU(2) link U_i = u0 - i (u1 s1 + u2 s2 + u3 s3),
 *   26 + 3 i + (a - 1): link momentum pi_B,i^a;
 * lphi4SU2U1 model: the same, then 35 phi_s, 36 pi_s, 37, 38 vphi_c, 39, 40 pi_vphi,c.
 * -1 for other models or a bad index. */
int clo_get_array(const clo_ctx* c, int a, double* out);
int clo_set_array(clo_ctx* c, int a, const double* in);
/* Doublet models: the momentum kernel K (pi' = K) of momentum array a (the
 * array order above) at the current state; -1 for other models or arrays. */
int clo_kernel(const clo_ctx* c, int a, double* out);
/* Gauss-law residual per site of generator g (0: the U(1) law; 1..3: the SU(2)
 * colour a = g, doublet model only): out[n] = (lattice divergence of the
 * electric field) - (charge density); -1 where the model has no such law. */
int clo_gauss_residual(const clo_ctx* c, int g, double* out);
/* exp(-i theta.sigma/2) as (u0, u1, u2, u3) in the link convention above. */
void clo_su2_exp(const double theta[3], double u[4]);
/* Gauge models: spectra of the modulus r = |phi| = sqrt(sum_c phi_c^2/2) of the charged
 * field (U(1) field or doublet) and of r' = sum_c phi_c phi_c'/(2 r), and the occupation
 * number of the canonical modulus rho = sqrt2 r (eq. OccuppationNum with
 * w^2 = k^2 + a^2 <V''(r)/2>, V = lam (r^2 - v^2)^2), on clo_spectrum's shells;
 * fo2 = (f_s/omega_s)^2.  -1 for scalar models, -2 if cap < nbins. */
int clo_norm_spectrum(const clo_ctx* c, double dk_bin, double fo2, double* k, double* df, double* dfp,
                      double* n, int64_t* mult, int cap, int* nbins);
/* which = 0: the model's charged field (as clo_norm_spectrum; the doublet of
 * lphi4SU2U1 with the mass q_G phi_s^2 + 2 q_H |vphi|^2 added); which = 1: the
 * U(1)-charged scalar vphi of lphi4SU2U1 (mass 2 q_H |Phi|^2).  -1 otherwise. */
int clo_norm_spectrum_of(const clo_ctx* c, int which, double dk_bin, double fo2, double* k, double* df,
                         double* dfp, double* n, int64_t* mult, int cap, int* nbins);
int clo_ic_sample(int model, int N, double kIR, double alpha, uint64_t seed, const clo_params* p,
                  int n, const int64_t* idx, double* out);

/* Discrete adjoint (scalar models; -2 for U(1)): from the current state, run
 * nsteps, evaluate the objective (0: chi energy fraction; 1: spectrum bin
 * `bin` of (field, what) with width dk), and return J, dJ/dq at a fixed
 * initial state (phi, pi, a, b), lam[(2f + w) V + n] = dJ/d(field f, what w)(n)
 * at the initial state, and, if dJdab is not NULL, dJdab[0..1] = dJ/da, dJ/db
 * at the initial state (zero unless the expansion is self-consistent).  The
 * state is restored. */
int clo_adjoint(clo_ctx* c, int nsteps, int objective, int field, int what, double dk, int bin,
                double* J, double* dJdq, double* lam, double* dJdab);
/* Chain lam (as above, at the initial conditions) to dJ/d|z_j| of each canonical
 * mode: out[(2f + j) V + n], j = 0, 1.  -2 with self-consistent expansion and
 * b0_mode 1 (the initial b then depends on the amplitudes). */
int clo_ic_amplitude_grad(const clo_ctx* c, const double* lam, double* out);
int clo_ic_draws(int model, int N, double kIR, double alpha, uint64_t seed, const clo_params* p, int n,
                 const int64_t* idx, double* out);

/* pieces exposed for the pin tests */
void clo_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);
double clo_u01(uint32_t hi, uint32_t lo);
int clo_gauss_modes(const clo_ctx* c, int n, const int64_t* idx, double* out); /* U(1) IC link momenta, Fourier */
int clo_draw_pairs(uint64_t seed, int n, const int64_t* idx, const int* f, const int* j,
                   double* out);  /* the IC draw pairs (u1, u2) */
int clo_fft3d(double* re, double* im, int N, int sign);      /* in place, unnormalised */
int clo_dft3d_naive(const double* re, const double* im, double* ore, double* oim, int N, int sign);
int clo_schedule(int integrator, double h, double* drifts, int cap);

#ifdef __cplusplus
}
#endif
#endif
