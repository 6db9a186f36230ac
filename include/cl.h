/*
 * cl.h -- C ABI of the GB300 (sm_103a) lattice kick-drift library.
 *
 * The library evolves interacting scalar fields, and U(1) gauge links, on a
 * periodic N^3 lattice in an expanding background, as described in the
 * CosmoLattice manual (arXiv:2102.01031): the Hamiltonian form of the field
 * and Friedmann equations in program variables (Sec. 3.5.2 for singlets,
 * Sec. 4.3 for the U(1) sector), advanced by velocity-Verlet / leapfrog
 * kick-drift steps and their symmetric compositions (VV4..VV10, Sec. 3.3.1
 * "evolver"), with vacuum-fluctuation initial conditions (Sec. 3.5.1 eqs.
 * fpr_influct, fpr_influct2, QuantumFlucts2; Sec. 4.4.1 for charged fields)
 * and the binned power spectrum of eq. discretePS.
 *
 * Conventions shared by every entry point
 *   - Status codes only (cl_status); nothing aborts or traps.  A failed call
 *     leaves a message retrievable with cl_last_error(ctx).
 *   - All device memory is owned by the context: allocated by cl_init,
 *     released by cl_free; the one exception is state memory the caller
 *     binds with cl_bind_buffers.  Host arrays passed in or out are owned by
 *     the caller and must hold the stated number of elements.
 *   - The state and gradient transfers (cl_get_state, cl_set_state and their
 *     cl_lattice_ forms, cl_get_array, cl_set_array, cl_upload_state,
 *     cl_download_state, cl_adjoint's dJ_dstate, cl_ic_amplitude_grad) also
 *     take device pointers (any address the CUDA runtime resolves through
 *     unified addressing, e.g. a torch CUDA tensor's data): the copy then
 *     stays on the GPU.  It is ordered on params.stream, so whatever writes a
 *     device input must be ordered before the call on that stream.
 *   - Lattice arrays are N^3 values, row major with x fastest: site
 *     (x, y, z) is element x + N*(y + N*z).
 *   - Field indices: scalar models: 0 .. nf-1 (phi, chi).  U(1) model:
 *     0, 1 = real components phi_0, phi_1 of phi = (phi_0 + i phi_1)/sqrt(2),
 *     2, 3, 4 = link fields A_x, A_y, A_z (stored non-compactly, the link is
 *     exp(-i gQ dx A_i)).  `what`: 0 = field, 1 = conjugate momentum
 *     (pi = a^{3-alpha} phi' for scalars, pi_A = a^{1-alpha} F_0i for links).
 *   - Work is enqueued on params.stream (a cudaStream_t, e.g. the current
 *     torch stream; NULL = legacy default stream).  cl_step only enqueues;
 *     every call that returns data to the host synchronises that stream.
 *   - Momenta run half a kick ahead of the fields between cl_step calls (the
 *     kicks of consecutive steps are merged); calls that observe the state
 *     first close the stream of kicks with a half kick (the manual's `sync`,
 *     Sec. 5.1), after which fields and momenta are at the same time.
 *   - One context is used by one host thread at a time.
 *   - A context holds one lattice (cl_init) or an ensemble of lattices
 *     (cl_ensemble_init); calls without a lattice argument act on lattice 0,
 *     except cl_step / cl_step_h / cl_sync / cl_set_scalars, which act on all.
 */
#ifndef CL_H
#define CL_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct cl_ctx cl_ctx;

typedef enum {
  CL_OK = 0,
  CL_EINVAL = 1,        /* bad argument */
  CL_ENOMEM = 2,        /* device allocation failed */
  CL_ECUDA = 3,         /* CUDA runtime error (message in cl_last_error) */
  CL_ESTATE = 4,        /* call not valid in the context's current state */
  CL_ETIMEOUT = 5,      /* a bounded device-side wait gave up; context unusable */
  CL_ENONFINITE = 6,    /* a measured quantity was NaN/Inf; data still returned */
  CL_EUNSUPPORTED = 7   /* combination of options not built */
} cl_status;

enum { CL_MODEL_LPHI4 = 1,      /* V = phi^4/4                              (eq. PotNat, chi = 0) */
       CL_MODEL_LPHI4_CHI = 2,  /* V = phi^4/4 + (q/2) phi^2 chi^2          (eq. PotNat) */
       CL_MODEL_U1_HIGGS = 3,   /* V = lam (|phi|^2 - v^2)^2 + U(1) links    (Sec. 4) */
       CL_MODEL_SU2U1_HIGGS = 4,   /* doublet Phi, V = lam (|Phi|^2 - v^2)^2, U(1) and SU(2)
                                      links: the gauge content of the lphi4SU2U1 example (Sec. 4) */
       CL_MODEL_LPHI4_SU2U1 = 5 }; /* the lphi4SU2U1 example (Sec. 4.5): the doublet and both gauge
                                      fields, a singlet phi_s and a U(1)-charged scalar vphi,
                                      V = lam (|Phi|^2 - v^2)^2 + qG |Phi|^2 phi_s^2
                                          + 2 qH |Phi|^2 |vphi|^2  (eq. PotGauge, lam = 1, v = 0) */

enum { CL_LF = 0, CL_VV2 = 2, CL_VV4 = 4, CL_VV6 = 6, CL_VV8 = 8, CL_VV10 = 10 };
enum { CL_FP64 = 0,             /* fields, momenta and arithmetic in FP64 */
       CL_FP32 = 1 };           /* fields and momenta stored and updated in FP32;
                                   reductions, a, b and constraints in FP64 */
enum { CL_EXP_OFF = 0, CL_EXP_SELF = 1, CL_EXP_FIXED = 2 };

/* Run parameters (subset of the manual's RunParameters and model variables,
 * Appendix "Parameters"; all in program units).  f_s, omega_s below are the
 * manual's f_* and omega_*. */
typedef struct {
  double dt;                    /* time step */
  double q;                     /* resonance parameter g^2/lambda (CL_MODEL_LPHI4_CHI) */
  double fluct_amp2;            /* (omega_s/f_s)^2 in eq. QuantumFlucts2; 0 = no fluctuations */
  double fstar_over_mp;         /* f_s/m_p in the Friedmann equations */
  double phi0[4];               /* homogeneous initial values (per field / component) */
  double dphi0[4];              /* homogeneous initial phi' */
  double lam, v;                /* gauge models: potential lam (|phi|^2 - v^2)^2 */
  double gQ;                    /* U(1) coupling times charge (g_A Q_A); doublet model: 0 = no U(1) field */
  double fstar_over_omegastar;  /* f_s/omega_s (gauge models) */
  double kcut;                  /* initial-spectrum cutoff (eq. kCutOff); < 0 = none */
  double omega_eos;             /* fixed background: equation of state w */
  double H0;                    /* fixed background: initial a'/a; <= 0 -> Hubble law */
  int integrator;               /* CL_LF, CL_VV2, CL_VV4 .. CL_VV10 */
  int expansion;                /* CL_EXP_OFF, CL_EXP_SELF, CL_EXP_FIXED */
  int b0_mode;                  /* 0: a'(t0) from homogeneous values (Sec. 5.2); 1: from averages */
  int precision;                /* CL_FP64 or CL_FP32 */
  void* stream;                 /* cudaStream_t */
  int autotune;                 /* nonzero: pick each lattice size's tile height by timing
                                   candidates on the device (cached per model, precision, N) */
  int tile_by;                  /* > 0: force this tile height (rows per CTA tile) for every
                                   lattice; 0: autotune or the built-in choice */
  double gQB;                   /* SU(2) coupling times charge (g_B Q_B), CL_MODEL_SU2U1_HIGGS */
  double qG, qH;                /* CL_MODEL_LPHI4_SU2U1: q_G = g^2/lambda, q_H = h^2/lambda (eq. PotGauge) */
  double Qc;                    /* CL_MODEL_LPHI4_SU2U1: U(1) charge of vphi in units of the doublet's
                                   (vphi hops with exp(-i Qc gQ dx A_i)); the singlet and vphi start
                                   with zero homogeneous values and vacuum fluctuations */
} cl_params;

/* Volume averages at a synchronised time (eqs. EK_EG_EV, energy-contrib). */
typedef struct {
  double eta, a, b;             /* time, scale factor, b = a' */
  double EK[4], EG[4];          /* kinetic / gradient energy per scalar species */
  double EV[4];                 /* potential energy per potential term */
  double EKA, EGA;              /* U(1) electric / magnetic energy */
  double rho;                   /* total energy density */
  double hubble_lhs, hubble_rhs, hubble_viol; /* a'^2, RHS of eq. NewFriedmannEQsI, (L-R)/(L+R) */
  double energy_cons;           /* 1 - rho/rho(t0) (meaningful without expansion) */
  double mean_phi[4], mean_phi2[4], mean_pi[4], mean_pi2[4];
  int64_t nonfinite;            /* number of non-finite momenta seen in the last measurement */
  double EKB, EGB;              /* SU(2) electric / magnetic energy (doublet model) */
} cl_energies_t;

/* Create a lattice of N^3 sites with kIR (so dx = 2 pi/(N kIR)), alpha of
 * eq. FieldSpaceTimeNaturalVariables, and vacuum fluctuations drawn from
 * `seed` (Sec. 3.5.1), all generated on the GPU.  N must be a multiple of 8,
 * at most 512, with no prime factor above 3.  Returns CL_EINVAL for bad
 * arguments, CL_ENOMEM / CL_ECUDA on device failure (*out is then NULL). */
cl_status cl_init(cl_ctx** out, int model, int N, double kIR, double alpha, uint64_t seed,
                  const cl_params* p);
cl_status cl_free(cl_ctx* ctx);

/* Enqueue n full time steps of params.dt (n >= 0); cl_step_h uses step h
 * (negative h runs the integrator backwards).  Asynchronous. */
cl_status cl_step(cl_ctx* ctx, int n);
cl_status cl_step_h(cl_ctx* ctx, int n, double h);

/* The kick and drift weights of the fused passes that cl_step_h launches (host
 * arithmetic only; needs no GPU and no context).  Each step is the integrator's
 * symmetric composition of Stoermer-Verlet substeps (Sec. 5.1; VV4..VV10 as
 * the triple-jump compositions of Yoshida 1990), every substep d a kick d/2, a
 * drift d and a kick d/2; a pass applies the kick-out of the previous substep,
 * the kick-in of the next and the next drift, so one pass per substep.  For
 * ncalls successive cl_step_h calls of steps_per_call[i] steps of size h on a
 * stream that starts closed, followed by the closing half kick (cl_sync or a
 * measurement), out receives 4 doubles per pass, in order:
 *   ck = wout + win (the total kick weight), wout (kick-out of the previous
 *   drift), win (kick-in of the next drift), dnext (that drift).
 * *npass receives the pass count; CL_EINVAL if it exceeds cap, or for an
 * unknown integrator, a negative count, more than 2^20 steps per call or a
 * non-finite h. */
cl_status cl_pass_weights(int integrator, double h, int ncalls, const int* steps_per_call, double* out, int cap,
                          int* npass);

/* Close the stream of kicks so that fields and momenta are at the same time
 * (the manual's `sync`).  Asynchronous; a no-op when already closed. */
cl_status cl_sync(cl_ctx* ctx);

/* Energies and means at the current (synchronised) time.  Synchronises the
 * stream.  Returns CL_ENONFINITE (with *out filled) if non-finite momenta were
 * seen. */
cl_status cl_energies(cl_ctx* ctx, cl_energies_t* out);

/* U(1) Gauss-law monitor (Sec. 4.5, average_gauss): LHS = sum_i grad^-_i pi_A,i,
 * RHS = (f_s/omega_s)^2 2 gQ Im[phi^* pi_phi]; rel = <|L-R|>/<|L+R|>.
 * Doublet model: the sums run over the U(1) law and the three SU(2) laws
 *   sum_i [pi_B,i^a(n) - (U_i^dag(n-i) pi_B,i(n-i) U_i(n-i))^a]/dx
 *     = (f_s/omega_s)^2 (gQB/2) Im[psi^dag sigma_a pi_psi],   psi = sqrt2 Phi,
 * with pi_B = pi_B^b sigma_b/2 and X^a = Tr[sigma_a X] (SU(N) toolkit,
 * eq. GaussSU2-eom on the lattice).
 * CL_EUNSUPPORTED for models without links.  Synchronises the stream. */
cl_status cl_gauss_constraint(cl_ctx* ctx, double* rel, double* lhs_abs, double* rhs_abs,
                              double* max_abs);

/* Binned power spectrum of eq. discretePS of field `field`, what = 0 (field)
 * or 1 (momentum), with bin width dk_bin in units of kIR: bins b =
 * floor(|n~|/dk_bin) over n~ != 0, k_b = kIR <|n~|>_b, delta_b =
 * k_b^3/(2 pi^2) (dx/N)^3 sum_b |f(n~)|^2 / (4 pi <|n~|>_b^2), mult_b = sites in
 * the bin.  Arrays k, delta, mult hold `cap` entries; *nbins receives the bin
 * count (CL_EINVAL if cap is too small).  Synchronises the stream. */
cl_status cl_spectrum(cl_ctx* ctx, int field, int what, double dk_bin, double* k, double* delta,
                      int64_t* mult, int cap, int* nbins);

/* Copy one lattice array to / from the host as FP64 (N^3 values).  Both
 * synchronise the kick stream first; set_state stores in the context's
 * precision.  Fields: scalar models f < nf; U(1) model 0,1 = phi_0, phi_1 and
 * 2,3,4 = A_i; doublet model 0..3 = the components of
 * Phi = (phi_0 + i phi_1, phi_2 + i phi_3)/sqrt2 and 4,5,6 = A_i;
 * CL_MODEL_LPHI4_SU2U1 as the doublet model, and 7 = phi_s, 8, 9 = the components
 * of vphi = (vphi_0 + i vphi_1)/sqrt2. */
cl_status cl_get_state(cl_ctx* ctx, int field, int what, double* host_out);
cl_status cl_set_state(cl_ctx* ctx, int field, int what, const double* host_in);

/* Gauge models (one lattice): spectra of the modulus of the charged field,
 * r = |phi| = sqrt(sum_c phi_c^2/2) (the U(1) field's two components or the
 * doublet's four), and of r' = sum_c phi_c phi_c'/(2 r) (phi_c' = a^{alpha-3} pi_c;
 * 0 where r = 0): df, dfp = eq. discretePS of r and r' on cl_spectrum's shells,
 * n = eq. OccuppationNum applied to the canonically normalised modulus
 * rho = sqrt2 r = sqrt(sum_c phi_c^2) with w_b^2 = k_b^2 + a^2 <d^2V/drho^2>,
 * V = lam (r^2 - v^2)^2, d^2V/drho^2 = V''(r)/2 = lam (6 r^2 - 2 v^2) (the manual's
 * spectrum outputs of the charged scalars, Sec. 4.5, with its `norm`: the
 * modulus, which is gauge invariant).  fo2 = (f_s/omega_s)^2; fo2 <= 0 takes 1/fluct_amp2.  k, df, dfp,
 * n, mult hold `cap` entries; *nbins receives the bin count.  CL_EUNSUPPORTED for
 * scalar models and ensembles.  Closes the stream of kicks; synchronises.  For
 * CL_MODEL_LPHI4_SU2U1 it is the doublet's (see cl_norm_spectrum_of). */
cl_status cl_norm_spectrum(cl_ctx* ctx, double dk_bin, double fo2, double* k, double* df, double* dfp, double* n,
                           int64_t* mult, int cap, int* nbins);
/* As cl_norm_spectrum for the charged field `which` (Sec. 4.5 outputs
 * spectra_norm_SU2Doublet_scalar and spectra_norm_cmplx_scalar): which = 0 the
 * model's charged field (cl_norm_spectrum); which = 1 the U(1)-charged scalar
 * vphi of CL_MODEL_LPHI4_SU2U1.  The mass of n is the potential's curvature
 * along the field's canonical modulus, averaged over the lattice (eq. PotGauge):
 * for lphi4SU2U1's doublet lam (6 <r^2> - 2 v^2) + q_G <phi_s^2> + 2 q_H <|vphi|^2>,
 * for its vphi 2 q_H <|Phi|^2>.  CL_EINVAL for which = 1 in other models. */
cl_status cl_norm_spectrum_of(cl_ctx* ctx, int which, double dk_bin, double fo2, double* k, double* df,
                              double* dfp, double* n, int64_t* mult, int cap, int* nbins);

/* Doublet model: whole arrays by index, in the order
 *   0..3 phi_c, 4..7 pi_c, 8..10 A_i, 11..13 pi_A,i,
 *   14 + 4 i + k: component u_k of the SU(2) link U_i(n) = u0 - i (u1 s1 + u2 s2 + u3 s3)
 *                 (s_a the Pauli matrices; U_i = exp(-i gQB dx B_i^a s_a/2)),
 *   26 + 3 i + (a - 1): link momentum pi_B,i^a,
 *   and for CL_MODEL_LPHI4_SU2U1: 35 phi_s, 36 pi_s, 37, 38 vphi_c, 39, 40 pi_vphi,c,
 * N^3 FP64 values, x fastest.  Links are stored as given (a caller that sets
 * them keeps them unitary).  CL_EUNSUPPORTED for other models, CL_EINVAL for
 * a bad index.  Both synchronise the kick stream first. */
cl_status cl_get_array(cl_ctx* ctx, int a, double* host_out);
cl_status cl_set_array(cl_ctx* ctx, int a, const double* host_in);

/* Scale factor, its derivative and the time.  cl_set_scalars also resets the
 * reference energy of energy_cons to the current state. */
cl_status cl_get_scalars(cl_ctx* ctx, double* eta, double* a, double* b);
cl_status cl_set_scalars(cl_ctx* ctx, double eta, double a, double b);

/* Raw state transfer in the storage precision, for end-to-end use: the whole
 * state (every array of lattice 0 in storage order: field then momentum per
 * field for the scalar and U(1) models, the order of cl_get_array for the
 * doublet model) is `*bytes` long.  Host buffers should be pinned for speed.
 * Both synchronise the kick stream first; the copies are enqueued on the
 * context stream (cl_download_state waits for its copy to finish). */
cl_status cl_state_bytes(cl_ctx* ctx, size_t* bytes);
cl_status cl_upload_state(cl_ctx* ctx, const void* host, size_t bytes);
cl_status cl_download_state(cl_ctx* ctx, void* host, size_t bytes);

/* Caller-owned state memory (the lattice state of Sec. 3: fields and momenta
 * on the sites, and for the gauge models the links and their momenta): lattice
 * `lat` keeps the two buffers a pass reads and writes in buf0 and buf1 instead
 * of in memory of its own, e.g. two torch CUDA tensors.  Each is a device
 * pointer on the context's device, 256-byte aligned, to `bytes` bytes, at least
 * the lattice's state (narr arrays of N^3 values in the storage precision,
 * array a at a * N^3 values, in the order of cl_upload_state; cl_state_bytes
 * gives the size for a single lattice); the two must not overlap.  The state
 * moves with the binding: both buffers are copied into buf0 and buf1 on the
 * context stream, and the lattice's own state memory is released.  buf0 = buf1 =
 * NULL moves the state back into new memory of the lattice's own.  The caller
 * keeps ownership; the buffers must stay allocated while bound (until cl_free or
 * a later cl_bind_buffers of the lattice) and must not be written while the
 * context uses them.  Synchronises the stream.  CL_EINVAL for a bad lattice
 * index, pointer, size, alignment or overlap (nothing changes); CL_ENOMEM when
 * memory of the lattice's own cannot be made again (the binding stays). */
cl_status cl_bind_buffers(cl_ctx* ctx, int lat, void* buf0, void* buf1, size_t bytes);
/* The buffer (0 or 1) that holds the state once the passes enqueued so far
 * have run: the one to read through a binding after the stream has reached
 * them (after cl_sync it holds what cl_get_state returns).  Each pass reads
 * one buffer and writes the other.  Host bookkeeping only. */
cl_status cl_state_buffer(cl_ctx* ctx, int* which);

/* Checkpoint and resume (single lattice): cl_checkpoint_save writes the state
 * arrays and the evolving scalars (a, a', eta, drift coefficients, carried sums,
 * the last measurement) to `path` through a temporary file that is renamed over
 * `path` once complete, so a failure leaves the previous checkpoint intact;
 * cl_checkpoint_load restores them into a context made with the same model, N,
 * precision, kIR and alpha, after which stepping continues exactly as the saved
 * run would (the kick stream is closed at both).  CL_EINVAL for an unreadable or
 * mismatched file, CL_EUNSUPPORTED for ensembles.  Both synchronise the stream. */
cl_status cl_checkpoint_save(cl_ctx* ctx, const char* path);
cl_status cl_checkpoint_load(cl_ctx* ctx, const char* path);

/* The autotuner's on-disk cache (cl_params.autotune): once a file is named,
 * tuned tile heights are read from it and new ones written to it (one line per
 * model, precision, N and device; rewritten through a temporary file), so later
 * processes skip the timing.  Each call forgets the heights tuned so far in
 * this process and takes the named file's entries; an entry whose height the
 * device cannot run is tuned afresh.  NULL or "" turns the file off.  A file
 * that cannot be written makes the autotuning cl_init fail with CL_EINVAL.
 * Process-wide; returns CL_OK. */
cl_status cl_set_tune_cache(const char* path);

int cl_nfields(const cl_ctx* ctx);           /* lattice arrays per kind (what=0 or 1) */
int64_t cl_kernel_launches(const cl_ctx* ctx); /* kernels this context has launched */
const char* cl_last_error(const cl_ctx* ctx);  /* never NULL; ctx may be NULL */

/* Timing hook for measurement tools: a CUDA event pair is recorded on the
 * context stream around every DK pass launch when enabled; the summed
 * device time of those passes (ms) and their count since the last reset are
 * returned by cl_pass_timing.  Disabled by default (no events recorded). */
cl_status cl_enable_pass_timing(cl_ctx* ctx, int enable);
cl_status cl_pass_timing(cl_ctx* ctx, double* ms_total, int64_t* passes, int reset);
/* The same for the reversed (adjoint) passes that cl_adjoint launches while
 * timing is enabled; cl_pass_timing counts only the forward DK passes. */
cl_status cl_adjoint_pass_timing(cl_ctx* ctx, double* ms_total, int64_t* passes, int reset);

/* ---------------------------------------------------------------------------
 * Ensembles (batched independent lattices).  `count` lattices of one model and
 * one set of run parameters, lattice l with its own size Ns[l] (any admissible
 * N, sizes may differ), kIRs[l] and seeds[l], evolved together: every DK pass
 * of cl_step covers all lattices in one persistent cooperative launch (the
 * plane tasks of all lattices split evenly by site count over the SMs, each
 * lattice with its own scale factor, volume averages and Friedmann update),
 * recorded in a CUDA graph on first use and replayed afterwards.  Lattice
 * results do not depend on the ensemble they are part of beyond the rounding
 * of their FP64 reductions.  The IC generator, spectra and transfers of
 * lattice l are those of a single lattice with (Ns[l], kIRs[l], seeds[l]).
 * Returns as cl_init; count must be 1 .. CL_MAX_LATTICES.
 */
#define CL_MAX_LATTICES 4096
cl_status cl_ensemble_init(cl_ctx** out, int model, int count, const int* Ns, const double* kIRs,
                           double alpha, const uint64_t* seeds, const cl_params* p);
int cl_ensemble_size(const cl_ctx* ctx);

/* Per-lattice forms of cl_energies, cl_get_state, cl_set_state and
 * cl_get_scalars (lat in 0 .. count-1, CL_EINVAL otherwise). */
cl_status cl_lattice_energies(cl_ctx* ctx, int lat, cl_energies_t* out);
cl_status cl_lattice_get_state(cl_ctx* ctx, int lat, int field, int what, double* host_out);
cl_status cl_lattice_set_state(cl_ctx* ctx, int lat, int field, int what, const double* host_in);
cl_status cl_lattice_scalars(cl_ctx* ctx, int lat, double* eta, double* a, double* b);

/* Tile shape the passes use for lattice `lat`: its N, its tile height BY
 * (rows of one CTA tile) and the context's number of ring stages.  The doublet
 * model's pass tiles x-y instead (BY reported as 0, 3 ring planes). */
cl_status cl_lattice_tile(cl_ctx* ctx, int lat, int* N, int* BY, int* stages);

/* Lattice occupation number of scalar field `field` (eq. OccuppationNum, with
 * the spectrum outputs of Sec. 5.3) per bin of cl_spectrum's shells:
 *   n_b = a^2 L^3/(2 N^6) (f_s/omega_s)^2 [ w_b <|phi_k|^2>_b
 *                                          + a^{2(1-alpha)}/w_b <|phi'_k + (a'/a) phi_k|^2>_b ],
 * <.>_b the mean over the bin's modes (k != 0), phi_k the forward DFT of the
 * field, phi' = a^{alpha-3} pi, L = N dx, w_b^2 = k_b^2 + a^2 <d^2V/dphi^2>
 * (k_b the bin's k, the volume average of the field's diagonal Hessian
 * element at the synchronised state).  fo2 = (f_s/omega_s)^2, the square of
 * the field over the frequency scale of the program units; fo2 <= 0 takes
 * 1/fluct_amp2 (the IC amplitude parameter is (omega_s/f_s)^2).  k and mult as
 * cl_spectrum; n_b is NaN where w_b^2 <= 0.  Single scalar lattices only
 * (CL_EUNSUPPORTED otherwise).  Synchronises the stream. */
cl_status cl_occupation(cl_ctx* ctx, int field, double dk_bin, double fo2, double* k, double* n,
                        int64_t* mult, int cap, int* nbins);

/* Gauge models (single lattice): binned spectrum of the U(1) electric (which = 0)
 * or magnetic (which = 1) field (eq. ElectricMagneticDefs, the gauge spectra of
 * the outputs of Sec. 5.3):  E_i = F_0i = a^{alpha-1} pi_A,i;
 * B_i = (1/2) eps_ijk F_jk with the compact F_jk = sin(theta_jk)/(gQ dx^2),
 * theta_jk(n) = gQ dx [A_j(n) + A_k(n+j) - A_j(n+k) - A_k(n)].  Doublet model
 * also the SU(2) electric (which = 2: E_i^a = a^{alpha-1} pi_B,i^a) and magnetic
 * (which = 3: B_i^a = (1/2) eps_ijk G_jk^a, G_jk^a = Tr[(i s_a/2)(U_jk - U_jk^dag)]/(gQB dx^2)
 * from the plaquette, SU(N) toolkit) fields.  delta_b is eq. discretePS with
 * |f(k)|^2 summed over the components (three, or nine with colour); k and mult as
 * cl_spectrum.  CL_EUNSUPPORTED for scalar models and for which = 1 with gQ = 0.
 * Synchronises the stream. */
cl_status cl_em_spectrum(cl_ctx* ctx, int which, double dk_bin, double* k, double* delta, int64_t* mult,
                         int cap, int* nbins);

/* Measured FP64 rate of the current device (FMA counted as two operations):
 * a full grid of independent FMA chains timed with CUDA events on `stream`
 * (a cudaStream_t, NULL = default), best of three after a warm-up.  The roof
 * of the FP64 plain pass, which is bound by FP64 arithmetic.  Needs no
 * context; returns CL_ECUDA / CL_ENOMEM on failure. */
cl_status cl_measure_fp64_rate(void* stream, double* flops_per_s);

/* Self-test of the bounded device waits that the persistent passes use (no
 * counterpart in the paper).  One GPU thread runs one wait with a limit of
 * limit_ns nanoseconds of device time (1 .. 1e10):
 *   kind 0: the inter-pass counter wait, on a device word holding 1 (satisfied)
 *           or 0 (nothing ever sets it);
 *   kind 1: the stage mbarrier wait, on a fresh barrier that expects one
 *           arrival, which the thread gives (satisfied) or not.
 * Returns CL_OK when the wait was satisfied, CL_ETIMEOUT when it ran out (the
 * status the passes record), CL_EINVAL for bad arguments, CL_ENOMEM /
 * CL_ECUDA on failure.  *elapsed_ns (may be NULL) receives the device time the
 * wait took.  Needs no context; synchronises `stream` (a cudaStream_t, NULL =
 * default). */
cl_status cl_selftest_wait(void* stream, int kind, int satisfied, uint64_t limit_ns, uint64_t* elapsed_ns);

/* The counter-based generator of the initial conditions, evaluated on the GPU
 * by the same device code cl_init uses (Philox4x32-10 of Salmon et al., SC'11,
 * keyed by the seed; the deviates of the Rayleigh amplitudes and uniform phases
 * of Sec. 3.5.1, eqs. fpr_influct and QuantumFlucts2), for checks against a
 * host implementation.  For element i of n (host arrays, caller-owned):
 *   mode 0: out[4i..4i+3] = Philox4x32-10(counter ctr[4i..4i+3], key key[2i..2i+1]);
 *           u[2i], u[2i+1] = the 53-bit deviates in (0, 1] made from words (0, 1)
 *           and (2, 3): (2^26 (w_hi >> 5) + (w_lo >> 6) + 1) 2^-53;
 *   mode 1: u[2i], u[2i+1] = the draw pair of the initial conditions at Fourier
 *           index ctr[4i] (x fastest), component ctr[4i+1], draw ctr[4i+2]
 *           (0 amplitudes, 1 phases) with seed key[2i] + 2^32 key[2i+1]
 *           (counter (index, component, draw, 0)); out is zeroed.
 * n in 0 .. 2^24.  Allocates device memory for the call; synchronises `stream`
 * (a cudaStream_t, NULL = default).  CL_EINVAL for bad arguments, CL_ENOMEM /
 * CL_ECUDA on failure.  Needs no context. */
cl_status cl_philox_draws(void* stream, int mode, int n, const uint32_t* ctr, const uint32_t* key, uint32_t* out,
                          double* u);

/* Ensemble-averaged binned spectrum: delta_b of cl_spectrum averaged over
 * the lattices lats[0 .. nl) (which must share N and kIR); k and mult as in
 * cl_spectrum (identical for those lattices).  Synchronises the stream. */
cl_status cl_ensemble_spectrum(cl_ctx* ctx, const int* lats, int nl, int field, int what,
                               double dk_bin, double* k, double* delta, int64_t* mult, int cap,
                               int* nbins);

/* ---------------------------------------------------------------------------
 * Adjoint (gradient of a final observable), for a single lattice of a scalar
 * model (CL_EUNSUPPORTED for U(1) and for ensembles), with any expansion mode.
 * cl_adjoint starts from the current (synchronised) state, runs nsteps steps
 * saving the fields every ckpt_every steps in device memory, evaluates the
 * objective at the synchronised end, then runs the passes backwards: each
 * reversed pass recovers the state before it (the time-reversible integrator
 * run backwards) and applies the transposed Jacobian of the pass (Sec. 3.5.2
 * Hamiltonian form: drift, field kick and, with CL_EXP_SELF, the Friedmann
 * kicks of b = a' and the drift of a) to the adjoint, and the saved fields
 * replace the recovered ones at the checkpoints (where FP32 rounding breaks
 * exact reversal).  Objectives:
 *   CL_OBJ_CHI_FRACTION: J = (E_K^chi + E_G^chi)/rho (CL_MODEL_LPHI4_CHI);
 *   CL_OBJ_SPECTRUM_BIN: J = delta_b of cl_spectrum(field, what, dk_bin), b = bin.
 * Returns J; dJ/dq at a fixed initial state (fields, momenta, a and b); if
 * dJ_dstate is not NULL, dJ/d(initial state) in 2 nf arrays of N^3 doubles
 * (field f: array 2f = d/dphi_f, 2f + 1 = d/dpi_f); and if dJ_dscale is not
 * NULL, dJ_dscale[0..1] = dJ/da, dJ/db at the start (both 0 unless the
 * expansion is CL_EXP_SELF, where a and b are evolved variables; a user whose
 * b(t0) follows from the state or from q adds dJ/db times that dependence).
 * The state, a, b and eta are left at the starting point.  Allocates
 * checkpoint storage for the duration of the call. */
enum { CL_OBJ_CHI_FRACTION = 0, CL_OBJ_SPECTRUM_BIN = 1 };
cl_status cl_adjoint(cl_ctx* ctx, int nsteps, int ckpt_every, int objective, int field, int what,
                     double dk_bin, int bin, double* J, double* dJ_dq, double* dJ_dstate,
                     double* dJ_dscale);

/* Chain dJ/d(initial state) (as returned by cl_adjoint started at the
 * initial conditions) through the IC map (Sec. 3.5.1) to the drawn mode
 * amplitudes: out[(2f + j) N^3 + n] = dJ/d|z_{j+1}| of field f at Fourier site
 * n (x fastest) for the drawn member of each (n, -n) pair; 0 elsewhere.
 * CL_EUNSUPPORTED with CL_EXP_SELF and b0_mode 1 (b(t0) then depends on the
 * amplitudes through the lattice averages). */
cl_status cl_ic_amplitude_grad(cl_ctx* ctx, const double* dJ_dstate, double* out);

/* ---------------------------------------------------------------------------
 * Volume averages without device allocation.  The paper has no counterpart:
 * this entry point exists for callers that cannot call cudaMalloc -- programs
 * that give the library all of their device memory up front (a fixed budget,
 * or another framework's memory pool) and loops that must not synchronise the
 * device, which cudaMalloc / cudaFree may do.  It computes, for a scalar-field
 * state (CL_MODEL_LPHI4 or CL_MODEL_LPHI4_CHI) held in the caller's device
 * memory, the same volume averages cl_energies reports, and calls no
 * cudaMalloc, cudaFree or other allocating routine.
 *
 *   arrays : host array of 2*nf device pointers {phi_0, pi_0[, phi_1, pi_1]},
 *            each N^3 values (x fastest) of float (CL_FP32) or double (CL_FP64).
 *   a      : scale factor of the state; kIR gives dx = 2 pi/(N kIR); q as in
 *            cl_params (used by CL_MODEL_LPHI4_CHI).
 *   out    : device pointer to CL_NOALLOC_OUT doubles, written in order
 *            E_K[2], E_G[2], E_V[2], <phi>[2], <phi^2>[2], <pi>[2], <pi^2>[2],
 *            rho, count of non-finite momenta (entries of absent fields are 0).
 *   stream : cudaStream_t the two kernels are enqueued on (asynchronous).
 *
 * Partial sums live in one file-scope device array of CL_NOALLOC_MAX_BLOCKS x
 * CL_NOALLOC_OUT doubles (128 KiB), held by every GPU that loads the library
 * until the process exits.  A call whose stream is not being captured looks up
 * that array's device address with the device current (so a device reset
 * cannot leave a stale address in use); a call during a stream capture reuses
 * the address the last uncaptured call on that device found, so make the first
 * call on a device before any stream capture.  Every call shares the array
 * (each row a call reads is written earlier in the same call), so calls that
 * overlap on the GPU race.
 * Returns CL_EINVAL for N > CL_NOALLOC_MAX_N (the no-allocation limit) or bad
 * arguments, CL_ECUDA if a launch or the address lookup fails. */
#define CL_NOALLOC_MAX_BLOCKS 1024
#define CL_NOALLOC_OUT 16
#define CL_NOALLOC_MAX_N 512
cl_status cl_volume_averages_noalloc(int model, int N, double kIR, double a, double q,
                                     int precision, const void* const* arrays, double* out,
                                     void* stream);

#ifdef __cplusplus
}
#endif
#endif
