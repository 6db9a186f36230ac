// capi.cu -- the C ABI of include/cl.h: contexts holding one lattice or an
// ensemble of lattices, the work list of the DK passes, the kick/drift
// schedule of the integrators, CUDA-graph replay of multi-pass launches, and
// the tile-shape autotuner.  Host code only marshals parameters and orders
// launches; every step of the method (initial conditions, FFTs, passes,
// reductions, Friedmann updates, spectra) runs in the kernels of this library.
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <tuple>
#include <vector>

#include "cl.h"
#include "common.cuh"
#include "checkpoint.h"
#include "su2_work.h"
#include "tune_cache.h"
#include "worklist.h"

namespace clg {

// kernels defined in the other translation units
typedef void (*PassKernel)(const PassArgs);

// The models run by the doublet pass: the SU(2) x U(1) doublet alone, or with
// the singlet and the U(1)-charged scalar of the lphi4SU2U1 example.
inline bool is_doublet(int model) { return model == CL_MODEL_SU2U1_HIGGS || model == CL_MODEL_LPHI4_SU2U1; }
PassKernel scalar_pass_kernel(int fp32, int nf, int red);
PassKernel u1_pass_kernel(int fp32, int red, int kd, int n256);
PassKernel su2_pass_kernel(int fp32, int red, int TX, int full);
size_t su2_smem_bytes(int TX, int TY, int esz, int full);
PassKernel su2_kd_pass_kernel(int fp32, int red, int TX, int TY, int full, int n256);
size_t su2_kd_smem_bytes(int TX, int TY, int esz, int full);
cudaError_t launch_su2_identity_links(int fp32, void* base, long long V, cudaStream_t st);
cudaError_t launch_su2_rho(int fp32, const LatConst* L, int parity, int g, double2* rho, long long V,
                           cudaStream_t st);
cudaError_t launch_su2_gauss_monitor(int fp32, const LatConst* L, int parity, double* part, int nblk,
                                     long long V, cudaStream_t st);
constexpr int SU2_PARTIALS = 30;  // partial sums per CTA of the doublet-model pass

cudaError_t launch_init_scalars(const LatConst*, LatScalars*, const ICArgs&, cudaStream_t);
cudaError_t launch_ic_modes(double2*, double2*, const LatConst*, const LatScalars*, const ICArgs&,
                            int, long long, cudaStream_t);
cudaError_t launch_ic_assemble(int, void*, void*, const double2*, const double2*, const LatConst*,
                               const LatScalars*, double, double, long long, cudaStream_t);
cudaError_t launch_fft_axis(double2*, const FftPlan&, cudaStream_t);
cudaError_t launch_fft_twiddles(double2*, int, cudaStream_t);
cudaError_t launch_real_spectrum(int fp32, const void* f, double2* H, const FftPlan& pl, double dk, int nb,
                                 int nblk, double* part, double kIR, double dx, double* out, cudaStream_t st,
                                 const int* bin_of, const double* geo);
cudaError_t launch_shell_geometry(int N, double dk, int nb, int nblk, int* bin_of, double* geo, double* part,
                                  cudaStream_t st);
int fft_batch(int N);
cudaError_t launch_to_complex(int, const void*, double2*, long long, cudaStream_t);
cudaError_t launch_bins(const double2*, int, double, int, int, double*, double, double, double*,
                        cudaStream_t, int raw = 0);
cudaError_t launch_combine_to_complex(int, const void*, double, const void*, double, double2*, long long,
                                      cudaStream_t);
cudaError_t launch_u1_plaquette_field(int, const void*, const void*, int, int, int, double, double, double2*,
                                      cudaStream_t);
cudaError_t launch_spec_mean(const double*, int, int, double*, cudaStream_t);
cudaError_t launch_su2_plaquette_field(int fp32, const void* Uj, const void* Ul, int j, int l, int a, int N,
                                       double inv_bdx2, double2* out, cudaStream_t st);
cudaError_t launch_norm_field(int fp32, const void* const* f, const void* const* p, int nc, double apm, double H,
                              int mode, double2* out, long long V, cudaStream_t st);
cudaError_t launch_convert(int, int, const void*, void*, long long, cudaStream_t);
cudaError_t launch_sum_sq(int fp32, const void* f0, const void* f1, const void* f2, double w0, double w1,
                          double w2, long long V, int nblk, double* part, cudaStream_t st);
cudaError_t launch_u1_gauss_init(const LatConst*, int, double2*, double2*, int, int, double, int,
                                 void*, long long, int, cudaStream_t);
cudaError_t launch_u1_gauss_monitor(const LatConst*, int, double*, int, long long, cudaStream_t);
__global__ void set_scalars_kernel(const LatConst*, LatScalars*, double, double, double);
__global__ void b_from_obs_kernel(const LatConst*, LatScalars*);
PassKernel adjoint_pass_kernel(int fp32, int nf, int self);
cudaError_t launch_seed_chi_fraction(int, const LatConst*, LatScalars*, int, void* const*, double*, int,
                                     double*, cudaStream_t);
cudaError_t launch_spectrum_seed(int, double2*, int, double, int, int, const double*, double, double, double*,
                                 int, void*, cudaStream_t);
cudaError_t launch_ic_amp_grad(const double2*, const double2*, double*, double*, const LatConst*,
                               const LatScalars*, const ICArgs&, int, long long, cudaStream_t);

}  // namespace clg

using namespace clg;

namespace {

// One lattice of a context (host view).
struct LatHost {
  int N = 0, BY = 0;
  long long V = 0;
  double kIR = 0.0, dx = 0.0;
  uint64_t seed = 0;
  void* slab = nullptr;  // 2 buffers x narr arrays of V values, array-major
  void* bound[2] = {nullptr, nullptr};  // caller-owned buffers (cl_bind_buffers), in place of slab
  ICArgs ic;             // what the initial conditions were drawn with
};

// Resources of the adjoint sweep (single scalar lattice), made on first use:
// the reversed-pass kernel's own tiling over the state and adjoint arrays.
struct AdjPlan {
  bool ready = false;
  int grid = 0, stages = 0;
  unsigned stage_bytes = 0;
  size_t smem = 0;
  bool coop = false;
  void* lam = nullptr;           // 2 buffers x 2 nf adjoint arrays
  LatConst* d_lat = nullptr;     // arrays: state (2 nf) then adjoint (2 nf), by buffer
  Seg* d_segs = nullptr;
  int* d_cta = nullptr;
  double* d_part = nullptr;
  unsigned* d_cnt = nullptr;
  double* d_out = nullptr;       // J and the explicit dJ/dq of the objective
  int nslot = 0;
  LatConst hl;                   // host copy of *d_lat
};

// A multi-pass launch recorded in a CUDA graph, replayed when the same
// passes are launched again from the same buffer parity.
struct GraphEntry {
  std::vector<PassStep> steps;
  int parity, red, write, set_rho0;
  const void* dev_steps;  // the device copy of the weights the graph reads
  cudaGraphExec_t exec;
};

}  // namespace

struct cl_ctx {
  int model = 0, nf = 0, narr = 0, fp32 = 0, esz = 0, nlat = 0;
  double alpha = 0.0;
  cl_params p;
  cudaStream_t stream = nullptr;      // the caller's stream (may be the legacy default stream)
  cudaStream_t cap_stream = nullptr;  // private stream that records graphs
  int dev = 0, nsm = 0;
  size_t smem_optin = 0;
  std::vector<LatHost> lats;
  std::vector<LatConst> hlat;
  long long vmax = 0;
  // device memory
  LatConst* d_lat = nullptr;       // [nlat]
  LatScalars* d_sc = nullptr;      // [nlat]
  Seg* d_segs = nullptr;
  int* d_cta = nullptr;
  double* d_part = nullptr;        // [nslot][NQ]
  unsigned* d_cnt = nullptr;       // [nlat]
  double* d_tmp = nullptr;         // scratch for conversions / monitors (vmax doubles)
  double2* d_cplx = nullptr;       // scratch complex (2 vmax)
  double2* d_tw = nullptr;         // FFT twiddle table (the largest lattice's N entries)
  double* d_spec = nullptr;        // spectrum scratch: block rows (3 x 2048 x nblk), per-lattice bins, mean
  int spec_lats = 0;               // lattices d_spec has room for
  int* d_bin_of = nullptr;         // cached shell geometry of (geo_N, geo_dk): bin of each |n|^2,
  double* d_geo = nullptr;         //   sum of |n| and count per bin (2 x 2048)
  int geo_N = 0;
  double geo_dk = 0.0;
  unsigned* d_gsync = nullptr;     // arrival counters of multi-pass launches
  bool coop = false;               // multi-pass cooperative launches possible
  bool graphs = true;              // record multi-pass launches in CUDA graphs
  std::vector<std::pair<std::vector<PassStep>, void*>> step_cache;
  std::vector<GraphEntry> graph_cache;
  AdjPlan adj;
  int grid = 0, nseg = 0, nslot = 0, stages = 0;
  unsigned stage_bytes = 0;
  size_t smem_bytes = 0;
  int su2_kd_ty = 8;                // doublet models: tile height of the kick-then-drift step pass (RED 0)
  int su2_tx = 0, su2_ty = 0;      // doublet model: CTA tile (x, y) of the pass
  // schedule state
  int parity = 0;
  bool open = false;
  double dprev = 0.0;
  bool obs_valid = false;
  long long launches = 0;
  // timing hook
  bool timing = false;
  std::vector<cudaEvent_t> ev_pool;
  std::vector<std::pair<cudaEvent_t, cudaEvent_t>> ev_pending;
  std::vector<int> ev_npass;
  std::vector<int> ev_kind;        // 0: DK passes, 1: adjoint passes
  double timing_ms = 0.0;
  long long timing_passes = 0;
  double adj_timing_ms = 0.0;
  long long adj_timing_passes = 0;
  std::string err;
};

namespace {

thread_local std::string g_init_err;

// NVTX range over a C-ABI call (visible in Nsight timelines; free without a tool attached).
struct Range {
  explicit Range(const char* name) { nvtxRangePushA(name); }
  ~Range() { nvtxRangePop(); }
  Range(const Range&) = delete;
  Range& operator=(const Range&) = delete;
};

cl_status fail(cl_ctx* c, cl_status s, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  if (c) c->err = buf;
  else g_init_err = buf;
  return s;
}

#define CU(call)                                                                         \
  do {                                                                                   \
    cudaError_t e_ = (call);                                                             \
    if (e_ != cudaSuccess)                                                               \
      return fail(c, e_ == cudaErrorMemoryAllocation ? CL_ENOMEM : CL_ECUDA, "%s: %s (%s:%d)", \
                  #call, cudaGetErrorString(e_), __FILE__, __LINE__);                    \
  } while (0)

#define CHECK_LAUNCH() CU(cudaGetLastError())

bool good_N(int N) {
  if (N < 8 || N > 512 || N % 8) return false;
  int m = N;
  while (m % 2 == 0) m /= 2;
  while (m % 3 == 0) m /= 3;
  return m == 1;
}

// Symmetric compositions: VV2 = one Stoermer-Verlet step; each higher order
// is the triple jump z1, 1 - 2 z1, z1 of the previous one, z1 = 1/(2 - 2^{1/(k+1)}).
void schedule(int order, double h, std::vector<double>& d) {
  if (order <= 2) {
    d.push_back(h);
    return;
  }
  const double z1 = 1.0 / (2.0 - std::pow(2.0, 1.0 / (double)(order - 1)));
  schedule(order - 2, z1 * h, d);
  schedule(order - 2, (1.0 - 2.0 * z1) * h, d);
  schedule(order - 2, z1 * h, d);
}

// Kick/drift weights of the passes of n steps of size h, appended to `steps`:
// the first pass of a closed stream only kicks (by half the first drift);
// later passes merge the kick-out of the previous drift with the kick-in of
// the next (first same as last).  `open` and `dprev` carry the stream across
// calls.
void append_pass_steps(int integrator, double h, int n, bool& open, double& dprev, std::vector<PassStep>& steps) {
  std::vector<double> d1;
  schedule(integrator == CL_LF ? 2 : integrator, h, d1);
  steps.reserve(steps.size() + (size_t)n * d1.size());
  for (int s = 0; s < n; ++s)
    for (double d : d1) {
      if (!open) {
        steps.push_back(PassStep{0.5 * d, 0.0, 0.5 * d, d});
        open = true;
      } else {
        steps.push_back(PassStep{0.5 * (dprev + d), 0.5 * dprev, 0.5 * d, d});
      }
      dprev = d;
    }
}

// The pass that closes a stream: the kick-out of the last drift, no drift.
PassStep closing_pass_step(double dprev) { return PassStep{0.5 * dprev, 0.5 * dprev, 0.0, 0.0}; }

void fft_radices(int N, FftPlan& pl) {
  pl.nrad = 0;
  int m = N;
  while (m % 4 == 0) { pl.rad[pl.nrad++] = 4; m /= 4; }
  while (m % 2 == 0) { pl.rad[pl.nrad++] = 2; m /= 2; }
  while (m % 3 == 0) { pl.rad[pl.nrad++] = 3; m /= 3; }
}

void* arr_ptr(cl_ctx* c, int lat, int parity, int a) {
  const LatHost& L = c->lats[lat];
  if (L.bound[0]) return (char*)L.bound[parity] + (size_t)a * L.V * c->esz;
  return (char*)L.slab + ((size_t)parity * c->narr + a) * (size_t)L.V * c->esz;
}

cl_status fft3d(cl_ctx* c, int N, double2* data, int sign) {
  FftPlan pl;
  pl.N = N;
  pl.sign = sign;
  pl.batch = fft_batch(N);
  pl.tw = c->d_tw;
  pl.pitch = pl.nu = N;
  fft_radices(N, pl);
  CU(launch_fft_twiddles(c->d_tw, N, c->stream));
  ++c->launches;
  for (int axis = 0; axis < 3; ++axis) {
    pl.axis = axis;
    CU(launch_fft_axis(data, pl, c->stream));
    ++c->launches;
  }
  return CL_OK;
}

// Doublet models without self-consistent expansion (a constant or fixed power-law
// background): kick-then-drift passes (pass_su2_kd.cu), which take no Friedmann
// sums (RED 1 only arises with self-consistent expansion).
bool su2_kd(const cl_ctx* c, int red) { return c->p.expansion != CL_EXP_SELF && red != 1; }
// Tile height of the kick-then-drift pass of measurement level red: the step pass's
// (16 rows for the FP32 lphi4SU2U1 model, else 8), the measurement pass's 8.
int kd_ty(const cl_ctx* c, int red) { return red == 0 ? c->su2_kd_ty : 8; }
// The FP32 32-wide kick-then-drift step pass on a 256^3 lattice runs the variant built for N = 256.
int kd_n256(const cl_ctx* c, int red) { return red == 0 && c->fp32 && c->su2_tx == 32 && c->lats[0].N == 256; }
size_t su2_launch_smem(const cl_ctx* c, int red) {
  return su2_kd(c, red) ? su2_kd_smem_bytes(c->su2_tx, kd_ty(c, red), c->esz, c->model == CL_MODEL_LPHI4_SU2U1)
                        : c->smem_bytes;
}
int su2_launch_ty(const cl_ctx* c, int red) { return su2_kd(c, red) ? kd_ty(c, red) : c->su2_ty; }

PassKernel pick_kernel(const cl_ctx* c, int red) {
  if (is_doublet(c->model)) {
    const int full = c->model == CL_MODEL_LPHI4_SU2U1;
    if (su2_kd(c, red)) return su2_kd_pass_kernel(c->fp32, red, c->su2_tx, kd_ty(c, red), full, kd_n256(c, red));
    return su2_pass_kernel(c->fp32, red, c->su2_tx, full);
  }
  // without self-consistent expansion the U(1) passes drift right after their
  // kick (the drift coefficient does not wait for the pass's sums)
  if (c->model == CL_MODEL_U1_HIGGS) {
    const bool n256 = c->nlat == 1 && c->lats[0].N == 256 && c->lats[0].BY == THREADS / (256 / u1_vx(c->esz));
    return u1_pass_kernel(c->fp32, red, c->p.expansion != CL_EXP_SELF, n256);
  }
  return scalar_pass_kernel(c->fp32, c->nf, red);
}

int tile_vx(int model, int esz) { return model == CL_MODEL_U1_HIGGS ? u1_vx(esz) : 16 / esz; }

// Bytes of one stage (BY + 2 rows of every array; with mown the momenta, the
// odd arrays, BY rows only), 128-byte aligned.
size_t stage_size(int N, int BY, int narr, int esz, bool mown = false) {
  const size_t rows = mown ? (size_t)(narr / 2) * (2 * BY + 2) : (size_t)(BY + 2) * narr;
  return (rows * N * esz + 127) / 128 * 128;
}

// The U(1) kick-then-drift passes (no self-consistent expansion) read the momenta at
// the own sites only, so their stages hold the momenta without halo rows.
bool ring_mown(const cl_ctx* c) { return c->model == CL_MODEL_U1_HIGGS && c->p.expansion != CL_EXP_SELF; }

// Tile heights BY admissible for N: BY divides N, the BY rows of N/VX
// threads fit in one CTA, and at least 3 stages fit in shared memory; the
// tallest first.
std::vector<int> tile_candidates(int model, int narr, int esz, int N, size_t smem_optin, bool mown = false) {
  std::vector<int> out;
  const int TX = N / tile_vx(model, esz);
  if (TX > THREADS) return out;
  for (int by = std::min(N, THREADS / TX); by >= 1; --by) {
    if (N % by) continue;
    if ((smem_optin - SM_TAIL_BYTES) / stage_size(N, by, narr, esz, mown) >= 3) out.push_back(by);
  }
  return out;
}

// Device copy of pass weights, cached by content.
cl_status device_steps(cl_ctx* c, const PassStep* st, int n, const PassStep** out) {
  std::vector<PassStep> key(st, st + n);
  for (auto& e : c->step_cache)
    if (e.first.size() == key.size() && memcmp(e.first.data(), key.data(), n * sizeof(PassStep)) == 0) {
      *out = static_cast<const PassStep*>(e.second);
      return CL_OK;
    }
  void* d = nullptr;
  if (c->step_cache.size() >= 8) {
    CU(cudaStreamSynchronize(c->stream));  // an evicted copy may still be read by a queued launch
    // graphs recorded with the evicted copy must not be replayed
    const void* gone = c->step_cache.front().second;
    for (size_t i = 0; i < c->graph_cache.size();) {
      if (c->graph_cache[i].dev_steps == gone) {
        cudaGraphExecDestroy(c->graph_cache[i].exec);
        c->graph_cache.erase(c->graph_cache.begin() + i);
      } else {
        ++i;
      }
    }
    cudaFree(c->step_cache.front().second);
    c->step_cache.erase(c->step_cache.begin());
  }
  CU(cudaMalloc(&d, n * sizeof(PassStep)));
  CU(cudaMemcpy(d, key.data(), n * sizeof(PassStep), cudaMemcpyHostToDevice));
  c->step_cache.push_back(std::make_pair(key, d));
  *out = static_cast<const PassStep*>(d);
  return CL_OK;
}

// The two nodes of a multi-pass launch: zero the arrival counters, then the
// cooperative kernel.
cl_status enqueue_multi(cl_ctx* c, PassKernel k, PassArgs& A, cudaStream_t st) {
  CU(cudaMemsetAsync(c->d_gsync, 0, 2 * sizeof(unsigned), st));
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(c->grid);
  cfg.blockDim = dim3(THREADS);
  cfg.dynamicSmemBytes = c->smem_bytes;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  CU(cudaLaunchKernelEx(&cfg, k, A));
  return CL_OK;
}

// Launch `n` passes of the given weights over every lattice of the context.
// One pass: a plain launch.  Several: one cooperative launch of the same
// kernel (all CTAs resident) that runs them back to back, reading the
// per-pass weights from a device copy; it is recorded in a CUDA graph the
// first time and the graph is replayed for the same passes later.
// Timing hook: an event pair from the context's pool around a launch of n
// passes of one kind (0 DK passes, 1 adjoint passes), read back by
// cl_pass_timing / cl_adjoint_pass_timing.
cl_status timing_begin(cl_ctx* c, cudaEvent_t* e0, cudaEvent_t* e1) {
  for (cudaEvent_t* e : {e0, e1}) {
    if (!c->ev_pool.empty()) {
      *e = c->ev_pool.back();
      c->ev_pool.pop_back();
    } else {
      CU(cudaEventCreate(e));
    }
  }
  CU(cudaEventRecord(*e0, c->stream));
  return CL_OK;
}

cl_status timing_end(cl_ctx* c, cudaEvent_t e0, cudaEvent_t e1, int n, int kind) {
  CU(cudaEventRecord(e1, c->stream));
  c->ev_pending.push_back(std::make_pair(e0, e1));
  c->ev_npass.push_back(n);
  c->ev_kind.push_back(kind);
  return CL_OK;
}

// Adds the pending event pairs to the per-kind totals (synchronises the stream).
cl_status timing_collect(cl_ctx* c) {
  CU(cudaStreamSynchronize(c->stream));
  for (size_t i = 0; i < c->ev_pending.size(); ++i) {
    auto& pr = c->ev_pending[i];
    float ms = 0.f;
    CU(cudaEventElapsedTime(&ms, pr.first, pr.second));
    if (c->ev_kind[i] == 1) {
      c->adj_timing_ms += ms;
      c->adj_timing_passes += c->ev_npass[i];
    } else {
      c->timing_ms += ms;
      c->timing_passes += c->ev_npass[i];
    }
    c->ev_pool.push_back(pr.first);
    c->ev_pool.push_back(pr.second);
  }
  c->ev_pending.clear();
  c->ev_npass.clear();
  c->ev_kind.clear();
  return CL_OK;
}

cl_status launch_passes(cl_ctx* c, const PassStep* st, int n, int red, int write, int set_rho0,
                        double* log = nullptr, long long log_base = 0) {
  PassKernel k = pick_kernel(c, red);
  if (!k) return fail(c, CL_EUNSUPPORTED, "no pass kernel for this configuration");
  PassArgs A;
  memset(&A, 0, sizeof(A));
  A.lat = c->d_lat;
  A.sc = c->d_sc;
  A.segs = c->d_segs;
  A.cta_seg = c->d_cta;
  A.partials = c->d_part;
  A.nslot = c->nslot;
  A.counters = c->d_cnt;
  A.ck = st[0].ck;
  A.wout = st[0].wout;
  A.win = st[0].win;
  A.dnext = st[0].dnext;
  A.parity = c->parity;
  A.write = write;
  A.set_rho0 = set_rho0;
  A.stages = c->stages;
  A.stage_bytes_max = c->stage_bytes;
  A.nlat = c->nlat;
  A.wait_limit_ns = 2000000000ull;  // 2 s
  A.steps = nullptr;
  A.npass = 1;
  A.gsync = nullptr;
  A.log = log;
  A.log_base = log_base;
  const bool su2 = is_doublet(c->model);
  const bool multi = n > 1 && c->coop && !su2;
  cudaGraphExec_t exec = nullptr;
  if (multi) {
    const PassStep* dev = nullptr;
    cl_status s = device_steps(c, st, n, &dev);
    if (s != CL_OK) return s;
    A.steps = dev;
    A.npass = n;
    A.gsync = c->d_gsync;
    if (c->graphs && !log) {
      for (auto& g : c->graph_cache)
        if (g.parity == c->parity && g.red == red && g.write == write && g.set_rho0 == set_rho0 &&
            g.dev_steps == (const void*)dev && g.steps.size() == (size_t)n &&
            memcmp(g.steps.data(), st, n * sizeof(PassStep)) == 0)
          exec = g.exec;
      if (!exec) {
        // record on the private stream; a failed recording falls back to direct launches
        cudaGraph_t graph = nullptr;
        bool ok = cudaStreamBeginCapture(c->cap_stream, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
        if (ok) {
          const bool enq = enqueue_multi(c, k, A, c->cap_stream) == CL_OK;
          ok = cudaStreamEndCapture(c->cap_stream, &graph) == cudaSuccess && enq;
        }
        if (ok) ok = cudaGraphInstantiate(&exec, graph, 0) == cudaSuccess;
        if (graph) cudaGraphDestroy(graph);
        cudaGetLastError();
        if (!ok) {
          if (exec) cudaGraphExecDestroy(exec);
          exec = nullptr;
          c->graphs = false;
        } else {
          if (c->graph_cache.size() >= 8) {
            CU(cudaStreamSynchronize(c->stream));
            cudaGraphExecDestroy(c->graph_cache.front().exec);
            c->graph_cache.erase(c->graph_cache.begin());
          }
          c->graph_cache.push_back(GraphEntry{std::vector<PassStep>(st, st + n), c->parity, red, write,
                                              set_rho0, (const void*)dev, exec});
        }
      }
    }
  }
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (c->timing) {
    cl_status s = timing_begin(c, &e0, &e1);
    if (s != CL_OK) return s;
  }
  if (multi && exec) {
    CU(cudaGraphLaunch(exec, c->stream));
  } else if (multi) {
    cl_status s = enqueue_multi(c, k, A, c->stream);
    if (s != CL_OK) return s;
  } else {
    for (int i = 0; i < n; ++i) {
      A.ck = st[i].ck;
      A.wout = st[i].wout;
      A.win = st[i].win;
      A.dnext = st[i].dnext;
      A.parity = c->parity ^ (write ? (i & 1) : 0);
      A.log_base = log_base + i;
      if (su2) k<<<c->grid, dim3(c->su2_tx, su2_launch_ty(c, red)), su2_launch_smem(c, red), c->stream>>>(A);
      else k<<<c->grid, THREADS, c->smem_bytes, c->stream>>>(A);
      CHECK_LAUNCH();
    }
  }
  c->launches += multi ? 1 : n;
  if (c->timing) {
    cl_status s = timing_end(c, e0, e1, n, 0);
    if (s != CL_OK) return s;
  }
  if (write && (n & 1)) c->parity ^= 1;
  return CL_OK;
}

cl_status run_pass(cl_ctx* c, double ck, double wout, double win, double dnext, int red, int write,
                   int set_rho0) {
  PassStep st = {ck, wout, win, dnext};
  return launch_passes(c, &st, 1, red, write, set_rho0);
}

int red_for_step(const cl_ctx* c) { return c->p.expansion == CL_EXP_SELF ? 1 : 0; }

cl_status close_stream(cl_ctx* c) {
  if (!c->open) return CL_OK;
  const PassStep cl = closing_pass_step(c->dprev);
  cl_status s = run_pass(c, cl.ck, cl.wout, cl.win, cl.dnext, 2, 1, 0);
  if (s != CL_OK) return s;
  c->open = false;
  c->obs_valid = true;
  return CL_OK;
}

cl_status measure(cl_ctx* c, int set_rho0) {
  cl_status s = close_stream(c);
  if (s != CL_OK) return s;
  if (!c->obs_valid || set_rho0) {
    s = run_pass(c, 0.0, 0.0, 0.0, 0.0, 2, 0, set_rho0);
    if (s != CL_OK) return s;
    c->obs_valid = true;
  }
  return CL_OK;
}

// Device-side status of every lattice (a bounded wait that gave up).
cl_status check_status(cl_ctx* c) {
  std::vector<LatScalars> h(c->nlat);
  CU(cudaMemcpyAsync(h.data(), c->d_sc, c->nlat * sizeof(LatScalars), cudaMemcpyDeviceToHost, c->stream));
  CU(cudaStreamSynchronize(c->stream));
  for (int l = 0; l < c->nlat; ++l)
    if (h[l].status == CL_ETIMEOUT)
      return fail(c, CL_ETIMEOUT, "a bounded device wait timed out (lattice %d)", l);
  return CL_OK;
}

}  // namespace

// Autotuner: the tile height of each (model, precision, N) is the candidate
// with the shortest measured DK pass on scratch lattices of that size (as
// many as it takes to give every SM work; two warm-up steps, then eight VV2
// steps timed with CUDA events), kept for the life of the process and, once
// cl_set_tune_cache names a file, on disk across processes (tune_cache.h; the
// device's SM count and compute capability are part of the key).
namespace {
std::mutex g_tune_mu;
std::map<TuneKey, int> g_tune;
std::string g_tune_path;
}  // namespace

static cl_status tune_tile(cl_ctx* c, int N, double kIR, int* by_out) {
  int ccmaj = 0, ccmin = 0;
  CU(cudaDeviceGetAttribute(&ccmaj, cudaDevAttrComputeCapabilityMajor, c->dev));
  CU(cudaDeviceGetAttribute(&ccmin, cudaDevAttrComputeCapabilityMinor, c->dev));
  const TuneKey key(c->model, c->esz, N, c->nsm, ccmaj, ccmin);
  std::vector<int> cand = tile_candidates(c->model, c->narr, c->esz, N, c->smem_optin, ring_mown(c));
  if (cand.empty()) return fail(c, CL_EUNSUPPORTED, "no tile shape fits shared memory for N=%d", N);
  {
    std::lock_guard<std::mutex> lock(g_tune_mu);
    if (!g_tune_path.empty()) tune_cache_load(g_tune_path, g_tune);
    auto it = g_tune.find(key);
    // a height this device cannot run (an edited or foreign file) is tuned afresh
    if (it != g_tune.end() && std::find(cand.begin(), cand.end(), it->second) != cand.end()) {
      *by_out = it->second;
      return CL_OK;
    }
  }
  if (cand.size() > 4) cand.resize(4);
  int best = cand[0];
  double best_t = 1e300;
  // enough identical scratch lattices to give every SM at least 8 plane tasks
  // with the tallest tile, so that the timing reflects throughput, not latency
  const long long tasks1 = (long long)(N / cand[0]) * N;
  const long long vbytes = (long long)N * N * N * c->narr * 2 * c->esz;
  int m = (int)std::min<long long>(64, std::max<long long>(1, (8LL * c->nsm + tasks1 - 1) / tasks1));
  m = (int)std::max<long long>(1, std::min<long long>(m, (1LL << 30) / std::max<long long>(1, vbytes)));
  const std::vector<int> Ns(m, N);
  const std::vector<double> kIRs(m, kIR);
  std::vector<uint64_t> seeds(m);
  for (int i = 0; i < m; ++i) seeds[i] = 1 + i;
  for (int by : cand) {
    cl_params q = c->p;
    q.autotune = 0;
    q.tile_by = by;
    q.integrator = CL_VV2;
    q.stream = c->stream;
    cl_ctx* t = nullptr;
    cl_status s = cl_ensemble_init(&t, c->model, m, Ns.data(), kIRs.data(), c->alpha, seeds.data(), &q);
    if (s != CL_OK) return fail(c, s, "autotune: %s", cl_last_error(nullptr));
    double ms = 0.0;
    int64_t np = 0;
    s = cl_step(t, 2);
    if (s == CL_OK) s = cl_enable_pass_timing(t, 1);
    if (s == CL_OK) s = cl_step(t, 8);
    if (s == CL_OK) s = cl_pass_timing(t, &ms, &np, 1);
    if (s == CL_OK) s = cl_sync(t);
    cl_free(t);
    if (s != CL_OK) return fail(c, s, "autotune: timing failed");
    const double per = np > 0 ? ms / (double)np : 1e300;
    if (per < best_t) {
      best_t = per;
      best = by;
    }
  }
  std::lock_guard<std::mutex> lock(g_tune_mu);
  if (!g_tune_path.empty()) tune_cache_load(g_tune_path, g_tune);  // entries other processes added meanwhile
  g_tune[key] = best;
  *by_out = best;
  if (!g_tune_path.empty()) {
    if (tune_cache_store(g_tune_path, g_tune) != 0)
      return fail(c, CL_EINVAL, "autotune: cannot write the cache %s", g_tune_path.c_str());
  }
  return CL_OK;
}

namespace clg {
// Small scalar kernels (host-side setup lives here to keep the ABI in one unit).
__global__ void set_scalars_kernel(const LatConst* Lc, LatScalars* S, double eta, double a, double b) {
  if (threadIdx.x | blockIdx.x) return;
  const double al = Lc->alpha;
  S->eta = eta;
  S->a = a;
  S->b = b;
  S->cd = S->cdA = 0.0;
  S->apow1 = pow(a, 1.0 + al);
  S->apow3 = pow(a, 3.0 + al);
  S->apowm1 = pow(a, al - 1.0);
}

// a' from the Hubble law (eq. NewFriedmannEQsI) with the measured averages.
__global__ void b_from_obs_kernel(const LatConst* Lc, LatScalars* S) {
  if (threadIdx.x | blockIdx.x) return;
  const double r = pow(S->a, 2.0 * Lc->alpha + 2.0) / 3.0 * Lc->fm2 * S->obs.rho;
  S->b = r > 0.0 ? sqrt(r) : 0.0;
}
}  // namespace clg

static cl_status init_impl(cl_ctx* c, const int* Ns, const double* kIRs, const uint64_t* seeds);
static cl_status su2_init(cl_ctx* c, int N, double kIR, uint64_t seed);
static cl_status init_finish(cl_ctx* c);

extern "C" {

cl_status cl_set_tune_cache(const char* path) {
  std::lock_guard<std::mutex> lock(g_tune_mu);
  g_tune_path = path ? path : "";
  g_tune.clear();  // from here on the file is the record
  if (!g_tune_path.empty()) tune_cache_load(g_tune_path, g_tune);
  return CL_OK;
}

const char* cl_last_error(const cl_ctx* c) { return c ? c->err.c_str() : g_init_err.c_str(); }

int cl_nfields(const cl_ctx* c) {
  if (!c) return -1;
  // doublet: 4 components + 3 U(1) link fields (+ the singlet and vphi's 2 components for lphi4SU2U1)
  return c->model == CL_MODEL_SU2U1_HIGGS ? 7 : (c->model == CL_MODEL_LPHI4_SU2U1 ? 10 : c->narr / 2);
}

int cl_ensemble_size(const cl_ctx* c) { return c ? c->nlat : -1; }

int64_t cl_kernel_launches(const cl_ctx* c) { return c ? (int64_t)c->launches : -1; }

cl_status cl_free(cl_ctx* c) {
  if (!c) return CL_OK;
  cudaStreamSynchronize(c->stream);
  for (auto& pr : c->ev_pending) {
    cudaEventDestroy(pr.first);
    cudaEventDestroy(pr.second);
  }
  for (cudaEvent_t e : c->ev_pool) cudaEventDestroy(e);
  for (auto& g : c->graph_cache) cudaGraphExecDestroy(g.exec);
  for (auto& L : c->lats) cudaFree(L.slab);
  cudaFree(c->d_lat);
  cudaFree(c->d_sc);
  cudaFree(c->d_segs);
  cudaFree(c->d_cta);
  cudaFree(c->d_part);
  cudaFree(c->d_cnt);
  cudaFree(c->d_tmp);
  cudaFree(c->d_cplx);
  cudaFree(c->d_tw);
  cudaFree(c->d_spec);
  cudaFree(c->d_bin_of);
  cudaFree(c->d_geo);
  cudaFree(c->d_gsync);
  cudaFree(c->adj.lam);
  cudaFree(c->adj.d_lat);
  cudaFree(c->adj.d_segs);
  cudaFree(c->adj.d_cta);
  cudaFree(c->adj.d_part);
  cudaFree(c->adj.d_cnt);
  cudaFree(c->adj.d_out);
  for (auto& e : c->step_cache) cudaFree(e.second);
  if (c->cap_stream) cudaStreamDestroy(c->cap_stream);
  delete c;
  return CL_OK;
}

cl_status cl_ensemble_init(cl_ctx** out, int model, int count, const int* Ns, const double* kIRs,
                           double alpha, const uint64_t* seeds, const cl_params* p) {
  Range range_("cl_init");
  if (!out) return fail(nullptr, CL_EINVAL, "out is NULL");
  *out = nullptr;
  if (!p || !Ns || !kIRs || !seeds) return fail(nullptr, CL_EINVAL, "NULL argument");
  if (count < 1 || count > CL_MAX_LATTICES)
    return fail(nullptr, CL_EINVAL, "count=%d: need 1..%d lattices", count, CL_MAX_LATTICES);
  if (model < CL_MODEL_LPHI4 || model > CL_MODEL_LPHI4_SU2U1)
    return fail(nullptr, CL_EINVAL, "unknown model %d", model);
  if (is_doublet(model) && count != 1)
    return fail(nullptr, CL_EUNSUPPORTED, "the doublet model runs one lattice per context");
  for (int l = 0; l < count; ++l) {
    if (!good_N(Ns[l]))
      return fail(nullptr, CL_EINVAL, "N=%d: need 8 <= N <= 512, N %% 8 == 0, factors 2,3", Ns[l]);
    if (!(kIRs[l] > 0.0) || !std::isfinite(kIRs[l])) return fail(nullptr, CL_EINVAL, "bad kIR");
  }
  if (!std::isfinite(alpha)) return fail(nullptr, CL_EINVAL, "bad alpha");
  if (p->precision != CL_FP64 && p->precision != CL_FP32)
    return fail(nullptr, CL_EINVAL, "unknown precision %d", p->precision);
  const int ig = p->integrator;
  if (!(ig == CL_LF || ig == CL_VV2 || ig == CL_VV4 || ig == CL_VV6 || ig == CL_VV8 || ig == CL_VV10))
    return fail(nullptr, CL_EINVAL, "unknown integrator %d", ig);
  if (p->expansion < CL_EXP_OFF || p->expansion > CL_EXP_FIXED)
    return fail(nullptr, CL_EINVAL, "unknown expansion mode %d", p->expansion);
  if (!(p->dt == p->dt)) return fail(nullptr, CL_EINVAL, "dt is NaN");
  if (model == CL_MODEL_U1_HIGGS && !(p->gQ != 0.0 && std::isfinite(p->gQ) && p->fstar_over_omegastar != 0.0))
    return fail(nullptr, CL_EINVAL, "U(1) needs a finite nonzero gQ and f*/omega*");
  if (is_doublet(model) &&
      !(p->gQB != 0.0 && std::isfinite(p->gQB) && std::isfinite(p->gQ) && p->fstar_over_omegastar != 0.0))
    return fail(nullptr, CL_EINVAL, "the doublet model needs a finite nonzero gQB, a finite gQ and f*/omega*");
  if (model == CL_MODEL_LPHI4_SU2U1 && !(std::isfinite(p->qG) && std::isfinite(p->qH) && std::isfinite(p->Qc)))
    return fail(nullptr, CL_EINVAL, "lphi4SU2U1 needs finite qG, qH and Qc");
  if (is_doublet(model) && Ns[0] % 16)
    return fail(nullptr, CL_EUNSUPPORTED, "the doublet model needs N a multiple of 16");
  if (p->tile_by < 0) return fail(nullptr, CL_EINVAL, "tile_by must be >= 0");
  cl_ctx* c = new cl_ctx();
  c->model = model;
  c->nf = model == CL_MODEL_LPHI4 ? 1 : (is_doublet(model) ? 4 : 2);
  c->narr = model == CL_MODEL_U1_HIGGS ? 10
            : (model == CL_MODEL_SU2U1_HIGGS ? 35 : (model == CL_MODEL_LPHI4_SU2U1 ? 41 : 2 * c->nf));
  c->fp32 = p->precision == CL_FP32;
  c->esz = c->fp32 ? 4 : 8;
  c->nlat = count;
  c->alpha = alpha;
  c->p = *p;
  c->stream = (cudaStream_t)p->stream;
  cl_status s = init_impl(c, Ns, kIRs, seeds);
  if (s != CL_OK) {
    g_init_err = c->err;
    cl_free(c);
    return s;
  }
  *out = c;
  return CL_OK;
}

cl_status cl_init(cl_ctx** out, int model, int N, double kIR, double alpha, uint64_t seed,
                  const cl_params* p) {
  return cl_ensemble_init(out, model, 1, &N, &kIR, alpha, &seed, p);
}

}  // extern "C"

static cl_status init_impl(cl_ctx* c, const int* Ns, const double* kIRs, const uint64_t* seeds) {
  CU(cudaGetDevice(&c->dev));
  CU(cudaDeviceGetAttribute(&c->nsm, cudaDevAttrMultiProcessorCount, c->dev));
  int optin = 0;
  CU(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, c->dev));
  c->smem_optin = (size_t)optin;
  CU(cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking));
  if (is_doublet(c->model)) {
    cl_status s = su2_init(c, Ns[0], kIRs[0], seeds[0]);
    if (s != CL_OK) return s;
    return init_finish(c);
  }
  const bool u1 = c->model == CL_MODEL_U1_HIGGS;
  // lattices and their tile heights: full x-rows of N/VX threads, BY rows
  // per CTA (BY divides N); given, autotuned, or the tallest that leaves at
  // least 3 stages of BY + 2 rows of every array in shared memory
  c->lats.resize(c->nlat);
  std::vector<LatTiles> tiles;
  size_t stage = 0;
  for (int l = 0; l < c->nlat; ++l) {
    LatHost& L = c->lats[l];
    L.N = Ns[l];
    L.V = (long long)L.N * L.N * L.N;
    L.kIR = kIRs[l];
    L.dx = 2.0 * M_PI / ((double)L.N * L.kIR);
    L.seed = seeds[l];
    c->vmax = std::max(c->vmax, L.V);
    const std::vector<int> cand = tile_candidates(c->model, c->narr, c->esz, L.N, c->smem_optin, ring_mown(c));
    if (cand.empty()) return fail(c, CL_EUNSUPPORTED, "no tile shape fits shared memory for N=%d", L.N);
    if (c->p.tile_by > 0) {
      if (std::find(cand.begin(), cand.end(), c->p.tile_by) == cand.end())
        return fail(c, CL_EINVAL, "tile_by=%d is not a tile height for N=%d", c->p.tile_by, L.N);
      L.BY = c->p.tile_by;
    } else if (c->p.autotune) {
      cl_status s = tune_tile(c, L.N, L.kIR, &L.BY);
      if (s != CL_OK) return s;
    } else {
      L.BY = cand[0];
    }
    tiles.push_back(LatTiles{L.N, L.BY, THREADS * tile_vx(c->model, c->esz)});
  }
  // work list: one CTA per SM, at least 8 plane tasks each
  long long tasks = 0;
  for (const LatTiles& t : tiles) tasks += (long long)(t.N / t.BY) * t.N;
  c->grid = (int)std::max<long long>(1, std::min<long long>(c->nsm, tasks / 8));
  std::vector<Seg> segs;
  std::vector<int> cta, sbeg, send;
  if (!build_worklist(tiles, c->grid, u1, segs, cta, sbeg, send)) {
    // tuned tiles too short for this mix of sizes: the tallest admissible ones
    bool ok = false;
    if (c->p.autotune && c->p.tile_by == 0) {
      for (int l = 0; l < c->nlat; ++l) {
        c->lats[l].BY = tile_candidates(c->model, c->narr, c->esz, c->lats[l].N, c->smem_optin, ring_mown(c))[0];
        tiles[l].BY = c->lats[l].BY;
      }
      ok = build_worklist(tiles, c->grid, u1, segs, cta, sbeg, send);
    }
    if (!ok)
      return fail(c, CL_EUNSUPPORTED, "work split needs more than %d segments per CTA", MAX_SEG_PER_CTA);
  }
  c->nseg = (int)segs.size();
  c->nslot = send[c->nlat - 1];
  // stage ring: the largest lattice stage, as many stages (3 .. 6) as fit
  for (const LatHost& L : c->lats) stage = std::max(stage, stage_size(L.N, L.BY, c->narr, c->esz, ring_mown(c)));
  const int S = (int)std::min<size_t>(6, (c->smem_optin - SM_TAIL_BYTES) / stage);
  if (S < 3) return fail(c, CL_EUNSUPPORTED, "shared memory too small for the stage ring");
  c->stages = S;
  c->stage_bytes = (unsigned)stage;
  c->smem_bytes = (size_t)S * stage + SM_TAIL_BYTES;
  for (int red = 0; red < 3; ++red) {
    PassKernel k = pick_kernel(c, red);
    if (!k && red == 1 && red_for_step(c) == 0) continue;  // Friedmann sums never taken here
    if (!k) return fail(c, CL_EUNSUPPORTED, "no pass kernel for this configuration");
    CU(cudaFuncSetAttribute((const void*)k, cudaFuncAttributeMaxDynamicSharedMemorySize,
                            (int)c->smem_bytes));
  }
  // device memory
  for (int l = 0; l < c->nlat; ++l) {
    LatHost& L = c->lats[l];
    const size_t bytes = 2 * (size_t)c->narr * L.V * c->esz;
    CU(cudaMalloc(&L.slab, bytes));
    CU(cudaMemsetAsync(L.slab, 0, bytes, c->stream));
  }
  CU(cudaMalloc(&c->d_lat, c->nlat * sizeof(LatConst)));
  CU(cudaMalloc(&c->d_sc, c->nlat * sizeof(LatScalars)));
  CU(cudaMemsetAsync(c->d_sc, 0, c->nlat * sizeof(LatScalars), c->stream));
  CU(cudaMalloc(&c->d_segs, segs.size() * sizeof(Seg)));
  CU(cudaMalloc(&c->d_cta, cta.size() * sizeof(int)));
  CU(cudaMalloc(&c->d_part, (size_t)c->nslot * NQ * sizeof(double)));
  CU(cudaMalloc(&c->d_cnt, c->nlat * sizeof(unsigned)));
  CU(cudaMemsetAsync(c->d_cnt, 0, c->nlat * sizeof(unsigned), c->stream));
  CU(cudaMalloc(&c->d_gsync, 2 * sizeof(unsigned)));
  {
    int coop = 0, nb = 0;
    CU(cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, c->dev));
    CU(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, (const void*)pick_kernel(c, red_for_step(c)),
                                                     THREADS, c->smem_bytes));
    c->coop = coop && (long long)nb * c->nsm >= c->grid;
  }
  c->hlat.resize(c->nlat);
  for (int l = 0; l < c->nlat; ++l) {
    const LatHost& H = c->lats[l];
    LatConst& L = c->hlat[l];
    memset(&L, 0, sizeof(L));
    L.N = H.N;
    L.BY = H.BY;
    L.YT = H.N / H.BY;
    L.model = c->model;
    L.nf = c->nf;
    L.narr = c->narr;
    L.expansion = c->p.expansion;
    L.slot_begin = sbeg[l];
    L.slot_end = send[l];
    L.esz = c->esz;
    L.int_alpha = (c->alpha == std::floor(c->alpha) && std::fabs(c->alpha) <= 4.0) ? 1 : 0;
    L.alpha_i = L.int_alpha ? (int)c->alpha : 0;
    L.inv_V = 1.0 / (double)H.V;
    L.inv_dx2 = 1.0 / (H.dx * H.dx);
    if (u1) {
      L.u1_gd = c->p.gQ * H.dx;
      L.u1_cJ = c->p.fstar_over_omegastar * c->p.fstar_over_omegastar * c->p.gQ / H.dx;
      L.u1_cC = 1.0 / (c->p.gQ * H.dx * H.dx * H.dx);
    }
    L.V = H.V;
    L.dx = H.dx;
    L.alpha = c->alpha;
    L.q = c->p.q;
    L.lam = c->p.lam;
    L.v = c->p.v;
    L.gQ = c->p.gQ;
    L.fo2 = c->p.fstar_over_omegastar * c->p.fstar_over_omegastar;
    L.fm2 = c->p.fstar_over_mp * c->p.fstar_over_mp;
    L.omega_eos = c->p.omega_eos;
    // one slab per lattice: array a of buffer p starts a * V values after
    // array 0 of that buffer (the U(1) pass relies on it)
    for (int par = 0; par < 2; ++par)
      for (int a = 0; a < c->narr; ++a) L.buf[par][a] = arr_ptr(c, l, par, a);
  }
  CU(cudaMemcpyAsync(c->d_lat, c->hlat.data(), c->nlat * sizeof(LatConst), cudaMemcpyHostToDevice,
                     c->stream));
  CU(cudaMemcpyAsync(c->d_segs, segs.data(), segs.size() * sizeof(Seg), cudaMemcpyHostToDevice, c->stream));
  CU(cudaMemcpyAsync(c->d_cta, cta.data(), cta.size() * sizeof(int), cudaMemcpyHostToDevice, c->stream));
  // initial conditions, lattice by lattice
  CU(cudaMalloc(&c->d_cplx, 2 * (size_t)c->vmax * sizeof(double2)));
  CU(cudaMalloc(&c->d_tw, 512 * sizeof(double2)));
  CU(cudaMalloc(&c->d_tmp, std::max<size_t>((size_t)c->vmax, 1 << 16) * sizeof(double)));
  for (int l = 0; l < c->nlat; ++l) {
    const LatHost& H = c->lats[l];
    const LatConst* dL = c->d_lat + l;
    LatScalars* dS = c->d_sc + l;
    ICArgs A;
    memset(&A, 0, sizeof(A));
    for (int k = 0; k < 4; ++k) {
      A.phi0[k] = c->p.phi0[k];
      A.dphi0[k] = c->p.dphi0[k];
    }
    A.amp2 = c->p.fluct_amp2;
    A.kcut = c->p.kcut;
    A.kIR = H.kIR;
    A.H0 = c->p.H0;
    A.q = c->p.q;
    A.lam = c->p.lam;
    A.v = c->p.v;
    A.seed = H.seed;
    A.model = c->model;
    A.nf = c->nf;
    c->lats[l].ic = A;
    CU(launch_init_scalars(dL, dS, A, c->stream));
    ++c->launches;
    double2* F = c->d_cplx;
    double2* G = c->d_cplx + H.V;
    for (int f = 0; f < c->nf; ++f) {
      CU(cudaMemsetAsync(c->d_cplx, 0, 2 * (size_t)H.V * sizeof(double2), c->stream));
      CU(launch_ic_modes(F, G, dL, dS, A, f, H.V, c->stream));
      ++c->launches;
      cl_status s = fft3d(c, H.N, F, +1);
      if (s != CL_OK) return s;
      s = fft3d(c, H.N, G, +1);
      if (s != CL_OK) return s;
      CU(launch_ic_assemble(c->fp32, arr_ptr(c, l, 0, 2 * f), arr_ptr(c, l, 0, 2 * f + 1), F, G, dL, dS,
                            c->p.phi0[f], c->p.dphi0[f], H.V, c->stream));
      ++c->launches;
    }
    if (u1) {
      // links start at zero (eq. Inflc1); their momenta solve the lattice Gauss law
      double2* rho = c->d_cplx;
      double2* E = c->d_cplx + H.V;
      CU(launch_u1_gauss_init(dL, 0, rho, E, H.N, 0, H.dx, c->fp32, nullptr, H.V, 0, c->stream));
      ++c->launches;
      cl_status s = fft3d(c, H.N, rho, -1);
      if (s != CL_OK) return s;
      for (int i = 0; i < 3; ++i) {
        CU(launch_u1_gauss_init(dL, 0, rho, E, H.N, i, H.dx, c->fp32, nullptr, H.V, 1, c->stream));
        ++c->launches;
        s = fft3d(c, H.N, E, +1);
        if (s != CL_OK) return s;
        CU(launch_u1_gauss_init(dL, 0, rho, E, H.N, i, H.dx, c->fp32, arr_ptr(c, l, 0, 2 * (2 + i) + 1),
                                H.V, 2, c->stream));
        ++c->launches;
      }
    }
  }
  return init_finish(c);
}

// Initial measurement (and, with b0_mode 1, a' from the lattice averages).
static cl_status init_finish(cl_ctx* c) {
  c->parity = 0;
  c->open = false;
  cl_status s = measure(c, 1);
  if (s != CL_OK) return s;
  if (c->p.expansion == CL_EXP_SELF && c->p.b0_mode == 1) {
    for (int l = 0; l < c->nlat; ++l) {
      b_from_obs_kernel<<<1, 32, 0, c->stream>>>(c->d_lat + l, c->d_sc + l);
      CHECK_LAUNCH();
      ++c->launches;
    }
    c->obs_valid = false;
    s = measure(c, 1);
    if (s != CL_OK) return s;
  }
  CU(cudaStreamSynchronize(c->stream));
  return check_status(c);
}


// Doublet model: one lattice, 35 arrays per buffer; the pass tiles x-y by
// TX x TY (TX = 32, or 16 when N is not a multiple of 32; TY = 8), cuts z into
// chunks and runs the resident CTAs over the (tile, chunk) items.  Initial conditions: the doublet's four
// components drawn like the U(1) field's (eqs. InConstr:1-2 for n = 0..3),
// links at the identity (eqs. Inflc1-2), and link momenta solving the U(1)
// and the three SU(2) lattice Gauss laws (eq. GaugeCurrentFluc with the
// backward-difference symbol; at the identity the laws are linear).
static cl_status su2_init(cl_ctx* c, int N, double kIR, uint64_t seed) {
  c->lats.resize(1);
  LatHost& H = c->lats[0];
  H.N = N;
  H.V = (long long)N * N * N;
  H.kIR = kIR;
  H.dx = 2.0 * M_PI / ((double)N * kIR);
  H.seed = seed;
  H.BY = 0;
  c->vmax = H.V;
  c->su2_tx = N % 32 == 0 ? 32 : 16;
  c->su2_ty = 8;
  const int full = c->model == CL_MODEL_LPHI4_SU2U1;
  // the FP32 lphi4SU2U1 step pass without expansion takes 32 x 16 tiles: one
  // 512-thread CTA per SM, with room for its momentum slot beside three stages
  c->su2_kd_ty = 8;
  if (full && c->fp32 && c->su2_tx == 32 && N % 16 == 0) {
    cudaFuncAttributes fa;
    CU(cudaFuncGetAttributes(&fa, (const void*)su2_kd_pass_kernel(1, 0, 32, 16, 1, 0)));
    if (su2_kd_smem_bytes(32, 16, 4, 1) + fa.sharedSizeBytes <= c->smem_optin) c->su2_kd_ty = 16;
  }
  c->smem_bytes = su2_smem_bytes(c->su2_tx, c->su2_ty, c->esz, full);
  if (std::max(c->smem_bytes, std::max(su2_launch_smem(c, 0), su2_launch_smem(c, 2))) > c->smem_optin)
    return fail(c, CL_EUNSUPPORTED, "shared memory too small for the pass");
  int smax = 0;
  CU(cudaDeviceGetAttribute(&smax, cudaDevAttrMaxSharedMemoryPerMultiprocessor, c->dev));
  for (int red = 0; red < 3; ++red) {
    CU(cudaFuncSetAttribute((const void*)su2_pass_kernel(c->fp32, red, c->su2_tx, full),
                            cudaFuncAttributeMaxDynamicSharedMemorySize, (int)c->smem_bytes));
    if (red != 1) {
      const int ty = kd_ty(c, red);
      const size_t sm = su2_kd_smem_bytes(c->su2_tx, ty, c->esz, full);
      const void* kk = (const void*)su2_kd_pass_kernel(c->fp32, red, c->su2_tx, ty, full, kd_n256(c, red));
      CU(cudaFuncSetAttribute(kk, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
      // the smallest shared-memory carve-out that holds the resident CTAs, so that
      // the rest of the SM's storage caches what the pass reads through L1
      cudaFuncAttributes fa;
      CU(cudaFuncGetAttributes(&fa, kk));
      const int per_cta = (int)(sm + fa.sharedSizeBytes) + 1024;
      const int by_regs = 65536 / std::max(1, fa.numRegs * c->su2_tx * ty);
      const int ctas = std::max(1, std::min(smax / per_cta, by_regs));
      const int pct = std::min(100, (int)((100LL * ctas * per_cta + smax - 1) / smax));
      CU(cudaFuncSetAttribute(kk, cudaFuncAttributePreferredSharedMemoryCarveout, pct));
    }
  }
  int nb = 0;
  const int rs = red_for_step(c);
  CU(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, (const void*)pick_kernel(c, rs),
                                                   c->su2_tx * su2_launch_ty(c, rs), su2_launch_smem(c, rs)));
  // work items (tile, z-chunk) over the resident CTAs (su2_work.h)
  const int ntiles = (N / c->su2_tx) * (N / su2_launch_ty(c, rs));
  const int R = c->nsm * std::max(nb, 1);
  const int nzc = su2_z_chunks(ntiles, N, R);
  c->grid = std::min(R, ntiles * nzc);
  c->nslot = c->grid;
  c->stages = 3;
  c->coop = false;
  const size_t bytes = 2 * (size_t)c->narr * H.V * c->esz;
  CU(cudaMalloc(&H.slab, bytes));
  CU(cudaMemsetAsync(H.slab, 0, bytes, c->stream));
  CU(cudaMalloc(&c->d_lat, sizeof(LatConst)));
  CU(cudaMalloc(&c->d_sc, sizeof(LatScalars)));
  CU(cudaMemsetAsync(c->d_sc, 0, sizeof(LatScalars), c->stream));
  CU(cudaMalloc(&c->d_part, (size_t)SU2_PARTIALS * c->grid * sizeof(double)));
  CU(cudaMalloc(&c->d_cnt, sizeof(unsigned)));
  CU(cudaMemsetAsync(c->d_cnt, 0, sizeof(unsigned), c->stream));
  c->hlat.resize(1);
  LatConst& L = c->hlat[0];
  memset(&L, 0, sizeof(L));
  L.N = N;
  L.model = c->model;
  L.nf = c->nf;
  L.narr = c->narr;
  L.expansion = c->p.expansion;
  L.slot_begin = 0;
  L.slot_end = c->grid;
  L.esz = c->esz;
  L.int_alpha = (c->alpha == std::floor(c->alpha) && std::fabs(c->alpha) <= 4.0) ? 1 : 0;
  L.alpha_i = L.int_alpha ? (int)c->alpha : 0;
  L.inv_V = 1.0 / (double)H.V;
  L.inv_dx2 = 1.0 / (H.dx * H.dx);
  L.V = H.V;
  L.dx = H.dx;
  L.alpha = c->alpha;
  L.q = c->p.q;
  L.lam = c->p.lam;
  L.v = c->p.v;
  L.gQ = c->p.gQ;
  L.gQB = c->p.gQB;
  L.qG = c->p.qG;
  L.qH = c->p.qH;
  L.Qc = c->p.Qc;
  L.su2_nzc = nzc;
  L.fo2 = c->p.fstar_over_omegastar * c->p.fstar_over_omegastar;
  L.fm2 = c->p.fstar_over_mp * c->p.fstar_over_mp;
  L.omega_eos = c->p.omega_eos;
  // the pass addresses array a of buffer p at buf[p][0] + a V
  for (int par = 0; par < 2; ++par)
    for (int a = 0; a < MAX_ARR; ++a) L.buf[par][a] = arr_ptr(c, 0, par, a);
  CU(cudaMemcpyAsync(c->d_lat, &L, sizeof(LatConst), cudaMemcpyHostToDevice, c->stream));
  CU(cudaMalloc(&c->d_cplx, 2 * (size_t)H.V * sizeof(double2)));
  CU(cudaMalloc(&c->d_tw, 512 * sizeof(double2)));
  CU(cudaMalloc(&c->d_tmp, std::max<size_t>((size_t)H.V, 1 << 16) * sizeof(double)));
  ICArgs A;
  memset(&A, 0, sizeof(A));
  for (int k = 0; k < 4; ++k) {
    A.phi0[k] = c->p.phi0[k];
    A.dphi0[k] = c->p.dphi0[k];
  }
  A.amp2 = c->p.fluct_amp2;
  A.kcut = c->p.kcut;
  A.kIR = H.kIR;
  A.H0 = c->p.H0;
  A.q = c->p.q;
  A.lam = c->p.lam;
  A.v = c->p.v;
  A.seed = H.seed;
  A.model = c->model;
  A.nf = c->nf;
  A.qG = c->p.qG;
  A.qH = c->p.qH;
  H.ic = A;
  CU(launch_init_scalars(c->d_lat, c->d_sc, A, c->stream));
  ++c->launches;
  double2* F = c->d_cplx;
  double2* G = c->d_cplx + H.V;
  // components: the doublet's four, and for lphi4SU2U1 the singlet (4) and vphi (5, 6),
  // which start at zero homogeneous values
  for (int f = 0; f < (full ? 7 : 4); ++f) {
    CU(cudaMemsetAsync(c->d_cplx, 0, 2 * (size_t)H.V * sizeof(double2), c->stream));
    CU(launch_ic_modes(F, G, c->d_lat, c->d_sc, A, f, H.V, c->stream));
    ++c->launches;
    cl_status s = fft3d(c, N, F, +1);
    if (s != CL_OK) return s;
    s = fft3d(c, N, G, +1);
    if (s != CL_OK) return s;
    const int af = f < 4 ? f : (f == 4 ? 35 : 37 + (f - 5));
    const int ap = f < 4 ? 4 + f : (f == 4 ? 36 : 39 + (f - 5));
    CU(launch_ic_assemble(c->fp32, arr_ptr(c, 0, 0, af), arr_ptr(c, 0, 0, ap), F, G, c->d_lat, c->d_sc,
                          f < 4 ? c->p.phi0[f] : 0.0, f < 4 ? c->p.dphi0[f] : 0.0, H.V, c->stream));
    ++c->launches;
  }
  CU(launch_su2_identity_links(c->fp32, arr_ptr(c, 0, 0, 0), H.V, c->stream));
  ++c->launches;
  double2* rho = c->d_cplx;
  double2* E = c->d_cplx + H.V;
  for (int g = 0; g < 4; ++g) {
    if (g == 0 && c->p.gQ == 0.0) continue;  // no U(1) field: its momenta stay zero
    CU(launch_su2_rho(c->fp32, c->d_lat, 0, g, rho, H.V, c->stream));
    ++c->launches;
    cl_status s = fft3d(c, N, rho, -1);
    if (s != CL_OK) return s;
    for (int i = 0; i < 3; ++i) {
      CU(launch_u1_gauss_init(c->d_lat, 0, rho, E, N, i, H.dx, c->fp32, nullptr, H.V, 1, c->stream));
      ++c->launches;
      s = fft3d(c, N, E, +1);
      if (s != CL_OK) return s;
      const int a = g == 0 ? 11 + i : 26 + 3 * i + (g - 1);
      CU(launch_u1_gauss_init(c->d_lat, 0, rho, E, N, i, H.dx, c->fp32, arr_ptr(c, 0, 0, a), H.V, 2,
                              c->stream));
      ++c->launches;
    }
  }
  return CL_OK;
}

extern "C" {

cl_status cl_step_h(cl_ctx* c, int n, double h) {
  Range range_("cl_step");
  if (!c) return fail(nullptr, CL_EINVAL, "ctx is NULL");
  if (n < 0 || !std::isfinite(h)) return fail(c, CL_EINVAL, "bad n/h");
  if (n == 0) return CL_OK;
  const int red = red_for_step(c);
  std::vector<PassStep> steps;
  append_pass_steps(c->p.integrator, h, n, c->open, c->dprev, steps);
  const int chunk = 4096;
  for (size_t b = 0; b < steps.size(); b += chunk) {
    const int m = (int)std::min<size_t>(chunk, steps.size() - b);
    cl_status st = launch_passes(c, steps.data() + b, m, red, 1, 0);
    if (st != CL_OK) return st;
  }
  c->obs_valid = false;
  return CL_OK;
}

cl_status cl_pass_weights(int integrator, double h, int ncalls, const int* steps_per_call, double* out, int cap,
                          int* npass) {
  if (!steps_per_call || !out || !npass || ncalls < 0 || !std::isfinite(h)) return CL_EINVAL;
  if (integrator != CL_LF && integrator != CL_VV2 && integrator != CL_VV4 && integrator != CL_VV6 &&
      integrator != CL_VV8 && integrator != CL_VV10)
    return CL_EINVAL;
  bool open = false;
  double dprev = 0.0;
  std::vector<PassStep> steps;
  for (int i = 0; i < ncalls; ++i) {
    if (steps_per_call[i] < 0 || steps_per_call[i] > (1 << 20)) return CL_EINVAL;
    append_pass_steps(integrator, h, steps_per_call[i], open, dprev, steps);
  }
  if (open) steps.push_back(closing_pass_step(dprev));
  *npass = (int)steps.size();
  if ((int)steps.size() > cap) return CL_EINVAL;
  for (size_t j = 0; j < steps.size(); ++j) {
    out[4 * j + 0] = steps[j].ck;
    out[4 * j + 1] = steps[j].wout;
    out[4 * j + 2] = steps[j].win;
    out[4 * j + 3] = steps[j].dnext;
  }
  return CL_OK;
}

cl_status cl_step(cl_ctx* c, int n) {
  if (!c) return fail(nullptr, CL_EINVAL, "ctx is NULL");
  return cl_step_h(c, n, c->p.dt);
}

cl_status cl_sync(cl_ctx* c) {
  if (!c) return fail(nullptr, CL_EINVAL, "ctx is NULL");
  return close_stream(c);
}

static cl_status bad_lat(cl_ctx* c, int lat) {
  return fail(c, CL_EINVAL, "lattice %d out of range (ensemble of %d)", lat, c->nlat);
}

cl_status cl_lattice_energies(cl_ctx* c, int lat, cl_energies_t* out) {
  Range range_("cl_energies");
  if (!c || !out) return fail(c, CL_EINVAL, "NULL argument");
  if (lat < 0 || lat >= c->nlat) return bad_lat(c, lat);
  cl_status s = measure(c, 0);
  if (s != CL_OK) return s;
  CU(cudaMemcpyAsync(out, &c->d_sc[lat].obs, sizeof(cl_energies_t), cudaMemcpyDeviceToHost, c->stream));
  s = check_status(c);
  if (s != CL_OK) return s;
  if (out->nonfinite > 0) return fail(c, CL_ENONFINITE, "%lld non-finite momenta", (long long)out->nonfinite);
  return CL_OK;
}

cl_status cl_energies(cl_ctx* c, cl_energies_t* out) { return cl_lattice_energies(c, 0, out); }

static cl_status array_index(cl_ctx* c, int field, int what, int* a) {
  if (what != 0 && what != 1) return fail(c, CL_EINVAL, "what must be 0 or 1");
  if (c->model == CL_MODEL_LPHI4_SU2U1 && field >= 7 && field <= 9) {  // singlet 7, vphi 8, 9
    *a = field == 7 ? 35 + what : 37 + (field - 8) + 2 * what;
    return CL_OK;
  }
  if (is_doublet(c->model)) {  // doublet components 0..3, U(1) link fields 4..6
    if (field < 0 || field > 6) return fail(c, CL_EINVAL, "field %d out of range", field);
    *a = field < 4 ? field + 4 * what : 8 + (field - 4) + 3 * what;
    return CL_OK;
  }
  if (field < 0 || field >= c->narr / 2) return fail(c, CL_EINVAL, "field %d out of range", field);
  *a = 2 * field + what;
  return CL_OK;
}

// Array a of lattice 0 to / from the host (FP64), converting the storage precision.
static cl_status copy_array(cl_ctx* c, int a, double* host_out, const double* host_in) {
  cl_status s = close_stream(c);
  if (s != CL_OK) return s;
  const long long V = c->lats[0].V;
  if (host_out) {
    CU(launch_convert(c->fp32, 1, arr_ptr(c, 0, c->parity, a), c->d_tmp, V, c->stream));
    ++c->launches;
    CU(cudaMemcpyAsync(host_out, c->d_tmp, (size_t)V * sizeof(double), cudaMemcpyDefault, c->stream));
    CU(cudaStreamSynchronize(c->stream));
    return check_status(c);
  }
  CU(cudaMemcpyAsync(c->d_tmp, host_in, (size_t)V * sizeof(double), cudaMemcpyDefault, c->stream));
  CU(launch_convert(c->fp32, 0, c->d_tmp, arr_ptr(c, 0, c->parity, a), V, c->stream));
  ++c->launches;
  CU(cudaStreamSynchronize(c->stream));
  c->obs_valid = false;
  return CL_OK;
}

cl_status cl_lattice_get_state(cl_ctx* c, int lat, int field, int what, double* host_out) {
  if (!c || !host_out) return fail(c, CL_EINVAL, "NULL argument");
  if (lat < 0 || lat >= c->nlat) return bad_lat(c, lat);
  int a = 0;
  cl_status s = array_index(c, field, what, &a);
  if (s != CL_OK) return s;
  s = close_stream(c);
  if (s != CL_OK) return s;
  const long long V = c->lats[lat].V;
  CU(launch_convert(c->fp32, 1, arr_ptr(c, lat, c->parity, a), c->d_tmp, V, c->stream));
  ++c->launches;
  CU(cudaMemcpyAsync(host_out, c->d_tmp, (size_t)V * sizeof(double), cudaMemcpyDefault, c->stream));
  CU(cudaStreamSynchronize(c->stream));
  return check_status(c);
}

cl_status cl_lattice_set_state(cl_ctx* c, int lat, int field, int what, const double* host_in) {
  if (!c || !host_in) return fail(c, CL_EINVAL, "NULL argument");
  if (lat < 0 || lat >= c->nlat) return bad_lat(c, lat);
  int a = 0;
  cl_status s = array_index(c, field, what, &a);
  if (s != CL_OK) return s;
  s = close_stream(c);
  if (s != CL_OK) return s;
  const long long V = c->lats[lat].V;
  CU(cudaMemcpyAsync(c->d_tmp, host_in, (size_t)V * sizeof(double), cudaMemcpyDefault, c->stream));
  CU(launch_convert(c->fp32, 0, c->d_tmp, arr_ptr(c, lat, c->parity, a), V, c->stream));
  ++c->launches;
  CU(cudaStreamSynchronize(c->stream));
  c->obs_valid = false;
  return CL_OK;
}

cl_status cl_get_state(cl_ctx* c, int field, int what, double* host_out) {
  return cl_lattice_get_state(c, 0, field, what, host_out);
}

cl_status cl_get_array(cl_ctx* c, int a, double* host_out) {
  if (!c || !host_out) return fail(c, CL_EINVAL, "NULL argument");
  if (!is_doublet(c->model)) return fail(c, CL_EUNSUPPORTED, "array access is for the doublet models");
  if (a < 0 || a >= c->narr) return fail(c, CL_EINVAL, "array %d out of range", a);
  return copy_array(c, a, host_out, nullptr);
}

cl_status cl_set_array(cl_ctx* c, int a, const double* host_in) {
  if (!c || !host_in) return fail(c, CL_EINVAL, "NULL argument");
  if (!is_doublet(c->model)) return fail(c, CL_EUNSUPPORTED, "array access is for the doublet models");
  if (a < 0 || a >= c->narr) return fail(c, CL_EINVAL, "array %d out of range", a);
  return copy_array(c, a, nullptr, host_in);
}

cl_status cl_set_state(cl_ctx* c, int field, int what, const double* host_in) {
  return cl_lattice_set_state(c, 0, field, what, host_in);
}

cl_status cl_lattice_scalars(cl_ctx* c, int lat, double* eta, double* a, double* b) {
  if (!c) return fail(nullptr, CL_EINVAL, "ctx is NULL");
  if (lat < 0 || lat >= c->nlat) return bad_lat(c, lat);
  cl_status s = close_stream(c);
  if (s != CL_OK) return s;
  double v[3];
  CU(cudaMemcpyAsync(v, &c->d_sc[lat], 3 * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  CU(cudaStreamSynchronize(c->stream));
  if (a) *a = v[0];
  if (b) *b = v[1];
  if (eta) *eta = v[2];
  return check_status(c);
}

cl_status cl_get_scalars(cl_ctx* c, double* eta, double* a, double* b) {
  return cl_lattice_scalars(c, 0, eta, a, b);
}

cl_status cl_set_scalars(cl_ctx* c, double eta, double a, double b) {
  if (!c) return fail(nullptr, CL_EINVAL, "ctx is NULL");
  if (!(a > 0.0)) return fail(c, CL_EINVAL, "a must be positive");
  cl_status s = close_stream(c);
  if (s != CL_OK) return s;
  for (int l = 0; l < c->nlat; ++l) {
    set_scalars_kernel<<<1, 32, 0, c->stream>>>(c->d_lat + l, c->d_sc + l, eta, a, b);
    CHECK_LAUNCH();
    ++c->launches;
  }
  c->obs_valid = false;
  s = measure(c, 1);
  if (s != CL_OK) return s;
  CU(cudaStreamSynchronize(c->stream));
  return check_status(c);
}

cl_status cl_lattice_tile(cl_ctx* c, int lat, int* N, int* BY, int* stages) {
  if (!c) return fail(nullptr, CL_EINVAL, "ctx is NULL");
  if (lat < 0 || lat >= c->nlat) return bad_lat(c, lat);
  if (N) *N = c->lats[lat].N;
  if (BY) *BY = c->lats[lat].BY;
  if (stages) *stages = c->stages;
  return CL_OK;
}

cl_status cl_ensemble_spectrum(cl_ctx* c, const int* lats, int nl, int field, int what, double dk_bin,
                               double* k, double* delta, int64_t* mult, int cap, int* nbins) {
  if (!c || !lats || !k || !delta || !mult || !nbins) return fail(c, CL_EINVAL, "NULL argument");
  if (nl < 1 || nl > c->nlat) return fail(c, CL_EINVAL, "need 1..%d lattices", c->nlat);
  if (!(dk_bin > 0.0)) return fail(c, CL_EINVAL, "dk_bin must be positive");
  for (int i = 0; i < nl; ++i) {
    if (lats[i] < 0 || lats[i] >= c->nlat) return bad_lat(c, lats[i]);
    const LatHost& A = c->lats[lats[i]];
    const LatHost& B = c->lats[lats[0]];
    if (A.N != B.N || A.kIR != B.kIR) return fail(c, CL_EINVAL, "averaged lattices differ in N or kIR");
  }
  int a = 0;
  cl_status s = array_index(c, field, what, &a);
  if (s != CL_OK) return s;
  const LatHost& H = c->lats[lats[0]];
  const int nb = (int)std::floor(std::sqrt(3.0) * (H.N / 2) / dk_bin) + 1;
  *nbins = nb;
  if (nb > cap) return fail(c, CL_EINVAL, "cap %d < %d bins", cap, nb);
  if (nb > 2048) return fail(c, CL_EINVAL, "too many bins (dk_bin too small)");
  s = close_stream(c);
  if (s != CL_OK) return s;
  const int nblk = 2 * c->nsm;
  if (c->spec_lats < nl) {
    CU(cudaStreamSynchronize(c->stream));
    cudaFree(c->d_spec);
    c->d_spec = nullptr;
    c->spec_lats = 0;
    CU(cudaMalloc(&c->d_spec, ((size_t)3 * 2048 * nblk + (size_t)(nl + 1) * 3 * 2048) * sizeof(double)));
    c->spec_lats = nl;
  }
  double* part = c->d_spec;
  double* bins = c->d_spec + (size_t)3 * 2048 * nblk;  // [nl][3 nb]: k, delta, mult
  double* mean = bins + (size_t)nl * 3 * nb;
  double2* F = c->d_cplx;
  // real fields: the half spectrum (row pairs along x, then the N/2 + 1 columns kept along y and z)
  FftPlan pl;
  pl.N = H.N;
  pl.sign = -1;
  pl.batch = fft_batch(H.N);
  pl.tw = c->d_tw;
  pl.pitch = pl.nu = H.N;
  pl.axis = 0;
  fft_radices(H.N, pl);
  CU(launch_fft_twiddles(c->d_tw, H.N, c->stream));
  ++c->launches;
  if (c->geo_N != H.N || c->geo_dk != dk_bin) {  // the shells of (N, dk_bin), kept for later calls
    CU(cudaStreamSynchronize(c->stream));
    cudaFree(c->d_bin_of);
    c->d_bin_of = nullptr;
    c->geo_N = 0;
    if (!c->d_geo) CU(cudaMalloc(&c->d_geo, 2 * 2048 * sizeof(double)));
    CU(cudaMalloc(&c->d_bin_of, ((size_t)3 * (H.N / 2) * (H.N / 2) + 1) * sizeof(int)));
    CU(launch_shell_geometry(H.N, dk_bin, nb, nblk, c->d_bin_of, c->d_geo, part, c->stream));
    c->launches += 3;
    c->geo_N = H.N;
    c->geo_dk = dk_bin;
  }
  for (int i = 0; i < nl; ++i) {
    const int l = lats[i];
    CU(launch_real_spectrum(c->fp32, arr_ptr(c, l, c->parity, a), F, pl, dk_bin, nb, nblk, part, H.kIR, H.dx,
                            bins + (size_t)i * 3 * nb, c->stream, c->d_bin_of, c->d_geo));
    c->launches += 5;
  }
  CU(launch_spec_mean(bins, nl, nb, mean, c->stream));
  ++c->launches;
  std::vector<double> h(3 * nb);
  CU(cudaMemcpyAsync(h.data(), mean, 3 * nb * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  CU(cudaStreamSynchronize(c->stream));
  for (int b = 0; b < nb; ++b) {
    k[b] = h[b];
    delta[b] = h[nb + b];
    mult[b] = (int64_t)h[2 * nb + b];
  }
  return check_status(c);
}

cl_status cl_spectrum(cl_ctx* c, int field, int what, double dk_bin, double* k, double* delta,
                      int64_t* mult, int cap, int* nbins) {
  Range range_("cl_spectrum");
  const int l0 = 0;
  return cl_ensemble_spectrum(c, &l0, 1, field, what, dk_bin, k, delta, mult, cap, nbins);
}

cl_status cl_occupation(cl_ctx* c, int field, double dk_bin, double fo2, double* k, double* n, int64_t* mult,
                        int cap, int* nbins) {
  Range range_("cl_occupation");
  if (!c || !k || !n || !mult || !nbins) return fail(c, CL_EINVAL, "NULL argument");
  if (c->nlat != 1 || c->model >= CL_MODEL_U1_HIGGS)
    return fail(c, CL_EUNSUPPORTED, "occupation numbers cover single scalar lattices");
  if (field < 0 || field >= c->nf) return fail(c, CL_EINVAL, "field %d out of range", field);
  if (!(dk_bin > 0.0)) return fail(c, CL_EINVAL, "dk_bin must be positive");
  if (!(fo2 > 0.0)) {
    if (!(c->p.fluct_amp2 > 0.0)) return fail(c, CL_EINVAL, "need (f*/omega*)^2 > 0 (fluct_amp2 is 0)");
    fo2 = 1.0 / c->p.fluct_amp2;
  }
  const LatHost& H = c->lats[0];
  const int nb = (int)std::floor(std::sqrt(3.0) * (H.N / 2) / dk_bin) + 1;
  *nbins = nb;
  if (nb > cap) return fail(c, CL_EINVAL, "cap %d < %d bins", cap, nb);
  if (nb > 2048) return fail(c, CL_EINVAL, "too many bins (dk_bin too small)");
  cl_status s = measure(c, 0);  // the synchronised state and its volume averages
  if (s != CL_OK) return s;
  LatScalars S;
  CU(cudaMemcpyAsync(&S, &c->d_sc[0], sizeof(S), cudaMemcpyDeviceToHost, c->stream));
  const int nblk = 2 * c->nsm;
  if (c->spec_lats < 1) {
    CU(cudaStreamSynchronize(c->stream));
    cudaFree(c->d_spec);
    c->d_spec = nullptr;
    CU(cudaMalloc(&c->d_spec, ((size_t)3 * 2048 * nblk + (size_t)2 * 3 * 2048) * sizeof(double)));
    c->spec_lats = 1;
  }
  double* part = c->d_spec;
  double* bins = c->d_spec + (size_t)3 * 2048 * nblk;  // [2][3 nb]: k, shell sum, mult
  double2* F = c->d_cplx;
  CU(cudaStreamSynchronize(c->stream));
  const double a = S.a, Hc = S.b / S.a, al = c->alpha;
  const void* phi = arr_ptr(c, 0, c->parity, 2 * field);
  const void* pi = arr_ptr(c, 0, c->parity, 2 * field + 1);
  // |phi_k|^2, then |phi'_k + (a'/a) phi_k|^2 with phi' = a^{alpha-3} pi, binned
  for (int r = 0; r < 2; ++r) {
    if (r == 0) CU(launch_to_complex(c->fp32, phi, F, H.V, c->stream));
    else CU(launch_combine_to_complex(c->fp32, pi, std::pow(a, al - 3.0), phi, Hc, F, H.V, c->stream));
    ++c->launches;
    s = fft3d(c, H.N, F, -1);
    if (s != CL_OK) return s;
    CU(launch_bins(F, H.N, dk_bin, nb, nblk, part, H.kIR, H.dx, bins + (size_t)r * 3 * nb, c->stream, 1));
    c->launches += 2;
  }
  std::vector<double> h(6 * nb);
  CU(cudaMemcpyAsync(h.data(), bins, 6 * nb * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  CU(cudaStreamSynchronize(c->stream));
  // volume average of the field's diagonal Hessian element (eq. PotNat), from the measured <phi_g^2>
  const double* p2 = S.obs.mean_phi2;
  double m2 = 0.0;
  if (c->model == CL_MODEL_LPHI4) m2 = 3.0 * p2[0];
  else m2 = field == 0 ? 3.0 * p2[0] + c->p.q * p2[1] : c->p.q * p2[0];
  const double V = (double)H.V, L = H.N * H.dx;
  const double C = a * a * L * L * L / (2.0 * V * V) * fo2, a2p = std::pow(a, 2.0 * (1.0 - al));
  for (int b = 0; b < nb; ++b) {
    const double cnt = h[2 * nb + b];
    k[b] = h[b];
    mult[b] = (int64_t)cnt;
    if (cnt == 0.0) {
      n[b] = 0.0;
      continue;
    }
    const double w2 = h[b] * h[b] + a * a * m2;
    if (!(w2 > 0.0)) {
      n[b] = std::nan("");
      continue;
    }
    const double w = std::sqrt(w2);
    n[b] = C * (w * h[nb + b] / cnt + a2p * h[3 * nb + nb + b] / (cnt * w));
  }
  return check_status(c);
}

cl_status cl_norm_spectrum(cl_ctx* c, double dk_bin, double fo2, double* k, double* df, double* dfp, double* n,
                           int64_t* mult, int cap, int* nbins) {
  return cl_norm_spectrum_of(c, 0, dk_bin, fo2, k, df, dfp, n, mult, cap, nbins);
}

cl_status cl_norm_spectrum_of(cl_ctx* c, int which, double dk_bin, double fo2, double* k, double* df, double* dfp,
                              double* n, int64_t* mult, int cap, int* nbins) {
  Range range_("cl_norm_spectrum");
  if (!c || !k || !df || !dfp || !n || !mult || !nbins) return fail(c, CL_EINVAL, "NULL argument");
  if (c->nlat != 1 || (c->model != CL_MODEL_U1_HIGGS && !is_doublet(c->model)))
    return fail(c, CL_EUNSUPPORTED, "modulus spectra cover single lattices of the gauge models");
  const bool full = c->model == CL_MODEL_LPHI4_SU2U1;
  if (which != 0 && !(which == 1 && full))
    return fail(c, CL_EINVAL, "which must be 0 (the charged field)%s", full ? " or 1 (vphi)" : "");
  if (!(dk_bin > 0.0)) return fail(c, CL_EINVAL, "dk_bin must be positive");
  if (!(fo2 > 0.0)) {
    if (!(c->p.fluct_amp2 > 0.0)) return fail(c, CL_EINVAL, "need (f*/omega*)^2 > 0 (fluct_amp2 is 0)");
    fo2 = 1.0 / c->p.fluct_amp2;
  }
  const LatHost& H = c->lats[0];
  const int nb = (int)std::floor(std::sqrt(3.0) * (H.N / 2) / dk_bin) + 1;
  *nbins = nb;
  if (nb > cap) return fail(c, CL_EINVAL, "cap %d < %d bins", cap, nb);
  if (nb > 2048) return fail(c, CL_EINVAL, "too many bins (dk_bin too small)");
  cl_status s = measure(c, 0);  // the synchronised state and its volume averages
  if (s != CL_OK) return s;
  LatScalars S;
  CU(cudaMemcpyAsync(&S, &c->d_sc[0], sizeof(S), cudaMemcpyDeviceToHost, c->stream));
  const int nblk = 2 * c->nsm;
  if (c->spec_lats < 3) {  // four rows of bins
    CU(cudaStreamSynchronize(c->stream));
    cudaFree(c->d_spec);
    c->d_spec = nullptr;
    c->spec_lats = 0;
    CU(cudaMalloc(&c->d_spec, ((size_t)3 * 2048 * nblk + (size_t)4 * 3 * 2048) * sizeof(double)));
    c->spec_lats = 3;
  }
  double* part = c->d_spec;
  double* bins = c->d_spec + (size_t)3 * 2048 * nblk;  // [4][3 nb]: k, delta or shell sum, mult
  double2* F = c->d_cplx;
  CU(cudaStreamSynchronize(c->stream));
  const double a = S.a, Hc = S.b / S.a, al = c->alpha;
  const bool u1 = c->model == CL_MODEL_U1_HIGGS;
  const int nc = u1 || which == 1 ? 2 : 4;
  const void* f[4];
  const void* p[4];
  for (int q = 0; q < nc; ++q) {
    // the U(1) model: phi_q, pi_q at 2q, 2q + 1; the doublet: 0..3, momenta 4..7;
    // lphi4SU2U1's vphi: 37, 38, momenta 39, 40
    f[q] = arr_ptr(c, 0, c->parity, which == 1 ? 37 + q : (u1 ? 2 * q : q));
    p[q] = arr_ptr(c, 0, c->parity, which == 1 ? 39 + q : (u1 ? 2 * q + 1 : 4 + q));
  }
  // lphi4SU2U1's doublet: the couplings' part of its mass, <q_G phi_s^2 + 2 q_H |vphi|^2>
  // (phi_s at 35), which the measurement does not keep
  double mfull = 0.0;
  if (full && which == 0) {
    const int nsum = 2 * c->nsm;
    CU(launch_sum_sq(c->fp32, arr_ptr(c, 0, c->parity, 35), arr_ptr(c, 0, c->parity, 37),
                     arr_ptr(c, 0, c->parity, 38), c->p.qG, c->p.qH, c->p.qH, H.V, nsum, part, c->stream));
    ++c->launches;
    std::vector<double> ps(nsum);
    CU(cudaMemcpyAsync(ps.data(), part, nsum * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    CU(cudaStreamSynchronize(c->stream));
    for (int b = 0; b < nsum; ++b) mfull += ps[b];
    mfull /= (double)H.V;
  }
  // rows: 0 Delta_r, 1 shell sums |r_k|^2, 2 Delta_r', 3 shell sums |r'_k + (a'/a) r_k|^2
  for (int mode = 0; mode < 3; ++mode) {
    CU(launch_norm_field(c->fp32, f, p, nc, std::pow(a, al - 3.0), Hc, mode, F, H.V, c->stream));
    ++c->launches;
    s = fft3d(c, H.N, F, -1);
    if (s != CL_OK) return s;
    if (mode == 0) {
      CU(launch_bins(F, H.N, dk_bin, nb, nblk, part, H.kIR, H.dx, bins, c->stream, 0));
      CU(launch_bins(F, H.N, dk_bin, nb, nblk, part, H.kIR, H.dx, bins + (size_t)3 * nb, c->stream, 1));
      c->launches += 4;
    } else {
      CU(launch_bins(F, H.N, dk_bin, nb, nblk, part, H.kIR, H.dx, bins + (size_t)(mode + 1) * 3 * nb, c->stream,
                     mode == 1 ? 0 : 1));
      c->launches += 2;
    }
  }
  std::vector<double> h(12 * nb);
  CU(cudaMemcpyAsync(h.data(), bins, 12 * nb * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  CU(cudaStreamSynchronize(c->stream));
  // n is that of the canonical modulus rho = sqrt2 r (|rho_k|^2 = 2 |r_k|^2), whose
  // mass is <d^2V/drho^2> = <V''(r)>/2: lam (6 <r^2> - 2 v^2), <r^2> = sum_c <phi_c^2>/2,
  // for the U(1) field and the doublet, plus <q_G phi_s^2 + 2 q_H |vphi|^2> for
  // lphi4SU2U1's doublet; 2 q_H <|Phi|^2> for its vphi (eq. PotGauge)
  double r2 = 0.0;
  for (int q = 0; q < (which == 1 ? 4 : nc); ++q) r2 += 0.5 * S.obs.mean_phi2[q];
  const double m2 = which == 1 ? 2.0 * c->p.qH * r2 : c->p.lam * (6.0 * r2 - 2.0 * c->p.v * c->p.v) + mfull;
  const double V = (double)H.V, L = H.N * H.dx;
  const double C = a * a * L * L * L / (2.0 * V * V) * fo2, a2p = std::pow(a, 2.0 * (1.0 - al));
  for (int b = 0; b < nb; ++b) {
    const double cnt = h[2 * nb + b];
    k[b] = h[b];
    mult[b] = (int64_t)cnt;
    df[b] = h[nb + b];
    dfp[b] = h[6 * nb + nb + b];
    if (cnt == 0.0) {
      n[b] = 0.0;
      continue;
    }
    const double w2 = h[b] * h[b] + a * a * m2;
    if (!(w2 > 0.0)) {
      n[b] = std::nan("");
      continue;
    }
    const double w = std::sqrt(w2);
    n[b] = 2.0 * C * (w * h[3 * nb + nb + b] / cnt + a2p * h[9 * nb + nb + b] / (cnt * w));
  }
  return check_status(c);
}

cl_status cl_em_spectrum(cl_ctx* c, int which, double dk_bin, double* k, double* delta, int64_t* mult, int cap,
                         int* nbins) {
  Range range_("cl_em_spectrum");
  if (!c || !k || !delta || !mult || !nbins) return fail(c, CL_EINVAL, "NULL argument");
  const bool su2 = is_doublet(c->model);
  if ((c->model != CL_MODEL_U1_HIGGS && !su2) || c->nlat != 1)
    return fail(c, CL_EUNSUPPORTED, "electric and magnetic spectra need a single gauge lattice");
  if (which < 0 || which > (su2 ? 3 : 1))
    return fail(c, CL_EINVAL, "which must be 0 (electric) or 1 (magnetic)%s", su2 ? ", 2 or 3 (SU(2))" : "");
  if (which == 1 && c->p.gQ == 0.0) return fail(c, CL_EUNSUPPORTED, "gQ = 0: no U(1) field");
  if (!(dk_bin > 0.0)) return fail(c, CL_EINVAL, "dk_bin must be positive");
  const LatHost& H = c->lats[0];
  const int nb = (int)std::floor(std::sqrt(3.0) * (H.N / 2) / dk_bin) + 1;
  *nbins = nb;
  if (nb > cap) return fail(c, CL_EINVAL, "cap %d < %d bins", cap, nb);
  if (nb > 2048) return fail(c, CL_EINVAL, "too many bins (dk_bin too small)");
  cl_status s = close_stream(c);
  if (s != CL_OK) return s;
  LatScalars S;
  CU(cudaMemcpyAsync(&S, &c->d_sc[0], sizeof(S), cudaMemcpyDeviceToHost, c->stream));
  const int nblk = 2 * c->nsm;
  if (c->spec_lats < 1) {
    CU(cudaStreamSynchronize(c->stream));
    cudaFree(c->d_spec);
    c->d_spec = nullptr;
    CU(cudaMalloc(&c->d_spec, ((size_t)3 * 2048 * nblk + (size_t)2 * 3 * 2048) * sizeof(double)));
    c->spec_lats = 1;
  }
  double* part = c->d_spec;
  double* bins = c->d_spec + (size_t)3 * 2048 * nblk;  // [3 nb]: k, shell sum, mult
  double2* F = c->d_cplx;
  CU(cudaStreamSynchronize(c->stream));
  const double gd = c->p.gQ * H.dx, ae = std::pow(S.a, c->alpha - 1.0);
  const double inv_gdx2 = which == 1 ? 1.0 / (c->p.gQ * H.dx * H.dx) : 0.0;
  const double inv_bdx2 = su2 ? 1.0 / (c->p.gQB * H.dx * H.dx) : 0.0;
  // U(1) model arrays: A_i = 4 + 2i, pi_A,i = 5 + 2i; doublet model: A_i = 8 + i,
  // pi_A,i = 11 + i, SU(2) link components 14 + 4i + k, pi_B,i^a = 26 + 3i + (a - 1)
  auto A_arr = [&](int i) { return su2 ? 8 + i : 4 + 2 * i; };
  auto pA_arr = [&](int i) { return su2 ? 11 + i : 5 + 2 * i; };
  std::vector<double> sum(nb, 0.0), kk(nb, 0.0), cnt(nb, 0.0), h(3 * nb);
  const int ncomp = which >= 2 ? 9 : 3;
  for (int comp = 0; comp < ncomp; ++comp) {
    const int i = which >= 2 ? comp / 3 : comp, a = comp % 3 + 1;
    const int j = (i + 1) % 3, l = (i + 2) % 3;  // B_i = F_jl with (i, j, l) cyclic
    if (which == 0) {
      const void* pa = arr_ptr(c, 0, c->parity, pA_arr(i));
      CU(launch_combine_to_complex(c->fp32, pa, ae, pa, 0.0, F, H.V, c->stream));
    } else if (which == 1) {
      CU(launch_u1_plaquette_field(c->fp32, arr_ptr(c, 0, c->parity, A_arr(j)), arr_ptr(c, 0, c->parity, A_arr(l)),
                                   j, l, H.N, gd, inv_gdx2, F, c->stream));
    } else if (which == 2) {
      const void* pb = arr_ptr(c, 0, c->parity, 26 + 3 * i + (a - 1));
      CU(launch_combine_to_complex(c->fp32, pb, ae, pb, 0.0, F, H.V, c->stream));
    } else {
      CU(launch_su2_plaquette_field(c->fp32, arr_ptr(c, 0, c->parity, 14 + 4 * j),
                                    arr_ptr(c, 0, c->parity, 14 + 4 * l), j, l, a, H.N, inv_bdx2, F, c->stream));
    }
    ++c->launches;
    s = fft3d(c, H.N, F, -1);
    if (s != CL_OK) return s;
    CU(launch_bins(F, H.N, dk_bin, nb, nblk, part, H.kIR, H.dx, bins, c->stream, 1));
    c->launches += 2;
    CU(cudaMemcpyAsync(h.data(), bins, 3 * nb * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    CU(cudaStreamSynchronize(c->stream));
    for (int b = 0; b < nb; ++b) sum[b] += h[nb + b];
    if (comp == 0)
      for (int b = 0; b < nb; ++b) {
        kk[b] = h[b];
        cnt[b] = h[2 * nb + b];
      }
  }
  // eq. discretePS on the summed shell sums
  const double pi = 3.14159265358979323846, fac = std::pow(H.dx / (double)H.N, 3.0);
  for (int b = 0; b < nb; ++b) {
    k[b] = kk[b];
    mult[b] = (int64_t)cnt[b];
    if (cnt[b] == 0.0) {
      delta[b] = 0.0;
      continue;
    }
    const double nbar = kk[b] / H.kIR;
    delta[b] = kk[b] * kk[b] * kk[b] / (2.0 * pi * pi) * fac * sum[b] / (4.0 * pi * nbar * nbar);
  }
  return check_status(c);
}

cl_status cl_gauss_constraint(cl_ctx* c, double* rel, double* lhs_abs, double* rhs_abs,
                              double* max_abs) {
  Range range_("cl_gauss_constraint");
  if (!c) return fail(nullptr, CL_EINVAL, "ctx is NULL");
  if (c->model != CL_MODEL_U1_HIGGS && !is_doublet(c->model))
    return fail(c, CL_EUNSUPPORTED, "model has no gauge field");
  cl_status s = close_stream(c);
  if (s != CL_OK) return s;
  const int nblk = 2 * c->nsm;
  double* part = c->d_tmp;
  if (is_doublet(c->model))
    CU(launch_su2_gauss_monitor(c->fp32, c->d_lat, c->parity, part, nblk, c->lats[0].V, c->stream));
  else
    CU(launch_u1_gauss_monitor(c->d_lat, c->parity, part, nblk, c->lats[0].V, c->stream));
  c->launches += 2;
  double h[4];
  CU(cudaMemcpyAsync(h, part + 3 * nblk, 4 * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  CU(cudaStreamSynchronize(c->stream));
  if (rel) *rel = h[0];
  if (lhs_abs) *lhs_abs = h[1];
  if (rhs_abs) *rhs_abs = h[2];
  if (max_abs) *max_abs = h[3];
  return check_status(c);
}

cl_status cl_state_bytes(cl_ctx* c, size_t* bytes) {
  if (!c || !bytes) return fail(c, CL_EINVAL, "NULL argument");
  *bytes = (size_t)c->narr * c->lats[0].V * c->esz;
  return CL_OK;
}

cl_status cl_bind_buffers(cl_ctx* c, int lat, void* buf0, void* buf1, size_t bytes) {
  Range range_("cl_bind_buffers");
  if (!c) return CL_EINVAL;
  if (lat < 0 || lat >= c->nlat) return fail(c, CL_EINVAL, "lattice %d of %d", lat, c->nlat);
  LatHost& L = c->lats[lat];
  const size_t need = (size_t)c->narr * L.V * c->esz;
  const bool unbind = !buf0 && !buf1;
  void* buf[2] = {buf0, buf1};
  if (!unbind) {
    if (!buf0 || !buf1) return fail(c, CL_EINVAL, "two buffers, or none");
    if (bytes < need) return fail(c, CL_EINVAL, "buffers of %zu bytes, the state needs %zu", bytes, need);
    const uintptr_t p0 = (uintptr_t)buf0, p1 = (uintptr_t)buf1;
    if (p0 % 256 || p1 % 256) return fail(c, CL_EINVAL, "buffers must be 256-byte aligned");
    if (p0 < p1 + need && p1 < p0 + need) return fail(c, CL_EINVAL, "the two buffers overlap");
    for (int k = 0; k < 2; ++k) {
      cudaPointerAttributes at;
      if (cudaPointerGetAttributes(&at, buf[k]) != cudaSuccess) {
        cudaGetLastError();
        return fail(c, CL_EINVAL, "buffer %d is not device memory", k);
      }
      if ((at.type != cudaMemoryTypeDevice && at.type != cudaMemoryTypeManaged) || at.device != c->dev)
        return fail(c, CL_EINVAL, "buffer %d is not memory of the context's device", k);
    }
  }
  void* fresh = nullptr;  // memory of the lattice's own, when the binding ends
  if (unbind) {
    if (!L.bound[0]) return CL_OK;
    CU(cudaMalloc(&fresh, 2 * need));
    buf[0] = fresh;
    buf[1] = (char*)fresh + need;
  }
  // the state moves with the binding: both buffers, on the context stream
  for (int par = 0; par < 2; ++par)
    CU(cudaMemcpyAsync(buf[par], arr_ptr(c, lat, par, 0), need, cudaMemcpyDeviceToDevice, c->stream));
  CU(cudaStreamSynchronize(c->stream));
  if (L.slab) CU(cudaFree(L.slab));
  L.slab = fresh;
  L.bound[0] = unbind ? nullptr : buf0;
  L.bound[1] = unbind ? nullptr : buf1;
  // every device-side copy of the array addresses (the doublet models keep the
  // first MAX_ARR and address the rest from array 0)
  LatConst& H = c->hlat[lat];
  for (int par = 0; par < 2; ++par)
    for (int a = 0; a < std::min(c->narr, MAX_ARR); ++a) H.buf[par][a] = arr_ptr(c, lat, par, a);
  CU(cudaMemcpyAsync(c->d_lat + lat, &H, sizeof(LatConst), cudaMemcpyHostToDevice, c->stream));
  if (c->adj.ready) {
    for (int par = 0; par < 2; ++par)
      for (int a = 0; a < 2 * c->nf; ++a) c->adj.hl.buf[par][a] = arr_ptr(c, 0, par, a);
    CU(cudaMemcpyAsync(c->adj.d_lat, &c->adj.hl, sizeof(LatConst), cudaMemcpyHostToDevice, c->stream));
  }
  for (auto& g : c->graph_cache) cudaGraphExecDestroy(g.exec);
  c->graph_cache.clear();
  CU(cudaStreamSynchronize(c->stream));
  return CL_OK;
}

cl_status cl_state_buffer(cl_ctx* c, int* which) {
  if (!c || !which) return fail(c, CL_EINVAL, "NULL argument");
  *which = c->parity;
  return CL_OK;
}

cl_status cl_checkpoint_save(cl_ctx* c, const char* path) {
  Range range_("cl_checkpoint_save");
  if (!c || !path) return fail(c, CL_EINVAL, "NULL argument");
  if (c->nlat != 1) return fail(c, CL_EUNSUPPORTED, "checkpoints cover single lattices");
  cl_status s = close_stream(c);
  if (s != CL_OK) return s;
  const LatHost& H = c->lats[0];
  const size_t ab = (size_t)H.V * c->esz, nb = (size_t)c->narr * ab;
  std::vector<char> state(nb);
  LatScalars S;
  for (int a = 0; a < c->narr; ++a)
    CU(cudaMemcpyAsync(state.data() + a * ab, arr_ptr(c, 0, c->parity, a), ab, cudaMemcpyDeviceToHost, c->stream));
  CU(cudaMemcpyAsync(&S, c->d_sc, sizeof(S), cudaMemcpyDeviceToHost, c->stream));
  CU(cudaStreamSynchronize(c->stream));
  s = check_status(c);
  if (s != CL_OK) return s;
  CkptHeader h;
  ckpt_init_header(h);
  h.model = c->model;
  h.N = H.N;
  h.narr = c->narr;
  h.esz = c->esz;
  h.kIR = H.kIR;
  h.alpha = c->alpha;
  h.seed = H.seed;
  h.scalars_bytes = sizeof(S);
  h.state_bytes = nb;
  const int rc = ckpt_write_atomic(path, h, &S, state.data());
  if (rc != 0) return fail(c, CL_EINVAL, "cannot write checkpoint %s", path);
  return CL_OK;
}

cl_status cl_checkpoint_load(cl_ctx* c, const char* path) {
  Range range_("cl_checkpoint_load");
  if (!c || !path) return fail(c, CL_EINVAL, "NULL argument");
  if (c->nlat != 1) return fail(c, CL_EUNSUPPORTED, "checkpoints cover single lattices");
  CkptHeader h;
  std::vector<char> sc, state;
  if (ckpt_read(path, h, sc, state) != 0) return fail(c, CL_EINVAL, "%s is not a readable checkpoint", path);
  const LatHost& H = c->lats[0];
  const size_t ab = (size_t)H.V * c->esz;
  if (h.model != c->model || h.N != H.N || h.narr != c->narr || h.esz != c->esz ||
      h.scalars_bytes != sizeof(LatScalars) || h.state_bytes != (size_t)c->narr * ab || h.kIR != H.kIR ||
      h.alpha != c->alpha)
    return fail(c, CL_EINVAL, "checkpoint %s does not match this context (model, N, precision, kIR, alpha)", path);
  cl_status s = close_stream(c);
  if (s != CL_OK) return s;
  for (int a = 0; a < c->narr; ++a)
    CU(cudaMemcpyAsync(arr_ptr(c, 0, c->parity, a), state.data() + a * ab, ab, cudaMemcpyHostToDevice, c->stream));
  CU(cudaMemcpyAsync(c->d_sc, sc.data(), sizeof(LatScalars), cudaMemcpyHostToDevice, c->stream));
  CU(cudaStreamSynchronize(c->stream));
  c->obs_valid = false;
  return CL_OK;
}

cl_status cl_upload_state(cl_ctx* c, const void* host, size_t bytes) {
  Range range_("cl_upload_state");
  if (!c || !host) return fail(c, CL_EINVAL, "NULL argument");
  const long long V = c->lats[0].V;
  if (bytes != (size_t)c->narr * V * c->esz) return fail(c, CL_EINVAL, "wrong byte count");
  cl_status s = close_stream(c);
  if (s != CL_OK) return s;
  const size_t ab = (size_t)V * c->esz;
  for (int a = 0; a < c->narr; ++a)
    CU(cudaMemcpyAsync(arr_ptr(c, 0, c->parity, a), (const char*)host + a * ab, ab, cudaMemcpyDefault,
                       c->stream));
  c->obs_valid = false;
  return CL_OK;
}

cl_status cl_download_state(cl_ctx* c, void* host, size_t bytes) {
  Range range_("cl_download_state");
  if (!c || !host) return fail(c, CL_EINVAL, "NULL argument");
  const long long V = c->lats[0].V;
  if (bytes != (size_t)c->narr * V * c->esz) return fail(c, CL_EINVAL, "wrong byte count");
  cl_status s = close_stream(c);
  if (s != CL_OK) return s;
  const size_t ab = (size_t)V * c->esz;
  for (int a = 0; a < c->narr; ++a)
    CU(cudaMemcpyAsync((char*)host + a * ab, arr_ptr(c, 0, c->parity, a), ab, cudaMemcpyDefault,
                       c->stream));
  CU(cudaStreamSynchronize(c->stream));
  return CL_OK;
}

cl_status cl_enable_pass_timing(cl_ctx* c, int enable) {
  if (!c) return fail(nullptr, CL_EINVAL, "ctx is NULL");
  c->timing = enable != 0;
  return CL_OK;
}

cl_status cl_pass_timing(cl_ctx* c, double* ms_total, int64_t* passes, int reset) {
  if (!c) return fail(nullptr, CL_EINVAL, "ctx is NULL");
  cl_status s = timing_collect(c);
  if (s != CL_OK) return s;
  if (ms_total) *ms_total = c->timing_ms;
  if (passes) *passes = c->timing_passes;
  if (reset) {
    c->timing_ms = 0.0;
    c->timing_passes = 0;
  }
  return CL_OK;
}

cl_status cl_adjoint_pass_timing(cl_ctx* c, double* ms_total, int64_t* passes, int reset) {
  if (!c) return fail(nullptr, CL_EINVAL, "ctx is NULL");
  cl_status s = timing_collect(c);
  if (s != CL_OK) return s;
  if (ms_total) *ms_total = c->adj_timing_ms;
  if (passes) *passes = c->adj_timing_passes;
  if (reset) {
    c->adj_timing_ms = 0.0;
    c->adj_timing_passes = 0;
  }
  return CL_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Adjoint sweep (gradient of a final observable).
// ---------------------------------------------------------------------------

// The reversed-pass kernel's tiling: its stage carries the state and the
// adjoint (4 nf arrays), so its tiles are shorter than the forward pass's.
static cl_status adjoint_plan(cl_ctx* c) {
  AdjPlan& A = c->adj;
  if (A.ready) return CL_OK;
  const LatHost& H = c->lats[0];
  const int narr = 4 * c->nf;
  const std::vector<int> cand = tile_candidates(c->model, narr, c->esz, H.N, c->smem_optin);
  if (cand.empty()) return fail(c, CL_EUNSUPPORTED, "no adjoint tile shape for N=%d", H.N);
  const int BY = cand[0];
  const long long tasks = (long long)(H.N / BY) * H.N;
  A.grid = (int)std::max<long long>(1, std::min<long long>(c->nsm, tasks / 8));
  std::vector<Seg> segs;
  std::vector<int> cta, sbeg, send;
  if (!build_worklist({LatTiles{H.N, BY, THREADS * tile_vx(c->model, c->esz)}}, A.grid, false, segs, cta, sbeg, send))
    return fail(c, CL_EUNSUPPORTED, "adjoint work split too fine");
  A.stage_bytes = (unsigned)stage_size(H.N, BY, narr, c->esz);
  A.stages = (int)std::min<size_t>(6, (c->smem_optin - SM_TAIL_BYTES) / A.stage_bytes);
  A.smem = (size_t)A.stages * A.stage_bytes + SM_TAIL_BYTES;
  PassKernel k = adjoint_pass_kernel(c->fp32, c->nf, c->p.expansion == CL_EXP_SELF);
  CU(cudaFuncSetAttribute((const void*)k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)A.smem));
  const size_t ab = (size_t)H.V * c->esz;
  CU(cudaMalloc(&A.lam, 2 * (size_t)(2 * c->nf) * ab));
  CU(cudaMalloc(&A.d_lat, sizeof(LatConst)));
  CU(cudaMalloc(&A.d_segs, segs.size() * sizeof(Seg)));
  CU(cudaMalloc(&A.d_cta, cta.size() * sizeof(int)));
  CU(cudaMalloc(&A.d_part, (size_t)send[0] * NQ * sizeof(double)));
  A.nslot = send[0];
  CU(cudaMalloc(&A.d_cnt, sizeof(unsigned)));
  CU(cudaMalloc(&A.d_out, 2 * sizeof(double) + 2 * c->nsm * sizeof(double)));
  CU(cudaMemsetAsync(A.d_cnt, 0, sizeof(unsigned), c->stream));
  LatConst L = c->hlat[0];
  L.BY = BY;
  L.YT = H.N / BY;
  L.narr = narr;
  L.slot_begin = sbeg[0];
  L.slot_end = send[0];
  for (int par = 0; par < 2; ++par)
    for (int a = 0; a < 2 * c->nf; ++a) {
      L.buf[par][a] = arr_ptr(c, 0, par, a);
      L.buf[par][2 * c->nf + a] = (char*)A.lam + ((size_t)par * 2 * c->nf + a) * ab;
    }
  A.hl = L;
  CU(cudaMemcpyAsync(A.d_lat, &A.hl, sizeof(L), cudaMemcpyHostToDevice, c->stream));
  CU(cudaMemcpyAsync(A.d_segs, segs.data(), segs.size() * sizeof(Seg), cudaMemcpyHostToDevice, c->stream));
  CU(cudaMemcpyAsync(A.d_cta, cta.data(), cta.size() * sizeof(int), cudaMemcpyHostToDevice, c->stream));
  int coop = 0, nb = 0;
  CU(cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, c->dev));
  CU(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, (const void*)k, THREADS, A.smem));
  A.coop = coop && (long long)nb * c->nsm >= A.grid;
  CU(cudaStreamSynchronize(c->stream));
  A.ready = true;
  return CL_OK;
}

// n reversed passes, coefficients dev_coef[ADJ_COEF_W i ..] for the i-th.
static cl_status launch_adjoint(cl_ctx* c, const double* dev_coef, int n) {
  AdjPlan& J = c->adj;
  PassKernel k = adjoint_pass_kernel(c->fp32, c->nf, c->p.expansion == CL_EXP_SELF);
  PassArgs A;
  memset(&A, 0, sizeof(A));
  A.lat = J.d_lat;
  A.sc = c->d_sc;
  A.segs = J.d_segs;
  A.cta_seg = J.d_cta;
  A.partials = J.d_part;
  A.nslot = J.nslot;
  A.counters = J.d_cnt;
  A.parity = c->parity;
  A.write = 1;
  A.stages = J.stages;
  A.stage_bytes_max = J.stage_bytes;
  A.nlat = 1;
  A.wait_limit_ns = 2000000000ull;
  A.adj = dev_coef;
  A.npass = 1;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (c->timing) {
    cl_status s = timing_begin(c, &e0, &e1);
    if (s != CL_OK) return s;
  }
  if (n > 1 && J.coop) {
    A.npass = n;
    A.gsync = c->d_gsync;
    CU(cudaMemsetAsync(c->d_gsync, 0, 2 * sizeof(unsigned), c->stream));
    void* args[] = {&A};
    CU(cudaLaunchCooperativeKernel((const void*)k, dim3(J.grid), dim3(THREADS), args, J.smem, c->stream));
    ++c->launches;
  } else {
    for (int i = 0; i < n; ++i) {
      A.adj = dev_coef + (size_t)ADJ_COEF_W * i;
      A.parity = c->parity ^ (i & 1);
      k<<<J.grid, THREADS, J.smem, c->stream>>>(A);
      CHECK_LAUNCH();
      ++c->launches;
    }
  }
  if (c->timing) {
    cl_status s = timing_end(c, e0, e1, n, 1);
    if (s != CL_OK) return s;
  }
  if (n & 1) c->parity ^= 1;
  return CL_OK;
}

extern "C" {

cl_status cl_adjoint(cl_ctx* c, int nsteps, int ckpt_every, int objective, int field, int what, double dk_bin,
                     int bin, double* J, double* dJ_dq, double* dJ_dstate, double* dJ_dscale) {
  Range range_("cl_adjoint");
  if (!c) return fail(nullptr, CL_EINVAL, "ctx is NULL");
  if (nsteps < 0 || ckpt_every < 1) return fail(c, CL_EINVAL, "need nsteps >= 0 and ckpt_every >= 1");
  if (c->nlat != 1 || c->model >= CL_MODEL_U1_HIGGS)
    return fail(c, CL_EUNSUPPORTED, "the adjoint covers single scalar lattices");
  const bool self = c->p.expansion == CL_EXP_SELF;
  if (objective == CL_OBJ_CHI_FRACTION) {
    if (c->model != CL_MODEL_LPHI4_CHI) return fail(c, CL_EINVAL, "the chi energy fraction needs two fields");
  } else if (objective == CL_OBJ_SPECTRUM_BIN) {
    if (field < 0 || field >= c->nf || (what != 0 && what != 1) || !(dk_bin > 0.0))
      return fail(c, CL_EINVAL, "bad spectrum objective");
    const int nb = (int)std::floor(std::sqrt(3.0) * (c->lats[0].N / 2) / dk_bin) + 1;
    if (bin < 0 || bin >= nb || nb > 2048) return fail(c, CL_EINVAL, "bin %d out of 0..%d", bin, nb - 1);
  } else {
    return fail(c, CL_EINVAL, "unknown objective %d", objective);
  }
  cl_status s = close_stream(c);
  if (s != CL_OK) return s;
  s = adjoint_plan(c);
  if (s != CL_OK) return s;
  const LatHost& H = c->lats[0];
  const int na = 2 * c->nf;
  const size_t ab = (size_t)H.V * c->esz;
  std::vector<double> dsub;
  schedule(c->p.integrator == CL_LF ? 2 : c->p.integrator, c->p.dt, dsub);
  const int nsub = (int)dsub.size();
  const int nchunk = (nsteps + ckpt_every - 1) / ckpt_every;
  const long long npass = (long long)nsteps * nsub + 1;  // with the closing half kick
  // the lattice's scalars (a, b, eta, ...) at the start, put back at the end
  LatScalars sc0;
  CU(cudaMemcpyAsync(&sc0, &c->d_sc[0], sizeof(sc0), cudaMemcpyDeviceToHost, c->stream));
  CU(cudaStreamSynchronize(c->stream));
  std::vector<PassStep> fw;  // every forward pass's weights, in order
  fw.reserve((size_t)npass);
  void* ckpt = nullptr;
  double* dlog = nullptr;
  double* dcoef = nullptr;
  auto cleanup = [&]() {
    cudaStreamSynchronize(c->stream);
    cudaFree(ckpt);
    cudaFree(dlog);
    cudaFree(dcoef);
  };
  auto copy_state = [&](void* dst_base, int ck, bool to_ckpt) -> cl_status {
    for (int a = 0; a < na; ++a) {
      char* cp = (char*)dst_base + ((size_t)ck * na + a) * ab;
      void* st = arr_ptr(c, 0, c->parity, a);
      CU(cudaMemcpyAsync(to_ckpt ? (void*)cp : st, to_ckpt ? st : (const void*)cp, ab, cudaMemcpyDeviceToDevice,
                         c->stream));
    }
    return CL_OK;
  };
#define ADJ_TRY(x)          \
  do {                      \
    cl_status s_ = (x);     \
    if (s_ != CL_OK) {      \
      cleanup();            \
      return s_;            \
    }                       \
  } while (0)
  if (cudaMalloc(&ckpt, (size_t)(nchunk + 1) * na * ab) != cudaSuccess ||
      cudaMalloc(&dlog, (size_t)npass * ADJ_LOG_W * sizeof(double)) != cudaSuccess ||
      cudaMalloc(&dcoef, (size_t)npass * ADJ_COEF_W * sizeof(double)) != cudaSuccess) {
    cleanup();
    return fail(c, CL_ENOMEM, "adjoint: checkpoint / log allocation failed");
  }
  CU(cudaMemsetAsync(dlog, 0, (size_t)npass * ADJ_LOG_W * sizeof(double), c->stream));
  // ---- forward: chunks of ckpt_every steps, the state saved after each ----
  ADJ_TRY(copy_state(ckpt, 0, true));
  std::vector<long long> chunk_first(nchunk + 1, 0);
  long long pc = 0;
  for (int ch = 0; ch < nchunk; ++ch) {
    const int m = std::min(ckpt_every, nsteps - ch * ckpt_every);
    std::vector<PassStep> steps;
    append_pass_steps(c->p.integrator, c->p.dt, m, c->open, c->dprev, steps);  // the forward plan of cl_step
    chunk_first[ch] = pc;
    fw.insert(fw.end(), steps.begin(), steps.end());
    for (size_t b = 0; b < steps.size(); b += 4096) {
      const int mm = (int)std::min<size_t>(4096, steps.size() - b);
      ADJ_TRY(launch_passes(c, steps.data() + b, mm, red_for_step(c), 1, 0, dlog, pc));
      pc += mm;
    }
    ADJ_TRY(copy_state(ckpt, ch + 1, true));
  }
  chunk_first[nchunk] = pc;
  if (c->open) {  // the closing half kick, which also measures
    PassStep st = closing_pass_step(c->dprev);
    fw.push_back(st);
    ADJ_TRY(launch_passes(c, &st, 1, 2, 1, 0, dlog, pc));
    ++pc;
    c->open = false;
    c->obs_valid = true;
  } else {
    ADJ_TRY(measure(c, 0));
  }
  const long long nrev = pc;  // passes to reverse
  // ---- seed: dJ/d(final state) and the objective (dJ/dq, dJ/da, dJ/db zeroed first) ----
  static_assert(offsetof(LatScalars, adjb) == offsetof(LatScalars, adjq) + 2 * sizeof(double),
                "adjq, adja, adjb are consecutive");
  CU(cudaMemsetAsync(&c->d_sc[0].adjq, 0, 3 * sizeof(double), c->stream));
  void* lam[4] = {nullptr, nullptr, nullptr, nullptr};
  for (int a = 0; a < na; ++a) lam[a] = (char*)c->adj.lam + ((size_t)c->parity * na + a) * ab;
  if (objective == CL_OBJ_CHI_FRACTION) {
    const int nblk = 2 * c->nsm;
    if (cudaSuccess != launch_seed_chi_fraction(c->fp32, c->d_lat, c->d_sc, c->parity, lam, c->adj.d_out + 2, nblk,
                                                c->adj.d_out, c->stream)) {
      cleanup();
      return fail(c, CL_ECUDA, "adjoint seed launch failed");
    }
    c->launches += 2;
  } else {
    for (int a = 0; a < na; ++a) CU(cudaMemsetAsync(lam[a], 0, ab, c->stream));
    const int nb = (int)std::floor(std::sqrt(3.0) * (H.N / 2) / dk_bin) + 1;
    const int nblk = 2 * c->nsm;
    if (c->spec_lats < 1) {
      cudaFree(c->d_spec);
      CU(cudaMalloc(&c->d_spec, ((size_t)3 * 2048 * nblk + (size_t)2 * 3 * 2048) * sizeof(double)));
      c->spec_lats = 1;
    }
    double* bins = c->d_spec + (size_t)3 * 2048 * nblk;
    double2* F = c->d_cplx;
    CU(launch_to_complex(c->fp32, arr_ptr(c, 0, c->parity, 2 * field + what), F, H.V, c->stream));
    ADJ_TRY(fft3d(c, H.N, F, -1));
    CU(launch_bins(F, H.N, dk_bin, nb, nblk, c->d_spec, H.kIR, H.dx, bins, c->stream));
    CU(launch_spectrum_seed(c->fp32, F, H.N, dk_bin, nb, bin, bins, H.kIR, H.dx, c->adj.d_out, 0, nullptr,
                            c->stream));
    ADJ_TRY(fft3d(c, H.N, F, +1));
    CU(launch_spectrum_seed(c->fp32, F, H.N, dk_bin, nb, bin, bins, H.kIR, H.dx, c->adj.d_out, 1,
                            lam[2 * field + what], c->stream));
    c->launches += 5;
  }
  // ---- reverse sweep: coefficients of the recorded passes, last first ----
  {
    std::vector<double> hlog((size_t)nrev * ADJ_LOG_W), hrev((size_t)nrev * ADJ_COEF_W, 0.0);
    CU(cudaMemcpyAsync(hlog.data(), dlog, hlog.size() * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    CU(cudaStreamSynchronize(c->stream));
    const double al = c->alpha, C = c->p.fstar_over_mp * c->p.fstar_over_mp / 3.0;
    const double iV = 1.0 / (double)H.V, idx2 = 1.0 / (H.dx * H.dx);
    for (long long i = 0; i < nrev; ++i) {
      const long long k = nrev - 1 - i;
      const double* lg = &hlog[(size_t)k * ADJ_LOG_W];
      double* rc = &hrev[(size_t)i * ADJ_COEF_W];
      for (int m = 0; m < 4; ++m) rc[m] = lg[m];
      if (!self) continue;
      // Friedmann kicks of forward pass k at a = a_k (K_a = C a^{2 alpha+1} [(alpha-2) E_K + alpha E_G
      // + (alpha+1) E_V]): dK_a/dpi = C (alpha-2) a^{2 alpha-5} pi/V, dK_a/dphi = C a^{2 alpha+1}
      // [-alpha Lap phi/(a^2 dx^2) + (alpha+1) dV/dphi]/V, dK_a/dq = C (alpha+1) a^{2 alpha+1} dV/dq/V
      const double a = lg[4], win = fw[(size_t)k].win, wout = fw[(size_t)k].wout;
      const double kpi = C * (al - 2.0) * std::pow(a, 2.0 * al - 5.0) * iV;
      rc[4] = win * kpi;
      rc[5] = wout * kpi;
      rc[6] = (win + wout) * C * (-al) * std::pow(a, 2.0 * al - 1.0) * idx2 * iV;
      rc[7] = (win + wout) * C * (al + 1.0) * std::pow(a, 2.0 * al + 1.0) * iV;
      rc[8] = 1.0 / a;
      rc[9] = lg[5];
      // the pass's drift: a_k = a_{k-1} + w b, cd = w abar^{alpha-3}, abar = (a_{k-1} + a_k)/2
      const double w = k > 0 ? fw[(size_t)k - 1].dnext : 0.0;
      if (w != 0.0) {
        const double abar = 0.5 * (hlog[(size_t)(k - 1) * ADJ_LOG_W + 4] + a);
        rc[10] = w * (al - 3.0) * std::pow(abar, al - 4.0);
        rc[11] = w;
      }
    }
    CU(cudaMemcpyAsync(dcoef, hrev.data(), hrev.size() * sizeof(double), cudaMemcpyHostToDevice, c->stream));
    // the closing pass, then chunk by chunk, each started from its saved end state
    long long done = 0;
    if (nrev > chunk_first[nchunk]) {
      ADJ_TRY(launch_adjoint(c, dcoef, 1));
      done = 1;
    }
    for (int ch = nchunk - 1; ch >= 0; --ch) {
      ADJ_TRY(copy_state(ckpt, ch + 1, false));
      long long left = chunk_first[ch + 1] - chunk_first[ch];
      while (left > 0) {
        const int mm = (int)std::min<long long>(4096, left);
        ADJ_TRY(launch_adjoint(c, dcoef + (size_t)ADJ_COEF_W * done, mm));
        done += mm;
        left -= mm;
      }
    }
    ADJ_TRY(copy_state(ckpt, 0, false));
  }
  double out[2] = {0.0, 0.0}, adj3[3] = {0.0, 0.0, 0.0};
  CU(cudaMemcpyAsync(out, c->adj.d_out, 2 * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  CU(cudaMemcpyAsync(adj3, &c->d_sc[0].adjq, 3 * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  if (dJ_dstate) {
    for (int a = 0; a < na; ++a) {
      const void* src = (char*)c->adj.lam + ((size_t)c->parity * na + a) * ab;
      CU(launch_convert(c->fp32, 1, src, c->d_tmp, H.V, c->stream));
      ++c->launches;
      CU(cudaMemcpyAsync(dJ_dstate + (size_t)a * H.V, c->d_tmp, H.V * sizeof(double), cudaMemcpyDefault,
                         c->stream));
    }
  }
  CU(cudaStreamSynchronize(c->stream));
  const cl_status st = check_status(c);
  if (st == CL_ETIMEOUT) sc0.status = CL_ETIMEOUT;  // kept for later calls
  CU(cudaMemcpyAsync(&c->d_sc[0], &sc0, sizeof(sc0), cudaMemcpyHostToDevice, c->stream));
  CU(cudaStreamSynchronize(c->stream));
  cleanup();
#undef ADJ_TRY
  c->obs_valid = false;
  if (J) *J = out[0];
  if (dJ_dq) *dJ_dq = out[1] + adj3[0];
  if (dJ_dscale) {
    dJ_dscale[0] = self ? adj3[1] : 0.0;
    dJ_dscale[1] = self ? adj3[2] : 0.0;
  }
  return st;
}

cl_status cl_ic_amplitude_grad(cl_ctx* c, const double* dJ_dstate, double* out) {
  if (!c || !dJ_dstate || !out) return fail(c, CL_EINVAL, "NULL argument");
  if (c->nlat != 1 || c->model >= CL_MODEL_U1_HIGGS)
    return fail(c, CL_EUNSUPPORTED, "amplitude gradients cover single scalar lattices");
  if (c->p.expansion == CL_EXP_SELF && c->p.b0_mode == 1)
    return fail(c, CL_EUNSUPPORTED, "with a' from lattice averages the initial b depends on the amplitudes");
  const LatHost& H = c->lats[0];
  double2* Lf = c->d_cplx;
  double2* Lp = c->d_cplx + H.V;
  double* dev_out = nullptr;
  CU(cudaMalloc(&dev_out, 2 * (size_t)H.V * sizeof(double)));
  cl_status s = CL_OK;
  for (int f = 0; f < c->nf && s == CL_OK; ++f) {
    for (int w = 0; w < 2 && s == CL_OK; ++w) {
      double2* dst = w == 0 ? Lf : Lp;
      if (cudaMemcpyAsync(c->d_tmp, dJ_dstate + (size_t)(2 * f + w) * H.V, H.V * sizeof(double),
                          cudaMemcpyDefault, c->stream) != cudaSuccess ||
          launch_to_complex(0, c->d_tmp, dst, H.V, c->stream) != cudaSuccess) {
        s = fail(c, CL_ECUDA, "amplitude gradient: transfer failed");
        break;
      }
      ++c->launches;
      s = fft3d(c, H.N, dst, +1);
    }
    if (s != CL_OK) break;
    if (launch_ic_amp_grad(Lf, Lp, dev_out, dev_out + H.V, c->d_lat, c->d_sc, H.ic, f, H.V, c->stream) !=
            cudaSuccess ||
        cudaMemcpyAsync(out + (size_t)(2 * f) * H.V, dev_out, 2 * (size_t)H.V * sizeof(double),
                        cudaMemcpyDefault, c->stream) != cudaSuccess) {
      s = fail(c, CL_ECUDA, "amplitude gradient: launch failed");
      break;
    }
    ++c->launches;
    if (cudaStreamSynchronize(c->stream) != cudaSuccess) s = fail(c, CL_ECUDA, "amplitude gradient: sync");
  }
  cudaStreamSynchronize(c->stream);
  cudaFree(dev_out);
  return s;
}

}  // extern "C"
