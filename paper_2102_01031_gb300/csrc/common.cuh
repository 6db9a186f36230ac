// common.cuh -- device-side structures and PTX helpers shared by the kernels
// of the lattice kick-drift library (sm_103a).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "worklist.h"  // Seg, MAX_SEG_PER_CTA

#include "cl.h"

namespace clg {

constexpr int NQ = 16;       // partial-sum slots per work segment
constexpr int MAX_ARR = 10;  // lattice arrays per buffer (U(1): 5 fields + 5 momenta)
constexpr int CONSUMER_WARPS = 16;           // warps per DK-pass CTA
constexpr int THREADS = 32 * CONSUMER_WARPS;
static_assert(CONSUMER_WARPS >= NQ, "the tail sums one slot per warp");

// Per-lattice constants, read-only during a pass.
struct LatConst {
  int N, BY, YT, model, nf, narr, expansion, esz;
  int slot_begin, slot_end;  // partial-sum slots of this lattice: [slot_begin, slot_end)
  int int_alpha, alpha_i;    // int_alpha: alpha is the integer alpha_i in [-4, 4] (powers by multiplication)
  long long V;
  double dx, alpha, q, lam, v, gQ, fo2, fm2, omega_eos;
  double inv_V, inv_dx2;
  double u1_gd, u1_cJ, u1_cC;  // U(1): gQ dx, (f_s/omega_s)^2 gQ/dx, 1/(gQ dx^3)
  double gQB;                  // doublet model: SU(2) coupling times charge
  double qG, qH, Qc;           // lphi4SU2U1: potential couplings, charge of vphi (units of the doublet's)
  int su2_nzc, su2_pad;        // doublet model: z-chunks of the pass's work items
  void* buf[2][MAX_ARR];  // ping-pong storage; array 2f = field f, 2f+1 = its momentum
};

// The evolving scalars of a lattice (the first members of LatScalars).
struct ScalarState {
  double a, b, eta;
  double cd, cdA;
  double apow1, apow3, apowm1;
  double a0, eta0, Hfix, rho0;
  double pi2, pi2A;
};

// Per-lattice evolving scalars (device resident, FP64).
struct LatScalars {
  double a, b, eta;
  double cd, cdA;                 // drift coefficients for the next pass (fields, links)
  double apow1, apow3, apowm1;    // a^{1+alpha}, a^{3+alpha}, a^{alpha-1} at the current a
  double a0, eta0, Hfix, rho0;
  double pi2;                     // sum of pi^2 after the last kick (the next kick's pre-kick sum)
  double pi2A;                    // the same for the U(1) link momenta
  cl_energies_t obs;              // last measurement
  double adjq;                    // adjoint sweep: accumulated dJ/dq of the passes
  double adja, adjb;              // adjoint sweep: dJ/da, dJ/db (self-consistent expansion)
  double H_ic;                    // a'/a the initial conditions were drawn with
  int status, pad;
};


// ---------------------------------------------------------------------------
// Sine and cosine of link and plaquette angles (the gauge passes).
// The library's FP32 sine and cosine, out of line: the passes take them only for
// angles beyond pi/4, and one copy keeps the kernels' code small (instruction cache).
static __device__ __noinline__ float sin_slow(float x) { return sinf(x); }
static __device__ __noinline__ void sincos_slow(float x, float* s, float* c) { sincosf(x, s, c); }

// FP32: for |x| <= pi/4 the Taylor series about 0 in Horner form (the first
// omitted terms, x^11/11! and x^12/12!, stay below 2e-9 there), else the
// library; link and plaquette angles are small in practice.  FP64: the library.
static __device__ __forceinline__ float sin_taylor(float x2) {  // sin(x)/x from x^2
  return fmaf(x2, fmaf(x2, fmaf(x2, fmaf(x2, 1.f / 362880.f, -1.f / 5040.f), 1.f / 120.f), -1.f / 6.f), 1.f);
}
static __device__ __forceinline__ float cos_taylor(float x2) {
  return fmaf(x2, fmaf(x2, fmaf(x2, fmaf(x2, fmaf(x2, -1.f / 3628800.f, 1.f / 40320.f), -1.f / 720.f), 1.f / 24.f),
              -0.5f),
              1.f);
}
static __device__ __forceinline__ void sincos_t(float x, float& s, float& c) {
  if (fabsf(x) <= 0.78539816f) {
    const float x2 = x * x;
    s = x * sin_taylor(x2);
    c = cos_taylor(x2);
  } else {
    sincos_slow(x, &s, &c);
  }
}
static __device__ __forceinline__ float sin_t(float x) {
  if (fabsf(x) <= 0.78539816f) return x * sin_taylor(x * x);
  return sin_slow(x);
}
static __device__ __forceinline__ void sincos_t(double x, double& s, double& c) { sincos(x, &s, &c); }
static __device__ __forceinline__ double sin_t(double x) { return sin(x); }

// Bring a line into L1 (no register, no wait).
template <typename T>
__device__ __forceinline__ void prefetch_l1(const T* p) {
  asm volatile("prefetch.global.L1 [%0];" ::"l"(p));
}

// Sites per thread along x in the U(1) pass (8-byte vectors in FP32, scalars in FP64).
constexpr int u1_vx(int esz) { return esz == 4 ? 2 : 1; }

// What a refill needs to know about a segment, cached in shared memory.
struct IssueInfo {
  int z0, nz, dir, ylo, N, rows, pad0, pad1;
  const void* src[2][MAX_ARR];  // by buffer parity
};

// Shared-memory layout behind the stage ring of a DK pass (byte offsets).
constexpr size_t SM_FULL = 0;                                   // 8 mbarriers
constexpr size_t SM_RELEASED = 64;                              // 8 release counts
constexpr size_t SM_OFF = 128;                                  // MAX_SEG_PER_CTA + 1 plane offsets
constexpr size_t SM_RED = (SM_OFF + 4 * (MAX_SEG_PER_CTA + 1) + 127) / 128 * 128;  // 33 x NQ doubles
constexpr size_t SM_FLAG = SM_RED + 33 * NQ * 8;                // 4 ints + pending tails
constexpr size_t SM_INFO = (SM_FLAG + 16 + 4 * MAX_SEG_PER_CTA + 127) / 128 * 128;  // IssueInfo[]
constexpr size_t SM_TAIL_BYTES = SM_INFO + MAX_SEG_PER_CTA * sizeof(IssueInfo);

// Kick/drift weights of one pass (see the schedule in capi.cu).
struct PassStep {
  double ck, wout, win, dnext;
};

struct PassArgs {
  const LatConst* lat;
  LatScalars* sc;
  const Seg* segs;
  const int* cta_seg;        // [gridDim.x + 1]
  double* partials;          // [NQ][nslot]: quantity-major, so a lattice's slots are contiguous
  unsigned* counters;        // [nlat]
  double ck, wout, win, dnext;
  int parity, write, set_rho0, stages;
  unsigned stage_bytes_max;  // bytes of one stage (max over lattices)
  int nlat;                  // lattices advanced by the launch
  int nslot;                 // partial-sum slots of the launch (all lattices)
  unsigned long long wait_limit_ns;  // bound of every wait
  // several passes in one cooperative launch (npass > 1): weights per pass and
  // two monotonic counters (writes arrived, tails done), zeroed before launch
  const PassStep* steps;
  int npass, pad2;
  unsigned* gsync;
  // forward passes: when set, what each pass used, for an adjoint sweep (one
  // lattice), ADJ_LOG_W words per pass at log + ADJ_LOG_W (log_base + pass):
  // block 0 writes cd, c_k, c_k a^{1+alpha}/dx^2, c_k a^{3+alpha}, a; the tail
  // writes the a-derivative of the pass's two Friedmann kicks,
  // w_in dK_a/da (post-kick momenta) + w_out dK_a/da (pre-kick momenta)
  double* log;
  long long log_base;
  // adjoint passes: ADJ_COEF_W coefficients per reversed pass (pass_adjoint.cu)
  const double* adj;
};
constexpr int ADJ_LOG_W = 6;
constexpr int ADJ_COEF_W = 12;

// Initial-condition parameters (program units).
struct ICArgs {
  double phi0[4], dphi0[4];
  double amp2, kcut, kIR, H0, q, lam, v;
  double qG, qH;  // lphi4SU2U1 potential couplings
  unsigned long long seed;
  int model, nf;
};

// One batched 1-D FFT along `axis` of an N^3 complex array.
struct FftPlan {
  int N, nrad, axis, sign;
  int rad[16];
  int batch;             // lines per CTA (a divisor of N)
  const double2* tw;     // tw[e] = exp(+2 pi i e/N), e < N
  int pitch;             // x extent of the array in memory (N; N/2 + 1 for a half spectrum)
  int nu;                // lines along the fastest other index (axes 1, 2: the columns kept, <= pitch)
};

// ---------------------------------------------------------------------------
// mbarrier + bulk async copy (TMA, 1-D) helpers, inline PTX.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count)
               : "memory");
}

__device__ __forceinline__ void fence_mbar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void fence_proxy_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void fence_proxy_async_global() {
  asm volatile("fence.proxy.async.global;" ::: "memory");
}

__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile(
      "{\n\t.reg .b64 st;\n\t"
      "mbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1;\n\t}" ::"r"(smem_u32(bar)),
      "r"(bytes)
      : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile(
      "{\n\t.reg .b64 st;\n\t"
      "mbarrier.arrive.shared::cta.b64 st, [%0];\n\t}" ::"r"(smem_u32(bar))
      : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// Bulk copy global -> shared, completion counted on `bar` (bytes % 16 == 0,
// both addresses 16-byte aligned).
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Bounded wait until the counter *c reaches `target` (other CTAs of a
// cooperative launch increment it); false after limit_ns.
__device__ __forceinline__ bool wait_counter(const unsigned* c, unsigned target,
                                             unsigned long long limit_ns) {
  if ((int)(ld_acquire_u32(c) - target) >= 0) return true;
  const unsigned long long t0 = global_ns();
  for (uint32_t i = 0; i < (1u << 30); ++i) {
    __nanosleep(64);
    if ((int)(ld_acquire_u32(c) - target) >= 0) return true;
    if ((i & 15u) == 15u && global_ns() - t0 > limit_ns) return false;
  }
  return false;
}

// Bounded wait on an mbarrier phase: gives up (returns false) after `limit_ns`
// nanoseconds or 2^30 unsuccessful try_wait rounds, whichever comes first.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity,
                                                  unsigned long long limit_ns) {
  if (mbar_try_wait(bar, parity)) return true;
  const unsigned long long t0 = global_ns();
  for (uint32_t i = 0; i < (1u << 30); ++i) {
    if (mbar_try_wait(bar, parity)) return true;
    if ((i & 63u) == 63u && global_ns() - t0 > limit_ns) return false;
  }
  return false;
}

// Fused multiply-add in the storage precision (fmaf for float, never promoted to double).
__device__ __forceinline__ float fmaT(float a, float b, float c) { return fmaf(a, b, c); }
__device__ __forceinline__ double fmaT(double a, double b, double c) { return fma(a, b, c); }

// Error-free transformation of a + b (Knuth's TwoSum): s + e == a + b exactly.
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = a + b;
  const float bb = s - a;
  e = (a - (s - bb)) + (b - bb);
}

// 16-byte vector of T
template <typename T> struct V16;
template <> struct V16<float> { typedef float4 type; static constexpr int n = 4; };
template <> struct V16<double> { typedef double2 type; static constexpr int n = 2; };

// Kahan-compensated accumulator (FP32 storage path) / plain (FP64 path).
template <typename T> struct Acc {
  T s, c;
  __device__ __forceinline__ void zero() { s = 0; c = 0; }
  __device__ __forceinline__ void add(T x) {
    T y = x - c;
    T t = s + y;
    c = (t - s) - y;
    s = t;
  }
  __device__ __forceinline__ double value() const { return (double)s - (double)c; }
};
template <> struct Acc<double> {
  double s;
  __device__ __forceinline__ void zero() { s = 0; }
  __device__ __forceinline__ void add(double x) { s += x; }
  __device__ __forceinline__ double value() const { return s; }
};

// Warp sum of one accumulator, returned on lane 0.  FP32 storage: the
// (sum, -compensation) pairs of the lanes are combined pairwise with TwoSum
// in FP32 and converted to FP64 once; FP64 storage: plain FP64 tree.
__device__ __forceinline__ double warp_sum(const Acc<float>& a) {
  float hi = a.s, lo = -a.c;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const float h2 = __shfl_down_sync(0xffffffffu, hi, o);
    const float l2 = __shfl_down_sync(0xffffffffu, lo, o);
    float s, e;
    two_sum(hi, h2, s, e);
    hi = s;
    lo = lo + l2 + e;
  }
  return (double)hi + (double)lo;
}
__device__ __forceinline__ double warp_sum(const Acc<double>& a) {
  double v = a.s;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}

// Fixed-order FP64 sum of part[begin .. end) over one warp (result on every
// lane): lane l adds slots begin + l, + 32, ..., all of its first eight loads
// issued before any add (one memory round trip for up to 256 slots), then a
// shuffle tree.  The values were written by other CTAs of the launch (read
// past L1).
__device__ __forceinline__ double warp_slot_sum(const double* part, int begin, int end, int lane) {
  double v[8];
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    const int k = begin + lane + 32 * i;
    v[i] = k < end ? __ldcg(part + k) : 0.0;
  }
  double s = 0.0;
#pragma unroll
  for (int i = 0; i < 8; ++i) s += v[i];
  for (int k = begin + lane + 256; k < end; k += 32) s += __ldcg(part + k);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  return s;
}

}  // namespace clg
