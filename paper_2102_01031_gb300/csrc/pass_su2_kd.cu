// pass_su2_kd.cu -- the doublet-model pass in kick-then-drift form (without
// self-consistent expansion): the kick of the SU(2) x U(1) doublet model (Sec. 4.3 Hamiltonian
// form in temporal gauge, links, plaquettes and covariant derivatives of the
// U(1) and SU(N) toolkits of Sec. 4.2), and of the lphi4SU2U1 model's singlet
// and U(1)-charged scalar (Sec. 4.5), each site's drift right after its kick.
//
// The equations are those of pass_su2.cu; what differs is where the work is
// done.  Without self-consistent expansion a(eta) is constant or a fixed power
// law, so the drift coefficient of a pass is known before its sums and the
// pass's own drift can follow its kick at each site (kick, then drift by the
// pass's dnext).  The values each site
// goes through are the same as with the drift deferred to the next pass, but
// no neighbour needs to be drifted on read: a stage holds the source buffer's
// raw fields.
//
// Kernel layout.  A work item is a TX x TY tile of x-y sites (32 or 16 wide, 8
// rows; 16 rows for the FP32 lphi4SU2U1 step pass) over a chunk of z-planes
// (su2_work.h); the CTA's items form one sequence of planes (each item adds the
// plane below its chunk) that a three-stage ring of shared memory streams in:
// per plane, every field array's tile rows plus a halo row on each side, each
// row from 16 bytes before the tile to 16 bytes after it, in 16-byte pieces the
// threads copy themselves with cp.async (each thread the same piece of a fixed
// list of arrays, its place on the lattice, periodic in x and y, found once per
// item).  A plane's copies are counted on its stage's "full" mbarrier; every
// warp arrives on the stage's "empty" mbarrier when done with it, and the
// copies of the plane two ahead go into a stage once it is empty: no CTA
// barrier.  Each thread's own momenta of the next plane are copied into a slot
// beside the stages (prefetched into L1 where the slot does not fit).
//
// Each plaquette is formed once per site (xy, xz, yz at n) and serves the
// staples of its links at n directly (P and P^dag); along z it also serves the
// two links it reaches from below, rotated by a link,
//     m(L_iz(n)) = m(U_z^dag(n-z) P_iz(n-z)^dag U_z(n-z)),
// which the thread forms at plane z - 1 and carries to plane z in registers.
// The lower staples across x and y are formed directly at each site (handing
// them on between lanes would leave the tile's edge column to one lane of a
// warp, which costs the whole warp the work).  The same goes for the compact
// U(1) plaquette sines and the backward hops W_i^dag(n-i) psi(n-i): carried
// along z, direct across x and y.  In the FP32 step passes the seven U(1)
// plaquette sines are evaluated two at a time and the six plaquette products and
// four lower staples are formed two at a time, in the packed two-lane FP32 form,
// each lane rounded as the single evaluation (trig2.cuh, Q2 below).
#include "su2_common.cuh"
#include "kd_drift.cuh"
#include "trig2.cuh"

namespace clg {

namespace {

template <typename T>
struct V3 {
  T x, y, z;
};

// vector part (a b)_{x,y,z} of a quaternion product
template <typename T>
__device__ __forceinline__ V3<T> qvec(const Q4<T>& a, const Q4<T>& b) {
  V3<T> r;
  r.x = fmaT(a.y, b.z, fmaT(-a.z, b.y, fmaT(b.w, a.x, a.w * b.x)));
  r.y = fmaT(a.z, b.x, fmaT(-a.x, b.z, fmaT(b.w, a.y, a.w * b.y)));
  r.z = fmaT(a.x, b.y, fmaT(-a.y, b.x, fmaT(b.w, a.z, a.w * b.z)));
  return r;
}
// scalar part (a b)_w
template <typename T>
__device__ __forceinline__ T qsca(const Q4<T>& a, const Q4<T>& b) {
  return fmaT(-a.z, b.z, fmaT(-a.y, b.y, fmaT(-a.x, b.x, a.w * b.w)));
}
// vector part of U^dag (v.s) U for a unit quaternion U = (u0, u): the rotation
// of v by U^dag,  v + 2 (u x t - u0 t),  t = u x v
template <typename T>
__device__ __forceinline__ V3<T> rotc(const Q4<T>& u, const V3<T>& v) {
  const T tx = fmaT(u.y, v.z, -u.z * v.y), ty = fmaT(u.z, v.x, -u.x * v.z), tz = fmaT(u.x, v.y, -u.y * v.x);
  const T wx = fmaT(u.y, tz, -u.z * ty), wy = fmaT(u.z, tx, -u.x * tz), wz = fmaT(u.x, ty, -u.y * tx);
  V3<T> r;
  r.x = fmaT(T(2), fmaT(-u.w, tx, wx), v.x);
  r.y = fmaT(T(2), fmaT(-u.w, ty, wy), v.y);
  r.z = fmaT(T(2), fmaT(-u.w, tz, wz), v.z);
  return r;
}
template <typename T>
__device__ __forceinline__ V3<T> neg(const V3<T>& v) {
  V3<T> r;
  r.x = -v.x;
  r.y = -v.y;
  r.z = -v.z;
  return r;
}

// Two independent quaternion products at once (FP32, the packed two-lane form):
// lane 0 and lane 1 of every component are the two products, each lane rounded
// exactly as qmul / qvec round one product (a conjugated operand enters by exact
// sign changes, (-a)(-b) = ab), so the pass's results are the same bits.
struct Q2 {
  float2 w, x, y, z;
};
struct P3 {
  float2 x, y, z;
};
__device__ __forceinline__ Q2 q2(const Q4<float>& a, const Q4<float>& b) {
  return Q2{make_float2(a.w, b.w), make_float2(a.x, b.x), make_float2(a.y, b.y), make_float2(a.z, b.z)};
}
__device__ __forceinline__ float2 ng(float2 v) { return make_float2(-v.x, -v.y); }
__device__ __forceinline__ Q4<float> lane_of(const Q2& a, int l) {
  return l ? Q4<float>{a.w.y, a.x.y, a.y.y, a.z.y} : Q4<float>{a.w.x, a.x.x, a.y.x, a.z.x};
}
__device__ __forceinline__ V3<float> lane_of(const P3& a, int l) {
  return l ? V3<float>{a.x.y, a.y.y, a.z.y} : V3<float>{a.x.x, a.y.x, a.z.x};
}
// a b (qmul)
__device__ __forceinline__ Q2 qmul2(const Q2& a, const Q2& b) {
  Q2 r;
  r.w = __ffma2_rn(ng(a.z), b.z, __ffma2_rn(ng(a.y), b.y, __ffma2_rn(ng(a.x), b.x, __fmul2_rn(a.w, b.w))));
  r.x = __ffma2_rn(a.y, b.z, __ffma2_rn(ng(a.z), b.y, __ffma2_rn(b.w, a.x, __fmul2_rn(a.w, b.x))));
  r.y = __ffma2_rn(a.z, b.x, __ffma2_rn(ng(a.x), b.z, __ffma2_rn(b.w, a.y, __fmul2_rn(a.w, b.y))));
  r.z = __ffma2_rn(a.x, b.y, __ffma2_rn(ng(a.y), b.x, __ffma2_rn(b.w, a.z, __fmul2_rn(a.w, b.z))));
  return r;
}
// a b^dag (qmul(a, qconj(b)))
__device__ __forceinline__ Q2 qmul2_cb(const Q2& a, const Q2& b) {
  Q2 r;
  r.w = __ffma2_rn(a.z, b.z, __ffma2_rn(a.y, b.y, __ffma2_rn(a.x, b.x, __fmul2_rn(a.w, b.w))));
  r.x = __ffma2_rn(ng(a.y), b.z, __ffma2_rn(a.z, b.y, __ffma2_rn(b.w, a.x, __fmul2_rn(ng(a.w), b.x))));
  r.y = __ffma2_rn(ng(a.z), b.x, __ffma2_rn(a.x, b.z, __ffma2_rn(b.w, a.y, __fmul2_rn(ng(a.w), b.y))));
  r.z = __ffma2_rn(ng(a.x), b.y, __ffma2_rn(a.y, b.x, __ffma2_rn(b.w, a.z, __fmul2_rn(ng(a.w), b.z))));
  return r;
}
// vector part of a b (qvec)
__device__ __forceinline__ P3 qvec2(const Q2& a, const Q2& b) {
  P3 r;
  r.x = __ffma2_rn(a.y, b.z, __ffma2_rn(ng(a.z), b.y, __ffma2_rn(b.w, a.x, __fmul2_rn(a.w, b.x))));
  r.y = __ffma2_rn(a.z, b.x, __ffma2_rn(ng(a.x), b.z, __ffma2_rn(b.w, a.y, __fmul2_rn(a.w, b.y))));
  r.z = __ffma2_rn(a.x, b.y, __ffma2_rn(ng(a.y), b.x, __ffma2_rn(b.w, a.z, __fmul2_rn(a.w, b.z))));
  return r;
}
// vector part of a b^dag (qvec(a, qconj(b)))
__device__ __forceinline__ P3 qvec2_cb(const Q2& a, const Q2& b) {
  const Q2 r = qmul2_cb(a, b);
  return P3{r.x, r.y, r.z};
}

// Asynchronous copies global -> shared by each thread (cp.async): 16 bytes (both
// addresses 16-byte aligned), or one element; completion either counted on an
// mbarrier (arrive once all of the thread's earlier copies landed) or awaited
// per thread by commit groups.
__device__ __forceinline__ void cp_async16(void* dst, const void* src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_u32(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_el(float* dst, const float* src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(smem_u32(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_el(double* dst, const double* src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(smem_u32(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_arrive(uint64_t* bar) {
  asm volatile("cp.async.mbarrier.arrive.noinc.shared::cta.b64 [%0];" ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_committed() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }

// Stage geometry: field array f of a stage holds HR = TY + 2 rows (the tile's
// and a halo row each side) of RW elements, from EPC = 16 B before the tile to
// 16 B after it; the tile's site (tx, ty) is element (ty + 1) RW + EPC + tx.
template <typename T, int TX, int TY, bool FULL>
struct KdGeom {
  static constexpr int EPC = 16 / (int)sizeof(T);
  static constexpr int RW = TX + 2 * EPC;
  static constexpr int HR = TY + 2;
  static constexpr int NFA = FULL ? 22 : 19;  // psi (4), A (3), U (12), [phi_s, vphi (2)]
  static constexpr int AE = HR * RW;
  static constexpr size_t STAGE = ((size_t)NFA * AE * sizeof(T) + 127) / 128 * 128;
  // a stage row in 16-byte pieces: NCOL per row, CPA per array
  static constexpr int NCOL = RW / EPC;
  static constexpr int CPA = HR * NCOL;
  // each thread's own momenta of the next plane in a slot after the stages (16
  // arrays, 19 for lphi4SU2U1); the lphi4SU2U1 pass with 8-row tiles, two CTAs
  // per SM, has no room for it and reads its momenta through L1
  static constexpr bool SLOT = !FULL || TY >= 16;
  static constexpr int NM = FULL ? 19 : 16;
  static constexpr size_t MSLOT = SLOT ? ((size_t)NM * TX * TY * sizeof(T) + 127) / 128 * 128 : 0;
  static constexpr size_t SMEM = 3 * STAGE + MSLOT;
};

// stage array f -> state array: psi 0..3, A 8..10, U 14..25, phi_s 35, vphi 37, 38
__device__ __forceinline__ int kd_state_array(int f) {
  return f < 4 ? f : (f < 7 ? f + 4 : (f < 19 ? f + 7 : (f == 19 ? SS : f + 17)));
}

enum : int { KF = 0, KA = 4, KU = 7, KS = 19, KV = 20 };  // stage arrays

}  // namespace

// RED: 0 = no sums, 2 = full measurement (the Friedmann sums of RED 1 are
// only needed with self-consistent expansion).  FULL: the lphi4SU2U1 model.  NC: 0 = the
// lattice size from the lattice constants; > 0 = built for N = NC (every array
// offset a compile-time constant).
template <typename T, int RED, int TX, int TY, bool FULL, int NC = 0>
__global__ void __launch_bounds__(TX * TY, (RED == 2 || sizeof(T) == 8) ? 1 : 2048 / (TX * TY * 4))
    kd_pass_su2(const PassArgs P) {
  using G = KdGeom<T, TX, TY, FULL>;
  constexpr int EPC = G::EPC, RW = G::RW, NFA = G::NFA, AE = G::AE;
  constexpr int nth = TX * TY, NW = nth / 32;
  constexpr bool SLOT = G::SLOT;
  constexpr int NACC = RED == 0 ? 1 : (FULL ? 29 : 23);
  static_assert(RED == 0 || RED == 2, "kick-then-drift passes take no Friedmann sums");
  extern __shared__ __align__(128) unsigned char smem[];
  __shared__ double red_s[SU2_NQ][9];
  __shared__ unsigned last_s;
  __shared__ __align__(8) uint64_t full_bar[3];   // per stage: every thread's copies of its plane landed
  __shared__ __align__(8) uint64_t empty_bar[3];  // per stage: every warp done with its plane
  __shared__ volatile int tflag;                   // a wait of this CTA ran out

  const LatConst& L = P.lat[0];
  const int N = NC ? NC : L.N;
  const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * TX + tx;
  const int lane = tid & 31, warp = tid >> 5;
  const long long NN = (long long)N * N, V = NC ? (long long)NC * NC * NC : L.V;
  const int parity = P.parity;
  const T* const src = reinterpret_cast<const T*>(L.buf[parity][0]);
  T* const dst = reinterpret_cast<T*>(L.buf[parity ^ 1][0]);
  // array a of the source and destination buffers, indexed by site (V < 2^32)
  auto sa = [&](int a) { return src + (size_t)a * (size_t)V; };
  auto da = [&](int a) { return dst + (size_t)a * (size_t)V; };
  const int ntx = N / TX, ntiles = ntx * (N / TY), nzc = L.su2_nzc, nitems = ntiles * nzc;

  // coefficients: FP64 products by one lane, broadcast in the storage precision
  T cf[17];
  if (lane == 0) {
    const LatScalars* SC = P.sc;
    const double ck = P.ck, ap1 = __ldcg(&SC->apow1), apm1 = __ldcg(&SC->apowm1), dx = L.dx;
    double kd, kdA;  // this pass's drift, after its kick
    kd_drift_coefficients(L, SC, P.dnext, kd, kdA);
    cf[0] = (T)kd;
    cf[1] = (T)kdA;
    cf[2] = (T)(0.5 * L.gQB * dx * kdA);                         // half the SU(2) drift angle per momentum
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
  const T kd = cf[0], kdA = cf[1], hB = cf[2], A1 = cf[3], A3 = cf[4], AJA = cf[5], ACA = cf[6], AJB = cf[7],
          AMB = cf[8], gd = cf[9], v2 = cf[10], lam = cf[11], lam2 = cf[12], qG = cf[13], qH = cf[14],
          gdc = cf[15], AJC = cf[16];

  if (tid == 0) {
    for (int s = 0; s < 3; ++s) {
      mbar_init(&full_bar[s], nth);
      mbar_init(&empty_bar[s], NW);
    }
    fence_mbar_init();
    tflag = 0;
  }
  __syncthreads();

  // The CTA's planes form one sequence of positions (item by item, each item's
  // planes z0 - 1 .. z0 + nz); position p lives in stage p mod 3.  produced: the
  // positions whose copies have gone out; ptot: the positions of the sequence.
  int produced = 0, ptot = 0;
  for (int it = blockIdx.x; it < nitems; it += gridDim.x) {
    const int chunk = it / ntiles;
    ptot += (chunk + 1) * N / nzc - chunk * N / nzc + 2;
  }
  // Each thread copies the same 16-byte piece (column pc, row pr) of a fixed set
  // of arrays of every plane: with room for two sets, the CTA's two halves
  // (warp-uniform) take the first and the second half of the arrays, else the
  // first CPA threads take all of them.  pso: the piece's offset in a plane of the
  // lattice for the producer's current item (periodic in x and y).
  constexpr int NH = 2 * G::CPA <= nth ? 2 : 1, FPH = (NFA + NH - 1) / NH;
  const int ph = tid / (nth / NH), pt = tid - ph * (nth / NH);
  const bool pcopy = pt < G::CPA;
  const int pr = pt / G::NCOL, pc = pt - pr * G::NCOL;
  // the producer's item (CTA-uniform): its z-chunk length and the plane the next
  // position copies (pzp) with its index in the item (pj)
  int pit = blockIdx.x, pnz = 0, pzp = 0, pj = 0;
  unsigned pso = 0u;
  auto producer_item = [&]() {
    if (pit >= nitems) return;
    const int chunk = pit / ntiles, tile = pit - chunk * ntiles;
    const int z0 = chunk * N / nzc;
    pnz = (chunk + 1) * N / nzc - z0;
    const int x0 = (tile % ntx) * TX, y0 = (tile / ntx) * TY;
    pzp = z0 == 0 ? N - 1 : z0 - 1;
    pj = 0;
    int gx = x0 - EPC + pc * EPC, gy = y0 - 1 + pr;
    gx = gx < 0 ? gx + N : (gx >= N ? gx - N : gx);
    gy = gy < 0 ? gy + N : (gy >= N ? gy - N : gy);
    pso = (unsigned)(gy * N + gx);
  };
  producer_item();
  // The copies of a position go out in two bursts (part 0, then part 1 later in
  // the step, so that a thread's pieces do not queue up at once); after part 1
  // the thread's arrival on the stage's full barrier (once all its copies have
  // landed) and a commit group.
  auto produce = [&](int part) {
    if (pit >= nitems) return;
    const int s = produced % 3;
    if (pcopy) {
      T* const d = reinterpret_cast<T*>(smem + (size_t)s * G::STAGE) + pr * RW + pc * EPC;
      const T* const g = src + (size_t)((unsigned)pzp * (unsigned)NN + pso);
      constexpr int H0 = FPH / 2, H1 = FPH + (NFA - FPH) / 2;
      if (ph == 0 && part == 0) {
#pragma unroll
        for (int f = 0; f < H0; ++f) cp_async16(d + f * AE, g + (size_t)kd_state_array(f) * (size_t)V);
      } else if (ph == 0) {
#pragma unroll
        for (int f = H0; f < FPH; ++f) cp_async16(d + f * AE, g + (size_t)kd_state_array(f) * (size_t)V);
      } else if (part == 0) {
#pragma unroll
        for (int f = FPH; f < H1; ++f) cp_async16(d + f * AE, g + (size_t)kd_state_array(f) * (size_t)V);
      } else {
#pragma unroll
        for (int f = H1; f < NFA; ++f) cp_async16(d + f * AE, g + (size_t)kd_state_array(f) * (size_t)V);
      }
    }
    if (part == 0) return;
    cp_async_arrive(&full_bar[s]);
    cp_async_commit();
    ++produced;
    pzp = pzp + 1 == N ? 0 : pzp + 1;
    if (++pj == pnz + 2) {
      pit += gridDim.x;
      producer_item();
    }
  };
  auto wait_bar = [&](uint64_t* bar, int phase) {
    if (tflag) return;
    if (!mbar_wait_bounded(bar, (uint32_t)(phase & 1), P.wait_limit_ns)) tflag = 1;
  };
  // Step p works on positions p and p + 1: the copies of position p + 2 go out
  // (into the stage position p - 1 held, once every warp is done with it), their
  // first part at the step's beginning, the second (produce(1)) within the step.
  auto step_begin = [&](int p) {
    if (p >= 1) wait_bar(&empty_bar[(p - 1) % 3], (p - 1) / 3);
    if (!tflag) produce(0);
    if (p == 0) wait_bar(&full_bar[0], 0);
    if (p + 1 < ptot) wait_bar(&full_bar[(p + 1) % 3], (p + 1) / 3);
  };
  auto step_end = [&](int p) {
    __syncwarp();
    if (lane == 0) mbar_arrive(&empty_bar[p % 3]);
  };
  for (int k = 0; k < 2; ++k) {
    produce(0);
    produce(1);
  }

  auto stage = [&](int q) { return reinterpret_cast<const T*>(smem + (size_t)(q % 3) * G::STAGE); };
  const int o = (ty + 1) * RW + EPC + tx;
  auto ld = [&](const T* st, int f, int dx, int dy) -> T { return st[f * AE + o + dy * RW + dx]; };
  auto ld4 = [&](const T* st, int f, int dx, int dy) {
    const T* p = st + f * AE + o + dy * RW + dx;
    Q4<T> q;
    q.w = p[0];
    q.x = p[AE];
    q.y = p[2 * AE];
    q.z = p[3 * AE];
    return q;
  };

  // own momentum a (one of SP.., SPA.., SPB.., and for lphi4SU2U1 SPS, SPC..) of
  // site g: from the slot, or from global memory (prefetched into L1)
  T* const mslot = reinterpret_cast<T*>(smem + 3 * G::STAGE);
  auto mom = [&](int a, unsigned g) -> T {
    if constexpr (!SLOT) {
      return __ldg(sa(a) + g);
    } else {
      const int m = a < SPA ? a - SP : (a < SU ? a - SPA + 4 : (a < SS ? a - SPB + 7 : (a == SPS ? 16 : a - SPC + 17)));
      return mslot[m * nth + tid];
    }
  };

  Acc<T> acc[NACC];
#pragma unroll
  for (int k = 0; k < NACC; ++k) acc[k].zero();
  float nonfinite = 0.f;

  // carried along z from the plane below: U(1) plaquette sines xz and yz at n - z,
  // the lower staples m(L_xz(n)), m(L_yz(n)), the backward hop W_z^dag(n-z) psi(n-z),
  // and (FULL) phi_s(n - z) and vphi's backward hop along z
  T c_sxz = T(0), c_syz = T(0), c_s = T(0), c_w0 = T(0), c_w1 = T(0);
  V3<T> c_xz = {T(0), T(0), T(0)}, c_yz = {T(0), T(0), T(0)};
  Q4<T> c_bz;
  c_bz.w = c_bz.x = c_bz.y = c_bz.z = T(0);

  int q = 0;  // position of the item's first plane in the CTA's sequence
  for (int it = blockIdx.x; it < nitems; it += gridDim.x) {
    const int chunk = it / ntiles, tile = it - chunk * ntiles;
    const int z0 = chunk * N / nzc, nz = (chunk + 1) * N / nzc - z0;
    const int x0 = (tile % ntx) * TX, y0 = (tile / ntx) * TY;
    const unsigned gown = (unsigned)((y0 + ty) * N + x0 + tx);
    // the momenta of own site g: into the thread's slot, or into L1 where the slot does not fit
    auto prefetch_momenta = [&](unsigned g) {
      if constexpr (SLOT) {
#pragma unroll
        for (int m = 0; m < G::NM; ++m)
          cp_async_el(mslot + m * nth + tid,
                      sa(m < 4 ? SP + m : (m < 7 ? SPA + m - 4 : (m < 16 ? SPB + m - 7 : (m == 16 ? SPS : SPC + m - 17)))) + g);
        cp_async_commit();
      } else {
#pragma unroll
        for (int m = 0; m < 4; ++m) prefetch_l1(sa(SP + m) + g);
#pragma unroll
        for (int m = 0; m < 3; ++m) prefetch_l1(sa(SPA + m) + g);
#pragma unroll
        for (int m = 0; m < 9; ++m) prefetch_l1(sa(SPB + m) + g);
        prefetch_l1(sa(SPS) + g);
        prefetch_l1(sa(SPC) + g);
        prefetch_l1(sa(SPC + 1) + g);
      }
    };

    // ---- the carries for plane z0 from plane z0 - 1 (position q) and z0 (q + 1) ----
    step_begin(q);
    prefetch_momenta((unsigned)z0 * (unsigned)NN + gown);
    {
      const T* C = stage(q);
      const T* Pn = stage(q + 1);
      const T ax = ld(C, KA, 0, 0), ay = ld(C, KA + 1, 0, 0), az = ld(C, KA + 2, 0, 0);
      c_sxz = sin_rn(gd * ((ax + ld(C, KA + 2, 1, 0)) - (ld(Pn, KA, 0, 0) + az)));
      c_syz = sin_rn(gd * ((ay + ld(C, KA + 2, 0, 1)) - (ld(Pn, KA + 1, 0, 0) + az)));
      const Q4<T> Ux = ld4(C, KU, 0, 0), Uy = ld4(C, KU + 4, 0, 0), Uz = ld4(C, KU + 8, 0, 0);
      const V3<T> pxz = qvec(qmul(Ux, ld4(C, KU + 8, 1, 0)), qconj(qmul(Uz, ld4(Pn, KU, 0, 0))));
      const V3<T> pyz = qvec(qmul(Uy, ld4(C, KU + 8, 0, 1)), qconj(qmul(Uz, ld4(Pn, KU + 4, 0, 0))));
      c_xz = neg(rotc(Uz, pxz));
      c_yz = neg(rotc(Uz, pyz));
      T s, c;
      sincos_t(gd * az, s, c);
      c_bz = udmul(Uz, ld4(C, KF, 0, 0));
      phase(c_bz, c, -s);
      if constexpr (FULL) {
        c_s = ld(C, KS, 0, 0);
        const T b0 = ld(C, KV, 0, 0), b1 = ld(C, KV + 1, 0, 0);
        sincos_t(gdc * az, s, c);
        c_w0 = c * b0 - s * b1;
        c_w1 = c * b1 + s * b0;
      }
    }
    if (!tflag) produce(1);
    step_end(q);

    for (int j = 1; j <= nz; ++j) {
      const int z = z0 + j - 1;
      const unsigned g = (unsigned)z * (unsigned)NN + gown;
      if (!SLOT && j < nz) prefetch_momenta(g + (unsigned)NN);
      step_begin(q + j);
      // this plane's momenta (the copies begun just now are not committed yet)
      if constexpr (SLOT) cp_async_wait_committed();
      const T* C = stage(q + j);
      const T* Pn = stage(q + j + 1);

      const Q4<T> psi = ld4(C, KF, 0, 0);
      const T ax = ld(C, KA, 0, 0), ay = ld(C, KA + 1, 0, 0), az = ld(C, KA + 2, 0, 0);

      // ---- compact U(1) plaquettes: sines at n, at n - x and n - y (direct), at n - z (carried) ----
      const T txy = gd * ((ax + ld(C, KA + 1, 1, 0)) - (ld(C, KA, 0, 1) + ay));
      const T txz = gd * ((ax + ld(C, KA + 2, 1, 0)) - (ld(Pn, KA, 0, 0) + az));
      const T tyz = gd * ((ay + ld(C, KA + 2, 0, 1)) - (ld(Pn, KA + 1, 0, 0) + az));
      const T axm = ld(C, KA, -1, 0);
      // the seven sines in one block (FP32: two at a time, one range check)
      const T ts[7] = {txy, txz, tyz, gd * ((axm + ay) - (ld(C, KA, -1, 1) + ld(C, KA + 1, -1, 0))),
                       gd * ((axm + az) - (ld(Pn, KA, -1, 0) + ld(C, KA + 2, -1, 0))),
                       gd * ((ld(C, KA, 0, -1) + ld(C, KA + 1, 1, -1)) - (ax + ld(C, KA + 1, 0, -1))),
                       gd * ((ld(C, KA + 1, 0, -1) + az) - (ld(Pn, KA + 1, 0, -1) + ld(C, KA + 2, 0, -1)))};
      T sn[7];
      sin_many(ts, sn);
      const T sxy = sn[0], sxz = sn[1], syz = sn[2], sxy_xm = sn[3], sxz_xm = sn[4], sxy_ym = sn[5], syz_ym = sn[6];
      const T Cc[3] = {(sxy - sxy_ym) + (sxz - c_sxz), (sxy_xm - sxy) + (syz - c_syz),
                       (sxz_xm - sxz) + (syz_ym - syz)};
      c_sxz = sxz;
      c_syz = syz;
      T s_mA = T(0);
      if constexpr (RED > 0) {
        const T h1 = sin_t(T(0.5) * txy), h2 = sin_t(T(0.5) * txz), h3 = sin_t(T(0.5) * tyz);
        s_mA = T(2) * (h1 * h1 + h2 * h2 + h3 * h3);
      }

      // ---- SU(2): the three plaquettes at n and the force vectors m(U_i S_i) ----
      const Q4<T> Ux = ld4(C, KU, 0, 0), Uy = ld4(C, KU + 4, 0, 0), Uz = ld4(C, KU + 8, 0, 0);
      V3<T> M[3];
      T s_mB = T(0);
      {
        V3<T> pxy, pxz, pyz, ryx, rzx, mxy, mzy;
        if constexpr (sizeof(T) == 4 && RED == 0) {
          // the step passes (FP32): products paired lane-wise, the same bits as below
          const Q2 UyUz = q2(Uy, Uz);
          const Q2 A = qmul2(q2(Ux, Ux), q2(ld4(C, KU + 4, 1, 0), ld4(C, KU + 8, 1, 0)));  // Axy, Axz
          const Q2 B = qmul2(UyUz, q2(ld4(C, KU, 0, 1), ld4(Pn, KU, 0, 0)));             // Bxy, Bxz (unconjugated)
          const Q2 Cp = qmul2(UyUz, q2(ld4(C, KU + 8, 0, 1), ld4(Pn, KU + 4, 0, 0)));    // Ayz, Byz (unconjugated)
          const P3 pp = qvec2_cb(A, B);
          pxy = lane_of(pp, 0);
          pxz = lane_of(pp, 1);
          pyz = qvec(lane_of(Cp, 0), qconj(lane_of(Cp, 1)));
          // lower staples in the x planes (of U_y, U_z) and in the y planes (of U_x, U_z)
          const Q4<T> uxm = ld4(C, KU, -1, 0), uym = ld4(C, KU + 4, 0, -1);
          const Q2 ix = qmul2(q2(ld4(C, KU + 4, -1, 0), ld4(C, KU + 8, -1, 0)), q2(ld4(C, KU, -1, 1), ld4(Pn, KU, -1, 0)));
          const P3 rr = qvec2(qmul2_cb(UyUz, ix), q2(uxm, uxm));
          const Q2 iy = qmul2(q2(ld4(C, KU, 0, -1), ld4(C, KU + 8, 0, -1)), q2(ld4(C, KU + 4, 1, -1), ld4(Pn, KU + 4, 0, -1)));
          const P3 mm = qvec2(qmul2_cb(q2(Ux, Uz), iy), q2(uym, uym));
          ryx = lane_of(rr, 0);
          rzx = lane_of(rr, 1);
          mxy = lane_of(mm, 0);
          mzy = lane_of(mm, 1);
        } else {
          const Q4<T> Axy = qmul(Ux, ld4(C, KU + 4, 1, 0)), Bxy = qconj(qmul(Uy, ld4(C, KU, 0, 1)));
          const Q4<T> Axz = qmul(Ux, ld4(C, KU + 8, 1, 0)), Bxz = qconj(qmul(Uz, ld4(Pn, KU, 0, 0)));
          const Q4<T> Ayz = qmul(Uy, ld4(C, KU + 8, 0, 1)), Byz = qconj(qmul(Uz, ld4(Pn, KU + 4, 0, 0)));
          pxy = qvec(Axy, Bxy);
          pxz = qvec(Axz, Bxz);
          pyz = qvec(Ayz, Byz);
          if constexpr (RED > 0) {
            s_mB = (pxy.x * pxy.x + pxy.y * pxy.y + pxy.z * pxy.z) / (T(1) + qsca(Axy, Bxy)) +
                   (pxz.x * pxz.x + pxz.y * pxz.y + pxz.z * pxz.z) / (T(1) + qsca(Axz, Bxz)) +
                   (pyz.x * pyz.x + pyz.y * pyz.y + pyz.z * pyz.z) / (T(1) + qsca(Ayz, Byz));
          }
          // lower staples of U_y(n), U_z(n) in the x planes, directly
          const Q4<T> uxm = ld4(C, KU, -1, 0);
          ryx = qvec(qmul(Uy, qconj(qmul(ld4(C, KU + 4, -1, 0), ld4(C, KU, -1, 1)))), uxm);
          rzx = qvec(qmul(Uz, qconj(qmul(ld4(C, KU + 8, -1, 0), ld4(Pn, KU, -1, 0)))), uxm);
          // lower staples of U_x(n), U_z(n) in the y planes, directly
          const Q4<T> uym = ld4(C, KU + 4, 0, -1);
          mxy = qvec(qmul(Ux, qconj(qmul(ld4(C, KU, 0, -1), ld4(C, KU + 4, 1, -1)))), uym);
          mzy = qvec(qmul(Uz, qconj(qmul(ld4(C, KU + 8, 0, -1), ld4(Pn, KU + 4, 0, -1)))), uym);
        }
        M[0].x = (pxy.x + pxz.x) + (mxy.x + c_xz.x);
        M[0].y = (pxy.y + pxz.y) + (mxy.y + c_xz.y);
        M[0].z = (pxy.z + pxz.z) + (mxy.z + c_xz.z);
        M[1].x = (pyz.x - pxy.x) + (ryx.x + c_yz.x);
        M[1].y = (pyz.y - pxy.y) + (ryx.y + c_yz.y);
        M[1].z = (pyz.z - pxy.z) + (ryx.z + c_yz.z);
        M[2].x = (rzx.x + mzy.x) - (pxz.x + pyz.x);
        M[2].y = (rzx.y + mzy.y) - (pxz.y + pyz.y);
        M[2].z = (rzx.z + mzy.z) - (pxz.z + pyz.z);
        // for plane z + 1: its lower staples of U_x, U_y in the z planes
        c_xz = neg(rotc(Uz, pxz));
        c_yz = neg(rotc(Uz, pyz));
      }
      if (!tflag) produce(1);

      // ---- hops, currents, link kicks and link drifts, direction by direction ----
      Q4<T> D;
      D.w = fmaT(T(-6), psi.w, c_bz.w);
      D.x = fmaT(T(-6), psi.x, c_bz.x);
      D.y = fmaT(T(-6), psi.y, c_bz.y);
      D.z = fmaT(T(-6), psi.z, c_bz.z);
      T s_g = T(0), s_pA = T(0), s_pB = T(0);
      // FULL: singlet Laplacian and vphi's covariant Laplacian, their gradient sums
      T xs0 = T(0), xc0 = T(0), xc1 = T(0), Ls = T(0), Dv0 = T(0), Dv1 = T(0), s_gs = T(0), s_gc = T(0);
      if constexpr (FULL) {
        xs0 = ld(C, KS, 0, 0);
        xc0 = ld(C, KV, 0, 0);
        xc1 = ld(C, KV + 1, 0, 0);
        Ls = fmaT(T(-6), xs0, c_s + (ld(C, KS, -1, 0) + ld(C, KS, 0, -1)));
        Dv0 = fmaT(T(-6), xc0, c_w0);
        Dv1 = fmaT(T(-6), xc1, c_w1);
        c_s = xs0;
      }
      const T av[3] = {ax, ay, az};
#pragma unroll
      for (int i = 0; i < 3; ++i) {
        const Q4<T> Ui = i == 0 ? Ux : (i == 1 ? Uy : Uz);
        const Q4<T> fn = i == 0 ? ld4(C, KF, 1, 0) : (i == 1 ? ld4(C, KF, 0, 1) : ld4(Pn, KF, 0, 0));
        T si, ci;
        sincos_t(gd * av[i], si, ci);
        Q4<T> chi = umul(Ui, fn);
        phase(chi, ci, si);
        qadd(D, chi);
        // the backward hop W_i^dag(n-i) psi(n-i): across x and y directly; along z the
        // thread's own W_z^dag(n) psi(n) is carried to plane z + 1
        if (i < 2) {
          T s, c;
          sincos_t(gd * (i == 0 ? axm : ld(C, KA + 1, 0, -1)), s, c);
          Q4<T> b = i == 0 ? udmul(ld4(C, KU, -1, 0), ld4(C, KF, -1, 0)) : udmul(ld4(C, KU + 4, 0, -1), ld4(C, KF, 0, -1));
          phase(b, c, -s);
          qadd(D, b);
        } else {
          c_bz = udmul(Ui, psi);
          phase(c_bz, ci, -si);
        }
        // psi = (p, q) = (w + i x, y + i z), chi = (c1, c2)
        const T ImA = fmaT(psi.w, chi.x, fmaT(-psi.x, chi.w, fmaT(psi.y, chi.z, -psi.z * chi.y)));  // Im psi^dag chi
        const T Im1 = fmaT(psi.w, chi.z, fmaT(-psi.x, chi.y, fmaT(psi.y, chi.x, -psi.z * chi.w)));  // Im psi^dag s1 chi
        const T Im2 = fmaT(psi.y, chi.w, fmaT(psi.z, chi.x, fmaT(-psi.w, chi.y, -psi.x * chi.z)));  // Im psi^dag s2 chi
        const T Im3 = fmaT(psi.w, chi.x, fmaT(-psi.x, chi.w, fmaT(-psi.y, chi.z, psi.z * chi.y)));  // Im psi^dag s3 chi
        if constexpr (RED > 0) {
          const T e0 = chi.w - psi.w, e1 = chi.x - psi.x, e2 = chi.y - psi.y, e3 = chi.z - psi.z;
          s_g += (e0 * e0 + e1 * e1) + (e2 * e2 + e3 * e3);
        }
        T pnA = mom(SPA + i, g) + (AJA * ImA + ACA * Cc[i]);
        if constexpr (FULL) {
          // singlet: forward neighbour along i (backward ones: x, y loaded above, z carried)
          const T sfw = i == 0 ? ld(C, KS, 1, 0) : (i == 1 ? ld(C, KS, 0, 1) : ld(Pn, KS, 0, 0));
          Ls += sfw;
          // vphi: forward hop Vc_i(n) vphi(n+i), Vc = exp(-i Qc gQ dx A)
          const T y0v = i == 0 ? ld(C, KV, 1, 0) : (i == 1 ? ld(C, KV, 0, 1) : ld(Pn, KV, 0, 0));
          const T y1v = i == 0 ? ld(C, KV + 1, 1, 0) : (i == 1 ? ld(C, KV + 1, 0, 1) : ld(Pn, KV + 1, 0, 0));
          T sc2, cc;
          sincos_t(gdc * av[i], sc2, cc);
          const T u0 = cc * y0v + sc2 * y1v, u1 = cc * y1v - sc2 * y0v;
          // backward hop Vc_i^*(n-i) vphi(n-i): across x and y directly; along z the
          // thread's own Vc_z^*(n) vphi(n) is carried to plane z + 1
          if (i < 2) {
            const T b0 = i == 0 ? ld(C, KV, -1, 0) : ld(C, KV, 0, -1);
            const T b1 = i == 0 ? ld(C, KV + 1, -1, 0) : ld(C, KV + 1, 0, -1);
            T sb, cb;
            sincos_t(gdc * (i == 0 ? axm : ld(C, KA + 1, 0, -1)), sb, cb);
            Dv0 += cb * b0 - sb * b1;
            Dv1 += cb * b1 + sb * b0;
          } else {
            c_w0 = cc * xc0 - sc2 * xc1;
            c_w1 = cc * xc1 + sc2 * xc0;
          }
          Dv0 += u0;
          Dv1 += u1;
          pnA += AJC * (xc0 * u1 - xc1 * u0);
          if constexpr (RED > 0) {
            const T gs = sfw - xs0, g0 = u0 - xc0, g1 = u1 - xc1;
            s_gs += gs * gs;
            s_gc += g0 * g0 + g1 * g1;
          }
        }
        const T Ims[3] = {Im1, Im2, Im3};
        const T Ms[3] = {M[i].x, M[i].y, M[i].z};
        T pnB[3];
#pragma unroll
        for (int a = 0; a < 3; ++a) pnB[a] = mom(SPB + 3 * i + a, g) + (AJB * Ims[a] + AMB * Ms[a]);
        if constexpr (RED > 0) {
          s_pA += pnA * pnA;
          s_pB += pnB[0] * pnB[0] + pnB[1] * pnB[1] + pnB[2] * pnB[2];
        }
        if (P.write) {
          // drift of the link fields: A_i += kdA pi_A,i, U_i <- exp(-i hB pi_B,i.s) U_i
          const T p1 = hB * pnB[0], p2 = hB * pnB[1], p3 = hB * pnB[2];
          T c, sc;
          cos_sinc(p1 * p1 + p2 * p2 + p3 * p3, c, sc);
          Q4<T> e;
          e.w = c;
          e.x = sc * p1;
          e.y = sc * p2;
          e.z = sc * p3;
          Q4<T> u = qmul(e, Ui);
          renorm(u);
          da(SA + i)[g] = fmaT(kdA, pnA, av[i]);
          da(SU + 4 * i)[g] = u.w;
          da(SU + 4 * i + 1)[g] = u.x;
          da(SU + 4 * i + 2)[g] = u.y;
          da(SU + 4 * i + 3)[g] = u.z;
          da(SPA + i)[g] = pnA;
#pragma unroll
          for (int a = 0; a < 3; ++a) da(SPB + 3 * i + a)[g] = pnB[a];
        }
      }
      // ---- doublet kick and drift ----
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
      for (int c2 = 0; c2 < 4; ++c2) pn[c2] = mom(SP + c2, g) + (A1 * Dc[c2] - A3 * gp * fc[c2]);
      T pns = T(0), pnc0 = T(0), pnc1 = T(0);
      if constexpr (FULL) {
        pns = mom(SPS, g) + (A1 * Ls - A3 * (T(2) * qG * r2) * xs0);
        pnc0 = mom(SPC, g) + (A1 * Dv0 - A3 * (T(2) * qH * r2) * xc0);
        pnc1 = mom(SPC + 1, g) + (A1 * Dv1 - A3 * (T(2) * qH * r2) * xc1);
      }
      if (P.write) {
#pragma unroll
        for (int c2 = 0; c2 < 4; ++c2) {
          da(SF + c2)[g] = fmaT(kd, pn[c2], fc[c2]);
          da(SP + c2)[g] = pn[c2];
        }
        if constexpr (FULL) {
          da(SS)[g] = fmaT(kd, pns, xs0);
          da(SC)[g] = fmaT(kd, pnc0, xc0);
          da(SC + 1)[g] = fmaT(kd, pnc1, xc1);
          da(SPS)[g] = pns;
          da(SPC)[g] = pnc0;
          da(SPC + 1)[g] = pnc1;
        }
      }
      if constexpr (RED == 2) {
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
      if (SLOT && j < nz) prefetch_momenta(g + (unsigned)NN);  // the slot is free again
      step_end(q + j);
    }
    step_begin(q + nz + 1);  // the item's last plane: nothing left to compute on it
    if (!tflag) produce(1);
    step_end(q + nz + 1);
    q += nz + 2;
  }

  __syncthreads();
  if (tflag) {  // a wait ran out: let this thread's copies in flight land, then report
    for (int p = produced > 3 ? produced - 3 : 0; p < produced; ++p)
      mbar_wait_bounded(&full_bar[p % 3], (uint32_t)((p / 3) & 1), 1000000ull);
    if (tid == 0) P.sc->status = CL_ETIMEOUT;
  }
  su2_pass_end<T, RED, FULL>(P, L, acc, nonfinite, red_s, last_s, tid, lane, warp, nth);
}

typedef void (*PassKernel)(const PassArgs);

// Kick-then-drift doublet passes (no self-consistent expansion): red 0 or 2, TX 16 or 32, tiles of
// 8 rows, and (FP32, 32 wide, red 0) of 16 rows with one 512-thread CTA per SM;
// n256: the FP32 32-wide step pass built for N = 256.
PassKernel su2_kd_pass_kernel(int fp32, int red, int TX, int TY, int full, int n256) {
  static const PassKernel tab[2][2][2][2] = {  // [full][TX == 32][fp32][red == 2]
      {{{kd_pass_su2<double, 0, 16, 8, false>, kd_pass_su2<double, 2, 16, 8, false>},
        {kd_pass_su2<float, 0, 16, 8, false>, kd_pass_su2<float, 2, 16, 8, false>}},
       {{kd_pass_su2<double, 0, 32, 8, false>, kd_pass_su2<double, 2, 32, 8, false>},
        {kd_pass_su2<float, 0, 32, 8, false>, kd_pass_su2<float, 2, 32, 8, false>}}},
      {{{kd_pass_su2<double, 0, 16, 8, true>, kd_pass_su2<double, 2, 16, 8, true>},
        {kd_pass_su2<float, 0, 16, 8, true>, kd_pass_su2<float, 2, 16, 8, true>}},
       {{kd_pass_su2<double, 0, 32, 8, true>, kd_pass_su2<double, 2, 32, 8, true>},
        {kd_pass_su2<float, 0, 32, 8, true>, kd_pass_su2<float, 2, 32, 8, true>}}}};
  if ((red != 0 && red != 2) || (TX != 16 && TX != 32)) return nullptr;
  if (n256 && (!fp32 || TX != 32 || red != 0)) return nullptr;
  if (TY == 16) {
    if (!fp32 || TX != 32 || red != 0) return nullptr;
    if (n256) return full ? kd_pass_su2<float, 0, 32, 16, true, 256> : kd_pass_su2<float, 0, 32, 16, false, 256>;
    return full ? kd_pass_su2<float, 0, 32, 16, true> : kd_pass_su2<float, 0, 32, 16, false>;
  }
  if (n256 && TY == 8) return full ? kd_pass_su2<float, 0, 32, 8, true, 256> : kd_pass_su2<float, 0, 32, 8, false, 256>;
  if (TY != 8) return nullptr;
  return tab[full ? 1 : 0][TX == 32 ? 1 : 0][fp32 ? 1 : 0][red == 2 ? 1 : 0];
}

// Dynamic shared memory of a kick-then-drift pass: three stages and the momentum slot.
size_t su2_kd_smem_bytes(int TX, int TY, int esz, int full) {
  if (TY == 16) return full ? KdGeom<float, 32, 16, true>::SMEM : KdGeom<float, 32, 16, false>::SMEM;
  if (TX == 32) {
    if (esz == 4) return full ? KdGeom<float, 32, 8, true>::SMEM : KdGeom<float, 32, 8, false>::SMEM;
    return full ? KdGeom<double, 32, 8, true>::SMEM : KdGeom<double, 32, 8, false>::SMEM;
  }
  if (esz == 4) return full ? KdGeom<float, 16, 8, true>::SMEM : KdGeom<float, 16, 8, false>::SMEM;
  return full ? KdGeom<double, 16, 8, true>::SMEM : KdGeom<double, 16, 8, false>::SMEM;
}

}  // namespace clg
