// worklist.h -- how the plane tasks of a DK pass are split over the CTAs of a
// persistent launch (host code, no CUDA; shared by the library and a CPU test).
//
// A task is one z-plane of one y-tile (BY full x-rows) of one lattice.  Each
// CTA marches a sequence of segments: runs of consecutive planes of one tile
// (plus one halo plane at each end, which the CTA loads but does not write).
// Each CTA accumulates one partial-sum slot per lattice it touches; slots are
// numbered lattice-major so that a lattice's slots are contiguous.
#pragma once

#include <algorithm>
#include <cmath>
#include <vector>

namespace clg {

// One work segment: planes [z0, z0+nz) of y-tile `ytile` of lattice `lat`,
// marched in direction dir (+1 up, -1 down).  Consecutive segments of one CTA
// on one lattice accumulate into partial-sum slot `slot`; `flush` marks the
// last segment of such a run.
struct Seg {
  int lat, ytile, z0, nz, dir, slot, flush, pad;
};
constexpr int MAX_SEG_PER_CTA = 64;

struct LatTiles {
  int N, BY;
  int min_sites;  // a plane task costs at least this many sites (a task runs one CTA however few of its threads work)
};

// Relative costs of the block-aligned split, measured on the FP32 scalar pass
// at 256^3: a plane of a tile whose halo rows wrap around y (the first and
// the last tile) takes one more bulk copy per array and about 6 % longer; a
// segment's two halo planes and its set-up cost about 0.8 of a plane.
constexpr double kWrapCost = 1.06;
constexpr double kSegCost = 0.8;

// Segments of the plane tasks [b, e) (numbered lattice-major, then y-tile,
// then z; a segment ends at a y-tile boundary), appended in march order.
inline void append_run(const std::vector<LatTiles>& lats, const std::vector<long long>& toff, long long b,
                       long long e, int dir, std::vector<Seg>& segs) {
  const size_t first = segs.size();
  size_t l = 0;
  for (long long t = b; t < e;) {
    while (t >= toff[l + 1]) ++l;
    const int N = lats[l].N;
    const long long u = t - toff[l];
    const int yt = (int)(u / N), z = (int)(u % N);
    const int len = (int)std::min<long long>(e - t, N - z);
    Seg sg;
    sg.lat = (int)l;
    sg.ytile = yt;
    sg.z0 = z;
    sg.nz = len;
    sg.dir = dir;
    sg.slot = -1;
    sg.flush = 0;
    sg.pad = 0;
    segs.push_back(sg);
    t += len;
  }
  if (dir < 0) std::reverse(segs.begin() + first, segs.end());
}

// Single lattice, block-aligned split.  z is cut into nb blocks, and CTA
// (block, y-tile) marches its tile through the block: every CTA of a block
// starts on the same plane in the same direction, so the y-halo rows a CTA
// reads are boundary rows its y-neighbours load at about the same time and
// come from L2.  Directions alternate by block so that the CTAs on both sides
// of a block boundary reach it together (all up for an up-only pass).  The planes left above the last
// block go, y-tile-major, to the remaining CTAs in runs of equal cost.  The
// block heights (Zb for interior tiles, Zw for the two wrap tiles, whose
// blocks then drift by a few planes) are chosen to minimise the largest
// per-CTA cost.  Returns false where the shape does not fit (then the
// cost-weighted contiguous split is used).
struct AlignedPlan {
  int Zb, Zw, nb, rest;
  double max_cost;
};

inline bool aligned_plan(const LatTiles& L, int grid, AlignedPlan& best) {
  const int N = L.N, YT = N / L.BY;
  if (YT < 2 || L.BY * N < L.min_sites || grid < YT) return false;
  const long long nt = (long long)YT * N;
  const int z0 = (int)((nt + grid - 1) / grid);
  auto wrap = [&](int t) { return t == 0 || t == YT - 1; };
  bool found = false;
  for (int Zb = std::max(1, z0 - 1); Zb <= z0 + 3; ++Zb) {
    const int nb = std::min(grid / YT, N / Zb);
    if (nb < 1) continue;
    const int rest = grid - nb * YT;
    for (int Zw = std::max(1, Zb - 8); Zw <= Zb; ++Zw) {
      if (nb * Zw > N) continue;
      double left_cost = 0.0;
      long long left_planes = 0;
      for (int t = 0; t < YT; ++t) {
        const int lt = N - nb * (wrap(t) ? Zw : Zb);
        left_planes += lt;
        left_cost += lt * (wrap(t) ? kWrapCost : 1.0);
      }
      if ((rest > 0) != (left_planes > 0)) continue;
      double mx = std::max((double)Zb, kWrapCost * Zw);
      if (rest > 0) {
        // leftover runs of equal plane cost, each with about
        // 1 + (its planes / the mean leftover column height) segments
        const double per = left_cost / rest;
        const double col = (double)left_planes / YT;
        mx = std::max(mx, per + kSegCost * (1.0 + per / std::max(col, 1.0)));
      }
      const bool better = !found || mx < best.max_cost - 1e-9 ||
                          (std::fabs(mx - best.max_cost) <= 1e-9 && Zw > best.Zw);
      if (better) {
        best = AlignedPlan{Zb, Zw, nb, rest, mx};
        found = true;
      }
    }
  }
  return found;
}

inline bool aligned_split(const LatTiles& L, int grid, bool up_only, std::vector<Seg>& segs,
                          std::vector<int>& cta_first) {
  AlignedPlan A;
  if (!aligned_plan(L, grid, A)) return false;
  const int N = L.N, YT = N / L.BY;
  auto wrap = [&](int t) { return t == 0 || t == YT - 1; };
  const std::vector<LatTiles> one = {L};
  const std::vector<long long> toff = {0, (long long)YT * N};
  segs.clear();
  cta_first.assign(grid + 1, 0);
  for (int cta = 0; cta < A.nb * YT; ++cta) {
    const int blk = cta / YT, yt = cta % YT;
    const int Z = wrap(yt) ? A.Zw : A.Zb;
    cta_first[cta] = (int)segs.size();
    const long long b = (long long)yt * N + (long long)blk * Z;
    append_run(one, toff, b, b + Z, (blk & 1) && !up_only ? -1 : +1, segs);
  }
  // leftover planes: tile t keeps [nb Z_t, N); runs of equal cost
  std::vector<double> cpre(YT + 1, 0.0);
  std::vector<int> lstart(YT);
  for (int t = 0; t < YT; ++t) {
    lstart[t] = A.nb * (wrap(t) ? A.Zw : A.Zb);
    cpre[t + 1] = cpre[t] + (N - lstart[t]) * (wrap(t) ? kWrapCost : 1.0);
  }
  // leftover position (tile, plane offset) where the running cost reaches c
  auto cut = [&](double c) -> std::pair<int, int> {
    if (c >= cpre[YT]) return {YT, 0};
    int t = 0;
    while (t + 1 < YT && cpre[t + 1] <= c) ++t;
    const double w = wrap(t) ? kWrapCost : 1.0;
    const int k = (int)std::llround((c - cpre[t]) / w);
    return {t, std::min(k, N - lstart[t])};
  };
  const int dir = (A.nb & 1) && !up_only ? -1 : +1;
  for (int c = 0; c < A.rest; ++c) {
    const int cta = A.nb * YT + c;
    cta_first[cta] = (int)segs.size();
    const auto pb = cut(cpre[YT] * c / A.rest), pe = cut(cpre[YT] * (c + 1) / A.rest);
    const size_t first = segs.size();
    for (int t = pb.first; t <= pe.first && t < YT; ++t) {
      const int k0 = t == pb.first ? pb.second : 0;
      const int k1 = t == pe.first ? pe.second : N - lstart[t];
      if (k1 <= k0) continue;
      const long long b = (long long)t * N + lstart[t] + k0;
      append_run(one, toff, b, b + (k1 - k0), +1, segs);
      segs.back().dir = dir;
    }
    if (dir < 0) std::reverse(segs.begin() + first, segs.end());
  }
  return true;
}

// The work list of a pass over `lats` on `grid` CTAs: the block-aligned split
// for a single lattice, else contiguous runs of equal cost
// (a task costs its sites, but at least a whole CTA's worth: a tile of a small
// lattice leaves threads idle and takes about as long as a full one), split
// into segments at y-tile and lattice boundaries; odd CTAs march down (and
// take their segments in reverse order) so that neighbouring runs reach their
// shared boundary plane at the same time, when halo planes come from L2
// (unless up_only: the U(1) pass carries values from the plane below).
// cta_first[c] is the first segment of CTA c; slot_begin/slot_end the slot
// range of each lattice.  Returns false if a CTA would get more than
// MAX_SEG_PER_CTA segments.
inline bool build_worklist(const std::vector<LatTiles>& lats, int grid, bool up_only, std::vector<Seg>& segs,
                           std::vector<int>& cta_first, std::vector<int>& slot_begin, std::vector<int>& slot_end) {
  const size_t nl = lats.size();
  std::vector<long long> toff(nl + 1, 0);
  std::vector<double> coff(nl + 1, 0.0);  // sites before each lattice
  for (size_t l = 0; l < nl; ++l) {
    const long long nt = (long long)(lats[l].N / lats[l].BY) * lats[l].N;
    toff[l + 1] = toff[l] + nt;
    coff[l + 1] = coff[l] + (double)nt * std::max(lats[l].BY * lats[l].N, lats[l].min_sites);
  }
  // first task of CTA k: where the running site count reaches k/grid of the total
  auto boundary = [&](int k) -> long long {
    if (k <= 0) return 0;
    if (k >= grid) return toff[nl];
    const double target = coff[nl] * (double)k / (double)grid;
    size_t l = 0;
    while (l + 1 < nl && coff[l + 1] <= target) ++l;
    const double per = (double)std::max(lats[l].BY * lats[l].N, lats[l].min_sites);
    const long long t = toff[l] + (long long)std::llround((target - coff[l]) / per);
    return std::min(std::max(t, toff[l]), toff[l + 1]);
  };
  if (!(nl == 1 && aligned_split(lats[0], grid, up_only, segs, cta_first))) {
    segs.clear();
    cta_first.assign(grid + 1, 0);
    for (int cta = 0; cta < grid; ++cta) {
      const long long b = boundary(cta), e = std::max(b, boundary(cta + 1));
      cta_first[cta] = (int)segs.size();
      append_run(lats, toff, b, e, (cta & 1) && !up_only ? -1 : +1, segs);
    }
  }
  for (int cta = 0; cta < grid; ++cta) {
    const int end = cta + 1 < grid ? cta_first[cta + 1] : (int)segs.size();
    if (end - cta_first[cta] > MAX_SEG_PER_CTA) return false;
    for (int i = cta_first[cta]; i < end; ++i)
      segs[i].flush = (i + 1 == end || segs[i + 1].lat != segs[i].lat) ? 1 : 0;
  }
  cta_first[grid] = (int)segs.size();
  slot_begin.assign(nl, 0);
  slot_end.assign(nl, 0);
  int next = 0;
  for (size_t l = 0; l < nl; ++l) {
    slot_begin[l] = next;
    for (int cta = 0; cta < grid; ++cta) {
      bool used = false;
      for (int i = cta_first[cta]; i < cta_first[cta + 1]; ++i)
        if (segs[i].lat == (int)l) {
          segs[i].slot = next;
          used = true;
        }
      if (used) ++next;
    }
    slot_end[l] = next;
  }
  return true;
}

}  // namespace clg
