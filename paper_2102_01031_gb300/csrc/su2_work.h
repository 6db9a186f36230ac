// su2_work.h -- how the doublet-model pass's work is split over its CTAs (host
// code, no CUDA; shared by the library and a CPU test).
//
// The pass takes work items (tile, z-chunk), numbered chunk-major
// (item = chunk * ntiles + tile), round-robin over R resident CTAs; chunk c
// covers planes [c N / nzc, (c + 1) N / nzc).  A round of items covers about one
// chunk of every tile, so neighbouring tiles march the same planes together.
#pragma once

#include <algorithm>
#include <cmath>

namespace clg {

// The number of z-chunks in 1 .. max(1, N/4) that minimises rounds x (planes
// per chunk + the 2 planes each item loads before its first kick).
inline int su2_z_chunks(int ntiles, int N, int R) {
  int nzc = 1;
  double best = 1e300;
  for (int k = 1; k <= std::max(1, N / 4); ++k) {
    const double rounds = std::ceil((double)ntiles * k / R);
    const double cost = rounds * ((double)N / k + 2.0);
    if (cost < best - 1e-9) {
      best = cost;
      nzc = k;
    }
  }
  return nzc;
}

}  // namespace clg
