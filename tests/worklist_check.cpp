// CPU check of the DK-pass work split (worklist.h): every plane task covered
// exactly once, segments inside their lattice, at most MAX_SEG_PER_CTA per
// CTA, slots contiguous per lattice and unique per (CTA, lattice), flush flags
// on the last segment of each run, and the balance of the block-aligned split.
// Prints one line per case: "OK <name> ..." or "FAIL <name>: <reason>".
#include <algorithm>
#include <cstdio>
#include <map>
#include <set>
#include <string>
#include <vector>

#include "su2_work.h"
#include "worklist.h"

using namespace clg;

static bool check(const char* name, const std::vector<LatTiles>& lats, int grid, bool up_only) {
  std::vector<Seg> segs;
  std::vector<int> cta, sb, se;
  if (!build_worklist(lats, grid, up_only, segs, cta, sb, se)) {
    std::printf("FAIL %s: build_worklist refused\n", name);
    return false;
  }
  auto fail = [&](const char* why) {
    std::printf("FAIL %s: %s\n", name, why);
    return false;
  };
  if ((int)cta.size() != grid + 1 || cta[0] != 0 || cta[grid] != (int)segs.size()) return fail("cta_first bounds");
  std::vector<std::vector<std::vector<int>>> cover(lats.size());
  for (size_t l = 0; l < lats.size(); ++l)
    cover[l].assign(lats[l].N / lats[l].BY, std::vector<int>(lats[l].N, 0));
  std::set<std::pair<int, int>> slot_owner;  // (slot, cta)
  std::map<int, int> slot_cta;
  double cost_max = 0.0, cost_sum = 0.0;
  for (int c = 0; c < grid; ++c) {
    if (cta[c + 1] < cta[c]) return fail("cta_first not monotonic");
    if (cta[c + 1] - cta[c] > MAX_SEG_PER_CTA) return fail("too many segments");
    double cost = 0.0;
    for (int i = cta[c]; i < cta[c + 1]; ++i) {
      const Seg& s = segs[i];
      if (s.lat < 0 || s.lat >= (int)lats.size()) return fail("lattice index");
      const int N = lats[s.lat].N, YT = N / lats[s.lat].BY;
      if (s.ytile < 0 || s.ytile >= YT || s.nz < 1 || s.z0 < 0 || s.z0 + s.nz > N) return fail("segment bounds");
      if (s.dir != 1 && s.dir != -1) return fail("direction");
      if (up_only && s.dir != 1) return fail("up_only segment marching down");
      for (int z = s.z0; z < s.z0 + s.nz; ++z) cover[s.lat][s.ytile][z] += 1;
      if (s.slot < sb[s.lat] || s.slot >= se[s.lat]) return fail("slot outside its lattice's range");
      auto it = slot_cta.find(s.slot);
      if (it != slot_cta.end() && it->second != c) return fail("slot shared by two CTAs");
      slot_cta[s.slot] = c;
      const bool last_of_run = i + 1 == cta[c + 1] || segs[i + 1].lat != s.lat;
      if ((s.flush != 0) != last_of_run) return fail("flush flag");
      const bool wrap = YT > 1 && (s.ytile == 0 || s.ytile == YT - 1);
      cost += s.nz * (wrap ? kWrapCost : 1.0) + kSegCost;
    }
    cost_max = std::max(cost_max, cost);
    cost_sum += cost;
  }
  for (size_t l = 0; l < lats.size(); ++l)
    for (auto& row : cover[l])
      for (int v : row)
        if (v != 1) return fail("a plane task covered other than once");
  for (size_t l = 0; l + 1 < lats.size(); ++l)
    if (se[l] != sb[l + 1]) return fail("slot ranges not contiguous");
  std::printf("OK %s segs %zu balance %.4f\n", name, segs.size(), cost_max / (cost_sum / grid));
  return true;
}

int main() {
  bool ok = true;
  // single lattices (block-aligned split where it fits)
  ok &= check("fp32_256_by8_g152", {{256, 8, 2048}}, 152, false);
  ok &= check("fp64_256_by4_g152", {{256, 4, 1024}}, 152, false);
  ok &= check("fp32_512_by4_g152", {{512, 4, 2048}}, 152, false);
  ok &= check("fp32_128_by16_g128", {{128, 16, 2048}}, 128, false);
  ok &= check("fp32_64_by32_g64", {{64, 32, 2048}}, 64, false);
  ok &= check("fp32_32_by32_g4", {{32, 32, 2048}}, 4, false);
  ok &= check("fp32_256_by8_g100", {{256, 8, 2048}}, 100, false);
  ok &= check("fp32_96_by16_g152", {{96, 16, 2048}}, 152, false);
  ok &= check("u1_256_by4_g152_up", {{256, 4, 1024}}, 152, true);
  ok &= check("adj_128_by8_g128", {{128, 8, 2048}}, 128, false);
  // ensembles of uneven sizes (contiguous cost-weighted split)
  std::vector<LatTiles> ens;
  for (int k = 0; k < 16; ++k) ens.push_back({32, 32, 2048});
  for (int k = 0; k < 16; ++k) ens.push_back({64, 32, 2048});
  for (int k = 0; k < 16; ++k) ens.push_back({96, 16, 2048});
  for (int k = 0; k < 16; ++k) ens.push_back({128, 16, 2048});
  ok &= check("ensemble_64_g152", ens, 152, false);
  ok &= check("ensemble_3_g7", {{16, 16, 2048}, {24, 24, 2048}, {32, 16, 2048}}, 7, false);
  // block-aligned split at 256^3: interior tiles of a block start together
  {
    std::vector<Seg> segs;
    std::vector<int> cta, sb, se;
    build_worklist({{256, 8, 2048}}, 152, false, segs, cta, sb, se);
    AlignedPlan A;
    aligned_plan({256, 8, 2048}, 152, A);
    bool al = A.nb * 32 <= 152;
    for (int b = 0; b < A.nb && al; ++b)
      for (int t = 1; t < 31; ++t) {
        const Seg& s = segs[cta[b * 32 + t]];
        if (cta[b * 32 + t + 1] - cta[b * 32 + t] != 1 || s.z0 != b * A.Zb || s.nz != A.Zb || s.ytile != t ||
            s.dir != ((b & 1) ? -1 : 1))
          al = false;
      }
    std::printf("%s aligned_blocks Zb %d Zw %d nb %d rest %d max_cost %.2f\n", al ? "OK" : "FAIL", A.Zb, A.Zw, A.nb,
                A.rest, A.max_cost);
    ok &= al;
  }
  // doublet-model items: chunk-major (tile, z-chunk) items cover every (tile,
  // plane) once with at least one plane each (the pass's chunk arithmetic), the
  // round-robin over R CTAs leaves no CTA idle, and at 256^3 (32 x 8 tiles, two
  // CTAs on 152 SMs) the chosen split is within 10 % of perfect balance
  struct Case {
    const char* name;
    int N, TX, TY, R;
  };
  for (const Case& cs : {Case{"su2_256_g304", 256, 32, 8, 304}, Case{"su2_128_g304", 128, 32, 8, 304},
                         Case{"su2_48_g304", 48, 16, 8, 304}, Case{"su2_16_g304", 16, 16, 8, 304},
                         Case{"su2_64_fp64_g152", 64, 32, 8, 152}}) {
    const int ntiles = (cs.N / cs.TX) * (cs.N / cs.TY);
    const int nzc = su2_z_chunks(ntiles, cs.N, cs.R);
    const int nitems = ntiles * nzc, grid = std::min(cs.R, nitems);
    std::vector<int> cover((size_t)ntiles * cs.N, 0);
    std::vector<long> per_cta(grid, 0);
    bool good = nzc >= 1 && nzc <= std::max(1, cs.N / 4);
    for (int item = 0; item < nitems; ++item) {
      const int tile = item % ntiles, chunk = item / ntiles;
      const int z0 = (int)((long long)chunk * cs.N / nzc);
      const int nz = (int)((long long)(chunk + 1) * cs.N / nzc) - z0;
      if (nz < 1) good = false;
      for (int z = z0; z < z0 + nz; ++z) cover[(size_t)tile * cs.N + z] += 1;
      per_cta[item % grid] += nz + 2;
    }
    for (int v : cover) good = good && v == 1;
    long mx = 0, sum = 0;
    for (long v : per_cta) {
      mx = std::max(mx, v);
      sum += v;
      good = good && v > 0;
    }
    const double bal = (double)mx * grid / (double)sum;
    if (cs.N == 256) good = good && bal < 1.10;
    std::printf("%s su2_items %s nzc %d grid %d balance %.3f\n", good ? "OK" : "FAIL", cs.name, nzc, grid, bal);
    ok &= good;
  }
  return ok ? 0 : 1;
}
