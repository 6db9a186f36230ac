// tune_cache.h -- the autotuner's on-disk cache of tile heights (host code, no
// CUDA; shared by the library and a CPU test).
//
// A text file, one entry per line:  model esz N sm_count cc_major cc_minor BY
// (the device's SM count and compute capability are part of the key, since the
// best tile height depends on the GPU).  Lines that do not parse are skipped.
// Stores rewrite the whole file through a temporary file of the writing process
// (`path.tmp.<pid>`) renamed over it, so a reader never sees a partial file and
// processes that store at the same time each replace the file whole.
#pragma once

#include <unistd.h>

#include <cstdio>
#include <map>
#include <string>
#include <tuple>

namespace clg {

typedef std::tuple<int, int, int, int, int, int> TuneKey;  // model, esz, N, sm_count, cc_major, cc_minor

// Adds the file's entries to `out` (entries already in `out` are kept); a
// missing file adds nothing.  Returns the number of entries read.
inline int tune_cache_load(const std::string& path, std::map<TuneKey, int>& out) {
  FILE* f = std::fopen(path.c_str(), "r");
  if (!f) return 0;
  int n = 0;
  char line[256];
  while (std::fgets(line, sizeof(line), f)) {
    int m, e, N, sm, ma, mi, by;
    char tail;
    if (std::sscanf(line, "%d %d %d %d %d %d %d %c", &m, &e, &N, &sm, &ma, &mi, &by, &tail) != 7) continue;
    if (N < 1 || by < 1 || N % by) continue;
    out.emplace(TuneKey(m, e, N, sm, ma, mi), by);
    ++n;
  }
  std::fclose(f);
  return n;
}

// Writes every entry of `entries` to `path` (temporary file, then rename).
// Returns 0 on success, -1 on an I/O error (the previous file is then intact).
inline int tune_cache_store(const std::string& path, const std::map<TuneKey, int>& entries) {
  const std::string tmp = path + ".tmp." + std::to_string((long)getpid());
  FILE* f = std::fopen(tmp.c_str(), "w");
  if (!f) return -1;
  bool ok = true;
  for (const auto& kv : entries) {
    const TuneKey& k = kv.first;
    ok = ok && std::fprintf(f, "%d %d %d %d %d %d %d\n", std::get<0>(k), std::get<1>(k), std::get<2>(k),
                            std::get<3>(k), std::get<4>(k), std::get<5>(k), kv.second) > 0;
  }
  ok = std::fclose(f) == 0 && ok;
  if (!ok || std::rename(tmp.c_str(), path.c_str()) != 0) {
    std::remove(tmp.c_str());
    return -1;
  }
  return 0;
}

}  // namespace clg
