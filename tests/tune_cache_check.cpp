// CPU check of the autotuner's on-disk cache (tune_cache.h): a missing file
// reads as empty, entries round-trip, loading keeps entries already known,
// malformed lines are skipped, and a store leaves no temporary file.
// Prints "OK <case>" or "FAIL <case>".
#include <cstdio>
#include <map>
#include <string>

#include "tune_cache.h"

using namespace clg;

int main(int argc, char** argv) {
  const std::string dir = argc > 1 ? argv[1] : ".";
  const std::string path = dir + "/tune.txt";
  bool all = true;
  auto report = [&](const char* name, bool ok) {
    std::printf("%s %s\n", ok ? "OK" : "FAIL", name);
    all = all && ok;
  };
  std::map<TuneKey, int> m;
  report("missing_file_is_empty", tune_cache_load(path, m) == 0 && m.empty());
  m[TuneKey(2, 4, 256, 152, 10, 3)] = 8;
  m[TuneKey(2, 8, 256, 152, 10, 3)] = 4;
  m[TuneKey(3, 4, 128, 152, 10, 3)] = 16;
  const bool stored = tune_cache_store(path, m) == 0;
  FILE* t = std::fopen((path + ".tmp").c_str(), "r");
  if (t) std::fclose(t);
  std::map<TuneKey, int> r;
  report("round_trip", stored && !t && tune_cache_load(path, r) == 3 && r == m);
  // a second process's view: an entry it already had is kept, others are added
  std::map<TuneKey, int> other;
  other[TuneKey(2, 4, 256, 152, 10, 3)] = 16;
  tune_cache_load(path, other);
  report("load_keeps_known_entries", other.size() == 3 && other[TuneKey(2, 4, 256, 152, 10, 3)] == 16 &&
                                         other[TuneKey(3, 4, 128, 152, 10, 3)] == 16);
  // malformed lines are skipped
  {
    FILE* f = std::fopen(path.c_str(), "a");
    std::fputs("garbage line\n1 4 100 152 10 3 7\n2 4 64 152 10 3 8 extra\n1 4 64 152 10 3 8\n", f);
    std::fclose(f);
  }
  std::map<TuneKey, int> g;
  report("skips_malformed_lines", tune_cache_load(path, g) == 4 && g.count(TuneKey(1, 4, 64, 152, 10, 3)) == 1 &&
                                      g.count(TuneKey(1, 4, 100, 152, 10, 3)) == 0);
  return all ? 0 : 1;
}
