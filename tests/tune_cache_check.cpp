// CPU check of the autotuner's on-disk cache (tune_cache.h): a missing file
// reads as empty, entries round-trip, loading keeps entries already known,
// malformed lines are skipped, a store leaves no temporary file, and two
// processes storing at the same time leave one of their files whole.
// Prints "OK <case>" or "FAIL <case>".
#include <dirent.h>
#include <sys/wait.h>
#include <unistd.h>

#include <cstdio>
#include <cstring>
#include <map>
#include <string>

#include "tune_cache.h"

using namespace clg;

// Number of directory entries other than `keep`, "." and "..".
static int stray_files(const std::string& dir, const char* keep) {
  DIR* d = opendir(dir.c_str());
  if (!d) return -1;
  int n = 0;
  while (dirent* e = readdir(d)) {
    if (!std::strcmp(e->d_name, ".") || !std::strcmp(e->d_name, "..") || !std::strcmp(e->d_name, keep)) continue;
    if (!std::strncmp(e->d_name, "tune.txt", 8)) ++n;
  }
  closedir(d);
  return n;
}

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
  std::map<TuneKey, int> r;
  report("round_trip", stored && stray_files(dir, "tune.txt") == 0 && tune_cache_load(path, r) == 3 && r == m);
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
  // two processes store different tables 300 times each at the same time: every
  // store succeeds and the file ends as one of the two tables, whole
  std::map<TuneKey, int> A, B;
  for (int i = 0; i < 40; ++i) A[TuneKey(1, 4, 8 * (i + 1), 152, 10, 3)] = 1;
  for (int i = 0; i < 25; ++i) B[TuneKey(2, 8, 16 * (i + 1), 148, 10, 0)] = 2;
  std::fflush(stdout);
  pid_t kids[2];
  for (int k = 0; k < 2; ++k) {
    kids[k] = fork();
    if (kids[k] == 0) {
      int bad = 0;
      for (int i = 0; i < 300; ++i) bad += tune_cache_store(path, k == 0 ? A : B) != 0;
      _exit(bad ? 1 : 0);
    }
  }
  bool kids_ok = true;
  for (int k = 0; k < 2; ++k) {
    int st = 0;
    kids_ok = kids_ok && kids[k] > 0 && waitpid(kids[k], &st, 0) == kids[k] && WIFEXITED(st) && WEXITSTATUS(st) == 0;
  }
  std::map<TuneKey, int> e;
  const int ne = tune_cache_load(path, e);
  report("concurrent_stores", kids_ok && stray_files(dir, "tune.txt") == 0 &&
                                  ((ne == 40 && e == A) || (ne == 25 && e == B)));
  return all ? 0 : 1;
}
