// CPU check of the checkpoint file (checkpoint.h): round trip, a failure
// between the write and the rename leaves the previous checkpoint, a stale
// temporary file from a crashed writer does not stop the next write, and short,
// long or foreign files are refused.  Prints "OK <case>" or "FAIL <case>".
#include <cstdio>
#include <string>
#include <vector>

#include "checkpoint.h"

using namespace clg;

static bool fail_hook(void*) { return false; }

static CkptHeader header(size_t nsc, size_t nst, int N) {
  CkptHeader h;
  ckpt_init_header(h);
  h.model = 2;
  h.N = N;
  h.narr = 4;
  h.esz = 4;
  h.kIR = 0.1;
  h.alpha = 1.0;
  h.seed = 7;
  h.scalars_bytes = nsc;
  h.state_bytes = nst;
  return h;
}

static bool same(const std::string& path, const CkptHeader& h, const std::vector<char>& sc,
                 const std::vector<char>& st) {
  CkptHeader r;
  std::vector<char> rs, rt;
  return ckpt_read(path, r, rs, rt) == 0 && r.N == h.N && rs == sc && rt == st;
}

static bool exists(const std::string& p) {
  FILE* f = std::fopen(p.c_str(), "rb");
  if (f) std::fclose(f);
  return f != nullptr;
}

int main(int argc, char** argv) {
  const std::string dir = argc > 1 ? argv[1] : ".";
  const std::string path = dir + "/ckpt.bin";
  bool all = true;
  auto report = [&](const char* name, bool ok) {
    std::printf("%s %s\n", ok ? "OK" : "FAIL", name);
    all = all && ok;
  };
  std::vector<char> scA(64, 'a'), stA(4096), scB(64, 'b'), stB(4096);
  for (size_t i = 0; i < stA.size(); ++i) {
    stA[i] = (char)(i * 7);
    stB[i] = (char)(i * 13 + 1);
  }
  const CkptHeader hA = header(scA.size(), stA.size(), 16), hB = header(scB.size(), stB.size(), 32);
  report("round_trip", ckpt_write_atomic(path, hA, scA.data(), stA.data()) == 0 && same(path, hA, scA, stA));
  // a failure after the data is written but before the rename
  const int rc = ckpt_write_atomic(path, hB, scB.data(), stB.data(), fail_hook, nullptr);
  report("failure_before_rename_keeps_previous", rc == -2 && same(path, hA, scA, stA) && !exists(path + ".tmp"));
  // a writer that died and left its temporary file behind
  {
    FILE* f = std::fopen((path + ".tmp").c_str(), "wb");
    std::fputs("partial", f);
    std::fclose(f);
  }
  report("stale_temporary_file", same(path, hA, scA, stA) &&
                                     ckpt_write_atomic(path, hB, scB.data(), stB.data()) == 0 &&
                                     same(path, hB, scB, stB) && !exists(path + ".tmp"));
  // short, long and foreign files are refused
  std::vector<char> bytes;
  {
    FILE* f = std::fopen(path.c_str(), "rb");
    int ch;
    while ((ch = std::fgetc(f)) != EOF) bytes.push_back((char)ch);
    std::fclose(f);
  }
  auto write_raw = [&](const std::string& p, const std::vector<char>& b) {
    FILE* f = std::fopen(p.c_str(), "wb");
    std::fwrite(b.data(), 1, b.size(), f);
    std::fclose(f);
  };
  CkptHeader r;
  std::vector<char> rs, rt;
  std::vector<char> shorter(bytes.begin(), bytes.end() - 10), longer = bytes, foreign = bytes;
  longer.push_back('x');
  foreign[0] = 'X';
  write_raw(dir + "/short.bin", shorter);
  write_raw(dir + "/long.bin", longer);
  write_raw(dir + "/foreign.bin", foreign);
  report("refuses_short_long_foreign", ckpt_read(dir + "/short.bin", r, rs, rt) != 0 &&
                                           ckpt_read(dir + "/long.bin", r, rs, rt) != 0 &&
                                           ckpt_read(dir + "/foreign.bin", r, rs, rt) != 0 &&
                                           ckpt_read(dir + "/missing.bin", r, rs, rt) != 0);
  return all ? 0 : 1;
}
