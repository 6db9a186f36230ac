// checkpoint.h -- the file format of a lattice checkpoint and its atomic write
// (host code, no CUDA; shared by the library and a CPU test).
//
// A checkpoint is a header, the lattice's evolving scalars (the device's
// LatScalars, bytes as stored) and its state arrays in storage order and
// precision.  It is written to `path.tmp`, flushed and synced to disk, and
// renamed over `path`, after which the directory is synced too, so that a
// failure at any point (of the process, or of the host once the data reached
// the disk) leaves either the previous checkpoint or the new one, never a
// partial file (the manual's backup keeps the old file until the new one is
// written, Sec. 5.3).  Reads check the magic, the version and every
// size against the file's length.
#pragma once

#include <cstdint>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include <fcntl.h>
#include <unistd.h>

namespace clg {

struct CkptHeader {
  char magic[8];                  // "CLGBCKP\0"
  uint32_t version, pad;
  int32_t model, N, narr, esz;    // model, lattice size, arrays per buffer, bytes per value
  double kIR, alpha;
  uint64_t seed;
  uint64_t scalars_bytes, state_bytes;
};

constexpr uint32_t kCkptVersion = 1;

inline void ckpt_init_header(CkptHeader& h) {
  std::memset(&h, 0, sizeof(h));
  std::memcpy(h.magic, "CLGBCKP", 8);
  h.version = kCkptVersion;
}

// Directory part of `path` ("." when it has none).
inline std::string ckpt_dir_of(const std::string& path) {
  const size_t s = path.find_last_of('/');
  if (s == std::string::npos) return ".";
  return s == 0 ? "/" : path.substr(0, s);
}

// Writes header, scalars and state to path + ".tmp", flushes and fsyncs it,
// renames it over `path` and fsyncs the directory, so that the rename cannot
// reach the disk before the data.  before_rename (may be null) runs between the flush and the
// rename; if it returns false the write is abandoned (the temporary file is
// removed, `path` is untouched) -- the hook the tests use to fail there.
// Returns 0 on success, -1 on an I/O error, -2 when abandoned by the hook.
inline int ckpt_write_atomic(const std::string& path, const CkptHeader& h, const void* scalars, const void* state,
                             bool (*before_rename)(void*) = nullptr, void* hook_arg = nullptr) {
  const std::string tmp = path + ".tmp";
  FILE* f = std::fopen(tmp.c_str(), "wb");
  if (!f) return -1;
  bool ok = std::fwrite(&h, sizeof(h), 1, f) == 1;
  ok = ok && (h.scalars_bytes == 0 || std::fwrite(scalars, h.scalars_bytes, 1, f) == 1);
  ok = ok && (h.state_bytes == 0 || std::fwrite(state, h.state_bytes, 1, f) == 1);
  ok = std::fflush(f) == 0 && ok;
  ok = ok && fsync(fileno(f)) == 0;
  ok = std::fclose(f) == 0 && ok;
  if (!ok) {
    std::remove(tmp.c_str());
    return -1;
  }
  if (before_rename && !before_rename(hook_arg)) {
    std::remove(tmp.c_str());
    return -2;
  }
  if (std::rename(tmp.c_str(), path.c_str()) != 0) {
    std::remove(tmp.c_str());
    return -1;
  }
  const int d = open(ckpt_dir_of(path).c_str(), O_RDONLY | O_DIRECTORY);
  if (d < 0) return -1;
  const bool synced = fsync(d) == 0;
  close(d);
  return synced ? 0 : -1;
}

// Reads a checkpoint; 0 on success, -1 when the file is missing, short, or not
// a checkpoint of this version.
inline int ckpt_read(const std::string& path, CkptHeader& h, std::vector<char>& scalars, std::vector<char>& state) {
  FILE* f = std::fopen(path.c_str(), "rb");
  if (!f) return -1;
  bool ok = std::fread(&h, sizeof(h), 1, f) == 1 && std::memcmp(h.magic, "CLGBCKP", 8) == 0 &&
            h.version == kCkptVersion && h.scalars_bytes < (1ull << 20) && h.state_bytes < (1ull << 40);
  if (ok) {
    scalars.resize(h.scalars_bytes);
    state.resize(h.state_bytes);
    ok = (h.scalars_bytes == 0 || std::fread(scalars.data(), h.scalars_bytes, 1, f) == 1) &&
         (h.state_bytes == 0 || std::fread(state.data(), h.state_bytes, 1, f) == 1);
    char extra;
    ok = ok && std::fread(&extra, 1, 1, f) == 0;  // nothing after the state
  }
  std::fclose(f);
  return ok ? 0 : -1;
}

}  // namespace clg
