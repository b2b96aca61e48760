// The autotuner's persisted cache (declared in include/csrc.h): one text line per decision,
// keyed by the matrix and the device. Host code only; no device work.
#include <sys/stat.h>
#include <unistd.h>

#include <cerrno>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <fstream>
#include <mutex>
#include <sstream>
#include <string>
#include <vector>

#include "internal.h"

namespace csrc {
namespace {

std::mutex g_tune_mutex;
constexpr const char* kTag = "csrc-tune-v1";

// The device field with blanks replaced, so that a line splits on whitespace.
std::string device_token(const char* d) {
  std::string s;
  for (size_t i = 0; i < 64 && d[i]; ++i) s += (d[i] == ' ' || d[i] == '\t' || d[i] == '\n') ? '_' : d[i];
  return s.empty() ? std::string("-") : s;
}

// The part of a line that identifies a decision (everything before the four values).
std::string key_text(const csrc_tune_key* k, int32_t kind, double param) {
  char buf[512];
  std::snprintf(buf, sizeof(buf), "%s %016llx %lld %lld %d %u %d %.17g %s", kTag,
                (unsigned long long)k->pattern_hash, (long long)k->n, (long long)k->nnz, (int)k->storage,
                (unsigned)k->flags, (int)kind, param, device_token(k->device).c_str());
  return buf;
}

bool mkdirs(const std::string& dir) {
  if (dir.empty()) return true;
  struct stat st;
  if (stat(dir.c_str(), &st) == 0) return S_ISDIR(st.st_mode);
  const size_t slash = dir.find_last_of('/');
  if (slash != std::string::npos && slash > 0 && !mkdirs(dir.substr(0, slash))) return false;
  return mkdir(dir.c_str(), 0755) == 0 || errno == EEXIST;
}

}  // namespace

int tune_mode() {
  const char* v = std::getenv("CSRC_TUNE");
  if (!v || !*v || std::strcmp(v, "cache") == 0) return TUNE_CACHE;
  if (std::strcmp(v, "off") == 0) return TUNE_OFF;
  if (std::strcmp(v, "full") == 0) return TUNE_FULL;
  return TUNE_CACHE;
}

std::string tune_cache_path() {
  if (const char* p = std::getenv("CSRC_TUNE_CACHE")) return p;
  if (const char* x = std::getenv("XDG_CACHE_HOME"))
    if (*x) return std::string(x) + "/csrc_gb300/tune.txt";
  if (const char* h = std::getenv("HOME"))
    if (*h) return std::string(h) + "/.cache/csrc_gb300/tune.txt";
  return std::string();
}

// FNV-1a 64 over n, the row pointers and the column indices.
uint64_t pattern_hash(int32_t n, const std::vector<int32_t>& ia, const std::vector<int32_t>& ja) {
  uint64_t hsh = 1469598103934665603ULL;
  auto mix = [&](const void* p, size_t bytes) {
    const unsigned char* c = static_cast<const unsigned char*>(p);
    for (size_t i = 0; i < bytes; ++i) {
      hsh ^= c[i];
      hsh *= 1099511628211ULL;
    }
  };
  mix(&n, sizeof(n));
  if (!ia.empty()) mix(ia.data(), ia.size() * sizeof(int32_t));
  if (!ja.empty()) mix(ja.data(), ja.size() * sizeof(int32_t));
  return hsh;
}

}  // namespace csrc

extern "C" {

csrc_status csrc_tune_cache_lookup(const csrc_tune_key* key, int32_t kind, double param, int32_t values[4]) {
  if (!key || !values || kind < 0 || kind > 2 || !std::isfinite(param)) return CSRC_ERR_INVALID_ARG;
  if (csrc::tune_mode() == csrc::TUNE_OFF) return CSRC_ERR_NOT_FOUND;
  const std::string path = csrc::tune_cache_path();
  if (path.empty()) return CSRC_ERR_NOT_FOUND;
  const std::string want = csrc::key_text(key, kind, param);
  std::lock_guard<std::mutex> lk(csrc::g_tune_mutex);
  std::ifstream in(path);
  std::string line;
  csrc_status st = CSRC_ERR_NOT_FOUND;
  while (std::getline(in, line)) {
    if (line.size() <= want.size() || line.compare(0, want.size(), want) != 0 || line[want.size()] != ' ') continue;
    std::istringstream rest(line.substr(want.size()));
    int32_t v[4];
    if (rest >> v[0] >> v[1] >> v[2] >> v[3]) {  // the last matching line wins
      std::memcpy(values, v, sizeof(v));
      st = CSRC_OK;
    }
  }
  return st;
}

csrc_status csrc_tune_cache_store(const csrc_tune_key* key, int32_t kind, double param, const int32_t values[4]) {
  if (!key || !values || kind < 0 || kind > 2 || !std::isfinite(param)) return CSRC_ERR_INVALID_ARG;
  if (csrc::tune_mode() == csrc::TUNE_OFF) return CSRC_OK;
  const std::string path = csrc::tune_cache_path();
  if (path.empty()) return CSRC_OK;  // nowhere to keep it
  const std::string want = csrc::key_text(key, kind, param);
  std::lock_guard<std::mutex> lk(csrc::g_tune_mutex);
  std::vector<std::string> lines;
  {
    std::ifstream in(path);
    std::string line;
    while (std::getline(in, line)) {
      const bool same = line.size() > want.size() && line.compare(0, want.size(), want) == 0 && line[want.size()] == ' ';
      if (!same && line.compare(0, std::strlen(csrc::kTag), csrc::kTag) == 0) lines.push_back(line);
    }
  }
  char vals[96];
  std::snprintf(vals, sizeof(vals), " %d %d %d %d", (int)values[0], (int)values[1], (int)values[2], (int)values[3]);
  lines.push_back(want + vals);
  const size_t slash = path.find_last_of('/');
  if (slash != std::string::npos && !csrc::mkdirs(path.substr(0, slash))) return CSRC_ERR_IO;
  const std::string tmp = path + ".tmp" + std::to_string((long long)getpid());
  {
    std::ofstream out(tmp, std::ios::trunc);
    if (!out) return CSRC_ERR_IO;
    for (const auto& l : lines) out << l << '\n';
    if (!out) return CSRC_ERR_IO;
  }
  if (std::rename(tmp.c_str(), path.c_str()) != 0) {
    std::remove(tmp.c_str());
    return CSRC_ERR_IO;
  }
  return CSRC_OK;
}

}  // extern "C"
