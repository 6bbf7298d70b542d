// Launch-shape autotuner of the operator kernels.
//
// A kernel family registers the launch parameters it can run with; the first time a shape key
// (the GPU's name, the grid and the column count) is met, the candidates are timed with CUDA
// events on the caller's stream and the fastest is kept, both in this process's table and in a
// JSON file, so later processes on the same GPU skip the measurement.  Every candidate the
// callers register produces bitwise-identical results (only the work split between blocks
// changes), so a choice never changes an answer.
//
// Cache file: $BIOT_TUNE_CACHE if set, else $XDG_CACHE_HOME/biot_gb300/tune.json, else
// $HOME/.cache/biot_gb300/tune.json.  Format: one JSON object {"key": value, ...}.  BIOT_TUNE=0
// disables measurement (the callers' heuristics then apply); an unreadable or malformed file
// is ignored and rewritten.  The file is read once per process and replaced as a whole: two
// processes tuning new shapes at the same time can each drop the other's new entry, which is
// then measured again by the next process that meets that shape.
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <sys/stat.h>
#include <unistd.h>

#include "../../include/biot.h"
#include "internal.h"

namespace biot {
namespace {

std::mutex g_tune_mu;
std::map<std::string, int> g_table;
bool g_loaded = false;

std::string cache_path() {
  if (const char* p = std::getenv("BIOT_TUNE_CACHE")) return p;
  std::string base;
  if (const char* x = std::getenv("XDG_CACHE_HOME")) base = x;
  else if (const char* h = std::getenv("HOME")) base = std::string(h) + "/.cache";
  else return "";
  return base + "/biot_gb300/tune.json";
}

// minimal reader of a flat {"key": int, ...} object (keys without quotes or backslashes)
void load_locked() {
  if (g_loaded) return;
  g_loaded = true;
  const std::string path = cache_path();
  if (path.empty()) return;
  FILE* f = std::fopen(path.c_str(), "rb");
  if (!f) return;
  std::string s;
  char buf[4096];
  size_t k;
  while ((k = std::fread(buf, 1, sizeof(buf), f)) > 0) s.append(buf, k);
  std::fclose(f);
  size_t i = 0;
  while (true) {
    const size_t q0 = s.find('"', i);
    if (q0 == std::string::npos) break;
    const size_t q1 = s.find('"', q0 + 1);
    if (q1 == std::string::npos) break;
    const size_t colon = s.find(':', q1);
    if (colon == std::string::npos) break;
    char* end = nullptr;
    const long v = std::strtol(s.c_str() + colon + 1, &end, 10);
    if (end == s.c_str() + colon + 1) break;  // malformed: keep what was read
    g_table[s.substr(q0 + 1, q1 - q0 - 1)] = (int)v;
    i = (size_t)(end - s.c_str());
  }
}

void mkdirs(const std::string& path) {
  for (size_t p = path.find('/', 1); p != std::string::npos; p = path.find('/', p + 1)) mkdir(path.substr(0, p).c_str(), 0755);
}

void save_locked() {
  const std::string path = cache_path();
  if (path.empty()) return;
  mkdirs(path);
  const std::string tmp = path + ".tmp" + std::to_string((long)getpid());
  FILE* f = std::fopen(tmp.c_str(), "wb");
  if (!f) return;
  std::fprintf(f, "{");
  bool first = true;
  for (const auto& kv : g_table) {
    std::fprintf(f, "%s\n  \"%s\": %d", first ? "" : ",", kv.first.c_str(), kv.second);
    first = false;
  }
  std::fprintf(f, "\n}\n");
  std::fclose(f);
  std::rename(tmp.c_str(), path.c_str());  // atomic replace
}

}  // namespace

bool tune_enabled() {
  const char* e = std::getenv("BIOT_TUNE");
  return !(e && e[0] == '0');
}

int tune_get(const std::string& key) {
  std::lock_guard<std::mutex> lk(g_tune_mu);
  load_locked();
  auto it = g_table.find(key);
  return it == g_table.end() ? -1 : it->second;
}

void tune_put(const std::string& key, int value) {
  std::lock_guard<std::mutex> lk(g_tune_mu);
  load_locked();
  g_table[key] = value;
  save_locked();
}

std::string tune_device_tag() {
  int dev = 0;
  cudaDeviceProp p;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaGetDeviceProperties(&p, dev) != cudaSuccess) return "unknown";
  std::string s = p.name;
  for (char& ch : s)
    if (ch == '"' || ch == '\\' || ch == ' ') ch = '_';
  return s + "_sm" + std::to_string(p.multiProcessorCount);
}

std::string tune_cache_path() { return cache_path(); }

}  // namespace biot

// Host-only access to the tuning table (no GPU needed): value of a key (-1 if absent), storing a
// value (also written to the cache file), and the cache file's path.
extern "C" int biot_tune_get(const char* key) { return key ? biot::tune_get(key) : -1; }
extern "C" int biot_tune_put(const char* key, int value) {
  if (!key || !*key || std::strchr(key, '"') || std::strchr(key, '\\')) return BIOT_EINVAL;
  biot::tune_put(key, value);
  return BIOT_OK;
}
extern "C" int biot_tune_cache_path(char* buf, int len) {
  const std::string p = biot::tune_cache_path();
  if (!buf || len < 1) return BIOT_EINVAL;
  std::snprintf(buf, (size_t)len, "%s", p.c_str());
  return (int)p.size() < len ? BIOT_OK : BIOT_EINVAL;
}
