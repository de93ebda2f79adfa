// Cache of the launch shapes the autotuners choose, kept as a JSON file so
// that a later process on the same GPU model and library build skips the
// timing.  Host code only.
//
// File: the path set by dvbe_set_autotune_cache, else $DVBE_AUTOTUNE_CACHE
// (empty: no cache), else $XDG_CACHE_HOME/dvbe/autotune.json, else
// $HOME/.cache/dvbe/autotune.json.  One entry per line:
//   "<key>": {"strip_rows": H, "warps_per_block": W, "blocks": B, "ms": T},
// The key names the kernel family, scheme, storage mode, the problem's size
// class, the GPU name with its SM count and the library build.  Writes go to
// a temporary file renamed over the old one, so readers never see half a
// file; a file that does not parse is treated as empty.
#include <sys/stat.h>

#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <unistd.h>

#include "capi_common.h"

#ifndef DVBE_BUILD_ID
#define DVBE_BUILD_ID "unversioned"
#endif

namespace dvbe {
namespace {

std::mutex g_mu;
bool g_init = false;
bool g_on = true;
std::string g_path;

void init_path_locked() {
  if (g_init) return;
  g_init = true;
  const char *e = std::getenv("DVBE_AUTOTUNE_CACHE");
  if (e) {
    g_on = *e != 0;
    g_path = e;
    return;
  }
  const char *x = std::getenv("XDG_CACHE_HOME");
  const char *h = std::getenv("HOME");
  if (x && *x)
    g_path = std::string(x) + "/dvbe/autotune.json";
  else if (h && *h)
    g_path = std::string(h) + "/.cache/dvbe/autotune.json";
  else
    g_on = false;
}

std::string clean(const std::string &s) {
  std::string o = s;
  for (char &c : o)
    if (c == '"' || c == '\\' || c == '\n' || (unsigned char)c < 32) c = '_';
  return o;
}

void read_locked(std::map<std::string, TuneEntry> &m) {
  FILE *f = std::fopen(g_path.c_str(), "r");
  if (!f) return;
  char line[1024];
  while (std::fgets(line, sizeof line, f)) {
    const char *q0 = std::strchr(line, '"');
    if (!q0) continue;
    const char *q1 = std::strstr(q0 + 1, "\": {");
    if (!q1) continue;
    TuneEntry t;
    if (std::sscanf(q1, "\": {\"strip_rows\": %d, \"warps_per_block\": %d, \"blocks\": %d, \"ms\": %lf",
                    &t.strip_rows, &t.warps_per_block, &t.blocks, &t.ms) == 4)
      m[std::string(q0 + 1, q1)] = t;
  }
  std::fclose(f);
}

void mkdirs(const std::string &path) {
  for (size_t i = 1; i < path.size(); ++i)
    if (path[i] == '/') mkdir(path.substr(0, i).c_str(), 0755);
}

} // namespace

void tune_set_path(const char *path) {
  std::lock_guard<std::mutex> lock(g_mu);
  g_init = true;
  if (!path) {
    g_on = false;
    return;
  }
  if (!*path) {
    g_init = false; // back to the environment / default path
    g_on = true;
    g_path.clear();
    init_path_locked();
    return;
  }
  g_on = true;
  g_path = path;
}

std::string tune_key(const std::string &what) {
  int dev = 0;
  cudaDeviceProp prop;
  std::string gpu = "unknown-gpu";
  if (cudaGetDevice(&dev) == cudaSuccess && cudaGetDeviceProperties(&prop, dev) == cudaSuccess)
    gpu = std::string(prop.name) + " sm" + std::to_string(prop.major) + std::to_string(prop.minor) +
          " x" + std::to_string(prop.multiProcessorCount);
  else
    cudaGetLastError();
  return clean(what + "|" + gpu + "|" + DVBE_BUILD_ID);
}

bool tune_lookup(const std::string &key, TuneEntry *out) {
  std::lock_guard<std::mutex> lock(g_mu);
  init_path_locked();
  if (!g_on) return false;
  std::map<std::string, TuneEntry> m;
  read_locked(m);
  auto it = m.find(key);
  if (it == m.end()) return false;
  *out = it->second;
  return true;
}

void tune_store(const std::string &key, const TuneEntry &e) {
  std::lock_guard<std::mutex> lock(g_mu);
  init_path_locked();
  if (!g_on) return;
  std::map<std::string, TuneEntry> m;
  read_locked(m);
  m[key] = e;
  mkdirs(g_path);
  const std::string tmp = g_path + ".tmp" + std::to_string((long long)getpid());
  FILE *f = std::fopen(tmp.c_str(), "w");
  if (!f) return;
  std::fprintf(f, "{\n  \"format\": \"dvbe autotune cache 1\",\n  \"entries\": {\n");
  size_t k = 0;
  for (auto &kv : m)
    std::fprintf(f, "    \"%s\": {\"strip_rows\": %d, \"warps_per_block\": %d, \"blocks\": %d, \"ms\": %.6g}%s\n",
                 kv.first.c_str(), kv.second.strip_rows, kv.second.warps_per_block, kv.second.blocks,
                 kv.second.ms, ++k < m.size() ? "," : "");
  std::fprintf(f, "  }\n}\n");
  const bool ok = std::fclose(f) == 0;
  if (ok)
    std::rename(tmp.c_str(), g_path.c_str());
  else
    std::remove(tmp.c_str());
}

} // namespace dvbe

extern "C" DVBE_API dvbe_status dvbe_set_autotune_cache(const char *path) {
  dvbe::tune_set_path(path);
  return DVBE_OK;
}
