// Project autotuner: for each (kernel, shape bucket) the fastest of the kernel's variants,
// measured on first use with CUDA events on the caller's stream and kept for the process.
//  - SC_AUTOTUNE_FILE=<path>: choices are read from this JSON object ({"key": variant, ...}) at
//    first use and the file is rewritten whenever a new choice is made;
//  - SC_TUNE_<KERNEL>=<variant> (e.g. SC_TUNE_TALL=1, SC_TUNE_SPMM=2) forces a variant of one
//    kernel for every shape;
//  - SC_AUTOTUNE=0 turns measuring off: unknown keys take the kernel's built-in default.
// Measuring runs each variant twice (the first run absorbs one-time setup such as function
// attributes) and keeps the faster second time; ties go to the lower variant index.  Nothing is
// measured while the stream is being captured into a CUDA graph.
#include <cuda_runtime.h>

#include <cctype>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <fstream>
#include <map>
#include <mutex>
#include <sstream>
#include <string>

#include "common.cuh"

namespace sc {
namespace {

struct TuneTable {
  std::mutex mu;
  bool loaded = false;
  std::map<std::string, int> choice;
};

TuneTable& table() {
  static TuneTable t;
  return t;
}

const char* tune_file() {
  const char* p = std::getenv("SC_AUTOTUNE_FILE");
  return (p && *p) ? p : nullptr;
}

// Reads {"key": int, ...}; anything else in the file is skipped.
void load_locked(TuneTable& t) {
  t.loaded = true;
  const char* path = tune_file();
  if (!path) return;
  std::ifstream f(path);
  if (!f) return;
  std::stringstream ss;
  ss << f.rdbuf();
  const std::string s = ss.str();
  size_t i = 0;
  while (true) {
    const size_t q0 = s.find('"', i);
    if (q0 == std::string::npos) break;
    const size_t q1 = s.find('"', q0 + 1);
    if (q1 == std::string::npos) break;
    const std::string key = s.substr(q0 + 1, q1 - q0 - 1);
    size_t c = s.find(':', q1);
    if (c == std::string::npos) break;
    ++c;
    while (c < s.size() && std::isspace((unsigned char)s[c])) ++c;
    char* end = nullptr;
    const long v = std::strtol(s.c_str() + c, &end, 10);
    if (end != s.c_str() + c && v >= 0 && v < 64) t.choice[key] = (int)v;
    i = end && end > s.c_str() + c ? (size_t)(end - s.c_str()) : q1 + 1;
  }
}

void save_locked(const TuneTable& t) {
  const char* path = tune_file();
  if (!path) return;
  const std::string tmp = std::string(path) + ".tmp";
  FILE* f = std::fopen(tmp.c_str(), "w");
  if (!f) return;
  std::fprintf(f, "{\n");
  size_t k = 0;
  for (const auto& kv : t.choice)
    std::fprintf(f, "  \"%s\": %d%s\n", kv.first.c_str(), kv.second,
                 ++k < t.choice.size() ? "," : "");
  std::fprintf(f, "}\n");
  std::fclose(f);
  std::rename(tmp.c_str(), path);
}

}  // namespace

int tune_override(const char* kernel) {
  std::string var = "SC_TUNE_";
  for (const char* c = kernel; *c; ++c) var += (char)std::toupper((unsigned char)*c);
  const char* v = std::getenv(var.c_str());
  if (!v || !*v) return -1;
  char* end = nullptr;
  const long x = std::strtol(v, &end, 10);
  return (end != v && x >= 0 && x < 64) ? (int)x : -1;
}

bool tune_measuring() {
  const char* v = std::getenv("SC_AUTOTUNE");
  return !(v && std::strcmp(v, "0") == 0);
}

int tune_lookup(const std::string& key) {
  TuneTable& t = table();
  std::lock_guard<std::mutex> lk(t.mu);
  if (!t.loaded) load_locked(t);
  auto it = t.choice.find(key);
  return it == t.choice.end() ? -1 : it->second;
}

void tune_store(const std::string& key, int v) {
  TuneTable& t = table();
  std::lock_guard<std::mutex> lk(t.mu);
  if (!t.loaded) load_locked(t);
  t.choice[key] = v;
  save_locked(t);
}

int tune_table_size() {
  TuneTable& t = table();
  std::lock_guard<std::mutex> lk(t.mu);
  if (!t.loaded) load_locked(t);
  return (int)t.choice.size();
}

int tune_pick(const std::string& key, const char* kernel, cudaStream_t st, int nvar,
              int fallback, const std::function<cudaError_t(int)>& run) {
  const int forced = tune_override(kernel);
  if (forced >= 0 && forced < nvar) return forced;
  const int known = tune_lookup(key);
  if (known >= 0 && known < nvar) return known;
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (!tune_measuring() || nvar < 2 || cudaStreamIsCapturing(st, &cs) != cudaSuccess ||
      cs != cudaStreamCaptureStatusNone)
    return fallback;
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess) return fallback;
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    return fallback;
  }
  int best = fallback;
  float best_ms = 0.f;
  bool any = false;
  for (int v = 0; v < nvar; ++v) {
    float ms = 0.f;
    bool ok = run(v) == cudaSuccess;  // first run: one-time setup
    ok = ok && cudaEventRecord(e0, st) == cudaSuccess;
    ok = ok && run(v) == cudaSuccess;
    ok = ok && cudaEventRecord(e1, st) == cudaSuccess;
    ok = ok && cudaEventSynchronize(e1) == cudaSuccess;
    ok = ok && cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess;
    if (!ok) {
      cudaGetLastError();  // a variant that cannot run (unsupported shape) is skipped
      continue;
    }
    if (!any || ms < best_ms) {
      best = v;
      best_ms = ms;
      any = true;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (any) tune_store(key, best);
  return best;
}

}  // namespace sc
