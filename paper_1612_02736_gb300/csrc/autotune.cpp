// Tile autotuner.  The first time a launch shape is met, every candidate configuration
// is run once on the caller's stream and timed with CUDA events; the fastest is kept for
// the rest of the process and, when a cache file is named, appended to it as one
// "key value" line so that later processes skip the trials.  Launch-timing records are
// suspended during the trials so that they do not count as work of the step.
#include <cstdio>
#include <fstream>
#include <map>
#include <mutex>
#include <set>
#include <sstream>

#include "hps_internal.h"

namespace hps {

namespace {

std::mutex g_mu;
std::map<std::string, int> g_choice;
std::map<std::string, std::set<std::string>> g_file_keys;  // path -> keys it holds

void load_file(const std::string& path) {
  if (path.empty() || g_file_keys.count(path)) return;
  std::set<std::string>& keys = g_file_keys[path];
  std::ifstream in(path);
  std::string line;
  while (std::getline(in, line)) {
    const size_t sp = line.rfind(' ');
    if (sp == std::string::npos || sp == 0) continue;
    try {
      g_choice[line.substr(0, sp)] = std::stoi(line.substr(sp + 1));
      keys.insert(line.substr(0, sp));
    } catch (...) {
      // a damaged line is skipped; its shape is tuned again
    }
  }
}

void append_file(const std::string& path, const std::string& key, int v) {
  if (path.empty() || g_file_keys[path].count(key)) return;
  g_file_keys[path].insert(key);
  std::ofstream out(path, std::ios::app);
  if (out) out << key << ' ' << v << '\n';
}

}  // namespace

float time_on_stream(cudaStream_t s, const std::function<void()>& run) {
  cudaEvent_t a = nullptr, b = nullptr;
  if (cudaEventCreate(&a) != cudaSuccess || cudaEventCreate(&b) != cudaSuccess) {
    cudaGetLastError();
    if (a) cudaEventDestroy(a);
    throw CudaError{HPS_ERR_CUDA, "autotune: cannot create timing events"};
  }
  timing_suspend(true);
  cudaEventRecord(a, s);
  try {
    run();
  } catch (...) {
    timing_suspend(false);
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    throw;
  }
  cudaEventRecord(b, s);
  timing_suspend(false);
  float ms = 0.0f;
  const cudaError_t e1 = cudaEventSynchronize(b);
  const cudaError_t e2 = e1 == cudaSuccess ? cudaEventElapsedTime(&ms, a, b) : e1;
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  if (e2 != cudaSuccess) {
    cudaGetLastError();
    throw CudaError{HPS_ERR_CUDA, std::string("autotune: ") + cudaGetErrorString(e2)};
  }
  return ms;
}

int tuned_choice(const std::string& key, const std::vector<int>& cands, const std::string& path,
                 const std::function<float(int)>& trial_ms) {
  if (cands.empty()) return 0;
  std::lock_guard<std::mutex> lk(g_mu);
  load_file(path);
  auto it = g_choice.find(key);
  if (it != g_choice.end()) {
    for (int c : cands)
      if (c == it->second) {
        append_file(path, key, c);  // a choice made earlier in this process, new to this file
        return c;
      }
    // a stored choice outside today's candidates (another build of the library) is retuned
  }
  if (cands.size() == 1) return cands[0];
  if (!trial_ms) return 0;  // lookup only (for example while a stream is being captured)
  int best = cands[0];
  float best_ms = 0.0f;
  for (size_t i = 0; i < cands.size(); ++i) {
    const float ms = trial_ms(cands[i]);
    if (i == 0 || ms < best_ms) {
      best = cands[i];
      best_ms = ms;
    }
  }
  g_choice[key] = best;
  append_file(path, key, best);
  return best;
}

}  // namespace hps
