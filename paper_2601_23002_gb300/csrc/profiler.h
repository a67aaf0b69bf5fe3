// Per-kernel launch counters and optional CUDA-event timing for one plan.
#pragma once
#include <cuda_runtime.h>

#include <cstring>
#include <map>
#include <string>
#include <vector>

namespace ofdft {

class Profiler {
 public:
  struct Stat { long long launches = 0; double ms = 0; double bytes = 0; };
  bool timing = false;

  ~Profiler() { release(); }

  void reset(bool t) {
    flush();
    stats_.clear();
    timing = t;
  }
  // call immediately before / after a launch on stream st
  // bytes: algorithmic DRAM bytes of this launch (each input read once,
  // each output written once)
  void begin(const char* name, cudaStream_t st, double bytes) {
    Stat& s = stats_[name];
    s.launches++;
    s.bytes += bytes;
    if (!timing) return;
    if (open_.size() > 4096) flush();   // only here: end() must find its pair
    cudaEvent_t a = get_event();
    if (a && cudaEventRecord(a, st) == cudaSuccess) open_.push_back({name, a, nullptr});
  }
  void end(cudaStream_t st) {
    if (!timing || open_.empty() || open_.back().b) return;
    cudaEvent_t b = get_event();
    if (b && cudaEventRecord(b, st) == cudaSuccess) open_.back().b = b;
  }
  // resolve recorded event pairs (waits for them)
  void flush() {
    for (auto& p : open_) {
      if (p.a && p.b) {
        cudaEventSynchronize(p.b);
        float ms = 0;
        if (cudaEventElapsedTime(&ms, p.a, p.b) == cudaSuccess) stats_[p.name].ms += ms;
      }
      if (p.a) pool_.push_back(p.a);
      if (p.b) pool_.push_back(p.b);
    }
    open_.clear();
  }
  const std::map<std::string, Stat>& stats() {
    flush();
    return stats_;
  }

 private:
  struct Pair { std::string name; cudaEvent_t a, b; };
  std::map<std::string, Stat> stats_;
  std::vector<Pair> open_;
  std::vector<cudaEvent_t> pool_;
  cudaEvent_t get_event() {
    if (!pool_.empty()) { cudaEvent_t e = pool_.back(); pool_.pop_back(); return e; }
    cudaEvent_t e = nullptr;
    if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
    return e;
  }
  void release() {
    flush();
    for (auto e : pool_) cudaEventDestroy(e);
    pool_.clear();
  }
};

}  // namespace ofdft
