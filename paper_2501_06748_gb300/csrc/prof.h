// Tracing of the library's own kernels: launch counts per phase, and (when
// enabled) device time per phase from CUDA event pairs recorded on the
// launching stream around each phase.
#pragma once

#include <cstdint>
#include <utility>
#include <vector>

#include <cuda_runtime.h>

namespace sbfwi {

enum Phase { kPhaseSetup = 0, kPhaseElement = 1, kPhaseSolve = 2, kPhaseOther = 3, kPhases = 4 };

struct Profiler {
  bool on = false;
  int64_t launches[kPhases] = {0, 0, 0, 0};
  double ms[kPhases] = {0, 0, 0, 0};
  int64_t intervals[kPhases] = {0, 0, 0, 0};
  std::vector<cudaEvent_t> pool;
  std::vector<std::pair<int, std::pair<cudaEvent_t, cudaEvent_t>>> pending;
  cudaEvent_t open_start[kPhases] = {nullptr, nullptr, nullptr, nullptr};

  cudaEvent_t take() {
    if (!pool.empty()) { cudaEvent_t e = pool.back(); pool.pop_back(); return e; }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
  }
  void begin(int ph, cudaStream_t st) {
    if (!on) return;
    open_start[ph] = take();
    cudaEventRecord(open_start[ph], st);
  }
  void end(int ph, cudaStream_t st) {
    if (!on || !open_start[ph]) return;
    cudaEvent_t e = take();
    cudaEventRecord(e, st);
    pending.push_back({ph, {open_start[ph], e}});
    open_start[ph] = nullptr;
  }
  // after the stream has been synchronised
  void resolve() {
    for (auto& p : pending) {
      float t = 0.f;
      if (cudaEventElapsedTime(&t, p.second.first, p.second.second) == cudaSuccess) {
        ms[p.first] += t;
        intervals[p.first] += 1;
      }
      pool.push_back(p.second.first);
      pool.push_back(p.second.second);
    }
    pending.clear();
  }
  void count(int ph, int64_t n = 1) { launches[ph] += n; }

  // Per-level wall time of the persistent global solve: block 0 stamps the global
  // timer after every grid barrier and adds the differences (ns) to level_acc
  // (device, [slots]); one slot per barrier-separated phase, forward levels first.
  unsigned long long* level_acc = nullptr;
  int level_slots = 0;
  int level_device = -1;
  int64_t level_steps = 0;
  // a zeroed accumulator of `slots` entries on the current device, or nullptr
  unsigned long long* level_trace(int slots, cudaStream_t st) {
    if (!on) return nullptr;
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) return nullptr;
    if (level_acc && (level_device != dev || level_slots != slots)) {
      cudaFree(level_acc);
      level_acc = nullptr;
    }
    if (!level_acc) {
      if (cudaMalloc(&level_acc, sizeof(unsigned long long) * slots) != cudaSuccess) {
        cudaGetLastError();
        level_acc = nullptr;
        return nullptr;
      }
      cudaMemsetAsync(level_acc, 0, sizeof(unsigned long long) * slots, st);
      level_slots = slots;
      level_device = dev;
      level_steps = 0;
    }
    return level_acc;
  }

  // Per-phase timing of the dataflow global solve: one row per solve (the last kFlowRows
  // solves kept), row = [earliest block start | per phase p (forward levels, then backward
  // levels): latest item finish, sum of item execution times (inputs ready -> finished),
  // sum of item waits (claimed -> inputs ready), items], global timer ns.
  static constexpr int kFlowRows = 64;
  unsigned long long* flow_acc = nullptr;
  int flow_stride = 0;
  int flow_device = -1;
  int64_t flow_steps = 0;
  // the zeroed row of the next solve on the current device, or nullptr
  unsigned long long* flow_trace(int phases, cudaStream_t st) {
    if (!on) return nullptr;
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) return nullptr;
    const int stride = 1 + 4 * phases;
    if (flow_acc && (flow_device != dev || flow_stride != stride)) {
      cudaFree(flow_acc);
      flow_acc = nullptr;
    }
    if (!flow_acc) {
      if (cudaMalloc(&flow_acc, sizeof(unsigned long long) * stride * kFlowRows) != cudaSuccess) {
        cudaGetLastError();
        flow_acc = nullptr;
        return nullptr;
      }
      flow_stride = stride;
      flow_device = dev;
      flow_steps = 0;
    }
    unsigned long long* row = flow_acc + (size_t)(flow_steps % kFlowRows) * stride;
    cudaMemsetAsync(row, 0xFF, sizeof(unsigned long long), st);          // start: a minimum
    cudaMemsetAsync(row + 1, 0, sizeof(unsigned long long) * (stride - 1), st);
    ++flow_steps;
    return row;
  }
};

Profiler& profiler();

}  // namespace sbfwi
