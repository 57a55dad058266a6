// Launch shapes chosen by measurement (the autotuner of the batched, many-angle workloads): the
// candidate shapes of a kernel family are timed on a short probe of the call's own launch (its
// pairs, a couple of steps) and the fastest is kept per shape key for the life of the process.
// Host code only, without CUDA, so the selection rule and the cache can be exercised on their own.
//
// Candidates are listed cheapest first (fewer SMs per (set, angle) pair, smaller tiles); a later
// candidate replaces an earlier one only if it is faster by more than a relative margin, so that
// timing noise does not flip a choice between shapes that perform alike.
#pragma once
#include <cmath>
#include <map>
#include <mutex>
#include <tuple>

namespace trh {
namespace tune {

// What is being chosen.
enum Kind : int {
  kWideTile = 0,     // tile edge of the wide FP64 kernel (candidates 64, 32)
  kColumnSplit = 1,  // one CTA per pair or two sharing its columns (candidates 1, 2)
};

// Index of the fastest of n probe times (ms); failed probes (time <= 0 or not finite) never win.
// Returns 0 when every probe failed.
inline int pick(const float* ms, int n, float rel_margin) {
  int best = -1;
  for (int i = 0; i < n; ++i) {
    if (!(ms[i] > 0.0f) || !std::isfinite(ms[i])) continue;
    if (best < 0 || ms[i] < ms[best] * (1.0f - rel_margin)) best = i;
  }
  return best < 0 ? 0 : best;
}

// (kind, precision, N, method, pairs per launch, steps): the shape a probe's result holds for.
using Key = std::tuple<int, int, int, int, long long, long long>;

// Time of a launch of L steps from probes of L1 < L2 steps (launch overhead plus a per-step cost,
// so that a short probe does not favour the shape with the cheaper set-up).
inline float extrapolate(float t1, int L1, float t2, int L2, int L) {
  if (!(t1 > 0.0f) || !(t2 > 0.0f) || L2 <= L1) return t1;
  return t1 + (t2 - t1) * (float)(L - L1) / (float)(L2 - L1);
}

class Cache {
 public:
  bool find(const Key& k, int* value) {
    std::lock_guard<std::mutex> lk(mu_);
    const auto it = map_.find(k);
    if (it == map_.end()) return false;
    *value = it->second;
    return true;
  }
  void put(const Key& k, int value) {
    std::lock_guard<std::mutex> lk(mu_);
    map_[k] = value;
  }
  size_t size() {
    std::lock_guard<std::mutex> lk(mu_);
    return map_.size();
  }

 private:
  std::mutex mu_;
  std::map<Key, int> map_;
};

}  // namespace tune
}  // namespace trh
