// Autotuner of size-dependent launch shapes (see tune.hpp).
#include "tune.hpp"

#include <algorithm>
#include <cmath>

namespace mgiga {

int tune_bucket(int64_t n) {
  if (n < 1) return 0;
  return (int)std::floor(2.0 * std::log2((double)n));
}

Tuner& Tuner::instance() {
  static Tuner t;
  return t;
}

bool Tuner::lookup(const TuneKey& key, int* choice) const {
  std::lock_guard<std::mutex> lock(mu_);
  const auto it = table_.find(key);
  if (it == table_.end()) return false;
  if (choice) *choice = it->second;
  return true;
}

int Tuner::choose(const TuneKey& key, int ncand, const std::function<double(int)>& measure, int reps) {
  int c = -1;
  if (lookup(key, &c)) return c;
  std::vector<double> t((size_t)std::max(ncand, 0), -1.0);
  int best = -1;
  for (int i = 0; i < ncand; ++i) {
    std::vector<double> m;
    for (int r = 0; r < std::max(reps, 1); ++r) {
      const double v = measure(i);
      if (v < 0.0) { m.clear(); break; }
      m.push_back(v);
    }
    if (m.empty()) continue;
    std::sort(m.begin(), m.end());
    t[(size_t)i] = m[m.size() / 2];
    if (best < 0 || t[(size_t)i] < t[(size_t)best]) best = i;
  }
  if (best < 0) best = 0;  // nothing could run: the first candidate, not remembered
  std::lock_guard<std::mutex> lock(mu_);
  last_ = t;
  if (best >= 0 && !t.empty() && t[(size_t)best] >= 0.0) table_[key] = best;
  return best;
}

void Tuner::clear() {
  std::lock_guard<std::mutex> lock(mu_);
  table_.clear();
  last_.clear();
}

size_t Tuner::size() const {
  std::lock_guard<std::mutex> lock(mu_);
  return table_.size();
}

std::vector<double> Tuner::last_times() const {
  std::lock_guard<std::mutex> lock(mu_);
  return last_;
}

}  // namespace mgiga
