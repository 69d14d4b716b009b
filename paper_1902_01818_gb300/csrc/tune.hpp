// Autotuner of the launch shapes that depend on problem size: each decision is taken once per
// size bucket by timing the candidates on the device and kept for the process (later handles of
// the same bucket reuse it).  The paper has no counterpart; the decisions change no result beyond
// the summation order of the FP32 parts of the preconditioner.
#pragma once

#include <cstdint>
#include <functional>
#include <map>
#include <mutex>
#include <tuple>
#include <vector>

namespace mgiga {

// what is tuned, in which problem class
struct TuneKey {
  int kind;        // TUNE_FD: contraction engine of the fast diagonalisation; TUNE_RESIDUAL: row blocking
  int dim, degree, precision;
  int bucket;      // size bucket (tune_bucket of the level's defining size)
  bool operator<(const TuneKey& o) const {
    return std::tie(kind, dim, degree, precision, bucket) < std::tie(o.kind, o.dim, o.degree, o.precision, o.bucket);
  }
};
enum { TUNE_FD = 0, TUNE_RESIDUAL = 1 };

// floor(2 log2(n)): buckets a factor sqrt(2) apart
int tune_bucket(int64_t n);

class Tuner {
 public:
  static Tuner& instance();
  // the index of the fastest of `ncand` candidates (measure(c): milliseconds of candidate c, or a
  // negative value when c cannot run); on a miss every runnable candidate is measured `reps` times
  // and the median taken, ties going to the lower index; on a hit measure is not called
  int choose(const TuneKey& key, int ncand, const std::function<double(int)>& measure, int reps = 3);
  bool lookup(const TuneKey& key, int* choice) const;
  void clear();
  size_t size() const;
  // the timings of the last miss (for the set-up log)
  std::vector<double> last_times() const;

 private:
  mutable std::mutex mu_;
  std::map<TuneKey, int> table_;
  std::vector<double> last_;
};

}  // namespace mgiga
