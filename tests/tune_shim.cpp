// Test-only C wrappers around the autotuner's selection logic (tune.cpp), compiled on the CPU with
// g++: the measurements are a table the test passes in, with a counter of the calls.
#include "tune.hpp"

extern "C" {

// choose among ncand candidates of key (kind, bucket); times[c * reps + r] is the r-th measurement
// of candidate c (negative: c cannot run); *calls receives the number of measurements taken
int tn_choose(int kind, int bucket, int ncand, int reps, const double* times, int* calls) {
  mgiga::TuneKey key{kind, 2, 3, 2, bucket};
  int n = 0;
  std::vector<int> next((size_t)ncand, 0);
  const int c = mgiga::Tuner::instance().choose(
      key, ncand,
      [&](int i) {
        ++n;
        return times[i * reps + next[(size_t)i]++];
      },
      reps);
  *calls = n;
  return c;
}

int tn_bucket(long long n) { return mgiga::tune_bucket(n); }
void tn_clear() { mgiga::Tuner::instance().clear(); }
int tn_size() { return (int)mgiga::Tuner::instance().size(); }
}
