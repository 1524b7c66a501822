// Checker for the serving loop's copy pool (paper_0809_0063_gb300/csrc/copy_pool.h), built and
// run by tests/test_copy_pool_cpu.py on the CPU.  For pools of 0 to 8 workers, many runs of
// random sizes (including 0 and 1) with uneven per-item work: every index must be handed out
// exactly once per run, every call must have returned when run() returns, and the pool must be
// reusable and stop cleanly.  Exit status 0 on success.
#include <atomic>
#include <cstdio>
#include <random>
#include <vector>

#include "copy_pool.h"

int main() {
  std::mt19937_64 rng(12345);
  for (int workers = 0; workers <= 8; ++workers) {
    fpd::CopyPool pool(workers);
    for (int rep = 0; rep < 300; ++rep) {
      const size_t n = rep < 4 ? (size_t)rep : (size_t)(rng() % 2000);
      std::vector<std::atomic<int>> hits(n);
      for (auto& h : hits) h.store(0);
      std::atomic<size_t> returned{0};
      const unsigned heavy = (unsigned)(rng() % 7);
      pool.run(n, [&](size_t i) {
        volatile unsigned x = 0;                        // uneven work: every heavy-th item is long
        const unsigned spin = (heavy && i % (heavy + 1) == 0) ? 20000u : 50u;
        for (unsigned k = 0; k < spin; ++k) x = x + k;
        hits[i].fetch_add(1);
        returned.fetch_add(1);
      });
      if (returned.load() != n) {
        std::printf("run returned early: %zu of %zu\n", returned.load(), n);
        return 1;
      }
      for (size_t i = 0; i < n; ++i)
        if (hits[i].load() != 1) {
          std::printf("index %zu handed out %d times (workers %d, n %zu)\n", i, hits[i].load(), workers, n);
          return 1;
        }
    }
  }
  std::printf("ok\n");
  return 0;
}
