// Checker for the serving loop's first-fit arena (paper_0809_0063_gb300/csrc/arena.h), built
// and run by tests/test_arena_cpu.py on the CPU.  Random allocations and releases are mirrored
// in a byte map of the arena.  After every step the allocator's free runs must be exactly the
// map's maximal free stretches (so adjacent free space is always merged), and an allocation
// must land at the lowest offset whose free stretch is large enough, or fail exactly when
// there is none.  Exit status 0 on success.
#include <cstdio>
#include <cstdlib>
#include <random>
#include <vector>

#include "arena.h"

namespace {

struct Block {
  size_t off, bytes;
};

bool runs_match_map(const fpd::FirstFitArena& a, const std::vector<char>& used) {
  std::vector<std::pair<size_t, size_t>> want;
  for (size_t i = 0; i < used.size();) {
    if (used[i]) { ++i; continue; }
    size_t j = i;
    while (j < used.size() && !used[j]) ++j;
    want.emplace_back(i, j - i);
    i = j;
  }
  if (want.size() != a.runs().size()) return false;
  size_t k = 0;
  for (const auto& r : a.runs())
    if (r.first != want[k].first || r.second != want[k++].second) return false;
  return true;
}

// Lowest offset of a free stretch of at least `bytes`, or size when there is none.
size_t first_fit(const std::vector<char>& used, size_t bytes) {
  for (size_t i = 0; i < used.size();) {
    if (used[i]) { ++i; continue; }
    size_t j = i;
    while (j < used.size() && !used[j]) ++j;
    if (j - i >= bytes) return i;
    i = j;
  }
  return used.size();
}

}  // namespace

int main() {
  const size_t sizes[] = {1, 64, 4096};
  for (size_t arena_bytes : sizes) {
    for (unsigned seed = 0; seed < 20; ++seed) {
      std::mt19937_64 rng(seed * 7919 + arena_bytes);
      fpd::FirstFitArena a;
      a.reset(arena_bytes);
      std::vector<char> used(arena_bytes, 0);
      std::vector<Block> live;
      for (int step = 0; step < 3000; ++step) {
        const bool do_alloc = live.empty() || (rng() % 100) < 55;
        if (do_alloc) {
          const size_t bytes = 1 + rng() % (arena_bytes < 256 ? arena_bytes : 256);
          const size_t expect = first_fit(used, bytes);
          size_t off = 0;
          const bool ok = a.alloc(bytes, &off);
          if (ok != (expect < arena_bytes) || (ok && off != expect)) {
            std::printf("alloc mismatch: arena %zu seed %u step %d bytes %zu ok %d off %zu expect %zu\n",
                        arena_bytes, seed, step, bytes, (int)ok, off, expect);
            return 1;
          }
          if (ok) {
            for (size_t i = off; i < off + bytes; ++i) used[i] = 1;
            live.push_back({off, bytes});
          }
        } else {
          const size_t k = rng() % live.size();
          const Block b = live[k];
          live[k] = live.back();
          live.pop_back();
          a.release(b.off, b.bytes);
          for (size_t i = b.off; i < b.off + b.bytes; ++i) used[i] = 0;
        }
        if (!runs_match_map(a, used)) {
          std::printf("free runs differ from the byte map: arena %zu seed %u step %d\n", arena_bytes, seed, step);
          return 1;
        }
      }
      // release everything: one run covering the whole arena again
      for (const Block& b : live) a.release(b.off, b.bytes);
      if (a.runs().size() != 1 || a.runs().begin()->first != 0 || a.runs().begin()->second != arena_bytes) {
        std::printf("arena %zu seed %u: not one free run after releasing everything\n", arena_bytes, seed);
        return 1;
      }
    }
  }
  // an empty arena refuses every allocation
  fpd::FirstFitArena z;
  z.reset(0);
  size_t off = 0;
  if (z.alloc(1, &off)) {
    std::printf("empty arena allocated\n");
    return 1;
  }
  std::printf("ok\n");
  return 0;
}
