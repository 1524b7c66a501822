// First-fit allocator over the serving loop's device arena (host bookkeeping only; plain C++,
// no CUDA).  The free space is kept as maximal runs, offset -> size: an allocation takes the
// lowest-offset run that is large enough and leaves its tail free; a release merges the block
// with the free runs that touch it on either side, so adjacent free space is always one run.
#pragma once

#include <cstddef>
#include <iterator>
#include <map>

namespace fpd {

class FirstFitArena {
 public:
  void reset(size_t bytes) {
    runs_.clear();
    if (bytes) runs_[0] = bytes;
  }
  // Offset of a block of `bytes` (> 0) in *off, or false when no free run is large enough.
  bool alloc(size_t bytes, size_t* off) {
    for (auto it = runs_.begin(); it != runs_.end(); ++it) {
      if (it->second >= bytes) {
        *off = it->first;
        const size_t rest = it->second - bytes, noff = it->first + bytes;
        runs_.erase(it);
        if (rest) runs_[noff] = rest;
        return true;
      }
    }
    return false;
  }
  // Give back a block that alloc returned (same offset and size).
  void release(size_t off, size_t bytes) {
    auto it = runs_.emplace(off, bytes).first;
    auto nx = std::next(it);
    if (nx != runs_.end() && it->first + it->second == nx->first) {
      it->second += nx->second;
      runs_.erase(nx);
    }
    if (it != runs_.begin()) {
      auto pv = std::prev(it);
      if (pv->first + pv->second == it->first) {
        pv->second += it->second;
        runs_.erase(it);
      }
    }
  }
  const std::map<size_t, size_t>& runs() const { return runs_; }

 private:
  std::map<size_t, size_t> runs_;
};

}  // namespace fpd
