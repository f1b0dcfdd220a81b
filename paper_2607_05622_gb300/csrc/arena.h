// Host-side first-fit allocator over one device slab (the service's HBM
// budget): blocks are rounded up to kAlign bytes, freed blocks merge with
// their neighbours.  Plain C++ (no CUDA), so the CPU tests compile it alone.
#pragma once
#include <algorithm>
#include <cstddef>
#include <iterator>
#include <map>

struct Arena {
  char *base = nullptr;
  size_t size = 0, used = 0, peak = 0;  // size: usable bytes, a multiple of kAlign
  std::map<size_t, size_t> free_;       // offset -> length
  static constexpr size_t kAlign = 256;
  static size_t rounded(size_t n) { return (n + kAlign - 1) / kAlign * kAlign; }
  // The usable size is the budget rounded down to whole blocks, so that a
  // request accepted by could_fit() can always be allocated once the arena
  // is empty (a request between the rounded-down and the raw budget would
  // otherwise wait at the head of the queue forever).
  void init(char *b, size_t budget) {
    base = b;
    size = budget / kAlign * kAlign;
    used = peak = 0;
    free_.clear();
    if (size) free_[0] = size;
  }
  bool could_fit(size_t n) const { return rounded(n) <= size; }
  bool alloc(size_t n, size_t *off) {
    n = rounded(n);
    for (auto it = free_.begin(); it != free_.end(); ++it) {
      if (it->second >= n) {
        *off = it->first;
        const size_t rest = it->second - n, o = it->first;
        free_.erase(it);
        if (rest) free_[o + n] = rest;
        used += n;
        peak = std::max(peak, used);
        return true;
      }
    }
    return false;
  }
  void release(size_t off, size_t n) {
    n = rounded(n);
    used -= n;
    auto it = free_.emplace(off, n).first;
    auto nx = std::next(it);
    if (nx != free_.end() && it->first + it->second == nx->first) {
      it->second += nx->second;
      free_.erase(nx);
    }
    if (it != free_.begin()) {
      auto pv = std::prev(it);
      if (pv->first + pv->second == it->first) {
        pv->second += it->second;
        free_.erase(it);
      }
    }
  }
};
