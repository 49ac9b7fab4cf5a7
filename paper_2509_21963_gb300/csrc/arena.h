// arena.h -- first-fit allocator over one byte range, coalescing on release.
// Host bookkeeping only: the server carves its device arena (and its wave
// descriptor area) with it.  Every block is rounded up to 256 bytes, so every
// offset handed out is a multiple of 256.  Not thread-safe (the server holds
// its lock around every call).
#pragma once

#include <algorithm>
#include <cstddef>
#include <iterator>
#include <map>

namespace cur {

inline size_t arena_round(size_t x) { return (x + 255) & ~(size_t)255; }

struct Arena {
  size_t cap = 0, used = 0, peak = 0;
  std::map<size_t, size_t> free_;  // offset -> bytes
  void init(size_t c) {
    cap = c;
    used = peak = 0;
    free_.clear();
    if (c) free_[0] = c;
  }
  // The lowest free block that holds `bytes` (rounded up); false if none.
  bool alloc(size_t bytes, size_t* off) {
    bytes = arena_round(bytes ? bytes : 1);
    for (auto it = free_.begin(); it != free_.end(); ++it) {
      if (it->second < bytes) continue;
      *off = it->first;
      const size_t rest = it->second - bytes, noff = it->first + bytes;
      free_.erase(it);
      if (rest) free_[noff] = rest;
      used += bytes;
      peak = std::max(peak, used);
      return true;
    }
    return false;
  }
  // Return a block (the offset and size it was allocated with); merges it
  // with free neighbours on both sides.
  void release(size_t off, size_t bytes) {
    bytes = arena_round(bytes ? bytes : 1);
    used -= std::min(used, bytes);
    auto it = free_.emplace(off, bytes).first;
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

}  // namespace cur
