// Drives the server's host-side arena allocator (csrc/arena.h) from a script
// on stdin, one operation per line:
//   I cap        init with `cap` bytes
//   A id bytes   allocate; prints "A id off" or "A id fail"
//   R id         release the block allocated as `id`
//   S            prints "S used peak nfree" and every free block "F off bytes"
#include <cstdio>
#include <map>

#include "arena.h"

int main() {
  cur::Arena a;
  std::map<long long, std::pair<size_t, size_t>> live;  // id -> (offset, requested bytes)
  char op;
  while (std::scanf(" %c", &op) == 1) {
    if (op == 'I') {
      size_t cap;
      if (std::scanf("%zu", &cap) != 1) return 2;
      a.init(cap);
    } else if (op == 'A') {
      long long id;
      size_t bytes, off = 0;
      if (std::scanf("%lld %zu", &id, &bytes) != 2) return 2;
      if (a.alloc(bytes, &off)) {
        live[id] = {off, bytes};
        std::printf("A %lld %zu\n", id, off);
      } else {
        std::printf("A %lld fail\n", id);
      }
    } else if (op == 'R') {
      long long id;
      if (std::scanf("%lld", &id) != 1) return 2;
      auto it = live.find(id);
      if (it == live.end()) return 3;
      a.release(it->second.first, it->second.second);
      live.erase(it);
    } else if (op == 'S') {
      std::printf("S %zu %zu %zu\n", a.used, a.peak, a.free_.size());
      for (const auto& f : a.free_) std::printf("F %zu %zu\n", f.first, f.second);
    } else {
      return 2;
    }
  }
  return 0;
}
