// Test infrastructure: checks the service's host-side arena allocator
// (paper_2607_05622_gb300/csrc/arena.h) without a GPU.  Built and run by
// tests/test_service_arena.py; exits non-zero with a message on the first
// failed check.
#include <cstdio>
#include <vector>

#include "arena.h"

#define CHECK(c)                                              \
  do {                                                        \
    if (!(c)) {                                               \
      std::fprintf(stderr, "check failed line %d: %s\n", __LINE__, #c); \
      return 1;                                               \
    }                                                         \
  } while (0)

int main() {
  const size_t MiB = size_t(1) << 20;
  // a budget that is not a multiple of the block size is rounded down
  Arena a;
  a.init(nullptr, MiB + 100);
  CHECK(a.size == MiB);
  // a request just under the raw budget but above the usable size is refused
  // up front (it could never be allocated)
  CHECK(!a.could_fit(MiB + 50));
  CHECK(!a.could_fit(MiB + 1));
  CHECK(a.could_fit(MiB));
  CHECK(a.could_fit(MiB - 255));
  size_t off = 0;
  CHECK(a.alloc(MiB, &off) && off == 0 && a.used == MiB);
  size_t o2 = 0;
  CHECK(!a.alloc(1, &o2));
  a.release(0, MiB);
  CHECK(a.used == 0 && a.free_.size() == 1 && a.free_.begin()->second == MiB);
  // every request that could_fit() accepts is allocatable in the empty arena
  for (size_t n : {size_t(1), size_t(255), size_t(256), size_t(257), MiB - 256, MiB - 1, MiB}) {
    Arena b;
    b.init(nullptr, MiB + 100);
    size_t o = 0;
    CHECK(b.could_fit(n) == b.alloc(n, &o));
  }
  // first fit, alignment, and coalescing of freed neighbours
  Arena c;
  c.init(nullptr, 10 * 256 + 17);
  std::vector<size_t> offs(5);
  for (int i = 0; i < 5; ++i) CHECK(c.alloc(2 * 256 - 3, &offs[i]));
  for (int i = 0; i < 5; ++i) CHECK(offs[i] == size_t(i) * 512);
  CHECK(c.used == 10 * 256 && c.peak == 10 * 256);
  c.release(offs[1], 2 * 256 - 3);
  c.release(offs[3], 2 * 256 - 3);
  CHECK(c.free_.size() == 2);
  c.release(offs[2], 2 * 256 - 3);
  CHECK(c.free_.size() == 1 && c.free_.begin()->first == 512 && c.free_.begin()->second == 3 * 512);
  CHECK(c.alloc(3 * 512, &o2) && o2 == 512);
  std::puts("arena ok");
  return 0;
}
