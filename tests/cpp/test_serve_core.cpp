// Unit test of the render server's host core (no GPU): range allocator,
// FIFO admission queue and latency percentiles.  Built and run by
// tests/test_serve_core.py.
#include <cassert>
#include <cstdio>
#include <random>
#include <vector>

#include "serve_core.h"

using adop::serve::AdmissionQueue;
using adop::serve::LatencyStats;
using adop::serve::RangeAllocator;

#define CHECK(c)                                                        \
  do {                                                                  \
    if (!(c)) {                                                         \
      std::printf("FAIL %s:%d: %s\n", __FILE__, __LINE__, #c);          \
      return 1;                                                         \
    }                                                                   \
  } while (0)

int main() {
  // allocator: alignment, exhaustion, merge on release
  RangeAllocator a(4096, 256);
  size_t o1 = a.alloc(100), o2 = a.alloc(1000), o3 = a.alloc(256);
  CHECK(o1 == 0 && o2 == 256 && o3 == 1280);
  CHECK(a.in_use() == 256 + 1024 + 256);
  CHECK(a.alloc(4096) == SIZE_MAX);
  CHECK(a.release(o2));
  CHECK(!a.release(o2));
  CHECK(a.alloc(1024) == 256);  // first fit reuses the hole
  CHECK(a.release(256) && a.release(o1) && a.release(o3));
  CHECK(a.in_use() == 0 && a.free_ranges() == 1 && a.largest_free() == 4096);
  CHECK(a.peak() == 1536);

  // random alloc/free never overlaps and always merges back
  std::mt19937 rng(1);
  RangeAllocator b(1 << 20, 256);
  std::vector<std::pair<size_t, size_t>> live;
  for (int it = 0; it < 20000; ++it) {
    if (live.empty() || rng() % 2) {
      size_t n = 1 + rng() % 20000;
      size_t o = b.alloc(n);
      if (o != SIZE_MAX) {
        size_t len = b.round(n);
        for (auto& lv : live) CHECK(o + len <= lv.first || lv.first + lv.second <= o);
        CHECK(o % 256 == 0 && o + len <= b.capacity());
        live.push_back({o, len});
      }
    } else {
      size_t k = rng() % live.size();
      CHECK(b.release(live[k].first));
      live.erase(live.begin() + k);
    }
  }
  for (auto& lv : live) CHECK(b.release(lv.first));
  CHECK(b.in_use() == 0 && b.free_ranges() == 1);

  // admission queue: FIFO and removal of a queued ticket
  AdmissionQueue<int> q;
  for (int i = 0; i < 5; ++i) q.push(i);
  CHECK(q.remove_if_first([](int v) { return v == 3; }));
  CHECK(!q.remove_if_first([](int v) { return v == 3; }));
  std::vector<int> order;
  while (!q.empty()) {
    order.push_back(q.front());
    q.pop();
  }
  CHECK((order == std::vector<int>{0, 1, 2, 4}));

  // latency percentiles (nearest rank)
  LatencyStats s;
  for (int i = 1; i <= 100; ++i) s.add((double)i);
  CHECK(s.percentile(50) == 50.0 && s.percentile(99) == 99.0 && s.percentile(100) == 100.0);
  CHECK(s.mean() == 50.5 && s.max() == 100.0 && s.count() == 100);
  std::printf("serve core: ok\n");
  return 0;
}
