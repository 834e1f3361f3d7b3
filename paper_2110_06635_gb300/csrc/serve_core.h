// Host-side core of the render server: a range allocator over the server's
// one device allocation, the admission queue bookkeeping and latency
// statistics.  Plain C++ (no CUDA), so it is unit-tested on the CPU.
#pragma once

#include <algorithm>
#include <cmath>
#include <cstddef>
#include <cstdint>
#include <deque>
#include <iterator>
#include <map>
#include <vector>

namespace adop {
namespace serve {

// First-fit allocator of byte ranges inside [0, capacity).  Offsets are
// multiples of `align`; freed ranges are merged with their neighbours.
class RangeAllocator {
 public:
  explicit RangeAllocator(size_t capacity = 0, size_t align = 256) : cap_(capacity), align_(align) {
    if (cap_ > 0) free_[0] = cap_;
  }
  size_t capacity() const { return cap_; }
  size_t in_use() const { return used_; }
  size_t peak() const { return peak_; }
  size_t round(size_t n) const { return (n + align_ - 1) / align_ * align_; }

  // Returns the offset, or SIZE_MAX if no free range is large enough.
  size_t alloc(size_t n) {
    n = round(n == 0 ? 1 : n);
    for (auto it = free_.begin(); it != free_.end(); ++it) {
      if (it->second >= n) {
        const size_t off = it->first, len = it->second;
        free_.erase(it);
        if (len > n) free_[off + n] = len - n;
        live_[off] = n;
        used_ += n;
        peak_ = std::max(peak_, used_);
        return off;
      }
    }
    return SIZE_MAX;
  }

  // Returns false for an offset that is not live.
  bool release(size_t off) {
    auto lv = live_.find(off);
    if (lv == live_.end()) return false;
    size_t len = lv->second;
    live_.erase(lv);
    used_ -= len;
    auto nx = free_.lower_bound(off);
    if (nx != free_.end() && off + len == nx->first) {
      len += nx->second;
      nx = free_.erase(nx);
    }
    if (nx != free_.begin()) {
      auto pv = std::prev(nx);
      if (pv->first + pv->second == off) {
        pv->second += len;
        return true;
      }
    }
    free_[off] = len;
    return true;
  }

  size_t largest_free() const {
    size_t m = 0;
    for (const auto& kv : free_) m = std::max(m, kv.second);
    return m;
  }
  size_t free_ranges() const { return free_.size(); }

 private:
  size_t cap_, align_;
  size_t used_ = 0, peak_ = 0;
  std::map<size_t, size_t> free_;  // offset -> length
  std::map<size_t, size_t> live_;  // offset -> length
};

// Latency samples (milliseconds) and percentiles by nearest rank.
class LatencyStats {
 public:
  void add(double ms) {
    samples_.push_back(ms);
    if (samples_.size() > kMax) samples_.erase(samples_.begin(), samples_.begin() + (samples_.size() - kMax));
  }
  size_t count() const { return samples_.size(); }
  double percentile(double q) const {
    if (samples_.empty()) return 0.0;
    std::vector<double> v(samples_.begin(), samples_.end());
    size_t k = (size_t)std::ceil(q / 100.0 * (double)v.size());
    k = k == 0 ? 0 : k - 1;
    if (k >= v.size()) k = v.size() - 1;
    std::nth_element(v.begin(), v.begin() + k, v.end());
    return v[k];
  }
  double mean() const {
    if (samples_.empty()) return 0.0;
    double s = 0.0;
    for (double x : samples_) s += x;
    return s / (double)samples_.size();
  }
  double max() const {
    double m = 0.0;
    for (double x : samples_) m = std::max(m, x);
    return m;
  }
  void clear() { samples_.clear(); }

 private:
  static constexpr size_t kMax = 1 << 20;
  std::deque<double> samples_;
};

// Admission: strict FIFO (no request overtakes an older one, so none starves);
// the head is admitted when a slot is free and its memory fits.
template <class Req>
class AdmissionQueue {
 public:
  void push(Req r) { q_.push_back(std::move(r)); }
  size_t size() const { return q_.size(); }
  bool empty() const { return q_.empty(); }
  Req& front() { return q_.front(); }
  void pop() { q_.pop_front(); }
  // Remove the request with this ticket if it is still queued.
  template <class Pred>
  bool remove_if_first(Pred p) {
    for (auto it = q_.begin(); it != q_.end(); ++it)
      if (p(*it)) {
        q_.erase(it);
        return true;
      }
    return false;
  }

 private:
  std::deque<Req> q_;
};

}  // namespace serve
}  // namespace adop
