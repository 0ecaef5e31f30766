// Host-side scheduling pieces of the request server (server.cu): the pool
// allocator, the work measure of a request, its stream priority level and the
// admission rule.  Plain C++17 with no CUDA dependency, so that the CPU tests
// build and exercise the same code with a host compiler.
#pragma once

#include <stddef.h>

#include <algorithm>
#include <iterator>
#include <map>
#include <vector>

#include "gp.h"

namespace gp {
namespace sched {

constexpr size_t kAlign = 256;

inline size_t align_up(size_t x) { return (x + kAlign - 1) & ~(kAlign - 1); }

// First-fit allocator over [0, size) with coalescing frees.  Block sizes are
// rounded up to kAlign; offsets are multiples of kAlign.
class PoolAllocator {
 public:
  explicit PoolAllocator(size_t size) : size_(size) {
    if (size_ > 0) free_[0] = size_;
  }
  bool alloc(size_t bytes, size_t* off) {
    bytes = align_up(bytes);
    for (auto it = free_.begin(); it != free_.end(); ++it) {
      if (it->second >= bytes) {
        *off = it->first;
        const size_t rest = it->second - bytes;
        const size_t start = it->first + bytes;
        free_.erase(it);
        if (rest > 0) free_[start] = rest;
        in_use_ += bytes;
        return true;
      }
    }
    return false;
  }
  void release(size_t off, size_t bytes) {
    bytes = align_up(bytes);
    in_use_ -= bytes;
    auto it = free_.emplace(off, bytes).first;
    auto next = std::next(it);
    if (next != free_.end() && it->first + it->second == next->first) {
      it->second += next->second;
      free_.erase(next);
    }
    if (it != free_.begin()) {
      auto prev = std::prev(it);
      if (prev->first + prev->second == it->first) {
        prev->second += it->second;
        free_.erase(it);
      }
    }
  }
  size_t in_use() const { return in_use_; }
  size_t size() const { return size_; }
  // Number of free extents (1 when everything has been released).
  size_t free_extents() const { return free_.size(); }

 private:
  size_t size_;
  size_t in_use_ = 0;
  std::map<size_t, size_t> free_;
};

// Entries x columns of the products a request issues (its CG, Lanczos and
// gradient passes, or its CG and the prediction product).
inline double request_work(const gp_request& r) {
  const double n = static_cast<double>(r.n);
  const int maxit = r.cg_maxit > 0 ? r.cg_maxit : 1000;
  if (r.kind == 0) {
    const int k = r.nlanczos > 0 ? r.nlanczos : 20;
    return n * n * (1.0 + r.nprobe) * (maxit + k + 1);
  }
  return n * n * maxit + n * static_cast<double>(r.m);
}

// Stream priority level (0 = highest) of a request: one level per decade of
// work above 1e9 entries x columns, clamped to the levels the device offers.
inline int priority_level(const gp_request& r, int levels) {
  const double w = request_work(r);
  int b = 0;
  for (double t = 1e10; w >= t && b < levels - 1; t *= 10.0) ++b;
  return b;
}

// Waiting time after which a queued request is admitted before any younger one
// (bounds how long the least-work-first order can hold a large request back).
constexpr double kAgeSeconds = 30.0;

// The admission rule over a queue in arrival order.  Entry i has work(i),
// submit time t_submit(i) and pool footprint bytes(i).  The oldest request
// goes first once it has waited kAgeSeconds (nothing starts while it does not
// fit); otherwise the request with the least work that fits, the earlier one
// among equal work.  Returns the admitted index and reserves its block in
// `pool` (*off), or -1 when nothing can start now.
template <class Work, class Submit, class Bytes>
long pick_next(size_t count, double now, PoolAllocator& pool, Work work, Submit t_submit,
               Bytes bytes, size_t* off) {
  if (count == 0) return -1;
  if (now - t_submit(0) >= kAgeSeconds) return pool.alloc(bytes(0), off) ? 0 : -1;
  std::vector<size_t> order(count);
  for (size_t i = 0; i < count; ++i) order[i] = i;
  std::stable_sort(order.begin(), order.end(), [&](size_t a, size_t b) { return work(a) < work(b); });
  for (size_t i : order)
    if (pool.alloc(bytes(i), off)) return static_cast<long>(i);
  return -1;
}

// Dimension class of a problem: the compile-time dimension template the
// products are instantiated for (1, 2, 3, 4; 5..8 -> 8; 9..16 -> 16).
inline int dim_class(int d) {
  if (d <= 4) return d;
  if (d <= 8) return 8;
  return 16;
}

// Requests that gp_loss_and_grad_batch can take: loss + gradient with FP32
// products and 1 + nprobe <= 64.
inline bool batchable(const gp_request& r) {
  const int slq = r.slq_prec == GP_PREC_SAME ? r.prec : r.slq_prec;
  return r.kind == 0 && r.prec == GP_PREC_FP32 && slq == GP_PREC_FP32 && 1 + r.nprobe <= 64;
}

// Two requests share a batch when both are batchable and agree on what one
// grouped launch needs in common: kernel, dimension class, nprobe, nlanczos.
inline bool same_batch(const gp_request& a, const gp_request& b) {
  const int ka = a.nlanczos > 0 ? a.nlanczos : 20, kb = b.nlanczos > 0 ? b.nlanczos : 20;
  return batchable(a) && batchable(b) && a.kernel == b.kernel && dim_class(a.d) == dim_class(b.d) &&
         a.nprobe == b.nprobe && ka == kb;
}

// Largest ratio between the work of two members of one batch: members advance
// together, so a much smaller member would wait for the larger ones.
constexpr double kBatchWorkRatio = 16.0;

// The batch of an admitted request `first` (not in the queue any more): up to
// max_extra queued requests k with compatible(k) and work within
// kBatchWorkRatio of first_work (either way), taken in order of increasing
// work (arrival order among equal work) while their blocks fit the pool; their
// blocks are reserved (offs) and their indices returned in that order.
template <class Compatible, class Work, class Bytes>
std::vector<size_t> pick_batch(size_t count, double first_work, int max_extra, PoolAllocator& pool,
                               Compatible compatible, Work work, Bytes bytes,
                               std::vector<size_t>* offs) {
  std::vector<size_t> order, chosen;
  for (size_t i = 0; i < count; ++i) {
    const double r = work(i) > first_work ? work(i) / first_work : first_work / work(i);
    if (compatible(i) && r <= kBatchWorkRatio) order.push_back(i);
  }
  std::stable_sort(order.begin(), order.end(), [&](size_t a, size_t b) { return work(a) < work(b); });
  for (size_t i : order) {
    if (static_cast<int>(chosen.size()) >= max_extra) break;
    size_t off = 0;
    if (pool.alloc(bytes(i), &off)) {
      chosen.push_back(i);
      offs->push_back(off);
    }
  }
  return chosen;
}

}  // namespace sched
}  // namespace gp
