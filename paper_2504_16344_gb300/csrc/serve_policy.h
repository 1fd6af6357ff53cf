// serve_policy.h -- admission and batching policy of the serving loop (host only).
//
// Requests (an arrival time, an event, an observation window) are admitted
// in arrival order.  The policy is work-conserving continuous batching at
// batch granularity: whenever the device is idle and requests are waiting,
// the oldest min(waiting, max_batch) of them start as one batch; requests
// that arrive while a batch runs wait for the next one.  `max_batch` is the
// number of slots the context reserved (tw_reserve_batch), chosen from free
// device memory, so admission by slots is admission by memory.
//
// The policy is separated from the CUDA calls so the same code drives the
// device loop (tw_serve_replay) and a virtual-clock simulation
// (tw_serve_simulate) that the host-only tests exercise.
#pragma once
#include <algorithm>
#include <cstddef>
#include <vector>

namespace twserve {

class Policy {
 public:
  Policy(int nreq, const double *arrival_s, int max_batch)
      : n_(nreq), arr_(arrival_s), max_batch_(max_batch) {}

  // requests with arrival <= now join the waiting queue (they arrive in order)
  void admit(double now) {
    while (next_ < n_ && arr_[next_] <= now) queue_end_ = ++next_;
  }
  bool waiting() const { return head_ < queue_end_; }
  bool all_admitted() const { return next_ >= n_; }
  double next_arrival() const { return next_ < n_ ? arr_[next_] : -1.0; }
  // the next batch: [first, first + count) in request order
  void take(int *first, int *count) {
    *first = head_;
    *count = std::min(max_batch_, queue_end_ - head_);
    head_ += *count;
  }
  bool done() const { return head_ >= n_; }

 private:
  int n_;
  const double *arr_;
  int max_batch_;
  int next_ = 0;        // first request not yet arrived
  int queue_end_ = 0;   // one past the last arrived request
  int head_ = 0;        // first waiting request
};

}  // namespace twserve
