// serve_policy.h -- admission and batching policy of the serving loop (host only).
//
// Requests (an arrival time, an event, an observation window) are admitted
// in arrival order into `lanes` independent batch slots sets ("lanes"; each
// holds up to max_batch right-hand sides).  Continuous batching: whenever a
// lane is free and requests are waiting, the oldest min(waiting, max_batch)
// of them start in that lane at once, while the batches of the other lanes
// are still running -- requests that arrive during a batch do not wait for
// it to finish, only for a free lane.  Batches start in request order; they
// may finish out of order.  The number of lanes is fixed per session from
// free device memory (each lane is a full set of batch workspaces), so
// admission by lanes and slots is admission by memory.
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
  Policy(int nreq, const double *arrival_s, int max_batch, int lanes)
      : n_(nreq), arr_(arrival_s), max_batch_(max_batch), busy_(lanes > 0 ? lanes : 1, 0) {}

  // requests with arrival <= now join the waiting queue (they arrive in order)
  void admit(double now) {
    while (next_ < n_ && arr_[next_] <= now) queue_end_ = ++next_;
  }
  bool waiting() const { return head_ < queue_end_; }
  bool all_taken() const { return head_ >= n_; }
  double next_arrival() const { return next_ < n_ ? arr_[next_] : -1.0; }
  int lanes() const { return (int)busy_.size(); }
  int in_flight() const { return (int)std::count(busy_.begin(), busy_.end(), 1); }
  // lowest free lane, -1 if all are busy
  int free_lane() const {
    for (int l = 0; l < lanes(); ++l)
      if (!busy_[l]) return l;
    return -1;
  }
  // the next batch, [first, first + count) in request order, into free lane l
  void take(int l, int *first, int *count) {
    *first = head_;
    *count = std::min(max_batch_, queue_end_ - head_);
    head_ += *count;
    busy_[l] = 1;
  }
  // lane l's batch has finished
  void release(int l) { busy_[l] = 0; }
  bool done() const { return all_taken() && in_flight() == 0; }

 private:
  int n_;
  const double *arr_;
  int max_batch_;
  std::vector<char> busy_;
  int next_ = 0;        // first request not yet arrived
  int queue_end_ = 0;   // one past the last arrived request
  int head_ = 0;        // first waiting request
};

}  // namespace twserve
