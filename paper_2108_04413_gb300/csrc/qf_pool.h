// A small persistent host worker pool for the per-call planning work of the C
// ABI (refilling thousands of block composites for new angles).  Created on
// first use with min(hardware threads, 16) - 1 workers; the calling thread
// takes part.  One job runs at a time: a call that finds the pool busy (another
// host thread inside the library), or runs in a process forked after the pool
// started, does the work itself.
#pragma once

#include <unistd.h>

#include <algorithm>
#include <atomic>
#include <condition_variable>
#include <cstddef>
#include <functional>
#include <mutex>
#include <thread>
#include <vector>

namespace qf {

class HostPool {
 public:
  static HostPool& get() {
    static HostPool* pool = new HostPool();  // never destroyed: workers may outlive static teardown
    return *pool;
  }

  // f(i) for i in [0, n), in chunks of `grain`, on the pool and the caller.
  void parallel_for(size_t n, size_t grain, const std::function<void(size_t)>& f) {
    if (n == 0) return;
    grain = std::max<size_t>(1, grain);
    std::unique_lock<std::mutex> busy(job_mu_, std::try_to_lock);
    if (!busy.owns_lock() || workers_.empty() || getpid() != pid_ || n <= grain) {
      for (size_t i = 0; i < n; ++i) f(i);
      return;
    }
    {
      std::lock_guard<std::mutex> lk(mu_);
      fn_ = &f;
      n_ = n;
      grain_ = grain;
      next_.store(0);
      pending_ = workers_.size();
      ++gen_;
    }
    cv_.notify_all();
    drain();
    std::unique_lock<std::mutex> lk(mu_);
    done_cv_.wait(lk, [&] { return pending_ == 0; });
    fn_ = nullptr;
  }

 private:
  HostPool() : pid_(getpid()) {
    const unsigned hw = std::max(1u, std::thread::hardware_concurrency());
    const unsigned nw = std::min(hw, 16u) - 1;
    for (unsigned i = 0; i < nw; ++i) workers_.emplace_back([this] { loop(); });
    for (auto& t : workers_) t.detach();
  }

  void drain() {
    for (;;) {
      const size_t b = next_.fetch_add(grain_);
      if (b >= n_) break;
      const size_t e = std::min(n_, b + grain_);
      for (size_t i = b; i < e; ++i) (*fn_)(i);
    }
  }

  void loop() {
    size_t seen = 0;
    for (;;) {
      {
        std::unique_lock<std::mutex> lk(mu_);
        cv_.wait(lk, [&] { return gen_ != seen; });
        seen = gen_;
      }
      drain();
      {
        std::lock_guard<std::mutex> lk(mu_);
        if (--pending_ == 0) done_cv_.notify_one();
      }
    }
  }

  pid_t pid_;
  std::vector<std::thread> workers_;
  std::mutex job_mu_;  // one job at a time
  std::mutex mu_;
  std::condition_variable cv_, done_cv_;
  size_t gen_ = 0, pending_ = 0, n_ = 0, grain_ = 1;
  std::atomic<size_t> next_{0};
  const std::function<void(size_t)>* fn_ = nullptr;
};

}  // namespace qf
