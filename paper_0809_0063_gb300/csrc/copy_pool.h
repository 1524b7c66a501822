// A small persistent pool of host threads for the serving loop's gather and scatter copies
// (plain C++, no CUDA: tested on the CPU by tests/test_copy_pool_cpu.py).
//
// run(n, fn) calls fn(i) exactly once for every i in [0, n), spread over the workers and the
// calling thread (which takes part), and returns when every call has returned.  Items are
// handed out one at a time from an atomic counter, so a few large items do not leave the other
// threads idle.  One run at a time (the serving loop is its only caller); the destructor stops
// and joins the workers.
#pragma once

#include <atomic>
#include <condition_variable>
#include <cstddef>
#include <cstdint>
#include <functional>
#include <mutex>
#include <thread>
#include <vector>

namespace fpd {

class CopyPool {
 public:
  explicit CopyPool(int workers) {
    for (int i = 0; i < workers; ++i) threads_.emplace_back([this] { worker(); });
  }
  ~CopyPool() {
    {
      std::lock_guard<std::mutex> lk(mu_);
      quit_ = true;
    }
    cv_.notify_all();
    for (auto& t : threads_) t.join();
  }
  CopyPool(const CopyPool&) = delete;
  CopyPool& operator=(const CopyPool&) = delete;

  int workers() const { return (int)threads_.size(); }

  void run(size_t n, const std::function<void(size_t)>& fn) {
    if (n == 0) return;
    if (threads_.empty() || n == 1) {
      for (size_t i = 0; i < n; ++i) fn(i);
      return;
    }
    {
      std::lock_guard<std::mutex> lk(mu_);
      job_ = &fn;
      n_ = n;
      next_.store(0);
      left_ = threads_.size();   // workers that have not yet finished this run
      ++gen_;
    }
    cv_.notify_all();
    drain();
    std::unique_lock<std::mutex> lk(mu_);
    done_.wait(lk, [this] { return left_ == 0; });
    job_ = nullptr;
  }

 private:
  void drain() {
    const std::function<void(size_t)>& fn = *job_;
    for (size_t i = next_.fetch_add(1); i < n_; i = next_.fetch_add(1)) fn(i);
  }

  void worker() {
    uint64_t seen = 0;
    for (;;) {
      {
        std::unique_lock<std::mutex> lk(mu_);
        cv_.wait(lk, [&] { return quit_ || gen_ != seen; });
        if (quit_) return;
        seen = gen_;
      }
      drain();
      {
        std::lock_guard<std::mutex> lk(mu_);
        if (--left_ == 0) done_.notify_one();
      }
    }
  }

  std::vector<std::thread> threads_;
  std::mutex mu_;
  std::condition_variable cv_, done_;
  const std::function<void(size_t)>* job_ = nullptr;
  size_t n_ = 0;
  std::atomic<size_t> next_{0};
  size_t left_ = 0;
  uint64_t gen_ = 0;
  bool quit_ = false;
};

}  // namespace fpd
