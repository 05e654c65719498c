// Host threads for the batched calls of the differentiable form.  Each image's
// kernels go to its own handle's stream; queuing them from one thread per image
// keeps the host's launch rate from serialising small images.  The pool is created
// on first use and lives until the process exits (its threads then sit idle on a
// condition variable).
#pragma once

#include <cuda_runtime.h>
#include <unistd.h>

#include <algorithm>
#include <condition_variable>
#include <cstdint>
#include <functional>
#include <mutex>
#include <thread>
#include <vector>

namespace dsg {

class HostPool {
  public:
    // Runs fn(0) .. fn(count - 1), each once, on the caller and the pool's threads with
    // the caller's CUDA device current; returns when every call has returned.  Calls
    // from different threads are taken one at a time; fn must not call run itself.
    static void run(int count, const std::function<void(int)>& fn) {
        if (count <= 0) return;
        if (count == 1) {
            fn(0);
            return;
        }
        instance().run_all(count, fn);
    }

  private:
    std::mutex run_mu_;  // one batch at a time
    std::mutex mu_;
    std::condition_variable work_cv_, done_cv_;
    std::vector<std::thread> threads_;
    const std::function<void(int)>* job_ = nullptr;
    int count_ = 0, next_ = 0, pending_ = 0, device_ = 0;
    uint64_t gen_ = 0;

    pid_t pid_ = getpid();

    // A child made by fork() has none of the parent's threads: it gets a fresh pool
    // (the parent's copy is abandoned, never destroyed).
    static HostPool& instance() {
        static std::mutex mu;
        static HostPool* p = nullptr;
        std::lock_guard<std::mutex> lk(mu);
        if (!p || p->pid_ != getpid()) p = new HostPool();
        return *p;
    }

    // takes tasks until none is left (mu_ held on entry and on return)
    void drain(std::unique_lock<std::mutex>& lk) {
        while (next_ < count_) {
            const int i = next_++;
            const std::function<void(int)>* f = job_;
            const int dev = device_;
            lk.unlock();
            cudaSetDevice(dev);
            (*f)(i);
            lk.lock();
            if (--pending_ == 0) done_cv_.notify_all();
        }
    }

    void loop() {
        uint64_t seen = 0;
        std::unique_lock<std::mutex> lk(mu_);
        for (;;) {
            work_cv_.wait(lk, [&] { return gen_ != seen; });
            seen = gen_;
            drain(lk);
        }
    }

    void run_all(int count, const std::function<void(int)>& fn) {
        std::lock_guard<std::mutex> serial(run_mu_);
        int dev = 0;
        cudaGetDevice(&dev);
        const int hw = (int)std::max(1u, std::thread::hardware_concurrency());
        const int want = std::min(std::min(count, hw) - 1, 15);
        std::unique_lock<std::mutex> lk(mu_);
        while ((int)threads_.size() < want) threads_.emplace_back([this] { loop(); });
        job_ = &fn;
        count_ = count;
        next_ = 0;
        pending_ = count;
        device_ = dev;
        ++gen_;
        work_cv_.notify_all();
        drain(lk);
        done_cv_.wait(lk, [&] { return pending_ == 0; });
        job_ = nullptr;
        count_ = 0;
    }
};

}  // namespace dsg
