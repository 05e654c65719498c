// Checks of the host thread pool used by the batched calls of the differentiable
// form: every index runs exactly once per batch, for batch sizes below, at and above
// the number of threads, over repeated batches and from two caller threads.  Needs no
// GPU (the pool's device calls only fail).  Prints "ok" and exits 0 on success.
#include <atomic>
#include <cstdio>
#include <thread>
#include <vector>

#include "host_pool.h"

static int check(int count, int reps) {
    std::vector<std::atomic<int>> hits(count);
    for (int r = 0; r < reps; ++r) {
        for (auto& h : hits) h.store(0);
        dsg::HostPool::run(count, [&](int i) { hits[i].fetch_add(1); });
        for (int i = 0; i < count; ++i)
            if (hits[i].load() != 1) {
                std::printf("count %d rep %d: index %d ran %d times\n", count, r, i, hits[i].load());
                return 1;
            }
    }
    return 0;
}

int main() {
    for (int count : {0, 1, 2, 3, 8, 17, 64})
        if (check(count, 20)) return 1;
    // two callers at once: their batches are taken one at a time
    int bad_a = 0, bad_b = 0;
    std::thread a([&] { bad_a = check(9, 50); });
    std::thread b([&] { bad_b = check(5, 50); });
    a.join();
    b.join();
    if (bad_a || bad_b) return 1;
    std::printf("ok\n");
    return 0;
}
