// Host scheduling of independent jobs under a memory budget: the admission policy
// of mg_batch_solve, free of CUDA so that it compiles and is tested on a host alone.
#pragma once

#include <algorithm>
#include <condition_variable>
#include <cstddef>
#include <mutex>
#include <numeric>
#include <thread>
#include <vector>

namespace mgsched {

// Runs jobs 0 .. n-1 on at most max_threads host threads (0: one per job) and puts
// run(i)'s result into status[i].
// * budget 0: every job may run at once, in index order; release is not called.
// * budget > 0: jobs start in order of decreasing est[i], each only while the
//   estimates of the running jobs and its own fit the budget (or when none runs);
//   release(i) is called when job i ends; a job whose result is retry_status is
//   run again alone, followed by release, after all others have ended.
// Returns false if the threads could not be started (the jobs that had started
// have ended; the others did not run).
template <class Run, class Release>
bool run_jobs(int n, const std::vector<size_t>& est, size_t budget, int max_threads, Run&& run, Release&& release,
              std::vector<int>& status, int retry_status) {
    std::vector<int> order(n);
    std::iota(order.begin(), order.end(), 0);
    if (budget) std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return est[a] > est[b]; });
    status.assign(n, 0);
    std::vector<int> retry;
    std::mutex mu;
    std::condition_variable cv;
    size_t in_use = 0;
    int running = 0, next = 0;
    auto worker = [&]() {
        for (;;) {
            std::unique_lock<std::mutex> lk(mu);
            if (next >= n) return;
            const int i = order[next++];
            if (budget) cv.wait(lk, [&] { return running == 0 || in_use + est[i] <= budget; });
            in_use += est[i];
            ++running;
            lk.unlock();
            const int s = run(i);
            if (budget) release(i);
            lk.lock();
            status[i] = s;
            in_use -= est[i];
            --running;
            if (budget && s == retry_status) retry.push_back(i);
            lk.unlock();
            cv.notify_all();
        }
    };
    const int nt = max_threads == 0 ? n : std::min(n, max_threads);
    std::vector<std::thread> pool;
    pool.reserve(nt);
    try {
        for (int t = 0; t < nt; ++t) pool.emplace_back(worker);
    } catch (...) {
        {
            std::lock_guard<std::mutex> lk(mu);
            next = n;  // no further job starts
        }
        cv.notify_all();
        for (auto& th : pool) th.join();
        return false;
    }
    for (auto& th : pool) th.join();
    for (int i : retry) {
        status[i] = run(i);
        release(i);
    }
    return true;
}

}  // namespace mgsched
