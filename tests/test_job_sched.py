"""Host logic of the concurrent-instance scheduler (csrc/job_sched.h), on the CPU.

mg_batch_solve admits independent solves under a device-memory budget: largest
estimate first, each only while the running ones' estimates and its own fit the
budget (or when none runs), work buffers released when a solve ends, and a solve
that ran out of memory next to others repeated alone at the end.  The policy is
CUDA-free C++; a small driver compiled here with g++ runs it on sleeping jobs and
reports what happened.
"""

import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1912_03106_gb300", "csrc")

DRIVER = r'''
#include <atomic>
#include <chrono>
#include <cstdio>
#include <cstdlib>
#include <mutex>
#include <random>
#include <thread>
#include <vector>
#include "job_sched.h"

// args: n budget max_threads seed enomem_job (-1: none)
int main(int argc, char** argv) {
    const int n = std::atoi(argv[1]);
    const size_t budget = (size_t)std::atoll(argv[2]);
    const int max_threads = std::atoi(argv[3]);
    std::mt19937 rng(std::atoi(argv[4]));
    const int enomem_job = std::atoi(argv[5]);
    std::vector<size_t> est(n);
    for (auto& e : est) e = 1 + rng() % 100;
    std::mutex mu;
    size_t in_use = 0, peak = 0, peak_over = 0;
    int running = 0, max_running = 0;
    std::vector<int> runs(n, 0), released(n, 0), start_order;
    auto run = [&](int i) {
        {
            std::lock_guard<std::mutex> lk(mu);
            in_use += est[i];
            ++running;
            max_running = std::max(max_running, running);
            peak = std::max(peak, in_use);
            if (budget && in_use > budget && running > 1) peak_over = std::max(peak_over, in_use);
            ++runs[i];
            start_order.push_back(i);
        }
        std::this_thread::sleep_for(std::chrono::milliseconds(1 + (i * 7) % 5));
        int s = 0;
        {
            std::lock_guard<std::mutex> lk(mu);
            if (i == enomem_job && running > 1) s = 9;  // out of memory next to others
            in_use -= est[i];
            --running;
        }
        return s;
    };
    auto release = [&](int i) {
        std::lock_guard<std::mutex> lk(mu);
        ++released[i];
    };
    std::vector<int> status;
    const bool ok = mgsched::run_jobs(n, est, budget, max_threads, run, release, status, 9);
    int bad_status = 0, bad_runs = 0, bad_release = 0, order_ok = 1;
    for (int i = 0; i < n; ++i) {
        bad_status += status[i] != 0;
        bad_runs += runs[i] != (i == enomem_job && budget && runs[i] == 2 ? 2 : 1);
        bad_release += budget ? released[i] != runs[i] : released[i] != 0;
    }
    if (max_threads == 1 && budget)
        for (size_t k = 1; k < (size_t)n; ++k)
            if (est[start_order[k]] > est[start_order[k - 1]]) order_ok = 0;
    size_t max_est = 0;
    for (auto e : est) max_est = std::max(max_est, e);
    std::printf("ok %d peak %zu peak_over %zu max_running %d bad_status %d bad_runs %d bad_release %d "
                "order_ok %d max_est %zu enomem_runs %d\n", ok, peak, peak_over, max_running, bad_status, bad_runs,
                bad_release, order_ok, max_est, enomem_job >= 0 ? runs[enomem_job] : 0);
    return 0;
}
'''


@pytest.fixture(scope="module")
def driver(tmp_path_factory):
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no C++ compiler")
    d = tmp_path_factory.mktemp("sched")
    src = d / "driver.cpp"
    src.write_text(DRIVER)
    exe = d / "driver"
    r = subprocess.run([cxx, "-std=c++17", "-O1", "-pthread", "-I", CSRC, str(src), "-o", str(exe)],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    return str(exe)


def run(driver, n, budget, threads, seed, enomem=-1):
    out = subprocess.run([driver, str(n), str(budget), str(threads), str(seed), str(enomem)], capture_output=True,
                         text=True, check=True, timeout=60).stdout.split()
    return {out[k]: int(out[k + 1]) for k in range(0, len(out), 2)}


@pytest.mark.parametrize("seed", [0, 1, 2])
@pytest.mark.parametrize("budget", [120, 300, 1000])
def test_running_estimates_stay_within_the_budget(driver, budget, seed):
    r = run(driver, 40, budget, 0, seed)
    assert r["ok"] == 1 and r["bad_status"] == 0 and r["bad_runs"] == 0 and r["bad_release"] == 0
    assert r["peak_over"] == 0  # only a job alone may exceed the budget
    assert r["peak"] <= max(budget, r["max_est"])


def test_a_budget_below_every_job_runs_them_one_at_a_time(driver):
    r = run(driver, 12, 1, 0, 5)
    assert r["ok"] == 1 and r["max_running"] == 1 and r["bad_runs"] == 0 and r["bad_release"] == 0


def test_no_budget_runs_everything_at_once_without_release(driver):
    r = run(driver, 16, 0, 0, 3)
    assert r["ok"] == 1 and r["bad_status"] == 0 and r["bad_runs"] == 0 and r["bad_release"] == 0
    assert r["max_running"] > 1


def test_largest_estimate_starts_first(driver):
    r = run(driver, 20, 10_000, 1, 4)
    assert r["ok"] == 1 and r["order_ok"] == 1 and r["max_running"] == 1


def test_out_of_memory_next_to_others_is_repeated_alone(driver):
    """Job 3 fails whenever another job runs beside it; it is run again alone at
    the end and succeeds, and its buffers are released after each run."""
    r = run(driver, 24, 10_000, 0, 6, enomem=3)
    assert r["ok"] == 1 and r["bad_status"] == 0 and r["bad_runs"] == 0 and r["bad_release"] == 0
    assert r["enomem_runs"] == 2
