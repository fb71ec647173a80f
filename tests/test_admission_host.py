"""The request server's admission policy (paper_1607_03777_gb300/csrc/admission.h),
host logic compiled on its own with g++ and checked without a GPU: arrival
order while the oldest request fits, backfilling past it while it does not,
at most ``max_bypass`` times, after which it is reserved; in a simulated
stream where small requests keep arriving, every large request runs within a
bounded wait and no request is passed more often than the bound."""
import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "..", "paper_1607_03777_gb300", "csrc")

HARNESS = r"""
#include "admission.h"
#include <cstdio>
#include <deque>
#include <random>
#include <vector>

struct R { long long bytes; int bypassed; int id; };

static int pick(const std::deque<R>& q, long long in_use, long long budget, int mb) {
    return sip::admission_pick(q, in_use, budget, mb);
}

int main() {
    std::deque<R> q;
    std::printf("empty %d\n", pick(q, 0, 10, 4));
    q = {{5, 0, 0}, {2, 0, 1}};
    std::printf("head_fits %d\n", pick(q, 0, 10, 4));
    std::printf("backfill %d\n", pick(q, 7, 10, 4));
    q[0].bypassed = 4;
    std::printf("reserved %d\n", pick(q, 7, 10, 4));
    q = {{5, 0, 0}, {4, 0, 1}, {3, 0, 2}};
    std::printf("none_fits %d\n", pick(q, 8, 10, 4));
    std::printf("first_that_fits %d\n", pick(q, 7, 10, 4));

    // arrivals: one small request (1 of a budget of 10) every tick for 400
    // ticks, each running 2 ticks (two in flight: within the 4 slots), and a
    // large one (the whole budget) every 50 ticks, running 5.  The large one
    // fits only when no small one runs, which the steady small stream never
    // allows: without the bound it would be passed until the arrivals stop
    const int slots = 4, mb = 4 * slots, ticks = 400;
    const long long budget = 10;
    std::deque<R> queue;
    struct Run { long long bytes; int left; };
    std::vector<Run> running;
    std::vector<int> arrived(ticks + ticks / 50 + 8, 0);
    long long in_use = 0;
    int next_id = 0, admitted = 0, max_bypassed = 0, order_violations = 0, max_large_wait = 0;
    for (int tick = 0; tick < ticks + 200; ++tick) {
        for (auto it = running.begin(); it != running.end();) {
            if (--it->left <= 0) { in_use -= it->bytes; it = running.erase(it); }
            else ++it;
        }
        if (tick < ticks) {
            if (tick % 50 == 0) { queue.push_back({10, 0, next_id}); arrived[next_id++] = tick; }
            queue.push_back({1, 0, next_id});
            arrived[next_id++] = tick;
        }
        while ((int)running.size() < slots) {
            const int i = pick(queue, in_use, budget, mb);
            if (i < 0) break;
            if (i > 0) {
                if (queue.front().bypassed >= mb) ++order_violations;   // passed a reserved head
                ++queue.front().bypassed;
            }
            R r = queue[i];
            queue.erase(queue.begin() + i);
            if (r.bypassed > max_bypassed) max_bypassed = r.bypassed;
            if (r.bytes == 10 && tick - arrived[r.id] > max_large_wait)
                max_large_wait = tick - arrived[r.id];
            running.push_back({r.bytes, r.bytes == 10 ? 5 : 2});
            in_use += r.bytes;
            ++admitted;
        }
    }
    std::printf("sim_arrived %d\n", next_id);
    std::printf("sim_admitted %d\n", admitted);
    std::printf("sim_max_bypassed %d\n", max_bypassed);
    std::printf("sim_order_violations %d\n", order_violations);
    std::printf("sim_max_large_wait %d\n", max_large_wait);
    std::printf("sim_bound %d\n", mb);
    return 0;
}
"""


def test_admission_policy(tmp_path):
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no C++ compiler")
    src = tmp_path / "harness.cpp"
    src.write_text(HARNESS)
    exe = tmp_path / "harness"
    subprocess.run([cxx, "-std=c++17", "-O1", "-I", CSRC, str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout
    got = {k: int(v) for k, v in (line.split() for line in out.strip().splitlines())}
    assert got["empty"] == -1
    assert got["head_fits"] == 0            # arrival order while the oldest fits
    assert got["backfill"] == 1             # a later request that fits runs ahead
    assert got["reserved"] == -1            # not once the oldest has been passed enough
    assert got["none_fits"] == -1
    assert got["first_that_fits"] == 2      # the first one that fits, not just the next
    assert got["sim_admitted"] == got["sim_arrived"]   # every request runs
    assert got["sim_max_bypassed"] <= got["sim_bound"]
    assert got["sim_order_violations"] == 0
    # a large request waits at most while the bound's worth of small ones
    # pass it and the running ones drain (a few ticks each), not until the
    # small arrivals stop (hundreds of ticks)
    assert got["sim_max_large_wait"] <= 25
