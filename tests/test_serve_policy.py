"""The serving loop's admission policy (``csrc/serve_policy.h``), compiled
on the CPU into a small driver exactly as the server includes it: which
waiting requests a free slot takes, which it leaves, which fail."""
import os
import shutil
import subprocess

import pytest

from paper_2403_14723_gb300 import build

DRIVER = r"""
#include <cstdio>
#include "serve_policy.h"
using namespace polylla::policy;
struct R { ReqView v; int id; };
int main() {
    SlotView s; int lane; int lane_on; double now, steal; long long cap; int n;
    if (std::scanf("%lld %lld %lld %d %d %d %lf %lf %lld %d", &s.V_cap, &s.T_cap, &s.H_cap, &s.n_cap, &lane,
                   &lane_on, &now, &steal, &cap, &n) != 10) return 2;
    s.lane = lane != 0;
    std::deque<R> q;
    for (int i = 0; i < n; i++) {
        R r; int small;
        if (std::scanf("%lld %lld %lld %d %lf", &r.v.V, &r.v.T, &r.v.H, &small, &r.v.t_submit) != 5) return 2;
        r.v.small = small != 0; r.id = i; q.push_back(r);
    }
    std::vector<R> take, failed;
    form_batch(q, s, lane_on != 0, now, steal, cap, [](const R &r) { return r.v; },
               [&](const R &r) { failed.push_back(r); }, take);
    std::printf("take"); for (auto &r : take) std::printf(" %d", r.id); std::printf("\n");
    std::printf("fail"); for (auto &r : failed) std::printf(" %d", r.id); std::printf("\n");
    std::printf("left"); for (auto &r : q) std::printf(" %d", r.id); std::printf("\n");
    return 0;
}
"""


@pytest.fixture(scope="module")
def driver(tmp_path_factory):
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no C++ compiler")
    d = tmp_path_factory.mktemp("policy")
    src = d / "driver.cpp"
    src.write_text(DRIVER)
    exe = d / "driver"
    subprocess.run([cxx, "-std=c++17", "-O1", "-I", build.CSRC, str(src), "-o", str(exe)], check=True,
                   capture_output=True)
    return str(exe)


def form(driver, slot, reqs, lane_on=False, now=1.0, steal=0.005, cap=0):
    """slot = (V_cap, T_cap, H_cap, n_cap, lane); reqs = [(V, T, H, small, t_submit)]."""
    head = " ".join(str(x) for x in (*slot[:4], int(slot[4]), int(lane_on), now, steal, cap, len(reqs)))
    body = "\n".join(" ".join(str(x) for x in (V, T, H, int(sm), t)) for V, T, H, sm, t in reqs)
    out = subprocess.run([driver], input=head + "\n" + body + "\n", capture_output=True, text=True, check=True).stdout
    res = {}
    for line in out.splitlines():
        k, *ids = line.split()
        res[k] = [int(i) for i in ids]
    return res


def req(T, small=False, t=0.99):
    return (T // 2 + 2, T, 3 * T + 8, small, t)


CE = (1_000_000, 1_000_000, 3_100_000, 4096, False)     # a copy-engine slot
LANE = (200_000, 200_000, 700_000, 4096, True)          # the lane slot


def test_fifo_until_the_first_request_that_does_not_fit(driver):
    r = form(driver, CE, [req(400_000), req(500_000), req(200_000), req(50_000)])
    # 400k + 500k fit; 200k would overflow: the batch stops there (no overtaking)
    assert r == {"take": [0, 1], "fail": [], "left": [2, 3]}


def test_mesh_count_limit(driver):
    slot = (1_000_000, 1_000_000, 3_100_000, 3, False)
    r = form(driver, slot, [req(10)] * 5)
    assert r["take"] == [0, 1, 2] and r["left"] == [3, 4]


def test_batch_triangle_cap_still_runs_one_larger_request(driver):
    r = form(driver, CE, [req(300_000), req(100_000)], cap=200_000)
    assert r["take"] == [0] and r["left"] == [1]
    r = form(driver, CE, [req(100_000), req(90_000), req(20_000)], cap=200_000)
    assert r["take"] == [0, 1] and r["left"] == [2]


def test_too_large_fails_unless_the_lane_can_take_it(driver):
    r = form(driver, CE, [req(2_000_000), req(10_000)])
    assert r == {"take": [1], "fail": [0], "left": []}
    small_ce = (100_000, 100_000, 310_000, 4096, False)    # tiny budget: a lane request larger than this slot
    r = form(driver, small_ce, [req(150_000, small=True, t=0.0)], lane_on=True)
    assert r == {"take": [], "fail": [], "left": [0]}


def test_lane_takes_lane_requests_only_in_order(driver):
    reqs = [req(5_000_000), req(20_000, True), req(3_000_000), req(30_000, True), req(10_000, True)]
    r = form(driver, LANE, reqs, lane_on=True)
    assert r == {"take": [1, 3, 4], "fail": [], "left": [0, 2]}


def test_copy_engine_slots_leave_lane_requests_for_a_while(driver):
    young, old = 0.999, 0.9           # submitted 1 ms and 100 ms before now = 1.0
    reqs = [req(20_000, True, young), req(400_000), req(20_000, True, old), req(30_000, True, young)]
    r = form(driver, CE, reqs, lane_on=True)
    assert r == {"take": [1, 2], "fail": [], "left": [0, 3]}


def test_without_lane_every_request_is_fifo(driver):
    reqs = [req(20_000), req(400_000), req(20_000)]
    r = form(driver, CE, reqs, lane_on=False)
    assert r["take"] == [0, 1, 2]


def test_policy_header_is_what_the_server_includes():
    src = open(os.path.join(build.CSRC, "polylla_server.cu")).read()
    assert '#include "serve_policy.h"' in src and "policy::form_batch(" in src
    assert os.path.join(build.CSRC, "serve_policy.h") in build.HEADERS
