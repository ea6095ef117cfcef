"""The serving loop's memory admission, on the CPU: how a device-memory
budget is split into the low-latency lane and the copy-engine slots
(``polylla_server_plan_slots`` is host arithmetic, the same the server's
create uses)."""
import pytest

from paper_2403_14723_gb300 import build, polylla

GiB = 1 << 30


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.build_library()


@pytest.mark.parametrize("budget", [64 << 20, 1 * GiB, 3 * GiB, 40 * GiB, 200 * GiB])
@pytest.mark.parametrize("n_slots", [1, 3, 8, 16])
@pytest.mark.parametrize("lane", [-1, 0, 4000])
def test_slots_fit_the_budget(budget, n_slots, lane):
    p = polylla.server_plan(budget, n_slots=n_slots, lane_triangles=lane)
    assert 0 < p["device_bytes"] <= budget
    assert p["slot_triangles"] >= 1
    # the budget is used, not left idle (under 0.1 % spare), unless a slot
    # reached the 500 M-triangle cap that keeps its half-edge indices in int32
    if p["slot_triangles"] < 500_000_000:
        assert budget - p["device_bytes"] < max(budget // 1000, 1 << 20)
    else:
        assert n_slots == 1 and budget > 100 * GiB
    if lane < 0:
        assert p["n_slots"] == n_slots and p["lane_triangles"] == 0 and p["lane_slot_triangles"] == 0
    else:
        want = lane or 65536
        assert p["n_slots"] == n_slots + 1
        assert 0 < p["lane_triangles"] <= want and p["lane_triangles"] <= p["lane_slot_triangles"]
        assert p["lane_slot_triangles"] <= 16 * want
        if p["lane_triangles"] < want:          # only a small budget cuts the lane's requests
            assert p["lane_slot_triangles"] == p["lane_triangles"]


def test_lane_is_small_beside_large_budgets():
    with_lane = polylla.server_plan(40 * GiB, n_slots=3)
    no_lane = polylla.server_plan(40 * GiB, n_slots=3, lane_triangles=-1)
    assert with_lane["lane_slot_triangles"] == 16 * 65536
    # the lane costs the copy-engine slots about 1 % of their capacity
    assert 0.98 * no_lane["slot_triangles"] < with_lane["slot_triangles"] < no_lane["slot_triangles"]
    # about 200-400 device bytes per triangle of slot capacity (arena, union, scratch, outputs)
    per_tri = no_lane["device_bytes"] / (3 * no_lane["slot_triangles"])
    assert 150 < per_tri < 400


def test_capacity_grows_with_budget_and_shrinks_with_slots():
    caps = [polylla.server_plan(b * GiB, n_slots=3)["slot_triangles"] for b in (1, 2, 4, 8, 16)]
    assert caps == sorted(caps) and caps[-1] > 15 * caps[0]
    per_slot = [polylla.server_plan(16 * GiB, n_slots=n)["slot_triangles"] for n in (1, 2, 4, 8, 16)]
    assert per_slot == sorted(per_slot, reverse=True)


def test_bad_options_are_rejected():
    for kw in ({"memory_budget": 0}, {"memory_budget": 1000}, {"memory_budget": GiB, "n_slots": 17},
               {"memory_budget": GiB, "n_slots": -1}, {"memory_budget": GiB, "max_batch_meshes": -2}):
        with pytest.raises(RuntimeError):
            polylla.server_plan(**kw)
