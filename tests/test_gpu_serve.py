"""The serving loop through the C ABI: requests batched continuously must
each get exactly the oracle's result for their mesh alone (bit-exact), the
same whether a request ran alone or in a mix, and a request too large for a
slot must fail cleanly."""
import numpy as np
import pytest

import oracle
from paper_2403_14723_gb300 import build, meshgen, polylla

pytestmark = pytest.mark.gpu


def _meshes():
    ms = [meshgen.two_triangle_square(), meshgen.exact_grid(6), meshgen.perturbed_grid(40, 0.3, seed=21)]
    for s in range(60):                        # meshes with barrier tips
        m = meshgen.random_delaunay(150, seed=7000 + s)
        if oracle.run_mesh(m).stats["tips"] >= 1:
            ms.append(m)
        if len(ms) >= 6:
            break
    ms += meshgen.random_batch(24, t_min=1000, t_max=50_000, seed=50)
    ms.append(meshgen.perturbed_grid(400, 0.3, seed=22))      # ~318k triangles
    return ms


def _check(mesh, info, res, r, tag):
    assert info["status"] == 0, tag
    assert info["n_polygons"] == r.n_polygons and info["n_frontier"] == r.he_list.shape[0], tag
    for k, want in (("seeds", r.seeds), ("offsets", r.offsets), ("he_list", r.he_list), ("v_list", r.v_list),
                    ("next", r.next_out), ("prev", r.prev_out)):
        assert np.array_equal(res[k], want), f"{tag}: {k} differs"


def test_served_requests_match_oracle_alone_and_in_the_mix():
    build.build_library()
    meshes = _meshes()
    oracle_res = [oracle.run_mesh(m) for m in meshes]
    with polylla.Server(memory_budget=3 << 30, n_slots=3, max_batch_meshes=16) as srv:
        # alone: one request at a time
        alone = []
        for i in (0, 4, len(meshes) - 1):
            hr = polylla.HostRequest(meshes[i])
            info = srv.wait(srv.submit(hr))
            assert info["batch_meshes"] == 1
            alone.append((i, hr.result(info)))
            _check(meshes[i], info, alone[-1][1], oracle_res[i], f"alone {meshes[i].name}")
        # in the mix: everything at once, so batches form and overlap
        reqs = [polylla.HostRequest(m) for m in meshes]
        tickets = [srv.submit(r) for r in reqs]
        infos = [srv.wait(t) for t in tickets]
        assert max(i["batch_meshes"] for i in infos) > 1, "no request was batched with another"
        for m, hr, info, r in zip(meshes, reqs, infos, oracle_res):
            _check(m, info, hr.result(info), r, f"mix {m.name}")
        for i, res in alone:
            mixed = reqs[i].result(infos[i])
            for k in res:
                assert np.array_equal(res[k], mixed[k]), f"{meshes[i].name}: {k} differs alone vs in the mix"
        st = srv.stats()
        assert st["requests_done"] == len(meshes) + 3 and st["batches"] >= 4
        assert st["device_bytes"] <= 3 << 30
        log = srv.batch_log()
        assert len(log) == st["batches"]
        assert sum(b["n_requests"] for b in log) == len(meshes) + 3
        assert sum(b["n_triangles"] for b in log) == sum(m.n_triangles for m in meshes) + \
            sum(meshes[i].n_triangles for i in (0, 4, len(meshes) - 1))
        for b in log:
            assert b["t_form"] <= b["t_enqueued"] <= b["t_meta_seen"] <= b["t_out_enqueued"] <= b["t_done"]
            assert min(b["in_ms"], b["run_ms"], b["idle_ms"], b["out_ms"]) >= 0 and 0 <= b["slot"] < st["n_slots"]
        assert srv.batch_log(2) == log[-2:]
        # small pinned requests ran in the lane (kernel copies), the large one outside it
        assert st["lane_triangles"] == 65536 and st["lane_batches"] >= 1
        assert st["n_slots"] == 4 and st["lane_slot_triangles"] >= 65536    # three copy-engine slots and the lane
        plan = polylla.server_plan(3 << 30, n_slots=3, max_batch_meshes=16)   # the same options, no GPU
        for k in ("n_slots", "slot_triangles", "lane_triangles", "lane_slot_triangles"):
            assert st[k] == plan[k], k
        assert any(b["lane"] == 1 for b in log) and any(b["lane"] == 0 for b in log)
        assert st["launches"] == 12 * st["lane_batches"] + 11 * (st["batches"] - st["lane_batches"])


def test_copy_paths_give_identical_results():
    """The same requests through the lane (kernel copies through host-mapped
    memory), through the copy engines (pageable buffers, or no lane), alone
    and mixed: every result is the oracle's, bit for bit."""
    build.build_library()
    meshes = [meshgen.exact_grid(7), meshgen.perturbed_grid(60, 0.3, seed=31)]
    meshes += meshgen.random_batch(10, t_min=500, t_max=60_000, seed=52)
    want = [oracle.run_mesh(m) for m in meshes]
    for lane, pinned in ((0, True), (0, False), (-1, True), (4000, True)):
        with polylla.Server(memory_budget=1 << 30, n_slots=3, lane_triangles=lane) as srv:
            reqs = [polylla.HostRequest(m, pinned=pinned) for m in meshes]
            infos = [srv.wait(t) for t in [srv.submit(r) for r in reqs]]
            st = srv.stats()
            log = srv.batch_log()
        tag = f"lane={lane} pinned={pinned}"
        for m, hr, info, r in zip(meshes, reqs, infos, want):
            _check(m, info, hr.result(info), r, f"{tag} {m.name}")
        n_lane = sum(b["n_requests"] for b in log if b["lane"])
        assert st["n_slots"] == (3 if lane < 0 else 4), tag
        if lane < 0 or not pinned:
            assert n_lane == 0 and st["lane_batches"] == 0, tag          # no lane, or nothing it may take
        else:
            limit = lane or 65536
            small = sum(m.n_triangles <= limit for m in meshes)
            assert 0 < n_lane <= small, tag                               # lane requests only (some may be taken by others)
            assert all(b["n_triangles"] <= limit * b["n_requests"] for b in log if b["lane"]), tag


def test_replay_poisson_trace():
    build.build_library()
    pool = meshgen.random_batch(16, t_min=1000, t_max=50_000, seed=51)
    hrs = [polylla.HostRequest(m) for m in pool]
    rng = np.random.default_rng(5)
    n = 400
    arrival = np.cumsum(rng.exponential(1 / 2000.0, size=n))
    pick = rng.integers(0, len(pool), size=n)
    with polylla.Server(memory_budget=2 << 30, n_slots=3) as srv:
        rc, lat, infos = srv.replay([hrs[i] for i in pick], arrival)
    assert rc == 0
    assert np.all(lat > 0) and np.all(np.isfinite(lat))
    r0 = oracle.run_mesh(pool[int(pick[-1])])
    assert infos[-1]["n_polygons"] == r0.n_polygons


def test_request_larger_than_a_slot_fails_cleanly():
    build.build_library()
    with polylla.Server(memory_budget=64 << 20, n_slots=2, max_batch_meshes=4) as srv:
        cap = srv.stats()["slot_triangles"]
        big = meshgen.perturbed_grid(int(np.sqrt(cap)) + 10, 0.3, seed=2)
        assert big.n_triangles > cap
        info = srv.wait(srv.submit(polylla.HostRequest(big)))
        assert info["status"] == -8
        small = meshgen.exact_grid(5)
        hr = polylla.HostRequest(small)
        info = srv.wait(srv.submit(hr))
        _check(small, info, hr.result(info), oracle.run_mesh(small), "after a rejected request")


def test_served_recipe_pool_matches_oracle():
    """The served workload's request pool (512 small + 32 large meshes, up
    to 8M triangles) through one second of its Poisson trace in the server
    configuration bench.py times: every pool mesh a request used gets the
    oracle's result."""
    import bench

    build.build_library()
    small, large = bench.serve_pool()
    pool = small + large
    hrs = [polylla.HostRequest(m) for m in pool]
    t, pick = bench.serve_trace(1.0, len(small), len(large), seed=11)
    with polylla.Server(memory_budget=bench.SERVE_RECIPE["budget"], n_slots=3) as srv:
        rc, lat, infos = srv.replay([hrs[i] for i in pick], t)
    assert rc == 0 and np.all(lat > 0)
    last = {}
    for k, i in enumerate(pick):
        last[int(i)] = infos[k]
    assert any(i >= len(small) for i in last), "no large request in the trace"
    for i, info in sorted(last.items()):
        _check(pool[i], info, hrs[i].result(info), oracle.run_mesh(pool[i]), f"pool mesh {i} ({pool[i].name})")


def test_malformed_request_fails_cleanly():
    """Indices outside a request's own mesh are caught by the longest-edge
    kernel's range checks, kept inside the mesh (no access leaves it) and
    reported as an invalid mesh; the server keeps serving."""
    build.build_library()
    good = meshgen.random_delaunay(300, seed=12)
    bad = meshgen.random_delaunay(300, seed=13)
    bad.twin = bad.twin.copy()
    bad.origin = bad.origin.copy()
    bad.twin[7] = 10 ** 9            # far outside the mesh
    bad.origin[11] = -5
    with polylla.Server(memory_budget=1 << 30, n_slots=2) as srv:
        info = srv.wait(srv.submit(polylla.HostRequest(bad)))
        assert info["status"] == -2
        hr = polylla.HostRequest(good)
        info = srv.wait(srv.submit(hr))
        _check(good, info, hr.result(info), oracle.run_mesh(good), "after a malformed request")
