"""Property-based pins of the oracle on random small triangulations
(hypothesis): the output invariants the method guarantees (each frontier
half-edge used once, next/prev inverse, no barrier tip left, polygon count
= seeds + chords, Euler characteristic, areas summing to the domain, every
triangle in one polygon) and the Lepp recursion hold for Delaunay meshes of
random point sets and for perturbed grids of random sizes and seeds."""
import numpy as np
import pytest

import oracle
from paper_2403_14723_gb300 import meshgen
from tests import checks
from tests import test_oracle_lepp as lepp_pins

hypothesis = pytest.importorskip("hypothesis")
from hypothesis import given, settings, strategies as st  # noqa: E402


def _invariants(mesh):
    r = oracle.run_mesh(mesh)
    checks.check_output_invariants(
        mesh, r.frontier1, r.next_out, r.prev_out, r.seeds, r.offsets, r.he_list, r.v_list,
        n_seeds_alg4=len(r.seed_list), n_distinct_chords=r.stats["distinct_chords"])
    checks.check_triangle_coverage(mesh, r.frontier1, r.he_list, r.offsets)
    lepp_pins.pin_lepp_recursion(mesh)


@settings(max_examples=40, deadline=None)
@given(n=st.integers(min_value=3, max_value=120), seed=st.integers(min_value=0, max_value=2 ** 31 - 1))
def test_random_delaunay_invariants(n, seed):
    _invariants(meshgen.random_delaunay(n, seed=seed))


@settings(max_examples=25, deadline=None)
@given(s=st.integers(min_value=2, max_value=30), seed=st.integers(min_value=0, max_value=2 ** 31 - 1),
       jitter=st.sampled_from([0.0, 0.1, 0.3, 0.45]))
def test_random_perturbed_grid_invariants(s, seed, jitter):
    _invariants(meshgen.perturbed_grid(s, jitter, seed=seed))
