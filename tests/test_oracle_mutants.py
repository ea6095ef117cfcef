"""The oracle pins are strong enough to catch plausible mistakes.

Each case compiles a copy of the oracle source with one planted mistake
(on the CPU, into a temporary directory) and checks that at least one pin
of ``test_oracle_pins`` fails on it.  The mistakes are the kind a reader of
the paper could make: a dropped term, a reversed rotation, an off-by-one
rotation count, the frontier condition as printed in Algorithm 3, a wrong
tie-break, a missing seed rule, output not started at the polygon minimum,
for the Lepp, the wrong half of a terminal edge or a path that stops
before the terminal edge's second triangle, and, for the convexification,
a flipped turn test, swapped cross-product operands, the nearest instead
of the farthest chord, and a chord with only one half on the frontier.
"""
import os
import shutil
import subprocess

import pytest

import oracle
from paper_2403_14723_gb300 import meshgen
from tests import test_oracle_convex as convex_pins
from tests import test_oracle_lepp as lepp_pins
from tests import test_oracle_pins as pins

SRC = os.path.join(os.path.dirname(oracle.__file__), "polylla_oracle.c")

MUTANTS = {
    "drop_dy_term": ("    return dx2 + dy2;", "    return dx2;"),
    "cw_is_ccw": ("static int32_t q_cw(const mesh_t *m, int32_t e) { return m->next[m->twin[e]]; }",
                  "static int32_t q_cw(const mesh_t *m, int32_t e) { return m->twin[m->prev[e]]; }"),
    "target_is_origin": ("static int32_t q_target(const mesh_t *m, int32_t e) { return m->origin[m->twin[e]]; }",
                         "static int32_t q_target(const mesh_t *m, int32_t e) { return m->origin[e]; }"),
    "tie_break_larger_id": ("(d == dbest && edge_id(m, cand[k]) < edge_id(m, best))",
                            "(d == dbest && edge_id(m, cand[k]) > edge_id(m, best))"),
    "frontier_as_printed": ("(!longest[e] && !longest[m->twin[e]])",
                            "(longest[e] || longest[m->twin[e]])"),
    "middle_edge_exclusive_loop": ("for (int32_t r = 0; r <= (d - 1) / 2; r++)",
                                   "for (int32_t r = 0; r < (d - 1) / 2; r++)"),
    "no_border_terminal_seeds": ("else if (border_terminal && e < HI) seed_list[n_seeds++] = e;",
                                 "else if (0) seed_list[n_seeds++] = e;"),
    "repair_skipped": ("            frontier1[e] = 1;\n            frontier1[tw] = 1;",
                       "            (void)tw;"),
    "output_from_next": ("        int32_t cur = e;\n        int64_t len = 0;",
                         "        int32_t cur = next_out[e];\n        int64_t len = 0;"),
    "lepp_terminal_larger_half": ("                terminal[t0] = e < tw ? e : tw;",
                                  "                terminal[t0] = e < tw ? tw : e;"),
    "lepp_border_half": ("                terminal[t0] = e;\n                break;",
                         "                terminal[t0] = tw;\n                break;"),
    "lepp_path_stops_before_terminal": ("        path[n++] = tw / 3;\n        if (longest[tw]) return n;",
                                        "        if (longest[tw]) return n;\n        path[n++] = tw / 3;"),
    # convexification (reading R9)
    "convex_reflex_sign_flipped": ("        if (!(cross2(ux, uy, wx, wy) > 0.0)) continue;",
                                   "        if (!(cross2(ux, uy, wx, wy) < 0.0)) continue;"),
    "convex_nearest_candidate": ("                    best = i;\n                    i++;\n                } else {",
                                 "                    best = i;\n                    i++;\n                    break;\n"
                                 "                } else {"),
    "convex_one_chord_half": ("            frontier2[twin[c]] = 1;\n", ""),
    "convex_cross_operands_swapped": ("    const double p = ax * by;\n    const double q = ay * bx;",
                                      "    const double p = ay * bx;\n    const double q = ax * by;"),
}


def _tip_mesh():
    for s in range(40):
        m = meshgen.random_delaunay(80, seed=1000 + s)
        if oracle.run_mesh(m).stats["tips"]:
            return m
    raise AssertionError("no mesh with a barrier tip found")


def _pins_hold(lib) -> bool:
    lat = None
    for s in range(3):
        try:
            lat = meshgen.lattice_delaunay(120, 14, seed=200 + s)
            break
        except ValueError:
            continue
    cases = [
        lambda: pins.pin_two_triangle_square(lib),
        lambda: pins.pin_exact_grid(5, lib),
        lambda: pins.pin_labels(meshgen.random_delaunay(130, seed=101), lib),
        lambda: pins.pin_labels(lat, lib),
        lambda: pins.pin_tips(_tip_mesh(), lib),
        lambda: pins.pin_invariants(meshgen.random_delaunay(500, seed=300), lib),
        lambda: pins.pin_relabelling(7, lib),
        lambda: lepp_pins.pin_lepp_terminal(meshgen.random_delaunay(130, seed=301), lib),
        lambda: lepp_pins.pin_lepp_recursion(meshgen.random_delaunay(200, seed=302), lib),
        lambda: lepp_pins.pin_lepp_grid(5, lib),
        lambda: convex_pins.pin_convex(meshgen.random_delaunay(300, seed=401), lib),
        lambda: convex_pins.pin_convex(meshgen.perturbed_grid(24, 0.3, seed=401), lib),
        lambda: convex_pins.pin_fixed_point(meshgen.random_delaunay(500, seed=430), lib),
    ]
    for c in cases:
        try:
            c()
        except (AssertionError, RuntimeError, IndexError, ValueError):
            return False
    return True


def test_unmutated_copy_passes(tmp_path):
    so = tmp_path / "liboracle_copy.so"
    subprocess.run(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fPIC", "-shared",
                    "-o", str(so), SRC], check=True)
    assert _pins_hold(oracle.load_variant(str(so)))


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_planted_mistake_is_caught(name, tmp_path):
    if shutil.which("gcc") is None:
        pytest.skip("gcc not available")
    old, new = MUTANTS[name]
    src = open(SRC).read()
    assert src.count(old) == 1, f"mutation site for {name} not found exactly once"
    mut = tmp_path / f"{name}.c"
    mut.write_text(src.replace(old, new))
    so = tmp_path / f"lib{name}.so"
    subprocess.run(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fPIC", "-shared",
                    "-o", str(so), str(mut)], check=True)
    assert not _pins_hold(oracle.load_variant(str(so))), f"pins did not catch mutant {name}"
