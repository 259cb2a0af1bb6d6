"""The oracle on the paper's own convergence problem (Sec. 4, Table 1):
rho = 1 - 0.9999 sin 2 pi x sin 2 pi y, u = (1, 0), p = 1, t = 0.02,
CFL 0.08, all limiters on, P2 on n x n periodic squares.

Facts that pin it, none taken from the oracle itself:

* Design order: the L2 error of the density falls as h^3 (the paper's order
  column: 2.99, 3.05, 2.97 on its finer grids).
* Near-best approximation: no P2 state is closer to the exact density in L2
  than the L2 projection of the exact solution (the "floor"); the oracle's
  error stays within 35 % of that floor on every grid checked.
* The printed errors are 3.5 to 4 times BELOW that floor on every grid, so
  they cannot be the plain L2 norm over the square: whatever norm the paper
  used, only the order and the ratio to the best approximation are
  comparable (recorded with the reading of Eq. LLF in the design notes).
* The literal reading of Eq. LLF (global s in the point flux's dissipation)
  loses an order on this problem, which the paper's table rules out.

The live runs take 42^2, 63^2 and 94^2 (about a minute on 8 cores); the
finer grids up to 212^2 are in ``golden/table1_oracle.txt``, written by
``golden/table1_oracle.py`` from the oracle, and one of its rows is checked
against a live run so that the file stays the current oracle's.
"""
import importlib.util
import os

import numpy as np
import pytest

HERE = os.path.dirname(os.path.abspath(__file__))


def _runner():
    spec = importlib.util.spec_from_file_location("table1_oracle", os.path.join(HERE, "golden", "table1_oracle.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def _printed():
    rows = [l.split() for l in open(os.path.join(HERE, "golden", "table1.txt")) if l.strip() and not l.startswith("#")]
    return {int(round(np.sqrt(float(r[1])))): float(r[2]) for r in rows if r[0] == "cart"}


def _order(a, b):
    return np.log(a["l2"] / b["l2"]) / np.log(b["n"] / a["n"])


@pytest.fixture(scope="module")
def local_runs(orc):
    t1 = _runner()
    return [t1.run(n) for n in (42, 63, 94)]


def test_table1_problem_third_order(local_runs):
    r = local_runs
    for a, b in zip(r[:-1], r[1:]):
        assert _order(a, b) >= 2.8, (a["n"], b["n"], _order(a, b))
    for x in r:
        assert x["n_mom"] == 0 and x["n_edge"] == 0      # the limiters turn off on these grids


def test_table1_problem_near_best_approximation(local_runs):
    printed = _printed()
    for x in local_runs:
        assert x["floor"] <= x["l2"] <= 1.35 * x["floor"], x
        # the printed error lies below the best P2 approximation by a fixed factor
        assert 3.5 < x["floor"] / printed[x["n"]] < 4.0, (x["n"], x["floor"], printed[x["n"]])


def test_table1_problem_literal_global_speed_loses_an_order(orc):
    t1 = _runner()
    a, b = t1.run(42, llf_global=True), t1.run(63, llf_global=True)
    assert _order(a, b) < 2.4
    assert b["l2"] > 5.0 * b["floor"]


def test_stored_fine_grid_table_is_the_current_oracle(orc):
    """The stored table (28^2 .. 212^2, both readings) comes from the oracle
    as it is: one of its rows equals a live run; its finer grids keep the
    third order (94^2 -> 141^2 -> 212^2) and the near-best ratio."""
    path = os.path.join(HERE, "golden", "table1_oracle.txt")
    rows = [l.split() for l in open(path) if l.strip() and not l.startswith("#")]
    tab = {(r[0], int(r[1])): {"n": int(r[1]), "l2": float(r[3]), "floor": float(r[4])} for r in rows}
    live = _runner().run(42)
    assert abs(tab[("local", 42)]["l2"] - live["l2"]) <= 1e-6 * live["l2"]
    fine = [tab[("local", n)] for n in (94, 141, 212)]
    for a, b in zip(fine[:-1], fine[1:]):
        assert _order(a, b) >= 2.8
    for x in fine:
        assert x["l2"] <= 1.35 * x["floor"]
