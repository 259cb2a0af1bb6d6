"""Pins of the oracle's flux limiter (Sec. 3.3 Steps 4-5) on its values,
not only on positivity.

* Hand-worked cells, one for each case of Step 4 (no, one, two, all edges
  with a negative density flux difference), the "enough mass" case, a
  quadrilateral, and a pressure case whose box corners are worked out by
  hand: the proposals must equal the numbers derived on paper.
* Tightness on random cells: where the density Lambda lies strictly in
  (0, 1), the corner of the final box with every negative edge at its
  proposal lands on the density floor; where some mu_c < 1, the lowest-
  pressure corner of the final box lands on the pressure floor.  An
  over-limiting variant (a Lambda smaller than needed) misses the floor.
* Each pin is shown to bite: over-limiting variants of the oracle, built
  here on the CPU from its source with one line changed, fail them.
"""
import ctypes as C
import os
import subprocess
import tempfile

import numpy as np
import pytest

import synth

G = 1.4
HERE = os.path.dirname(os.path.abspath(__file__))
ORACLE_SRC = os.path.join(os.path.dirname(HERE), "oracle", "lxw_oracle.c")


def pressure(q):
    q = np.asarray(q, dtype=np.float64)
    return (G - 1) * (q[..., 3] - 0.5 * (q[..., 1] ** 2 + q[..., 2] ** 2) / q[..., 0])


def _cell(rho, e):
    """Per-edge flux rows (rho, m, n, E) with only density and energy set."""
    f = np.zeros((len(rho), 4))
    f[:, 0] = rho
    f[:, 3] = e
    return f


def hand_cases():
    """(name, E, area, dt, qbar, fW, fF, expected proposals, eps0).

    Density cases: qbar = (1, 0, 0, 10), area = dt = 1, f^LxF of density 0.2
    per edge, so Gamma^rho = 1 - 0.6 = 0.4, rho^LxF = 0.4 and the floor is
    eps = min(1e-12, 0.2) = 1e-12.  The energy is large and no energy flux
    moves, so the pressure never binds (mu = 1).  Every negative edge gets
    the largest common Lambda with rho >= eps at the corner that takes all of
    them: rho^LxF - Lambda |sum of negatives| = eps."""
    q = np.array([1.0, 0.0, 0.0, 10.0])
    ff3 = _cell([0.2, 0.2, 0.2], [0, 0, 0])
    L2 = (0.4 - 1e-12) / 0.8
    cases = [
        ("no negative edge", 3, 1.0, 1.0, q, _cell([0.1, 0.2, 0.0], [0, 0, 0]), ff3, [1.0, 1.0, 1.0], 1e-12),
        ("one negative edge", 3, 1.0, 1.0, q, _cell([1.0, 0.2, 0.1], [0, 0, 0]), ff3, [L2, 1.0, 1.0], 1e-12),
        ("two negative edges", 3, 1.0, 1.0, q, _cell([0.5, 0.7, 0.1], [0, 0, 0]), ff3, [L2, L2, 1.0], 1e-12),
        ("three negative edges", 3, 1.0, 1.0, q, _cell([0.3, 0.4, 0.5], [0, 0, 0]), ff3,
         [(0.4 - 1e-12) / 0.6] * 3, 1e-12),
        ("enough mass", 3, 1.0, 1.0, q, _cell([0.25, 0.2, 0.2], [0, 0, 0]), ff3, [1.0, 1.0, 1.0], 1e-12),
        # quadrilateral: Gamma^rho = 1 - 0.4 = 0.6, negatives -0.4 and -0.3
        ("quadrilateral", 4, 1.0, 1.0, q, _cell([0.5, 0.1, 0.4, 0.0], [0, 0, 0, 0]),
         _cell([0.1] * 4, [0] * 4), [(0.6 - 1e-12) / 0.7, 1.0, (0.6 - 1e-12) / 0.7, 1.0], 1e-12),
    ]
    # Pressure case: qbar = (1, 0, 0, 1), f^LxF = 0, density fluxes equal
    # (Lambda = 1), energy outflows 0.6, 0.6 and inflow 0.5.  With rho = 1
    # and no momentum p = 0.4 E; the corners' energies are 1 - (0.6, 0.6,
    # -0.5 over the edges they take): {0} 0.4, {1} 0.4, {2} 1.5, {0,1} -0.2,
    # {0,2} 0.9, {1,2} 0.9, {0,1,2} 0.3.  Only {0,1} falls below the floor
    # eps_p = min(1e-12, 0.4/2); its mu solves 0.4 (1 - 1.2 mu) = 1e-12.
    # Edges 0 and 1 take that mu; edge 2 lies in no failing corner.
    mu = (1.0 - 1e-12 / 0.4) / 1.2
    cases.append(("pressure corner", 3, 1.0, 1.0, np.array([1.0, 0.0, 0.0, 1.0]),
                  _cell([0, 0, 0], [0.6, 0.6, -0.5]), _cell([0, 0, 0], [0, 0, 0]), [mu, mu, 1.0], 1e-12))
    return cases


def random_cells(E, count, seed, which):
    """Random cells in the style of the brute-force positivity test.
    which = "density": the two fluxes differ only in density and the energy
    is raised by 1e4, so only the density limits (the proposals are Lambda);
    which = "pressure": the two fluxes have the same density component
    (Lambda = 1), so only the pressure limits (the proposals are the min of
    mu over the corners holding the edge)."""
    rng = np.random.default_rng(seed)
    out = []
    for trial in range(count):
        qbar = synth.random_modal_state(1, 1, seed=seed * 1000 + trial, rho_range=(0.01, 2.0),
                                        p_range=(1e-3, 2.0))[0, :, 0]
        T, dt = rng.uniform(0.5, 2.0), rng.uniform(0.05, 0.3)
        qlxf = synth.random_modal_state(1, 1, seed=seed * 7000 + trial, rho_range=(1e-4, 1.0),
                                        p_range=(1e-5, 1.0))[0, :, 0]
        if which == "density":
            qbar = qbar.copy(); qbar[3] += 1e4; qlxf = qlxf.copy(); qlxf[3] += 1e4
        fF = rng.normal(size=(E, 4))
        fF += ((qbar - qlxf) * T / dt - fF.sum(0)) / E
        fW = fF + rng.normal(size=(E, 4)) * np.abs(qbar) * T / dt * rng.uniform(0.05, 1.0)
        if which == "density":
            fW[:, 1:] = fF[:, 1:]
        else:
            fW[:, 0] = fF[:, 0]
        out.append((T, dt, qbar, fW, fF))
    return out


def box_corner(qbar, T, dt, fW, fF, alpha):
    """q^n+1 for theta_k = alpha_k on each edge (Sec. 3.3 Step 6)."""
    return qbar - dt / T * (alpha @ fW + (1.0 - alpha) @ fF)


def pin_failures(flc, eps0=1e-3):
    """Runs every pin against a flux-limiter implementation
    flc(gamma, eps0, area, dt, qbar, fW, fF) -> (proposals, cfl_bad) and
    returns the pins it fails (an empty list for a correct one)."""
    fails = []
    for name, E, T, dt, qbar, fW, fF, want, e0 in hand_cases():
        prop, bad = flc(G, e0, T, dt, qbar, fW, fF)
        if bad or not np.allclose(prop, want, rtol=1e-13, atol=1e-15):
            fails.append("hand: %s: %s != %s" % (name, list(prop), want))
    # density: where Lambda is in (0, 1), the corner taking every negative
    # edge at its proposal has exactly the floor density min(eps0, rho^LxF/2)
    hits = 0
    for E in (3, 4):
        for (T, dt, qbar, fW, fF) in random_cells(E, 150, 11 + E, "density"):
            prop, bad = flc(G, eps0, T, dt, qbar, fW, fF)
            neg = (fF[:, 0] - fW[:, 0]) < 0
            if bad or not neg.any() or not (0.0 < prop[neg].max() < 1.0):
                continue
            hits += 1
            rho_lxf = box_corner(qbar, T, dt, fW, fF, np.zeros(E))[0]
            floor = min(eps0, 0.5 * rho_lxf)
            rho_c = box_corner(qbar, T, dt, fW, fF, np.where(neg, prop, 0.0))[0]
            if abs(rho_c - floor) > 1e-12 * (abs(qbar[0]) + dt / T * np.abs(fW[:, 0]).sum()):
                fails.append("density tightness: corner rho %.6e, floor %.6e" % (rho_c, floor))
                break
    if hits < 50:
        fails.append("density tightness: only %d limited cells" % hits)
    # pressure: every corner of the final box keeps p >= the floor
    # min(eps0, p^LxF/2), and where an edge was cut below 1 the lowest corner
    # sits on the floor (the corner with the smallest mu keeps its mu on all
    # its edges, so it is the segment point that solves for the floor)
    hits = 0
    for E in (3, 4):
        corners = np.array([[(c >> k) & 1 for k in range(E)] for c in range(1 << E)], dtype=float)
        for (T, dt, qbar, fW, fF) in random_cells(E, 300, 41 + E, "pressure"):
            q_lxf = box_corner(qbar, T, dt, fW, fF, np.zeros(E))
            if not (q_lxf[0] > 0 and pressure(q_lxf) > 0):
                continue
            prop, bad = flc(G, eps0, T, dt, qbar, fW, fF)
            floor = min(eps0, 0.5 * pressure(q_lxf))
            qc = np.array([box_corner(qbar, T, dt, fW, fF, c * prop) for c in corners])
            pmin = pressure(qc).min()
            tol = 1e-11 * (abs(qbar[3]) + dt / T * np.abs(fW[:, 3]).sum())
            if pmin < floor - tol:
                fails.append("pressure positivity: lowest corner p %.6e below floor %.6e" % (pmin, floor))
                break
            if prop.min() < 1.0:
                if prop.min() == 0.0:
                    continue
                hits += 1
                if abs(pmin - floor) > tol:
                    fails.append("pressure tightness: lowest corner p %.6e, floor %.6e" % (pmin, floor))
                    break
    if hits < 30:
        fails.append("pressure tightness: only %d limited cells" % hits)
    return fails


def test_flux_limiter_hand_cases_and_tightness(orc):
    fails = pin_failures(orc.flux_limit_cell)
    assert fails == [], fails


MUTANTS = {
    # Lambda = 0 on every edge with a negative density difference
    "lambda_zero": ("Lam[k] = df[k] < 0.0 ? lneg : 1.0;", "Lam[k] = df[k] < 0.0 ? 0.0 : 1.0;"),
    # half the largest admissible Lambda
    "lambda_half": ("Lam[k] = df[k] < 0.0 ? lneg : 1.0;", "Lam[k] = df[k] < 0.0 ? 0.5 * lneg : 1.0;"),
    # min of mu over every corner, not only the corners holding the edge
    "mu_all_corners": ("if ((c >> k) & 1 && mu < mmin[k]) mmin[k] = mu;", "if (mu < mmin[k]) mmin[k] = mu;"),
    # the pressure step over the single-edge corners only
    "mu_singletons": ("for (int c = 1; c < (1 << E); ++c) {\n    double qc[4];",
                      "for (int c = 1; c < (1 << E); c <<= 1) {\n    double qc[4];"),
}


def _build_mutant(tmp, name):
    old, new = MUTANTS[name]
    src = open(ORACLE_SRC).read()
    assert src.count(old) == 1, name
    path = os.path.join(tmp, name + ".c")
    open(path, "w").write(src.replace(old, new))
    lib = os.path.join(tmp, name + ".so")
    inc = os.path.dirname(ORACLE_SRC)
    subprocess.run(["gcc", "-O2", "-fPIC", "-shared", "-ffp-contract=off", "-std=gnu11", "-I", inc,
                    "-o", lib, path, "-lm"], check=True, capture_output=True)
    L = C.CDLL(lib)
    dp = C.POINTER(C.c_double)
    L.orc_flux_limit_cell.argtypes = [C.c_double, C.c_double, C.c_int, C.c_double, C.c_double, dp, dp, dp, dp]

    def flc(gamma, eps0, area, dt, qbar, fW, fF):
        qbar = np.ascontiguousarray(qbar, dtype=np.float64)
        fW = np.ascontiguousarray(fW, dtype=np.float64); fF = np.ascontiguousarray(fF, dtype=np.float64)
        prop = np.zeros(fW.shape[0])
        bad = L.orc_flux_limit_cell(gamma, eps0, fW.shape[0], area, dt, qbar.ctypes.data_as(dp),
                                    fW.ctypes.data_as(dp), fF.ctypes.data_as(dp), prop.ctypes.data_as(dp))
        return prop, bad
    return flc


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_over_limiting_variants_fail_the_pins(name):
    """A planted over-limiting mistake in the oracle's flux limiter (built
    here from its source with one line changed) fails the pins above."""
    with tempfile.TemporaryDirectory() as tmp:
        flc = _build_mutant(tmp, name)
        assert pin_failures(flc) != []
