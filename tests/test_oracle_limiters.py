"""Pins of the oracle's positivity machinery (Sec. 3) by brute force on small
random inputs: the moment limiter (Sec. 3.1), the mu quadratic (Sec. 3.3
Step 5b), the positivity of every state in the final theta box (Steps 4-6)
and the invariants of the shock-capturing limiter (Sec. 4.1)."""
import os

import numpy as np
import pytest

import synth

G = 1.4


def pressure(q):
    return (G - 1) * (q[..., 3] - 0.5 * (q[..., 1] ** 2 + q[..., 2] ** 2) / q[..., 0])


def small_meshes(orc):
    yield orc.Mesh.cartesian(5, 4, (0.0, 1.0, 0.0, 0.8))
    xy, tv = synth.structured_triangles(3, jitter=0.2, seed=5)
    yield orc.Mesh.triangles(xy, tv)


@pytest.mark.parametrize("deg", [2, 3])
def test_moment_limiter_positivity_and_feasibility(orc, deg):
    for mesh in small_meshes(orc):
        sol = orc.Solver(mesh, deg, gamma=G)
        Q0 = synth.random_modal_state(mesh.N, sol.ML, seed=100 + deg, amp=1.2)
        Q0[::2, :, 1:] *= 0.02 * np.arange(1, mesh.N + 1, 2)[:, None, None] / mesh.N
        Q = Q0.copy()
        th, st = sol.moment_limit(Q)
        assert st == 0
        assert np.array_equal(Q[:, :, 0], Q0[:, :, 0])               # averages untouched
        assert np.all((th >= 0) & (th <= 1)) and np.any(th < 1) and np.any(th == 1)
        assert np.allclose(Q[:, :, 1:], th[:, None, None] * Q0[:, :, 1:], rtol=1e-15, atol=0)
        q = sol.eval_limiter_points(Q)
        rbar = Q0[:, 0, 0]; pbar = pressure(Q0[:, :, 0])
        eps_r = np.minimum(1e-12, rbar / 2); eps_p = np.minimum(1e-12, pbar / 2)
        scale = np.abs(Q0[:, :, 0]).max(axis=1)
        assert np.all(q[..., 0] >= eps_r[:, None] - 1e-14 * scale[:, None])
        assert np.all(pressure(q) >= eps_p[:, None] - 1e-13 * scale[:, None])
        # brute force: every theta' <= theta is feasible, and theta is not
        # larger than the largest feasible value found on a dense grid
        qu = sol.eval_limiter_points(Q0)
        qb = Q0[:, :, 0][:, None, :]
        grid = np.linspace(0.0, 1.0, 2001)
        for i in range(mesh.N):
            qs = qb[i] + grid[:, None, None] * (qu[i] - qb[i])[None]
            ok = np.all(qs[..., 0] >= eps_r[i] * (1 - 1e-9), axis=1) & np.all(pressure(qs) >= eps_p[i] * (1 - 1e-9), axis=1)
            star = grid[np.argmin(ok)] if not ok.all() else 1.0
            assert th[i] <= star + 1e-12
            assert ok[grid <= th[i] - 1e-12].all()


@pytest.mark.parametrize("deg", [2, 3])
def test_moment_limiter_exact_root_is_the_largest_feasible_theta(orc, deg):
    """The exact-root variant (Sec. 3.1 remarks that the optimal theta can be
    computed exactly): theta equals the supremum of the feasible set
    {theta: rho >= eps_rho and p >= eps_p at every point}, found here by
    bisection of that set (an interval [0, theta*]: density is linear and
    pressure concave in theta), and is never below Lemma 1's secant."""
    for mesh in small_meshes(orc):
        exact = orc.Solver(mesh, deg, gamma=G, moment_exact=True)
        secant = orc.Solver(mesh, deg, gamma=G)
        Q0 = synth.random_modal_state(mesh.N, exact.ML, seed=200 + deg, amp=1.2)
        Q0[::2, :, 1:] *= 0.02 * np.arange(1, mesh.N + 1, 2)[:, None, None] / mesh.N
        Qe, Qs = Q0.copy(), Q0.copy()
        te, st = exact.moment_limit(Qe)
        ts, _ = secant.moment_limit(Qs)
        assert st == 0
        assert np.all(te >= ts - 1e-15) and np.any(te > ts + 1e-6)
        assert np.array_equal(Qe[:, :, 0], Q0[:, :, 0])
        qu = exact.eval_limiter_points(Q0)
        rbar = Q0[:, 0, 0]; pbar = pressure(Q0[:, :, 0])
        eps_r = np.minimum(1e-12, rbar / 2); eps_p = np.minimum(1e-12, pbar / 2)
        for i in range(mesh.N):
            qb = Q0[i, :, 0]

            def feasible(t):
                qs = qb[None] + t * (qu[i] - qb[None])
                return bool(np.all(qs[:, 0] >= eps_r[i]) and np.all(pressure(qs) >= eps_p[i]))

            if feasible(1.0):
                assert te[i] == 1.0
                continue
            lo, hi = 0.0, 1.0
            for _ in range(200):
                mid = 0.5 * (lo + hi)
                lo, hi = (mid, hi) if feasible(mid) else (lo, mid)
            assert abs(te[i] - lo) <= 1e-9 * max(lo, 1e-3), (i, te[i], lo, ts[i])


def test_mu_solve_matches_bisection(orc):
    rng = np.random.default_rng(3)
    hits = 0
    for _ in range(400):
        ql = synth.random_modal_state(1, 1, seed=int(rng.integers(1 << 30)))[0, :, 0]
        qc = ql + rng.normal(size=4) * np.abs(ql) * rng.uniform(0.1, 3)
        qc[0] = abs(qc[0]) + 1e-3                        # corner densities are positive
        mu = orc.mu_solve(G, 1e-12, ql, qc)
        eps_p = min(1e-12, 0.5 * pressure(ql))
        f = lambda m: pressure(ql + m * (qc - ql)) - eps_p
        if f(1.0) >= 0:
            assert mu == 1.0
            continue
        lo, hi = 0.0, 1.0
        for _ in range(200):
            mid = 0.5 * (lo + hi)
            lo, hi = (mid, hi) if f(mid) >= 0 else (lo, mid)
        assert abs(mu - lo) < 1e-12
        assert f(mu) >= -1e-12 * abs(ql[3])
        hits += 1
    assert hits > 50


@pytest.mark.parametrize("E", [3, 4])
def test_flux_limiter_box_positivity_brute_force(orc, E):
    """Steps 4-5 on random cells: every state of the box [0, Lambda'] has
    rho >= 0 and p > 0 (sampled densely, corners included)."""
    rng = np.random.default_rng(E)
    limited = 0
    for trial in range(300):
        qbar = synth.random_modal_state(1, 1, seed=1000 * E + trial, rho_range=(0.01, 2.0), p_range=(1e-3, 2.0))[0, :, 0]
        T, dt = rng.uniform(0.5, 2.0), rng.uniform(0.05, 0.3)
        # a positive low-order state q^LxF fixes sum_k f^LxF_k
        qlxf = synth.random_modal_state(1, 1, seed=7000 * E + trial, rho_range=(1e-4, 1.0), p_range=(1e-5, 1.0))[0, :, 0]
        fF = rng.normal(size=(E, 4))
        fF += ((qbar - qlxf) * T / dt - fF.sum(0)) / E
        fW = fF + rng.normal(size=(E, 4)) * np.abs(qbar) * T / dt * rng.uniform(0.05, 1.0)
        prop, bad = orc.flux_limit_cell(G, 1e-12, T, dt, qbar, fW, fF)
        assert bad == 0 and np.all((prop >= 0) & (prop <= 1))
        limited += np.any(prop < 1)
        samp = rng.uniform(0, 1, (400, E)) * prop[None, :]
        corners = np.array([[(c >> k) & 1 for k in range(E)] for c in range(1 << E)]) * prop[None, :]
        samp = np.vstack([samp, corners])
        qn = qbar[None, :] - dt / T * (samp @ fW + (1 - samp) @ fF)
        assert np.all(qn[:, 0] >= 0)
        assert np.all(pressure(qn) > 0)
    assert limited > 100


@pytest.mark.parametrize("case", ["random_literal_llf", "rarefaction"])
def test_step_uses_edge_min_of_proposals(orc, case):
    """Through a full step: the new averages equal the blended update at
    theta_e, and theta_e keeps every state of the box positive.  Random data
    wakes the flux limiter when the point flux dissipates with the global s
    (the literal reading of Eq. LLF); with the local speed (default) a strong
    rarefaction (u = -+3, p = 0.01) at CFL 0.6 does."""
    if case == "random_literal_llf":
        mesh = orc.Mesh.cartesian(10, 10, bc=(2, 2, 2, 2))
        sol = orc.Solver(mesh, 2, gamma=G, shock_limiter=False, llf_global=True)
        Q = synth.random_modal_state(mesh.N, sol.ML, seed=78, amp=0.3, rho_range=(0.01, 3.0), p_range=(0.001, 3.0))
        cfl, warm = 0.9, 0
    else:
        mesh = orc.Mesh.cartesian(16, 4, bc=(2, 2, 0, 0))
        sol = orc.Solver(mesh, 2, gamma=G, shock_limiter=False)
        Q = sol.project_fn(lambda x, y: (np.ones_like(x), np.where(x < 0.5, -3.0, 3.0), 0 * x, 0.01 + 0 * x))
        cfl, warm = 0.6, 20
    for _ in range(warm + 1):
        Qlim = Q.copy(); sol.moment_limit(Qlim)
        d = sol.step(Q, cfl=cfl, want_theta=True)
        if d["n_edge"] > 0:
            break
    assert d["status"] == 0 and d["n_edge"] > 0
    fw, ff, dt = sol.last_fluxes()
    area = mesh.geometry()[0]
    rng = np.random.default_rng(0)
    for i in range(mesh.N):
        th = d["theta_edge"][i]
        samp = np.vstack([rng.uniform(0, 1, (300, mesh.E)) * th[None, :], th[None, :]])
        qn = Qlim[i, :, 0][None, :] - dt / area[i] * (samp @ fw[i] + (1 - samp) @ ff[i])
        assert np.all(qn[:, 0] >= 0) and np.all(pressure(qn) > 0)
        assert np.allclose(qn[-1], Q[i, :, 0], rtol=1e-13, atol=1e-14)


def test_shock_limiter_invariants(orc):
    n = 8
    mesh = orc.Mesh.cartesian(n, n)
    sol = orc.Solver(mesh, 2, gamma=G, alpha0=5.0)
    Q0 = synth.random_modal_state(mesh.N, sol.ML, seed=21, amp=0.6)
    Q = Q0.copy()
    th = sol.shock_limit(Q)
    assert np.array_equal(Q[:, :, 0], Q0[:, :, 0])
    assert np.all((th >= 0) & (th <= 1)) and np.any(th < 1)
    assert np.allclose(Q[:, :, 1:], th[:, None, None] * Q0[:, :, 1:], rtol=1e-15, atol=0)
    # density is linear in Q: its limited point values lie in [m_i, M_i]
    alpha = 5.0 * (1.0 / n) ** 1.5
    rb = Q0[:, 0, 0].reshape(n, n)
    nb = np.stack([np.roll(rb, 1, 0), np.roll(rb, -1, 0), np.roll(rb, 1, 1), np.roll(rb, -1, 1)])
    Mx = np.maximum(rb + alpha, nb.max(0)).ravel(); Mn = np.minimum(rb - alpha, nb.min(0)).ravel()
    r = sol.eval_limiter_points(Q)[..., 0]
    assert np.all(r <= Mx[:, None] + 1e-13) and np.all(r >= Mn[:, None] - 1e-13)
    # smooth, well-resolved data is left alone
    sm = orc.Solver(orc.Mesh.cartesian(32, 32), 2, gamma=G)
    Qs = sm.project_fn(synth.ic_smooth)
    assert np.all(sm.shock_limit(Qs.copy()) == 1.0)


def shock_tightness_failures(orc):
    """Failures of the density-tightness pin of the shock limiter (G14, Sec.
    4.1) for the oracle module as it is loaded now; [] when it holds."""
    n = 8
    alpha0 = 5.0
    mesh = orc.Mesh.cartesian(n, n)
    sol = orc.Solver(mesh, 2, gamma=G, alpha0=alpha0)
    Q0 = synth.random_modal_state(mesh.N, sol.ML, seed=22, amp=0.6)
    # in half of the cells velocity and pressure are constant over the cell
    # (momentum and energy modes follow the density's), so there only the
    # density can bind
    u = Q0[:, 1, 0] / Q0[:, 0, 0]; v = Q0[:, 2, 0] / Q0[:, 0, 0]
    half = np.arange(mesh.N) % 2 == 0
    Q0[half, 1, 1:] = u[half, None] * Q0[half, 0, 1:]
    Q0[half, 2, 1:] = v[half, None] * Q0[half, 0, 1:]
    Q0[half, 3, 1:] = 0.5 * (u[half, None] ** 2 + v[half, None] ** 2) * Q0[half, 0, 1:]
    Q = Q0.copy()
    th = sol.shock_limit(Q)
    alpha = alpha0 * (1.0 / n) ** 1.5
    rb = Q0[:, 0, 0].reshape(n, n)
    nb = np.stack([np.roll(rb, 1, 0), np.roll(rb, -1, 0), np.roll(rb, 1, 1), np.roll(rb, -1, 1)])
    Mx = np.maximum(rb + alpha, nb.max(0)).ravel(); Mn = np.minimum(rb - alpha, nb.min(0)).ravel()
    r0 = sol.eval_limiter_points(Q0)[..., 0]
    rbar = Q0[:, 0, 0]
    hx, hn = r0.max(axis=1), r0.min(axis=1)
    th_rho = np.ones(mesh.N)
    up, dn = hx > rbar, hn < rbar
    th_rho[up] = np.minimum(th_rho[up], (Mx[up] - rbar[up]) / (hx[up] - rbar[up]))
    th_rho[dn] = np.minimum(th_rho[dn], (rbar[dn] - Mn[dn]) / (rbar[dn] - hn[dn]))
    th_rho = np.clip(th_rho, 0.0, 1.0)
    out = []
    if not np.all(th <= th_rho + 1e-14):
        out.append("theta above the density's ratio")
    # cells where only the density varies (and stays positive at every
    # point): theta is the density's ratio, and the limited density reaches
    # its bound at the extreme point
    binding = half & (th_rho < 1.0) & (r0.min(axis=1) > 0.0)
    if binding.sum() < 3:
        out.append("fewer than 3 density-bound cells")
    if binding.any() and np.abs(th[binding] - th_rho[binding]).max() > 1e-13:
        out.append("theta differs from the density's ratio by %.2e" % np.abs(th[binding] - th_rho[binding]).max())
    r = sol.eval_limiter_points(Q)[..., 0]
    gap = np.minimum(np.abs(r.max(axis=1) - Mx), np.abs(r.min(axis=1) - Mn))
    if binding.any() and gap[binding].max() > 1e-12:
        out.append("over-limited: the limited density stays %.2e inside its bound" % gap[binding].max())
    if not np.allclose(Q[:, :, 1:], th[:, None, None] * Q0[:, :, 1:], rtol=1e-15, atol=0):
        out.append("the higher modes are not scaled by theta")
    return out


def test_shock_limiter_is_tight_on_the_density(orc):
    """G14 takes theta_sc as the smallest of four ratios, one per primitive;
    the density is linear in theta, so where only its ratio binds the limited
    density reaches its bound exactly at the extreme point (no
    over-limiting), and theta_sc never exceeds the density's ratio."""
    assert shock_tightness_failures(orc) == []


SHOCK_MUTANTS = {
    # half the theta
    "half_theta": ("  if (th < 0.0) th = 0.0;\n  return th;", "  if (th < 0.0) th = 0.0;\n  return 0.5 * th;"),
    # bounds from the cell alone (the neighbours' averages ignored)
    "no_neighbours": ("    if (!(qj[0] > 0.0)) continue;\n    double wj[4];",
                      "    if (1) continue;\n    double wj[4];"),
    # bounds without alpha
    "no_alpha": ("  for (int c = 0; c < 4; ++c) { Mx[c] = wbar[c] + alpha; Mn[c] = wbar[c] - alpha; }",
                 "  for (int c = 0; c < 4; ++c) { Mx[c] = wbar[c]; Mn[c] = wbar[c]; }"),
}


@pytest.mark.parametrize("name", sorted(SHOCK_MUTANTS))
def test_over_limiting_shock_variants_fail_the_pin(orc, name):
    """A planted over-limiting mistake in the oracle's shock limiter (built
    here from its source with one line changed) fails the tightness pin."""
    import subprocess
    import tempfile
    src_path = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "oracle", "lxw_oracle.c")
    old, new = SHOCK_MUTANTS[name]
    src = open(src_path).read()
    assert src.count(old) == 1, name
    with tempfile.TemporaryDirectory() as tmp:
        path = os.path.join(tmp, name + ".c")
        open(path, "w").write(src.replace(old, new))
        so = os.path.join(tmp, name + ".so")
        subprocess.run(["gcc", "-O2", "-fPIC", "-shared", "-ffp-contract=off", "-std=gnu11", "-I",
                        os.path.dirname(src_path), "-o", so, path, "-lm"], check=True, capture_output=True)
        with orc.use_library(so):
            assert shock_tightness_failures(orc) != []
