"""Pins of the oracle's masked Cartesian meshes and inflow boundaries (the
shock-diffraction setting of Sec. 4) against facts that do not come from the
oracle's own formulas:

- a masked mesh whose left-out cells only cut the grid short is the smaller
  grid with a wall there, step for step (also across a periodic side);
- a left-out column in the middle splits the domain into two channels that
  evolve independently, mirror images for mirrored data;
- an inflow face is, for one whole step, a ghost column holding the steady
  inflow state;
- a Mach 5.09 shock driven by the inflow: mass, momentum and energy grow at
  exactly the boundary fluxes the Euler equations fix, and the shock sits at
  x_s + 5.09 t (Rankine-Hugoniot)."""
import numpy as np
import pytest

import synth

G = 1.4
T_, R_ = 2, 1   # transparent, reflective


def riemann_2d(x, y):
    """Two-dimensional data with a density jump and a tilted velocity field."""
    r = np.where(x + 0.3 * y < 0.45, 1.6, 0.7)
    u = 0.4 * np.cos(3.0 * y) + 0.1
    v = 0.3 * np.sin(5.0 * x)
    p = np.where(x < 0.4, 1.5, 0.5) + 0.1 * y
    return r, u, v, p


def conserved(prim):
    r, u, v, p = prim
    return np.array([r, r * u, r * v, p / (G - 1.0) + 0.5 * r * (u * u + v * v)])


def run(sol, Q, steps, dt):
    for _ in range(steps):
        d = sol.step(Q, dt=dt)
        assert d["status"] == 0
        assert d["min_rho"] > 0 and d["min_p"] > 0
    return d


def test_masked_column_is_a_wall(orc):
    """8 x 6 cells with the last column left out and mask_bc reflective give
    the 7 x 6 grid whose right side is a wall."""
    mask = np.ones((6, 8), bool); mask[:, 7] = False
    bc = (T_, T_, R_, R_)
    A = orc.Solver(orc.Mesh.cartesian_masked(8, 6, (0.0, 1.0, 0.0, 0.75), bc, mask, mask_bc=R_), 2, gamma=G)
    B = orc.Solver(orc.Mesh.cartesian(7, 6, (0.0, 0.875, 0.0, 0.75), (T_, R_, R_, R_)), 2, gamma=G)
    assert A.N == B.N == 42
    QA = A.project_fn(riemann_2d); QB = B.project_fn(riemann_2d)
    assert np.array_equal(QA, QB)
    run(A, QA, 25, 2e-3); run(B, QB, 25, 2e-3)
    assert np.abs(QA - QB).max() <= 1e-13 * np.abs(QB).max()


def test_masked_column_across_a_periodic_side(orc):
    """Left-out column 0 of a grid periodic in x: the faces that reach it
    across the seam and directly both become walls (the 5-column grid with
    reflective sides)."""
    mask = np.ones((4, 6), bool); mask[:, 0] = False
    A = orc.Solver(orc.Mesh.cartesian_masked(6, 4, (0.0, 0.75, 0.0, 0.5), (0, 0, R_, R_), mask, mask_bc=R_), 2, gamma=G)
    B = orc.Solver(orc.Mesh.cartesian(5, 4, (0.125, 0.75, 0.0, 0.5), (R_, R_, R_, R_)), 2, gamma=G)
    QA = A.project_fn(riemann_2d); QB = B.project_fn(riemann_2d)
    assert np.array_equal(QA, QB)
    run(A, QA, 20, 2e-3); run(B, QB, 20, 2e-3)
    assert np.abs(QA - QB).max() <= 1e-13 * np.abs(QB).max()


def test_masked_middle_column_splits_into_mirrored_channels(orc):
    """9 x 4 cells on [0, 1.125] without column 4: two channels with a wall
    between them.  Mirror-image data stays mirrored, and the left channel is
    the 4 x 4 grid run on its own."""
    mask = np.ones((4, 9), bool); mask[:, 4] = False
    A = orc.Solver(orc.Mesh.cartesian_masked(9, 4, (0.0, 1.125, 0.0, 0.5), (T_, T_, R_, R_), mask, mask_bc=R_), 2, gamma=G)
    B = orc.Solver(orc.Mesh.cartesian(4, 4, (0.0, 0.5, 0.0, 0.5), (T_, R_, R_, R_)), 2, gamma=G)

    def left(x, y):
        return riemann_2d(x / 0.5 * 0.9, y)

    def both(x, y):
        r, u, v, p = left(np.where(x < 0.5625, x, 1.125 - x), y)
        return r, np.where(x < 0.5625, u, -u), v, p

    QA = A.project_fn(both); QB = B.project_fn(left)
    run(A, QA, 25, 2e-3); run(B, QB, 25, 2e-3)
    QA = QA.reshape(4, 8, 4, 6)
    L = QA[:, :4]; Rt = QA[:, 4:][:, ::-1]
    sc = np.abs(QB).max()
    assert np.abs(L.reshape(16, 4, 6) - QB).max() <= 1e-13 * sc
    # mirror x -> -x on the quadrilateral modes 1, L1(x), L1(y), L1(x)L1(y), L2(x), L2(y):
    # odd in x flips the sign of modes 1 and 3, and x-momentum flips as a whole
    sgn = np.array([1, -1, 1, -1, 1, 1.0])
    M = Rt * sgn
    M[..., 1, :] *= -1
    assert np.abs(L - M).max() <= 1e-13 * sc


def test_inflow_face_is_a_ghost_column_with_the_steady_state(orc):
    """An inflow side acts as one more column, on the left, that holds the
    inflow state as a constant polynomial: one whole step without the shock
    limiter (moment limiter, CK traces, f^LxW and f^LxF at the face, flux
    limiter, update) gives the same fluxes and state; the shock limiter and the
    gate features, which read the neighbour average, see the same bounds."""
    prim_in = (2.0, 0.5, 0.0, 1.0)
    qin = conserved(prim_in)
    nx, ny, h = 6, 4, 0.125
    bcA, bcB = (orc.INFLOW, T_, R_, R_), (T_, T_, R_, R_)
    boxA, boxB = (0.0, nx * h, 0.0, ny * h), (-h, nx * h, 0.0, ny * h)

    def data(x, y):
        # a strong jump inside the first column wakes the moment and shock limiters there
        r, u, v, p = riemann_2d(x, y)
        right = x > 0.0625
        return np.where(right, 0.1 * r, r), u, v, np.where(right, 0.05 * p, p)

    def with_ghost(QA):
        QB = np.zeros((ny, nx + 1, 4, 6))
        QB[:, 1:] = QA.reshape(ny, nx, 4, 6)
        QB[:, 0, :, 0] = qin
        return QB.reshape(-1, 4, 6).copy()

    def inner(X, k=None):
        return X.reshape((ny, nx + 1) + X.shape[1:])[:, 1:].reshape((-1,) + X.shape[1:])

    A = orc.Solver(orc.Mesh.cartesian(nx, ny, boxA, bcA), 2, gamma=G, shock_limiter=False)
    B = orc.Solver(orc.Mesh.cartesian(nx + 1, ny, boxB, bcB), 2, gamma=G, shock_limiter=False)
    A.set_inflow(prim_in)
    QA = A.project_fn(data)
    QB = with_ghost(QA)
    assert A.wave_speed(QA) == B.wave_speed(QB)   # the inflow state is not the fastest
    dA = A.step(QA, dt=4e-3, want_theta=True); dB = B.step(QB, dt=4e-3, want_theta=True)
    assert dA["status"] == dB["status"] == 0 and dA["n_mom"] > 0
    sc = np.abs(QA).max()
    assert np.abs(QA - inner(QB)).max() <= 1e-13 * sc
    assert np.array_equal(dA["theta_mom"], inner(dB["theta_mom"]))
    assert np.array_equal(dA["theta_edge"], inner(dB["theta_edge"]))
    fwA, ffA, _ = A.last_fluxes(); fwB, ffB, _ = B.last_fluxes()
    for a_, b_ in ((fwA, fwB), (ffA, ffB)):
        assert np.abs(a_ - inner(b_)).max() <= 1e-13 * np.abs(b_).max()
    # the inflow face's f^LxF differs from the copy (transparent) one: the test sees the face
    At = orc.Solver(orc.Mesh.cartesian(nx, ny, boxA, (T_, T_, R_, R_)), 2, gamma=G, shock_limiter=False)
    Qt = At.project_fn(data); At.step(Qt, dt=4e-3)
    assert np.abs(At.last_fluxes()[1][::nx, 3] - ffA[::nx, 3]).max() > 1e-3

    # shock limiter and features on the stepped state, the ghost holding q_in again
    A2 = orc.Solver(orc.Mesh.cartesian(nx, ny, boxA, bcA), 2, gamma=G, alpha0=2.0)
    B2 = orc.Solver(orc.Mesh.cartesian(nx + 1, ny, boxB, bcB), 2, gamma=G, alpha0=2.0)
    A2.set_inflow(prim_in)
    QB = with_ghost(QA)
    assert np.abs(A2.features(QA) - inner(B2.features(QB))).max() <= 1e-13
    tA = A2.shock_limit(QA); tB = B2.shock_limit(QB)
    assert np.sum(tA[::nx] < 1.0) >= 3          # the first column is limited against q_in
    assert np.abs(tA - inner(tB)).max() <= 1e-13
    assert np.abs(QA - inner(QB)).max() <= 1e-13 * sc


def test_inflow_driven_mach_5_09_shock(orc):
    """Post-shock state of a Mach 5.09 shock into gas at rest (rho 1.4, p 1)
    prescribed on the left of a channel: the shock moves at 5.09 (c0 = 1);
    the integrals of mass, momentum and energy change at exactly the inflow
    minus outflow fluxes while the shock is inside.  The shock starts 40
    cells from the inflow: the LLF dissipation (global s = 6.5) lets the
    start-up disturbance leak upstream by about (s - (u - c)) / (s + (u - c))
    = 0.6 per cell, which 40 cells bring below rounding."""
    post = synth.normal_shock_state(5.09)
    q1, q0 = conserved(post), conserved((1.4, 0.0, 0.0, 1.0))
    nx, ny, Lx, H, xs = 96, 2, 3.0, 0.0625, 1.25
    sol = orc.Solver(orc.Mesh.cartesian(nx, ny, (0.0, Lx, 0.0, H), (orc.INFLOW, T_, R_, R_)), 2, gamma=G)
    sol.set_inflow(post)
    a, _, cx, _ = sol.mesh.geometry()
    Q = np.zeros((sol.N, 4, sol.ML))
    Q[:, :, 0] = np.where((cx < xs)[:, None], q1[None, :], q0[None, :])
    tot0 = a @ Q[:, :, 0]
    dt, n = 2e-4, 400
    for k in range(n):
        d = sol.step(Q, dt=dt)
        assert d["status"] == 0 and d["min_rho"] > 0 and d["min_p"] > 0, (k, d)
    t = n * dt
    F1 = np.array([q1[1], q1[1] * post[1] + post[3], 0.0, post[1] * (q1[3] + post[3])])
    F0 = np.array([0.0, 1.0, 0.0, 0.0])
    tot = a @ Q[:, :, 0]
    expect = tot0 + (F1 - F0) * H * t
    for v in (0, 1, 3):
        assert abs(tot[v] - expect[v]) <= 1e-13 * abs(expect[v]), (v, tot[v], expect[v])
    assert abs(tot[2]) <= 1e-12
    # shock position: where the density crosses the mid value (one row)
    rho = Q[:nx, 0, 0]
    xm = cx[:nx]
    k = int(np.argmax(rho < 0.5 * (post[0] + 1.4)))
    x_half = xm[k - 1] + (xm[k] - xm[k - 1]) * (0.5 * (post[0] + 1.4) - rho[k - 1]) / (rho[k] - rho[k - 1])
    assert abs(x_half - (xs + 5.09 * t)) < 1.5 * Lx / nx, (x_half, xs + 5.09 * t)
    # the inflow side stays the exact steady state
    assert np.abs(Q[0, :, 0] - q1).max() <= 1e-13 * np.abs(q1).max()
    assert np.abs(Q[nx - 1, :, 0] - q0).max() <= 1e-12 * np.abs(q0).max()


def test_diffraction_mesh_and_first_steps(orc):
    """The step geometry at 1/10 of the paper's resolution, its boundaries
    (inflow above the step, walls on the step, transparent elsewhere): cell
    count and positivity over the first steps."""
    nx, ny = 39, 33
    mask = synth.diffraction_mask(nx, ny)
    assert mask.sum() == nx * ny - 3 * 18
    mesh = orc.Mesh.cartesian_masked(nx, ny, synth.DIFFRACTION_BOX, synth.DIFFRACTION_BC, mask, mask_bc=R_)
    sol = orc.Solver(mesh, 2, gamma=G)
    sol.set_inflow(synth.normal_shock_state(synth.DIFFRACTION_MACH))
    Q = sol.project_fn(synth.ic_diffraction)
    for k in range(30):
        d = sol.step(Q, cfl=0.1)
        assert d["status"] == 0 and d["min_rho"] > 0 and d["min_p"] > 0, (k, d)
