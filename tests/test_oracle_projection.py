"""Pins of the oracle's L2 projection of the initial data (Sec. 1.2: the
modal expansion) and of its global wave speed (Eq. LLF) against closed forms:
a state whose conserved variables are polynomials of the element's degree is
reproduced exactly at arbitrary points, its cell averages are the exact
integrals over the cell, and a uniform state's speed is |u| + c."""
import numpy as np
import pytest

import synth

G = 1.4


def poly_state(deg):
    """rho and E polynomials of total degree deg, at rest (so the projected
    conserved variables are exactly those polynomials)."""
    def f(x, y):
        rho = 1.5 + 0.3 * x - 0.2 * y + 0.1 * x * y + 0.15 * x * x
        e = 2.0 - 0.1 * x + 0.25 * y * y - 0.05 * x * y
        if deg == 3:
            rho = rho + 0.05 * x ** 3 - 0.04 * x * y * y
            e = e + 0.03 * y ** 3
        z = 0.0 * x
        return rho, z, z, (G - 1.0) * e
    return f


def meshes(orc):
    xy, tv = synth.structured_triangles(5, jitter=0.2, seed=9)
    return [orc.Mesh.cartesian(4, 3, (0.0, 1.0, 0.0, 0.75), (2, 2, 2, 2)), orc.Mesh.triangles(xy, tv)]


@pytest.mark.parametrize("deg", [2, 3])
def test_projection_reproduces_polynomials(orc, deg):
    f = poly_state(deg)
    for mesh in meshes(orc):
        sol = orc.Solver(mesh, deg, gamma=G)
        Q = sol.project_fn(f)
        # at the limiter points (interior and edge quadrature points): the same polynomial
        xy = sol.limiter_points()
        q = sol.eval_limiter_points(Q)
        r, _, _, p = f(xy[..., 0], xy[..., 1])
        assert np.abs(q[..., 0] - r).max() < 1e-13
        assert np.abs(q[..., 3] - p / (G - 1.0)).max() < 1e-13
        assert np.abs(q[..., 1:3]).max() < 1e-15


def test_projection_averages_are_cell_integrals(orc):
    """rho = 1 + x^2 y on axis-aligned cells: the average is the exact integral
    over the cell divided by its area (closed form)."""
    nx, ny = 4, 3
    sol = orc.Solver(orc.Mesh.cartesian(nx, ny, (0.0, 1.0, 0.0, 0.75), (2, 2, 2, 2)), 2, gamma=G)
    Q = sol.project_fn(lambda x, y: (1.0 + x * x * y, 0 * x, 0 * x, 1.0 + 0 * x))
    hx, hy = 1.0 / nx, 0.75 / ny
    for iy in range(ny):
        for ix in range(nx):
            x0, x1, y0, y1 = ix * hx, (ix + 1) * hx, iy * hy, (iy + 1) * hy
            exact = 1.0 + (x1 ** 3 - x0 ** 3) / 3.0 * (y1 ** 2 - y0 ** 2) / 2.0 / (hx * hy)
            assert abs(Q[iy * nx + ix, 0, 0] - exact) < 1e-14


def test_wave_speed_of_uniform_and_bounded_states(orc):
    sol = orc.Solver(orc.Mesh.cartesian(5, 5), 2, gamma=G)
    rho, u, v, p = 1.3, 0.3, -0.2, 0.8
    Q = sol.project_fn(synth.ic_uniform(rho, u, v, p))
    assert abs(sol.wave_speed(Q) - (np.hypot(u, v) + np.sqrt(G * p / rho))) < 1e-14
    # any state: s is at least every average's speed and every point's speed
    Q = synth.random_modal_state(sol.N, sol.ML, seed=3, amp=0.05)
    s = sol.wave_speed(Q)
    qb = Q[:, :, 0]
    pb = (G - 1) * (qb[:, 3] - 0.5 * (qb[:, 1] ** 2 + qb[:, 2] ** 2) / qb[:, 0])
    sb = np.hypot(qb[:, 1], qb[:, 2]) / qb[:, 0] + np.sqrt(G * pb / qb[:, 0])
    q = sol.eval_limiter_points(Q)
    pp = (G - 1) * (q[..., 3] - 0.5 * (q[..., 1] ** 2 + q[..., 2] ** 2) / q[..., 0])
    sp = np.hypot(q[..., 1], q[..., 2]) / q[..., 0] + np.sqrt(G * np.maximum(pp, 0) / q[..., 0])
    assert s >= sb.max() - 1e-14 and abs(s - max(sb.max(), sp.max())) < 1e-13
