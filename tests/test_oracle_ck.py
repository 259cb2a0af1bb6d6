"""Closed-form pin of the oracle's Cauchy-Kovalevskaya time-averaged flux
(Sec. 2.2, Eqs. fluxderivs-a/b and taylor3-flux).

For a density wave with constant velocity and pressure, whose density is a
quadratic polynomial inside the element, the conserved variables and the
flux are exactly quadratic, every projection in the CK chain is exact, and
the exact solution rho0(x - u t) is quadratic in t, so the truncated series
F + dt/2 F_t + dt^2/6 F_tt equals the exact time average
(1/dt) Int_0^dt F(q(x, t)) dt at every point.  A dropped or mis-signed term
of F_t or F_tt, or a wrong Hessian, breaks this identity.
"""
import numpy as np
import numpy.polynomial.legendre as npleg
import pytest

import synth

G = 1.4
U, V, P = 0.7, -0.4, 1.1


def rho0(x, y):
    return 1.0 + 0.3 * x - 0.2 * y + 0.4 * x * x + 0.1 * x * y - 0.3 * y * y


def ic(x, y):
    return rho0(x, y), U * np.ones_like(x), V * np.ones_like(x), P * np.ones_like(x)


def exact_time_average(orc, x, y, dt):
    t, w = npleg.leggauss(4)
    tau = 0.5 * dt * (t + 1.0)
    FT = np.zeros((len(x), 4)); GT = np.zeros((len(x), 4))
    for k in range(4):
        r = rho0(x - U * tau[k], y - V * tau[k])
        for p in range(len(x)):
            q = np.array([r[p], r[p] * U, r[p] * V, P / (G - 1) + 0.5 * r[p] * (U * U + V * V)])
            F, Gf = orc.flux(G, q)
            FT[p] += 0.5 * w[k] * F; GT[p] += 0.5 * w[k] * Gf
    return FT, GT


def meshes(orc):
    yield "quad", orc.Mesh.cartesian(3, 3, (0.0, 0.9, 0.0, 0.9))
    xy, tv = synth.structured_triangles(3, jitter=0.2, seed=11, box=(0.0, 0.9, 0.0, 0.9))
    yield "tri", orc.Mesh.triangles(xy, tv)


@pytest.mark.parametrize("deg", [2, 3])
def test_ck_flux_equals_exact_time_average(orc, deg):
    for name, mesh in meshes(orc):
        sol = orc.Solver(mesh, deg, gamma=G)
        Q = sol.project_fn(ic)
        xy = sol.limiter_points()
        for i in (0, 4, mesh.N - 1):
            for dt in (0.01, 0.05):
                out = sol.ck_element(Q, i, dt)
                FT, GT = exact_time_average(orc, xy[i, :, 0], xy[i, :, 1], dt)
                assert np.allclose(out["FT"], FT, rtol=1e-12, atol=1e-12), (name, i, dt)
                assert np.allclose(out["GT"], GT, rtol=1e-12, atol=1e-12), (name, i, dt)
                # q_t of the density is -u . grad rho exactly
                x, y = xy[i, :, 0], xy[i, :, 1]
                drdx = 0.3 + 0.8 * x + 0.1 * y
                drdy = -0.2 + 0.1 * x - 0.6 * y
                assert np.allclose(out["qt"][:, 0], -(U * drdx + V * drdy), atol=1e-12)


def rho3(x, y):
    return 1.0 + 0.3 * x - 0.2 * y + 0.4 * x * x + 0.1 * x * y - 0.3 * y * y + 0.2 * x ** 3 - 0.1 * x * y * y + 0.15 * y ** 3


def ic3(x, y):
    return rho3(x, y), U * np.ones_like(x), V * np.ones_like(x), P * np.ones_like(x)


def exact_time_average3(orc, x, y, dt):
    t, w = npleg.leggauss(4)
    tau = 0.5 * dt * (t + 1.0)
    FT = np.zeros((len(x), 4)); GT = np.zeros((len(x), 4))
    for k in range(4):
        r = rho3(x - U * tau[k], y - V * tau[k])
        for p in range(len(x)):
            q = np.array([r[p], r[p] * U, r[p] * V, P / (G - 1) + 0.5 * r[p] * (U * U + V * V)])
            F, Gf = orc.flux(G, q)
            FT[p] += 0.5 * w[k] * F; GT[p] += 0.5 * w[k] * Gf
    return FT, GT


def test_fourth_order_ck_flux_equals_exact_time_average_for_a_cubic_wave(orc):
    """P3 elements, density cubic in space with constant velocity and
    pressure: rho0(x - u t) is cubic in t, so the series through dt^3/24
    F_ttt is the exact time average at every point; the third-order series
    misses the dt^3 term (here by more than 1e-9)."""
    for name, mesh in meshes(orc):
        s4 = orc.Solver(mesh, 3, gamma=G, ck_order=4)
        s3 = orc.Solver(mesh, 3, gamma=G)
        Q = s4.project_fn(ic3)
        xy = s4.limiter_points()
        for i in (0, 4, mesh.N - 1):
            for dt in (0.02, 0.05):
                FT, GT = exact_time_average3(orc, xy[i, :, 0], xy[i, :, 1], dt)
                out = s4.ck_element(Q, i, dt)
                assert np.allclose(out["FT"], FT, rtol=1e-12, atol=1e-12), (name, i, dt)
                assert np.allclose(out["GT"], GT, rtol=1e-12, atol=1e-12), (name, i, dt)
                o3 = s3.ck_element(Q, i, dt)
                assert np.abs(o3["FT"] - FT).max() > 1e-9 and np.abs(o3["GT"] - GT).max() > 1e-9, (name, i, dt)


def test_third_and_mixed_flux_derivatives(orc):
    """The third directional derivative against finite differences of the
    second one and of the flux itself; zero along q (Euler homogeneity) and
    along a density-wave direction (the flux is affine there); the mixed
    second derivative is symmetric and equals the second directional
    derivative on the diagonal."""
    rng = np.random.default_rng(11)
    for trial in range(10):
        q = synth.random_modal_state(1, 1, seed=500 + trial)[0, :, 0]
        w = rng.normal(size=4) * np.abs(q) * 0.3
        F3, G3 = orc.flux_d3(G, q, w)
        h = 1e-4
        Fp, Gp = orc.flux_d2(G, q + h * w, w); Fm, Gm = orc.flux_d2(G, q - h * w, w)
        sc = 1 + np.abs(F3).max() + np.abs(G3).max()
        assert np.allclose(F3, (Fp - Fm) / (2 * h), atol=1e-6 * sc)
        assert np.allclose(G3, (Gp - Gm) / (2 * h), atol=1e-6 * sc)
        h = 1e-2
        f = [np.concatenate(orc.flux(G, q + k * h * w)) for k in (-2, -1, 1, 2)]
        fd = (f[3] - 2 * f[2] + 2 * f[1] - f[0]) / (2 * h ** 3)
        assert np.allclose(np.concatenate([F3, G3]), fd, atol=1e-3 * sc)
        Z = orc.flux_d3(G, q, q)
        assert np.abs(np.concatenate(Z)).max() < 1e-12 * (1 + np.abs(q).max() ** 2)
        u, v = q[1] / q[0], q[2] / q[0]
        dw = np.array([1.0, u, v, 0.5 * (u * u + v * v)])
        assert np.abs(np.concatenate(orc.flux_d3(G, q, dw))).max() < 1e-12 * sc
        a, b = rng.normal(size=4), rng.normal(size=4)
        Fab, Gab = orc.flux_d11(G, q, a, b); Fba, Gba = orc.flux_d11(G, q, b, a)
        assert np.allclose(Fab, Fba, atol=1e-13 * sc) and np.allclose(Gab, Gba, atol=1e-13 * sc)
        F2, G2 = orc.flux_d2(G, q, a); Faa, Gaa = orc.flux_d11(G, q, a, a)
        assert np.allclose(F2, Faa, atol=1e-13 * sc) and np.allclose(G2, Gaa, atol=1e-13 * sc)


def test_fourth_order_flux_at_a_transparent_boundary(orc):
    """At a transparent side the exterior state copies the interior one, so
    f^LxW there is the interior's own time-averaged flux, fourth-order term
    included: (1/2) sum_p w_p n.F_T(x_p) over the edge's Gauss points."""
    n, h, dt = 4, 0.25, 2e-3
    mesh = orc.Mesh.cartesian(n, n, bc=(2, 2, 2, 2))
    sol = orc.Solver(mesh, 3, gamma=G, ck_order=4, shock_limiter=False)
    Q = synth.random_modal_state(mesh.N, sol.ML, seed=8, amp=0.05)
    Q0 = Q.copy()
    sol.step(Q, dt=dt)
    fw, _, _ = sol.last_fluxes()
    gx, gw = orc.gauss_legendre(4)
    nq = sol.npts - 4 * 4
    normals = [(0.0, -h), (h, 0.0), (0.0, h), (-h, 0.0)]   # edges bottom, right, top, left
    checked = 0
    for i in range(mesh.N):
        iy, ix = divmod(i, n)
        ck = sol.ck_element(Q0, i, dt)
        for k, bnd in enumerate((iy == 0, ix == n - 1, iy == n - 1, ix == 0)):
            if not bnd:
                continue
            sl = slice(nq + 4 * k, nq + 4 * (k + 1))
            nx, ny = normals[k]
            want = 0.5 * (gw[:, None] * (nx * ck["FT"][sl] + ny * ck["GT"][sl])).sum(axis=0)
            assert np.allclose(fw[i, k], want, rtol=1e-12, atol=1e-14), (i, k)
            checked += 1
    assert checked == 4 * n
