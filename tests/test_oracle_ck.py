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
