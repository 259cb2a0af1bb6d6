"""Pins of the oracle's Euler flux and its directional derivatives
(Eqs. 1-2 and fluxderivs-a/b): special states, rotational invariance,
homogeneity, the characteristic speeds and finite differences."""
import numpy as np
import pytest

G = 1.4


def cons(rho, u, v, p, g=G):
    return np.array([rho, rho * u, rho * v, p / (g - 1) + 0.5 * rho * (u * u + v * v)])


def rand_states(n, seed=0):
    rng = np.random.default_rng(seed)
    return [cons(rng.uniform(0.2, 3), rng.uniform(-2, 2), rng.uniform(-2, 2), rng.uniform(0.1, 4)) for _ in range(n)]


def test_flux_at_rest_is_pressure(orc):
    q = cons(1.7, 0.0, 0.0, 2.3)
    F, Gf = orc.flux(G, q)
    assert np.allclose(F, [0, 2.3, 0, 0], atol=1e-15)
    assert np.allclose(Gf, [0, 0, 2.3, 0], atol=1e-15)


def test_flux_uniform_motion(orc):
    """A state moving with velocity (u,0) carries mass u rho, momentum
    u rho u + p and energy u (E + p) through a unit x-face."""
    rho, u, p = 0.9, 1.3, 0.7
    q = cons(rho, u, 0.0, p)
    F, Gf = orc.flux(G, q)
    E = q[3]
    assert np.allclose(F, [rho * u, rho * u * u + p, 0.0, u * (E + p)], rtol=1e-14)
    assert np.allclose(Gf, [0.0, 0.0, p, 0.0], atol=1e-14)


@pytest.mark.parametrize("ang", [0.3, 1.1, 2.5, -0.7])
def test_rotational_invariance(orc, ang):
    """n.F(q) = T^-1 F_x(T q) with T rotating the momentum into the n frame."""
    c, s = np.cos(ang), np.sin(ang)
    for q in rand_states(5, 3):
        F, Gf = orc.flux(G, q)
        nF = c * F + s * Gf
        Tq = q.copy(); Tq[1] = c * q[1] + s * q[2]; Tq[2] = -s * q[1] + c * q[2]
        Fr, _ = orc.flux(G, Tq)
        back = Fr.copy(); back[1] = c * Fr[1] - s * Fr[2]; back[2] = s * Fr[1] + c * Fr[2]
        assert np.allclose(nF, back, rtol=1e-13, atol=1e-13)


def test_homogeneity_identities(orc):
    """F is homogeneous of degree 1: F'(q) q = F(q) and F''(q)(q,q) = 0."""
    for q in rand_states(10, 1):
        F, Gf = orc.flux(G, q)
        F1, G1 = orc.flux_d1(G, q, q)
        F2, G2 = orc.flux_d2(G, q, q)
        assert np.allclose(F1, F, rtol=1e-13, atol=1e-13) and np.allclose(G1, Gf, rtol=1e-13, atol=1e-13)
        assert np.allclose(F2, 0, atol=1e-12) and np.allclose(G2, 0, atol=1e-12)


def test_directional_derivatives_match_finite_differences(orc):
    rng = np.random.default_rng(7)
    for q in rand_states(10, 2):
        w = rng.normal(size=4) * np.abs(q) * 0.3
        h = 1e-4
        Fp, Gp = orc.flux(G, q + h * w); Fm, Gm = orc.flux(G, q - h * w); F0, G0 = orc.flux(G, q)
        F1, G1 = orc.flux_d1(G, q, w)
        F2, G2 = orc.flux_d2(G, q, w)
        sc = 1 + np.abs(F0).max() + np.abs(G0).max()
        assert np.allclose(F1, (Fp - Fm) / (2 * h), atol=1e-7 * sc)
        assert np.allclose(G1, (Gp - Gm) / (2 * h), atol=1e-7 * sc)
        assert np.allclose(F2, (Fp - 2 * F0 + Fm) / h ** 2, atol=1e-5 * sc)
        assert np.allclose(G2, (Gp - 2 * G0 + Gm) / h ** 2, atol=1e-5 * sc)


def test_jacobian_eigenvalues_are_characteristic_speeds(orc):
    """n.F'(q) has eigenvalues u.n - c, u.n, u.n, u.n + c."""
    for q in rand_states(6, 4):
        rho, u, v = q[0], q[1] / q[0], q[2] / q[0]
        p = (G - 1) * (q[3] - 0.5 * rho * (u * u + v * v))
        c = np.sqrt(G * p / rho)
        for ang in (0.0, 0.8, 2.0):
            n = np.array([np.cos(ang), np.sin(ang)])
            A = np.zeros((4, 4))
            for j in range(4):
                e = np.zeros(4); e[j] = 1.0
                F1, G1 = orc.flux_d1(G, q, e)
                A[:, j] = n[0] * F1 + n[1] * G1
            ev = np.sort(np.linalg.eigvals(A).real)
            un = u * n[0] + v * n[1]
            assert np.allclose(ev, np.sort([un - c, un, un, un + c]), atol=1e-10)
