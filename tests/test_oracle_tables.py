"""Pins of the oracle's quadrature rules and modal basis (Sec. 1.2).

Each check compares against something other than the oracle's own formula:
numpy's Gauss-Legendre and Legendre routines, closed-form monomial integrals,
and orthonormality measured with an independent high-order rule.
"""
import math

import numpy as np
import numpy.polynomial.legendre as npleg
import pytest

QUAD, TRI = 0, 1


@pytest.mark.parametrize("n", [1, 2, 3, 4, 5, 6, 8])
def test_gauss_legendre_matches_numpy(orc, n):
    x, w = orc.gauss_legendre(n)
    xr, wr = npleg.leggauss(n)
    assert np.allclose(x, xr, atol=1e-15, rtol=0)
    assert np.allclose(w, wr, atol=1e-15, rtol=0)
    assert np.array_equal(x, -x[::-1])            # exact mirror symmetry
    # exact for degree 2n-1, not for 2n
    for d in range(2 * n):
        exact = 2.0 / (d + 1) if d % 2 == 0 else 0.0
        assert abs(np.sum(w * x ** d) - exact) < 1e-14
    assert abs(np.sum(w * x ** (2 * n)) - 2.0 / (2 * n + 1)) > 1e-6


@pytest.mark.parametrize("n", [2, 3, 4, 5])
def test_quad_rule_exact_monomials(orc, n):
    xi, eta, w = orc.interior_rule(QUAD, n)
    assert abs(w.sum() - 1.0) < 1e-15
    for a in range(2 * n):
        for b in range(2 * n):
            ex = (2.0 / (a + 1) if a % 2 == 0 else 0.0) * (2.0 / (b + 1) if b % 2 == 0 else 0.0) / 4.0
            assert abs(np.sum(w * xi ** a * eta ** b) - ex) < 1e-14


@pytest.mark.parametrize("n", [2, 3, 4, 5])
def test_triangle_rule_exact_to_degree_2n_minus_2(orc, n):
    xi, eta, w = orc.interior_rule(TRI, n)
    assert abs(w.sum() - 1.0) < 1e-15
    assert np.all(xi >= 0) and np.all(eta >= 0) and np.all(xi + eta <= 1 + 1e-15)
    for a in range(2 * n - 1):
        for b in range(2 * n - 1 - a):
            # (1/|T0|) Int x^a y^b = 2 a! b! / (a+b+2)!
            ex = 2.0 * math.factorial(a) * math.factorial(b) / math.factorial(a + b + 2)
            assert abs(np.sum(w * xi ** a * eta ** b) - ex) < 1e-14, (a, b)


@pytest.mark.parametrize("kind", [QUAD, TRI])
@pytest.mark.parametrize("deg", [1, 2, 3])
def test_basis_orthonormal_and_first_mode_one(orc, kind, deg):
    xi, eta, w = orc.interior_rule(kind, 8)
    phi, dx, dy = orc.basis_eval(kind, deg, xi, eta)
    assert phi.shape[1] == (deg + 1) * (deg + 2) // 2
    G = phi.T @ (w[:, None] * phi)
    assert np.allclose(G, np.eye(phi.shape[1]), atol=1e-13)
    assert np.allclose(phi[:, 0], 1.0, atol=1e-15)       # phi^(1) == 1: Q^(1) is the average
    assert np.allclose(dx[:, 0], 0.0) and np.allclose(dy[:, 0], 0.0)


def test_quad_basis_is_tensor_legendre(orc):
    """Mode order documented for quadrilaterals: 1, L1(x), L1(y), L1L1, L2(x),
    L2(y), L3(x), L2(x)L1(y), L1(x)L2(y), L3(y), with (1/2) Int L_n^2 = 1."""
    rng = np.random.default_rng(1)
    x = rng.uniform(-1, 1, 50); y = rng.uniform(-1, 1, 50)
    phi, dx, dy = orc.basis_eval(QUAD, 3, x, y)
    order = [(0, 0), (1, 0), (0, 1), (1, 1), (2, 0), (0, 2), (3, 0), (2, 1), (1, 2), (0, 3)]
    for l, (a, b) in enumerate(order):
        ca = np.zeros(a + 1); ca[a] = math.sqrt(2 * a + 1)
        cb = np.zeros(b + 1); cb[b] = math.sqrt(2 * b + 1)
        ref = npleg.legval(x, ca) * npleg.legval(y, cb)
        rdx = npleg.legval(x, npleg.legder(ca)) * npleg.legval(y, cb)
        rdy = npleg.legval(x, ca) * npleg.legval(y, npleg.legder(cb))
        assert np.allclose(phi[:, l], ref, atol=1e-13)
        assert np.allclose(dx[:, l], rdx, atol=1e-12)
        assert np.allclose(dy[:, l], rdy, atol=1e-12)


def test_triangle_basis_hierarchical_and_gradients(orc):
    """Gram-Schmidt order: phi_l lies in span(1, x, y, x^2, ...)[:l+1]; its
    gradient matches central differences."""
    rng = np.random.default_rng(2)
    u = rng.uniform(0, 1, 80); v = rng.uniform(0, 1, 80)
    x = np.where(u + v <= 1, u, 1 - u); y = np.where(u + v <= 1, v, 1 - v)
    phi, dx, dy = orc.basis_eval(TRI, 3, x, y)
    mono = [(0, 0), (1, 0), (0, 1), (2, 0), (1, 1), (0, 2), (3, 0), (2, 1), (1, 2), (0, 3)]
    M = np.stack([x ** a * y ** b for a, b in mono], axis=1)
    for l in range(10):
        c, res, *_ = np.linalg.lstsq(M[:, : l + 1], phi[:, l], rcond=None)
        assert np.allclose(M[:, : l + 1] @ c, phi[:, l], atol=1e-10)
        assert c[-1] > 0                                  # positive leading coefficient
    h = 1e-6
    pp, _, _ = orc.basis_eval(TRI, 3, x + h, y); pm, _, _ = orc.basis_eval(TRI, 3, x - h, y)
    assert np.allclose((pp - pm) / (2 * h), dx, atol=1e-6)
    pp, _, _ = orc.basis_eval(TRI, 3, x, y + h); pm, _, _ = orc.basis_eval(TRI, 3, x, y - h)
    assert np.allclose((pp - pm) / (2 * h), dy, atol=1e-6)
