"""Pins of the oracle's learned-indicator network (FP64): the gradient
against central finite differences and the loss against its definition on a
network whose output is constant."""
import numpy as np


def test_mlp_gradient_matches_finite_differences(orc):
    rng = np.random.default_rng(0)
    P = rng.normal(size=orc.MLP_PARAMS) * 0.2
    X = rng.normal(size=(7, 24))
    y = rng.uniform(0, 1, size=7)
    loss, g, _ = orc.mlp_loss_grad(P, X, y)
    h = 1e-6
    idx = np.concatenate([rng.integers(0, orc.MLP_PARAMS, 60), [orc.MLP_PARAMS - 1]])
    for k in idx:
        Pp = P.copy(); Pp[k] += h
        Pm = P.copy(); Pm[k] -= h
        fd = (orc.mlp_loss_grad(Pp, X, y)[0] - orc.mlp_loss_grad(Pm, X, y)[0]) / (2 * h)
        assert abs(fd - g[k]) < 1e-7 * (1 + abs(g[k])), (k, fd, g[k])


def test_mlp_constant_network_loss():
    """All weights zero: the output is sigmoid(b3) for every input."""
    from oracle import oracle as orc
    P = np.zeros(orc.MLP_PARAMS); P[-1] = 0.7
    y = np.array([0.1, 0.9, 0.5])
    loss, g, yh = orc.mlp_loss_grad(P, np.ones((3, 24)), y)
    s = 1 / (1 + np.exp(-0.7))
    assert np.allclose(yh, s)
    assert abs(loss - np.mean((s - y) ** 2)) < 1e-15
    assert abs(g[-1] - np.mean(2 * (s - y) * s * (1 - s))) < 1e-15


def test_features_of_flat_and_sheared_cells(orc):
    """A flat state has only its energy-fraction and alpha features; the
    neighbour features see a density jump."""
    n = 40
    sol = orc.Solver(orc.Mesh.cartesian(n, n), 2)
    Q = sol.new_state()
    Q[:, 0, 0] = 1.0; Q[:, 3, 0] = 2.5            # rho = 1, u = 0, p = 1
    F = sol.features(Q)
    assert np.allclose(F[:, :22], 0.0)
    assert np.allclose(F[:, 22], 500.0 * (1.0 / n) ** 1.5)      # alpha / rho (below the clip at 8)
    assert np.allclose(F[:, 23], 1.0)
    Q[:n, 0, 0] = 2.0; Q[:n, 3, 0] = 2.5          # bottom row denser
    F = sol.features(Q)
    i = n + 1                                     # a cell of the second row
    assert abs(F[i, 14] - 1.0) < 1e-15            # bottom neighbour: rho_j/rho - 1 = 1
