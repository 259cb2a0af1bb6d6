"""The 3D Cartesian FP64 form (lxw3_*) against the 3D oracle.

The GPU kernels and the oracle derive the flux derivatives independently
(hand-derived Jacobian products on the GPU, Taylor-series arithmetic in the
oracle) and sum in different orders, so FP64 states agree to round-off:
1e-13 relative per step, amplified by the limiters' discontinuous decisions
only when one flips (the tests count the decisions on both sides).
"""
import numpy as np
import pytest

import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
G = 1.4


@pytest.fixture(scope="module")
def L():
    if not torch.cuda.is_available():
        pytest.fail("GPU tests need CUDA")
    from paper_1601_08145_gb300 import build
    build.build()
    from paper_1601_08145_gb300 import lxw
    return lxw


@pytest.fixture(scope="module")
def O():
    from oracle import oracle
    oracle.lib()
    return oracle


def pair(L, O, n3, box, bc, deg, **opt):
    o = L.lxw_options_default()
    for k, v in opt.items():
        setattr(o, k, v)
    s = L.lxw3_solver_create(*n3, box, bc, deg, o, stream=torch.cuda.current_stream())
    so = O.Solver3(O.Mesh3(*n3, box, bc), deg, gamma=G, alpha0=o.alpha0, shock_limiter=bool(o.shock_limiter),
                   llf_global=bool(o.llf_global))
    assert s.N == so.N and s.ML == so.ML and s.nproj == so.nproj
    return s, so


def rel(a, b):
    return float(np.abs(a - b).sum() / np.abs(b).sum())


def test_projection_matches_oracle(L, O):
    box = (0.0, 1.0, -0.5, 0.5, 0.0, 0.7)
    for deg in (1, 2):
        s, so = pair(L, O, (5, 4, 3), box, (0, 0, 1, 1, 2, 2), deg)
        xyz = L.lxw3_projection_points(s)
        assert np.allclose(xyz, so.projection_points(), rtol=0, atol=1e-14)
        fn = lambda x, y, z: (1 + 0.3 * np.sin(3 * x) * np.cos(2 * y + z), 0.2 + x * y, -0.1 * z, 0.3 * np.cos(x),  # noqa: E731
                              1.0 + 0.2 * y * y)
        vals = fn(xyz[..., 0], xyz[..., 1], xyz[..., 2])
        prim = torch.from_numpy(np.stack(np.broadcast_arrays(*vals), axis=-1).copy()).cuda()
        Q = torch.zeros(s.state_shape, dtype=torch.float64, device="cuda")
        L.lxw3_project(s, prim, Q)
        assert np.allclose(Q.cpu().numpy(), so.project_fn(fn), rtol=1e-13, atol=1e-14)


@pytest.mark.parametrize("deg,n3,bc,llf", [(1, (7, 5, 6), (2, 2, 1, 1, 0, 0), 0), (2, (5, 6, 7), (1, 1, 0, 0, 2, 2), 0),
                                           (2, (4, 3, 5), (0, 0, 0, 0, 0, 0), 1)])
def test_one_step_with_every_limiter_against_oracle(L, O, deg, n3, bc, llf):
    """Random near-vacuum data (N not a multiple of the block): the moment,
    flux and shock limiters act; the state, s, dt, the face thetas and the
    limiter counts match the oracle."""
    box = (0.0, 1.0, 0.0, 1.2, -0.3, 0.6)
    s, so = pair(L, O, n3, box, bc, deg, alpha0=50.0, llf_global=llf)
    assert s.N % 128 != 0
    Q0 = synth.random_modal_state3(s.N, s.ML, seed=300 + deg, amp=0.3, rho_range=(0.01, 2.0), p_range=(0.005, 2.0))
    Qo = Q0.copy()
    do = so.step(Qo, cfl=0.6, want_theta=True)
    Q = torch.from_numpy(Q0).cuda()
    tf = torch.zeros((s.N, 6), dtype=torch.float64, device="cuda")
    d = L.lxw3_step(s, Q, 0.0, 0.6, diag=True, theta_face=tf)
    assert d["status"] == do["status"]
    assert abs(d["s"] / do["s"] - 1) < 1e-14 and abs(d["dt"] / do["dt"] - 1) < 1e-14
    assert do["n_mom"] > 0 and do["n_sc"] > 0
    for k in ("n_mom", "n_face", "n_sc"):
        assert d[k] == do[k], (k, d[k], do[k])
    Qg = Q.cpu().numpy()
    assert rel(Qg, Qo) < 1e-12
    sc = np.abs(Qo).max(axis=0, keepdims=True) + 1e-12
    assert (np.abs(Qg - Qo) / sc).max() < 1e-10
    assert np.abs(tf.cpu().numpy() - do["theta_face"]).max() < 1e-9
    for key, k in (("mass", 0), ("momx", 1), ("momy", 2), ("momz", 3), ("energy", 4)):
        vol = so.mesh.geometry()[0]
        assert abs(d[key] - (vol * Qo[:, k, 0]).sum()) <= 1e-12 * (1 + abs(d[key]))


def test_flux_limiter_acts_and_matches(L, O):
    """The literal global dissipation speed at a large CFL number wakes the
    six-face flux limiter; its counts and the state match the oracle."""
    s, so = pair(L, O, (6, 5, 4), (0, 1, 0, 1, 0, 1), (2,) * 6, 2, llf_global=1)
    Q0 = synth.random_modal_state3(s.N, s.ML, seed=77, amp=0.3, rho_range=(0.01, 2.0), p_range=(0.005, 2.0))
    Qo = Q0.copy()
    do = so.step(Qo, cfl=1.5)
    Q = torch.from_numpy(Q0).cuda()
    d = L.lxw3_step(s, Q, 0.0, 1.5, diag=True)
    assert do["n_face"] > 0 and d["n_face"] == do["n_face"]
    assert rel(Q.cpu().numpy(), Qo) < 1e-12


def test_blast_multi_step_and_run(L, O):
    """A point-energy blast in a walled box, 12 steps: the GPU (graph-replayed
    lxw3_run and single lxw3_step calls, bit for bit the same) against the
    oracle, and mass conserved to round-off."""
    n = 9
    box = (-1.0, 1.0, -1.0, 1.0, -1.0, 1.0)
    s, so = pair(L, O, (n, n, n), box, (1,) * 6, 2)

    def ic(x, y, z):
        r2 = x * x + y * y + z * z
        return (1.0 + 0 * x, 0 * x, 0 * x, 0 * x, np.where(r2 < 0.09, 40.0, 0.1))
    Qo = so.project_fn(ic)
    Q = torch.from_numpy(Qo.copy()).cuda()
    Q2 = Q.clone()
    for _ in range(12):
        do = so.step(Qo, cfl=0.2)
    L.lxw3_run(s, Q, 12, 0.2)
    for _ in range(12):
        d = L.lxw3_step(s, Q2, 0.0, 0.2, diag=True)
    assert torch.equal(Q, Q2)
    assert d["status"] == 0 and d["min_p"] > 0 and do["n_mom"] + do["n_sc"] > 0
    assert rel(Q.cpu().numpy(), Qo) < 1e-11
    vol = so.mesh.geometry()[0]
    assert abs(d["mass"] - (vol * so.project_fn(ic)[:, 0, 0]).sum()) < 1e-12
    assert L.lxw3_step_launches(s) == 6


def test_full_size_step_against_oracle(L, O):
    """48^3 P2 cells (110,592) from near-vacuum random data, one step."""
    s, so = pair(L, O, (48, 48, 48), (0, 1, 0, 1, 0, 1), (0,) * 6, 2)
    Q0 = synth.random_modal_state3(s.N, s.ML, seed=4848, amp=0.3, rho_range=(0.01, 2.0), p_range=(0.005, 2.0))
    Qo = Q0.copy()
    do = so.step(Qo, cfl=0.4)
    Q = torch.from_numpy(Q0).cuda()
    d = L.lxw3_step(s, Q, 0.0, 0.4, diag=True)
    assert do["n_mom"] > 0 and d["n_mom"] == do["n_mom"] and d["n_sc"] == do["n_sc"]
    assert rel(Q.cpu().numpy(), Qo) < 1e-12
    ms = L.lxw3_profile_step(s, Q, 0.4)
    assert set(ms) == {"moment", "ck", "face", "update", "shock"} and all(v > 0 for v in ms.values())
