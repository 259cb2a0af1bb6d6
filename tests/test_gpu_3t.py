"""The tetrahedral FP64 form (lxw3_solver_create_tets + lxw3_*) against the
3D oracle on the same meshes.

As for the hexahedra, the GPU kernels and the oracle derive the flux
derivatives independently and sum in different orders, and the GPU builds
its own rules, basis (Cholesky of the exact Gram matrix against the oracle's
Gram-Schmidt) and face tables: FP64 states agree to round-off, amplified by
the limiters' discontinuous decisions only when one flips (the tests count
the decisions on both sides).
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


def pair(L, O, n, deg, periodic=False, jitter=0.0, bc=2, seed=1, walls=None, permute=False, **opt):
    """GPU and oracle solvers on one Kuhn mesh of 6 n^3 cells; bc: the code of
    every unmatched face, or walls: a function of the face centroid's
    position giving it per face; permute renumbers each cell's vertices."""
    xyz, tets, vid = synth.tet_mesh(n, periodic=periodic, jitter=jitter, seed=seed, permute=permute)
    fbc = np.full((len(tets), 4), bc, dtype=np.int32)
    if walls is not None:
        for i, t in enumerate(tets):
            for k in range(4):
                fbc[i, k] = walls(xyz[np.delete(t, k)].mean(axis=0))
    o = L.lxw_options_default()
    for k, v in opt.items():
        setattr(o, k, v)
    s = L.lxw3_solver_create_tets(xyz, tets, vid, deg, face_bc=fbc, options=o, stream=torch.cuda.current_stream())
    so = O.Solver3(O.Mesh3.tets(xyz, tets, vid, fbc), deg, gamma=G, alpha0=o.alpha0,
                   shock_limiter=bool(o.shock_limiter), llf_global=bool(o.llf_global))
    assert s.N == so.N == 6 * n ** 3 and s.ML == so.ML and s.nproj == so.nproj and s.E == 4
    return s, so


def rel(a, b):
    return float(np.abs(a - b).sum() / np.abs(b).sum())


def test_projection_matches_oracle(L, O):
    for deg in (1, 2):
        s, so = pair(L, O, 3, deg, jitter=0.2)
        xyz = L.lxw3_projection_points(s)
        assert np.allclose(xyz, so.projection_points(), rtol=0, atol=1e-14)
        fn = lambda x, y, z: (1 + 0.3 * np.sin(3 * x) * np.cos(2 * y + z), 0.2 + x * y, -0.1 * z, 0.3 * np.cos(x),  # noqa: E731
                              1.0 + 0.2 * y * y)
        vals = fn(xyz[..., 0], xyz[..., 1], xyz[..., 2])
        prim = torch.from_numpy(np.stack(np.broadcast_arrays(*vals), axis=-1).copy()).cuda()
        Q = torch.zeros(s.state_shape, dtype=torch.float64, device="cuda")
        L.lxw3_project(s, prim, Q)
        assert np.allclose(Q.cpu().numpy(), so.project_fn(fn), rtol=1e-13, atol=1e-14)


def test_step_exact_for_advected_quadratic(L, O):
    """A quadratic density advected at constant velocity and pressure stays
    in P2 and is quadratic in t: one GPU step reproduces the projection of
    the exact solution (a check of the geometry, the face pairing and the
    CK terms that needs no oracle)."""
    s, _ = pair(L, O, 3, 2, jitter=0.2, bc=2, seed=4, shock_limiter=0)
    U = np.array([0.7, -0.4, 0.3]); P = 1.1
    rho0 = lambda x, y, z: 1.0 + 0.3 * x - 0.2 * y + 0.1 * z + 0.4 * x * x + 0.1 * x * y - 0.3 * y * z + 0.2 * z * z  # noqa: E731
    xyz = torch.from_numpy(L.lxw3_projection_points(s)).cuda()

    def proj(t):
        x, y, z = xyz[..., 0] - U[0] * t, xyz[..., 1] - U[1] * t, xyz[..., 2] - U[2] * t
        prim = torch.stack([rho0(x, y, z), 0 * x + U[0], 0 * x + U[1], 0 * x + U[2], 0 * x + P], dim=-1).contiguous()
        Q = torch.zeros(s.state_shape, dtype=torch.float64, device="cuda")
        L.lxw3_project(s, prim, Q)
        return Q
    for dt in (0.01, 0.03):
        Q = proj(0.0)
        d = L.lxw3_step(s, Q, dt, 0.0, diag=True)
        assert d["n_mom"] == 0 and d["n_face"] == 0
        assert (Q - proj(dt)).abs().max().item() < 5e-14


@pytest.mark.parametrize("deg,n,periodic,llf", [(1, 5, False, 0), (2, 5, False, 0), (2, 3, True, 1)])
def test_one_step_with_every_limiter_against_oracle(L, O, deg, n, periodic, llf):
    """Random near-vacuum data on jittered (or periodic) meshes whose sides
    are walls below x = 1/2 and transparent above: the moment, flux and
    shock limiters act; state, s, dt, face thetas and counts match.  s and
    dt agree to 1e-12 relative rather than the hexahedra's 1e-14: the
    tetrahedral basis values carry the rounding of the Gram-Schmidt
    coefficients (entries up to ~30 at P2), and |u| + c at densities of 0.01
    amplifies it."""
    walls = None if periodic else (lambda c: 1 if c[0] < 0.5 else 2)
    s, so = pair(L, O, n, deg, periodic=periodic, jitter=0.0 if periodic else 0.2, walls=walls, alpha0=50.0,
                 llf_global=llf)
    assert s.N % 128 != 0
    Q0 = synth.random_modal_state3(s.N, s.ML, seed=400 + deg, amp=0.3, rho_range=(0.01, 2.0), p_range=(0.005, 2.0))
    Qo = Q0.copy()
    do = so.step(Qo, cfl=0.5, want_theta=True)
    Q = torch.from_numpy(Q0).cuda()
    tf = torch.zeros((s.N, 4), dtype=torch.float64, device="cuda")
    d = L.lxw3_step(s, Q, 0.0, 0.5, diag=True, theta_face=tf)
    assert d["status"] == do["status"]
    assert abs(d["s"] / do["s"] - 1) < 1e-12 and abs(d["dt"] / do["dt"] - 1) < 1e-12
    assert do["n_mom"] > 0 and do["n_sc"] > 0
    for k in ("n_mom", "n_face", "n_sc"):
        assert d[k] == do[k], (k, d[k], do[k])
    Qg = Q.cpu().numpy()
    assert rel(Qg, Qo) < 1e-12
    sc = np.abs(Qo).max(axis=0, keepdims=True) + 1e-12
    assert (np.abs(Qg - Qo) / sc).max() < 1e-10
    assert np.abs(tf.cpu().numpy() - do["theta_face"]).max() < 1e-9
    vol = so.mesh.geometry()[0]
    for key, k in (("mass", 0), ("momx", 1), ("momy", 2), ("momz", 3), ("energy", 4)):
        assert abs(d[key] - (vol * Qo[:, k, 0]).sum()) <= 1e-12 * (1 + abs(d[key]))


def test_flux_limiter_acts_and_matches(L, O):
    """The literal global dissipation speed at a large CFL number wakes the
    four-face flux limiter; its counts and the state match the oracle."""
    s, so = pair(L, O, 4, 2, jitter=0.15, bc=2, llf_global=1)
    Q0 = synth.random_modal_state3(s.N, s.ML, seed=78, amp=0.3, rho_range=(0.01, 2.0), p_range=(0.005, 2.0))
    Qo = Q0.copy()
    do = so.step(Qo, cfl=1.2)
    Q = torch.from_numpy(Q0).cuda()
    d = L.lxw3_step(s, Q, 0.0, 1.2, diag=True)
    assert do["n_face"] > 0 and d["n_face"] == do["n_face"]
    assert rel(Q.cpu().numpy(), Qo) < 1e-12


def test_blast_multi_step_and_run(L, O):
    """A point-energy blast in a walled box of jittered tetrahedra, 10 steps:
    graph-replayed lxw3_run and single lxw3_step calls agree bit for bit, the
    oracle to round-off, mass is conserved."""
    s, so = pair(L, O, 5, 2, jitter=0.15, bc=1)

    def ic(x, y, z):
        r2 = (x - 0.5) ** 2 + (y - 0.5) ** 2 + (z - 0.5) ** 2
        return (1.0 + 0 * x, 0 * x, 0 * x, 0 * x, np.where(r2 < 0.04, 40.0, 0.1))
    Qo = so.project_fn(ic)
    Q = torch.from_numpy(Qo.copy()).cuda()
    Q2 = Q.clone()
    for _ in range(10):
        do = so.step(Qo, cfl=0.2)
    L.lxw3_run(s, Q, 10, 0.2)
    for _ in range(10):
        d = L.lxw3_step(s, Q2, 0.0, 0.2, diag=True)
    assert torch.equal(Q, Q2)
    assert d["status"] == 0 and d["min_p"] > 0 and do["n_mom"] + do["n_sc"] > 0
    assert rel(Q.cpu().numpy(), Qo) < 1e-11
    vol = so.mesh.geometry()[0]
    assert abs(d["mass"] - (vol * so.project_fn(ic)[:, 0, 0]).sum()) < 1e-12
    assert L.lxw3_step_launches(s) == 6


def test_full_size_step_against_oracle(L, O):
    """24^3 boxes = 82,944 periodic P2 tetrahedra from near-vacuum random
    data, one step."""
    s, so = pair(L, O, 24, 2, periodic=True)
    Q0 = synth.random_modal_state3(s.N, s.ML, seed=2424, amp=0.3, rho_range=(0.01, 2.0), p_range=(0.005, 2.0))
    Qo = Q0.copy()
    do = so.step(Qo, cfl=0.4)
    Q = torch.from_numpy(Q0).cuda()
    d = L.lxw3_step(s, Q, 0.0, 0.4, diag=True)
    assert do["n_mom"] > 0 and d["n_mom"] == do["n_mom"] and d["n_sc"] == do["n_sc"]
    assert rel(Q.cpu().numpy(), Qo) < 1e-12
    ms = L.lxw3_profile_step(s, Q, 0.4)
    assert set(ms) == {"moment", "ck", "face", "update", "shock"} and all(v > 0 for v in ms.values())


@pytest.mark.parametrize("deg,periodic", [(1, False), (2, False), (2, True)])
def test_renumbered_cells_against_oracle(L, O, deg, periodic):
    """Cells whose vertices are renumbered by random even permutations, so
    that the two cells of a face list its vertices in unrelated orders and
    every one of the six face-point tables per face is used: one step from
    near-vacuum random data with the limiters acting matches the oracle (and
    the advected quadratic stays exact on the GPU)."""
    walls = None if periodic else (lambda c: 1 if c[2] < 0.5 else 2)
    s, so = pair(L, O, 5 if not periodic else 3, deg, periodic=periodic, jitter=0.0 if periodic else 0.2,
                 walls=walls, permute=True, alpha0=50.0, seed=11)
    Q0 = synth.random_modal_state3(s.N, s.ML, seed=600 + deg, amp=0.3, rho_range=(0.01, 2.0), p_range=(0.005, 2.0))
    Qo = Q0.copy()
    do = so.step(Qo, cfl=0.5, want_theta=True)
    Q = torch.from_numpy(Q0).cuda()
    tf = torch.zeros((s.N, 4), dtype=torch.float64, device="cuda")
    d = L.lxw3_step(s, Q, 0.0, 0.5, diag=True, theta_face=tf)
    assert d["status"] == do["status"] and do["n_mom"] > 0
    for k in ("n_mom", "n_face", "n_sc"):
        assert d[k] == do[k], (k, d[k], do[k])
    assert rel(Q.cpu().numpy(), Qo) < 1e-12
    assert np.abs(tf.cpu().numpy() - do["theta_face"]).max() < 1e-9
