"""The mixed 3D forms (precision = LXW_PREC_MIXED on hexahedra and on
tetrahedra): the Cauchy-Kovalevskaya kernel in FP32, the state, averages,
face fluxes and all limiters in FP64.

Budget: the FP32 kernel's traces and volume terms carry a relative rounding
of ~1e-7, which enters the averages through the face fluxes times the CFL
number and the higher moments through dt times the volume term, so one step
agrees with the FP64 oracle to ~1e-7 relative L1.  The moment limiter's
FP32 screen clears a cell only when its FP64 values provably clear the
thresholds, so its decisions equal the oracle's; the wave speed of cleared
cells is the FP32 one (s, and dt, to ~1e-7).  Conservation is exact (both
cells of a face use the same stored traces).
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


def solvers(L, O, kind, deg, mixed=True, **opt):
    o = L.lxw_options_default(precision=L.PREC_MIXED if mixed else L.PREC_FP64)
    for k, v in opt.items():
        setattr(o, k, v)
    st = torch.cuda.current_stream()
    if kind == "hex":
        n3, box, bc = (7, 6, 5), (0.0, 1.0, 0.0, 1.0, 0.0, 1.0), (1,) * 6   # walls: totals conserved exactly
        s = L.lxw3_solver_create(*n3, box, bc, deg, o, stream=st)
        so = O.Solver3(O.Mesh3(*n3, box, bc), deg, gamma=G, alpha0=o.alpha0, shock_limiter=bool(o.shock_limiter))
    else:
        xyz, tets, vid = synth.tet_mesh(5, jitter=0.2, seed=9)
        fbc = np.full((len(tets), 4), 1, dtype=np.int32)
        s = L.lxw3_solver_create_tets(xyz, tets, vid, deg, face_bc=fbc, options=o, stream=st)
        so = O.Solver3(O.Mesh3.tets(xyz, tets, vid, fbc), deg, gamma=G, alpha0=o.alpha0,
                       shock_limiter=bool(o.shock_limiter))
    return s, so


def rel(a, b):
    return float(np.abs(a - b).sum() / np.abs(b).sum())


@pytest.mark.parametrize("kind", ["hex", "tet"])
@pytest.mark.parametrize("deg", [1, 2])
def test_one_step_near_vacuum_against_oracle(L, O, kind, deg):
    """Near-vacuum random data with every limiter acting: the moment-limiter
    count equals the oracle's, s agrees to 1e-6, the state to 1e-6 relative
    L1, totals of mass and energy to 1e-12."""
    s, so = solvers(L, O, kind, deg, alpha0=50.0)
    Q0 = synth.random_modal_state3(s.N, s.ML, seed=500 + deg, amp=0.3, rho_range=(0.01, 2.0), p_range=(0.005, 2.0))
    Qo = Q0.copy()
    do = so.step(Qo, cfl=0.4)
    Q = torch.from_numpy(Q0).cuda()
    d = L.lxw3_step(s, Q, 0.0, 0.4, diag=True)
    assert d["status"] == 0 and d["min_rho"] > 0 and d["min_p"] > 0
    assert d["n_mom"] == do["n_mom"] > 0
    assert abs(d["s"] / do["s"] - 1) < 1e-6
    assert rel(Q.cpu().numpy(), Qo) < 1e-6
    assert abs(d["mass"] - do["mass"]) < 1e-12 * abs(do["mass"])
    assert abs(d["energy"] - do["energy"]) < 1e-12 * abs(do["energy"])


@pytest.mark.parametrize("kind", ["hex", "tet"])
def test_walled_blast_positive_and_conservative(L, O, kind):
    """20 graph-replayed steps of a point-energy blast with walls: positive
    averages, mass and energy conserved to 1e-12, and within 1e-4 (relative
    L1) of the FP64 GPU form, whose limiter decisions it may flip where a
    proposal sits on a threshold."""
    s, _ = solvers(L, O, kind, 2)
    s64, so = solvers(L, O, kind, 2, mixed=False)

    def ic(x, y, z):
        r2 = (x - 0.5) ** 2 + (y - 0.5) ** 2 + (z - 0.5) ** 2
        return (1.0 + 0 * x, 0 * x, 0 * x, 0 * x, np.where(r2 < 0.04, 40.0, 0.1))
    Q0 = so.project_fn(ic)
    vol = so.mesh.geometry()[0]
    m0, e0 = (vol * Q0[:, 0, 0]).sum(), (vol * Q0[:, 4, 0]).sum()
    Q = torch.from_numpy(Q0.copy()).cuda()
    Q64 = Q.clone()
    d = L.lxw3_run(s, Q, 20, 0.2, diag=True)
    L.lxw3_run(s64, Q64, 20, 0.2)
    assert d["status"] == 0 and d["min_rho"] > 0 and d["min_p"] > 0
    assert abs(d["mass"] - m0) < 1e-12 * m0 and abs(d["energy"] - e0) < 1e-12 * e0
    assert rel(Q.cpu().numpy(), Q64.cpu().numpy()) < 1e-4


@pytest.mark.parametrize("kind", ["hex", "tet"])
def test_equal_error_on_smooth_advection(L, O, kind):
    """The smooth periodic 3D advection (rho = 1 + 0.2 sin 2 pi (x + y + z),
    u = (1, 0.5, 0.25), p = 1) to t = 0.05: the mixed form's L2 density error
    equals the FP64 form's within 0.1 %."""
    U = np.array([1.0, 0.5, 0.25])
    ex = lambda x, y, z, t: 1 + 0.2 * np.sin(2 * np.pi * ((x - U[0] * t) + (y - U[1] * t) + (z - U[2] * t)))  # noqa: E731
    errs = {}
    for mixed in (False, True):
        o = L.lxw_options_default(precision=L.PREC_MIXED if mixed else L.PREC_FP64)
        if kind == "hex":
            s = L.lxw3_solver_create(10, 10, 10, (0.0, 1.0) * 3, (0,) * 6, 2, o, stream=torch.cuda.current_stream())
            vol = np.full(s.N, 1e-3)
        else:
            xyz, tets, vid = synth.tet_mesh(6, periodic=True)
            s = L.lxw3_solver_create_tets(xyz, tets, vid, 2, options=o, stream=torch.cuda.current_stream())
            vol = np.full(s.N, 1.0 / s.N)
        P = L.lxw3_projection_points(s)
        prim = np.stack(np.broadcast_arrays(ex(P[..., 0], P[..., 1], P[..., 2], 0.0), U[0], U[1], U[2], 1.0), axis=-1)
        Q = torch.zeros(s.state_shape, dtype=torch.float64, device="cuda")
        L.lxw3_project(s, torch.from_numpy(prim.copy()).cuda(), Q)
        t = 0.0
        while t < 0.05 - 1e-14:
            Qc = Q.clone()
            d = L.lxw3_step(s, Qc, 0.0, 0.2, diag=True)
            if t + d["dt"] >= 0.05:
                L.lxw3_step(s, Q, 0.05 - t, 0.0)
                t = 0.05
            else:
                Q = Qc
                t += d["dt"]
        # L2 error of the density from the modal coefficients' projection of the exact solution
        prim_e = np.stack(np.broadcast_arrays(ex(P[..., 0], P[..., 1], P[..., 2], 0.05), U[0], U[1], U[2], 1.0), axis=-1)
        Qe = torch.zeros(s.state_shape, dtype=torch.float64, device="cuda")
        L.lxw3_project(s, torch.from_numpy(prim_e.copy()).cuda(), Qe)
        diff = (Q[:, 0, :] - Qe[:, 0, :]).cpu().numpy()
        errs[mixed] = float(np.sqrt((vol[:, None] * diff ** 2).sum()))
    assert abs(errs[True] / errs[False] - 1) < 1e-3, errs
