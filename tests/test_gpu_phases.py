"""Phase-by-phase parity of one GPU step with the oracle, on meshes of
several CTAs: moment limiter and wave speed (Sec. 3.1), CK traces and volume
integral (Sec. 2.2-2.3), edge fluxes f^LxW / f^LxF (Sec. 3.3 Step 3), the
blended update (Step 6) and the shock limiter (Sec. 4.1)."""
import numpy as np
import pytest

import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

QUAD, TRI = 0, 1


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


def setup(L, O, kind, deg, n, shock):
    if kind == QUAD:
        X = np.linspace(0.0, 1.0, n + 1)
        om = O.Mesh.cartesian(n, n, bc=(2, 2, 2, 2)); lm = L.lxw_mesh_cartesian(n, n, bc=(2, 2, 2, 2))
        verts = []
        for iy in range(n):
            for ix in range(n):
                verts.append([(X[ix], X[iy]), (X[ix + 1], X[iy]), (X[ix + 1], X[iy + 1]), (X[ix], X[iy + 1])])
        verts = np.array(verts)
    else:
        xy, tv = synth.structured_triangles(n, jitter=0.2, seed=99)
        om = O.Mesh.triangles(xy, tv); lm = L.lxw_mesh_triangles(xy, tv)
        verts = xy[tv]
    os_ = O.Solver(om, deg, shock_limiter=shock)
    ls = L.lxw_solver_create(lm, deg, L.lxw_options_default(shock_limiter=int(shock)),
                             stream=torch.cuda.current_stream())
    E = verts.shape[1]
    nrm = np.stack([verts[:, (np.arange(E) + 1) % E, 1] - verts[:, :, 1],
                    -(verts[:, (np.arange(E) + 1) % E, 0] - verts[:, :, 0])], axis=-1)   # [N][E][2]
    return os_, ls, nrm


@pytest.mark.parametrize("kind,deg", [(QUAD, 2), (QUAD, 3), (TRI, 2), (TRI, 3)])
def test_each_phase_matches_oracle(L, O, kind, deg):
    os_, ls, nrm = setup(L, O, kind, deg, 16 if kind == QUAD else 12, shock=True)
    N, E, ML = os_.N, os_.E, os_.ML
    Q0 = synth.random_modal_state(N, ML, seed=1234, amp=0.3)
    cfl = 0.1
    # phase 1: moment limiter and wave speed
    Ql = Q0.copy(); os_.moment_limit(Ql)
    so = os_.wave_speed(Ql)
    a = os_.mesh.geometry()
    dt = cfl * np.min(2 * a[0] / a[1]) / so
    Qg = torch.from_numpy(Q0.copy()).cuda()
    L.lxw_step_phases(ls, Qg, 0.0, cfl, 1)
    sd = L.lxw_workspace_copy(ls, 3)
    assert abs(sd[0] - so) <= 1e-14 * so and abs(sd[1] - dt) <= 1e-14 * dt
    assert np.abs(Qg.cpu().numpy() - Ql).max() < 1e-13 * np.abs(Q0).max()
    # phase 2: traces (q, n.F_T at edge points) and the volume integral
    Qg = torch.from_numpy(Q0.copy()).cuda()
    L.lxw_step_phases(ls, Qg, 0.0, cfl, 2)
    tr = L.lxw_workspace_copy(ls, 0)                   # [E][MQ][8][N]
    MQ = tr.shape[1]
    NQ = os_.npts - E * MQ
    Qv = Ql.copy()
    for i in range(N):
        ck = os_.ck_element(Ql, i, dt)
        for k in range(E):
            sl = slice(NQ + k * MQ, NQ + (k + 1) * MQ)
            qo = ck["q"][sl]
            Fn = nrm[i, k, 0] * ck["FT"][sl] + nrm[i, k, 1] * ck["GT"][sl]
            sc = np.abs(ck["FT"]).max() + np.abs(ck["GT"]).max() + 1.0
            assert np.abs(tr[k, :, 0:4, i] - qo).max() < 1e-12 * (np.abs(qo).max() + 1), (i, k)
            assert np.abs(tr[k, :, 4:8, i] - Fn).max() < 1e-12 * sc, (i, k)
        Qv[i, :, 1:] += dt / a[0][i] * ck["V"][1:].T
    assert np.abs(Qg.cpu().numpy() - Qv).max() < 1e-12 * np.abs(Q0).max()
    # phases 3-4: edge fluxes and the blended update (oracle step without the shock limiter)
    os2, ls2, _ = setup(L, O, kind, deg, 16 if kind == QUAD else 12, shock=False)
    Qo = Q0.copy(); d = os2.step(Qo, cfl=cfl, want_theta=True)
    fw, ff, dto = os2.last_fluxes()
    Qg = torch.from_numpy(Q0.copy()).cuda()
    L.lxw_step_phases(ls2, Qg, 0.0, cfl, 3)
    fl = L.lxw_workspace_copy(ls2, 1)                  # [E][8][N]
    fs = np.abs(fw).max() + np.abs(ff).max()
    assert np.abs(np.transpose(fl[:, 0:4, :], (2, 0, 1)) - fw).max() < 1e-12 * fs
    assert np.abs(np.transpose(fl[:, 4:8, :], (2, 0, 1)) - ff).max() < 1e-12 * fs
    assert np.abs(Qg.cpu().numpy()[:, :, 1:] - Qo[:, :, 1:]).max() < 1e-12 * np.abs(Q0).max()
    Qg = torch.from_numpy(Q0.copy()).cuda()
    L.lxw_step_phases(ls2, Qg, 0.0, cfl, 4)
    assert np.abs(Qg.cpu().numpy() - Qo).max() < 1e-12 * np.abs(Q0).max()
    # phase 5: shock limiter on top
    Qo = Q0.copy(); os_.step(Qo, cfl=cfl)
    Qg = torch.from_numpy(Q0.copy()).cuda()
    L.lxw_step_phases(ls, Qg, 0.0, cfl, 5)
    assert np.abs(Qg.cpu().numpy() - Qo).max() < 1e-12 * np.abs(Q0).max()
