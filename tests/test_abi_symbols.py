"""CPU checks of the C ABI library: it builds, loads without a GPU, and
exports every entry point include/lxw.h declares (no compute calls)."""
import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    src = open(os.path.join(ROOT, "include", "lxw.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = set(re.findall(r"\b(lxw3?_[a-z_0-9]+)\s*\(", src))
    return sorted(names)


@pytest.fixture(scope="module")
def libpath():
    from paper_1601_08145_gb300 import build
    return build.build()


def test_every_declared_symbol_is_exported(libpath):
    L = ctypes.CDLL(libpath)
    names = declared_symbols()
    assert len(names) >= 15
    for n in names:
        assert hasattr(L, n), n


def test_binding_covers_the_header():
    from paper_1601_08145_gb300 import lxw
    assert sorted(lxw.EXPORTS) == declared_symbols()


def test_host_side_errors_without_gpu(libpath):
    """Argument validation happens on the host and needs no device."""
    from paper_1601_08145_gb300 import lxw
    with pytest.raises(lxw.LxwError) as e:
        lxw.lxw_mesh_cartesian(0, 4)
    assert e.value.code == lxw.ERR_ARG
    with pytest.raises(lxw.LxwError) as e:
        lxw.lxw_mesh_cartesian(4, 4, bc=(lxw.BC_PERIODIC, lxw.BC_REFLECT, 0, 0))
    assert e.value.code == lxw.ERR_ARG
    import numpy as np
    xy = np.array([[0, 0], [1, 0], [0, 1]], dtype=float)
    with pytest.raises(lxw.LxwError) as e:
        lxw.lxw_mesh_triangles(xy, np.array([[0, 2, 1]]))       # clockwise
    assert e.value.code == lxw.ERR_ARG
    with pytest.raises(lxw.LxwError) as e:
        lxw.lxw_mesh_triangles(xy, np.array([[0, 1, 5]]))
    assert e.value.code == lxw.ERR_BOUNDS
    m = lxw.lxw_mesh_cartesian(3, 2)
    assert m.N == 6
    o = lxw.lxw_options_default()
    assert o.gamma == 1.4 and o.eps0 == 1e-12 and o.alpha0 == 500.0 and o.shock_limiter == 1


@pytest.mark.parametrize("kind,deg", [(0, 2), (0, 3), (1, 2), (1, 3)])
def test_basis_eval_matches_the_oracle_basis(kind, deg):
    """lxw_basis_eval (host only, no GPU) against the oracle's independently
    built basis (long-double Gram-Schmidt vs the library's Cholesky for
    triangles) at random reference points."""
    from oracle import oracle as orc
    from paper_1601_08145_gb300 import lxw as L
    rng = np.random.default_rng(3 + kind + deg)
    if kind == 0:
        ref = rng.uniform(-1.0, 1.0, size=(200, 2))
    else:
        ref = rng.uniform(0.0, 1.0, size=(400, 2))
        ref = ref[ref.sum(axis=1) <= 1.0][:200]
    phi = L.lxw_basis_eval(kind, deg, ref)
    po = orc.basis_eval(kind, deg, ref[:, 0].copy(), ref[:, 1].copy())[0]
    assert phi.shape == po.shape
    assert np.abs(phi - po).max() < 1e-12


def test_masked_mesh_and_boundary_codes_host_side(libpath):
    """The mesh builders run on the host: masked grids keep the cells of the
    mask (row order) and reject bad codes; triangle meshes accept the inflow
    code on boundary edges and reject unknown ones."""
    import numpy as np
    import synth
    from paper_1601_08145_gb300 import lxw
    mask = synth.diffraction_mask(39, 33)
    m = lxw.lxw_mesh_cartesian_masked(39, 33, synth.DIFFRACTION_BOX, synth.DIFFRACTION_BC, mask)
    assert m.N == int(mask.sum()) == 39 * 33 - 3 * 18
    full = lxw.lxw_mesh_cartesian_masked(5, 4, (0, 1, 0, 1), (0, 0, 1, 1), np.ones((4, 5), bool))
    assert full.N == 20
    for bad in (dict(mask_bc=0), dict(mask_bc=4)):
        with pytest.raises(lxw.LxwError) as e:
            lxw.lxw_mesh_cartesian_masked(5, 4, (0, 1, 0, 1), (2, 2, 2, 2), np.ones((4, 5), bool), **bad)
        assert e.value.code == lxw.ERR_ARG
    with pytest.raises(lxw.LxwError) as e:
        lxw.lxw_mesh_cartesian(4, 4, bc=(4, 2, 2, 2))
    assert e.value.code == lxw.ERR_ARG
    xy, tv = synth.structured_triangles(4, jitter=0.2, seed=1)
    t = lxw.lxw_mesh_triangles(xy, tv, np.full((len(tv), 3), lxw.BC_INFLOW, np.int32))
    assert t.N == len(tv)
    with pytest.raises(lxw.LxwError) as e:
        lxw.lxw_mesh_triangles(xy, tv, np.full((len(tv), 3), 7, np.int32))
    assert e.value.code == lxw.ERR_ARG


def test_3d_argument_errors_without_gpu(libpath):
    """The 3D solver validates its arguments on the host, before any CUDA call."""
    from paper_1601_08145_gb300 import lxw
    box = (0.0, 1.0, 0.0, 1.0, 0.0, 1.0)
    bad = [dict(nx=0), dict(degree=3), dict(bc=(0, 1, 0, 0, 0, 0)), dict(bc=(4,) * 6), dict(box=(0, 1, 0, 1, 1, 1)),
           dict(options=lxw.lxw_options_default(precision=7)),
           dict(options=lxw.lxw_options_default(ck_order=4)), dict(options=lxw.lxw_options_default(block_threads=48))]
    for b in bad:
        kw = dict(nx=3, degree=2, bc=(0,) * 6, box=box, options=None)
        kw.update(b)
        with pytest.raises(lxw.LxwError) as e:
            lxw.lxw3_solver_create(kw["nx"], 3, 3, kw["box"], kw["bc"], kw["degree"], kw["options"])
        assert e.value.code == lxw.ERR_ARG, b


def test_tet_argument_errors_without_gpu(libpath):
    """The tetrahedral solver validates its mesh on the host, before any
    CUDA call: indices, repeated ids, orientation, over-shared faces and the
    boundary codes of unmatched faces."""
    from paper_1601_08145_gb300 import lxw
    import synth
    xyz, tets, vid = synth.tet_mesh(2, jitter=0.1, seed=1)
    flipped = tets.copy()
    flipped[0, [1, 2]] = flipped[0, [2, 1]]
    out_of_range = tets.copy()
    out_of_range[3, 2] = len(xyz)
    repeated = vid.copy()
    repeated[tets[0, 1]] = vid[tets[0, 0]]
    tripled = np.concatenate([tets, tets[:1]])
    bad = [dict(degree=3), dict(tets=flipped), dict(tets=out_of_range), dict(vid=repeated), dict(tets=tripled),
           dict(face_bc=np.zeros((len(tets), 4), dtype=np.int32)),
           dict(options=lxw.lxw_options_default(precision=7))]
    for b in bad:
        kw = dict(xyz=xyz, tets=tets, vid=vid, degree=2, face_bc=None, options=None)
        kw.update(b)
        with pytest.raises(lxw.LxwError) as e:
            lxw.lxw3_solver_create_tets(kw["xyz"], kw["tets"], kw["vid"], kw["degree"], face_bc=kw["face_bc"],
                                        options=kw["options"])
        assert e.value.code == lxw.ERR_ARG, b
