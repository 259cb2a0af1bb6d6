"""Planted mistakes in the tetrahedral oracle fail its pins.

Each case builds the 3D oracle from its source with one line changed (a
plausible mistake: an unoriented face normal, face points not put in the
shared vertex-id order, the inverse Jacobian transposed in the q_t
projection, a Gauss-Jacobi rule for the wrong weight, the face area off by
two) and runs a short set of the tetrahedral pins of test_oracle_3d.py on
it on meshes whose cells list shared faces in unrelated vertex orders: the
exact step of an advected quadratic, free stream through transparent
sides, conservation of all five totals on a periodic mesh.  Each mutant must fail at least
one of them, while the unchanged source passes them all.
"""
import os
import subprocess
import tempfile

import numpy as np
import pytest

import synth

HERE = os.path.dirname(os.path.abspath(__file__))
ODIR = os.path.join(HERE, "..", "oracle")
SRC2 = os.path.join(ODIR, "lxw_oracle.c")
SRC3 = os.path.join(ODIR, "lxw_oracle3d.c")
G = 1.4

MUTANTS = {
    # face normals always from the canonical vertex order, never flipped outward
    "normal_unoriented": ("double sg = side > 0.0 ? -1.0 : 1.0;", "double sg = 1.0;"),
    # face points placed from the cell's own vertex order, not the shared id order
    "face_order_local": ("if (vid[v[lv[b]]] < vid[v[lv[a]]]) { int t = lv[a]; lv[a] = lv[b]; lv[b] = t; }",
                         "if (0) { int t = lv[a]; lv[a] = lv[b]; lv[b] = t; }"),
    # the physical gradient of the q_t projection with the inverse Jacobian transposed
    "jacobian_transposed": (
        "double gd = Ji[0 * 3 + d] * s->dref[k][0][m] + Ji[1 * 3 + d] * s->dref[k][1][m] + "
        "Ji[2 * 3 + d] * s->dref[k][2][m];",
        "double gd = Ji[d * 3 + 0] * s->dref[k][0][m] + Ji[d * 3 + 1] * s->dref[k][1][m] + "
        "Ji[d * 3 + 2] * s->dref[k][2][m];"),
    # the collapsed rule's first direction with the weight (1 - u) instead of (1 - u)^2
    "jacobi_weight": ("gauss_jacobi01(n, 2.0, ua, uw);", "gauss_jacobi01(n, 1.0, ua, uw);"),
    # the face area from the cross product without its factor 1/2
    "area_double": ("n[0] = 0.5 * (e1[1] * e2[2] - e1[2] * e2[1]);", "n[0] = (e1[1] * e2[2] - e1[2] * e2[1]);"),
}


def _build(tmp, name):
    src = open(SRC3).read()
    if name is not None:
        old, new = MUTANTS[name]
        assert src.count(old) == 1, name
        src = src.replace(old, new)
    path = os.path.join(tmp, "mut3d.c")
    open(path, "w").write(src)
    lib = os.path.join(tmp, "liborc_%s.so" % (name or "base"))
    subprocess.run(["gcc", "-O2", "-fPIC", "-shared", "-ffp-contract=off", "-std=gnu11", "-I", ODIR, "-o", lib,
                    SRC2, path, "-lm"], check=True, capture_output=True)
    return lib


def pin_failures(orc):
    """The tetrahedral pins of the short set that fail on the loaded oracle."""
    fails = []
    U = np.array([0.7, -0.4, 0.3]); P = 1.1
    rho0 = lambda x, y, z: 1.0 + 0.3 * x - 0.2 * y + 0.1 * z + 0.4 * x * x + 0.1 * x * y - 0.3 * y * z + 0.2 * z * z  # noqa: E731
    xyz, tets, vid = synth.tet_mesh(3, jitter=0.2, seed=4, permute=True)   # cells list shared faces in unrelated orders
    try:
        m = orc.Mesh3.tets(xyz, tets, vid, np.full((len(tets), 4), 2, dtype=np.int32))
        s = orc.Solver3(m, 2, gamma=G, shock_limiter=False)
        ic = lambda t: (lambda x, y, z: (rho0(x - U[0] * t, y - U[1] * t, z - U[2] * t), U[0] + 0 * x,  # noqa: E731
                                         U[1] + 0 * x, U[2] + 0 * x, P + 0 * x))
        Q = s.project_fn(ic(0.0))
        s.step(Q, dt=0.02)
        if not np.abs(Q - s.project_fn(ic(0.02))).max() < 5e-14:
            fails.append("exact_quadratic")
        Q = s.project_fn(lambda x, y, z: (1.3 + 0 * x, 0.4 + 0 * x, -0.2 + 0 * x, 0.7 + 0 * x, 0.9 + 0 * x))
        Q0 = Q.copy()
        s.step(Q, cfl=0.3)
        if not np.allclose(Q, Q0, atol=1e-13):
            fails.append("free_stream")
        # a periodic, renumbered mesh: every face is matched, all five totals conserved
        m = orc.Mesh3.tets(*synth.tet_mesh(3, periodic=True, seed=6, permute=True), None)
        s = orc.Solver3(m, 2, gamma=G, alpha0=50.0)
        Q = synth.random_modal_state3(m.N, s.ML, seed=13, amp=0.3, rho_range=(0.02, 2.0), p_range=(0.01, 2.0))
        vol = m.geometry()[0]
        t0 = (vol[:, None] * Q[:, :, 0]).sum(axis=0)
        d = s.step(Q, cfl=0.3)
        t1 = (vol[:, None] * Q[:, :, 0]).sum(axis=0)
        if d["status"] != 0 or not np.allclose(t1, t0, rtol=1e-13, atol=1e-13):
            fails.append("conservation")
    except Exception as e:   # a mutant may break the mesh or the step outright
        fails.append("error: %s" % str(e)[:60])
    return fails


def test_unchanged_source_passes():
    from oracle import oracle as orc
    with tempfile.TemporaryDirectory() as tmp:
        with orc.use_library(_build(tmp, None)):
            assert pin_failures(orc) == []


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_planted_mistakes_fail_the_pins(name):
    from oracle import oracle as orc
    with tempfile.TemporaryDirectory() as tmp:
        with orc.use_library(_build(tmp, name)):
            assert pin_failures(orc) != [], name


# ---------------------------------------------------------------- hexahedra
HEX_MUTANTS = {
    # neighbour index with the y and z strides confused
    "neighbour_strides": ("m->nbr[6 * i + k] = (cc[2] * ny + cc[1]) * nx + cc[0];",
                          "m->nbr[6 * i + k] = (cc[1] * nz + cc[2]) * nx + cc[0];"),
    # face normals pointing inward
    "normal_inward": ("n[d] = (k % 2 ? 1.0 : -1.0) * m->vol[i] / h[d];", "n[d] = (k % 2 ? -1.0 : 1.0) * m->vol[i] / h[d];"),
    # the reference-to-physical derivative without its factor 2
    "jacobian_half": ("m->Ji[9 * i + 4 * d] = 2.0 / h[d];", "m->Ji[9 * i + 4 * d] = 1.0 / h[d];"),
    # Legendre polynomials without their normalisation (the basis no longer orthonormal)
    "legendre_unnormalised": ("v[k] = sqrt(2.0 * k + 1.0) * p[k];", "v[k] = p[k];"),
    # the periodic wrap one cell off
    "periodic_wrap_off": ("if (bc[k] == B3_PERIODIC) cc[d] = (cc[d] + n3[d]) % n3[d];",
                          "if (bc[k] == B3_PERIODIC) cc[d] = (cc[d] + n3[d] + 1) % n3[d];"),
}


def _build_hex(tmp, name):
    src = open(SRC3).read()
    if name is not None:
        old, new = HEX_MUTANTS[name]
        assert src.count(old) == 1, name
        src = src.replace(old, new)
    path = os.path.join(tmp, "mut3d.c")
    open(path, "w").write(src)
    lib = os.path.join(tmp, "liborc_hex_%s.so" % (name or "base"))
    subprocess.run(["gcc", "-O2", "-fPIC", "-shared", "-ffp-contract=off", "-std=gnu11", "-I", ODIR, "-o", lib,
                    SRC2, path, "-lm"], check=True, capture_output=True)
    return lib


def hex_pin_failures(orc):
    """The hexahedral pins of the short set that fail on the loaded oracle:
    the exact step of an advected quadratic on non-cubic cells with ny != nz,
    free stream, conservation of all five totals on a periodic mesh."""
    fails = []
    U = np.array([0.7, -0.4, 0.3]); P = 1.1
    rho0 = lambda x, y, z: 1.0 + 0.3 * x - 0.2 * y + 0.1 * z + 0.4 * x * x + 0.1 * x * y - 0.3 * y * z + 0.2 * z * z  # noqa: E731
    try:
        m = orc.Mesh3(3, 2, 4, (0.0, 0.9, 0.0, 0.6, 0.0, 0.7), (2,) * 6)
        s = orc.Solver3(m, 2, gamma=G, shock_limiter=False)
        ic = lambda t: (lambda x, y, z: (rho0(x - U[0] * t, y - U[1] * t, z - U[2] * t), U[0] + 0 * x,  # noqa: E731
                                         U[1] + 0 * x, U[2] + 0 * x, P + 0 * x))
        Q = s.project_fn(ic(0.0))
        s.step(Q, dt=0.02)
        if not np.abs(Q - s.project_fn(ic(0.02))).max() < 5e-14:
            fails.append("exact_quadratic")
        Q = s.project_fn(lambda x, y, z: (1.3 + 0 * x, 0.4 + 0 * x, -0.2 + 0 * x, 0.7 + 0 * x, 0.9 + 0 * x))
        Q0 = Q.copy()
        s.step(Q, cfl=0.3)
        if not np.allclose(Q, Q0, atol=1e-13):
            fails.append("free_stream")
        m = orc.Mesh3(4, 3, 5, (0.0, 1.0, 0.0, 0.8, 0.0, 1.2), (0,) * 6)
        s = orc.Solver3(m, 2, gamma=G, alpha0=50.0)
        Q = synth.random_modal_state3(m.N, s.ML, seed=21, amp=0.3, rho_range=(0.02, 2.0), p_range=(0.01, 2.0))
        vol = m.geometry()[0]
        t0 = (vol[:, None] * Q[:, :, 0]).sum(axis=0)
        d = s.step(Q, cfl=0.3)
        t1 = (vol[:, None] * Q[:, :, 0]).sum(axis=0)
        if d["status"] != 0 or not np.allclose(t1, t0, rtol=1e-13, atol=1e-13):
            fails.append("conservation")
    except Exception as e:
        fails.append("error: %s" % str(e)[:60])
    return fails


def test_unchanged_source_passes_hex():
    from oracle import oracle as orc
    with tempfile.TemporaryDirectory() as tmp:
        with orc.use_library(_build_hex(tmp, None)):
            assert hex_pin_failures(orc) == []


@pytest.mark.parametrize("name", sorted(HEX_MUTANTS))
def test_planted_hex_mistakes_fail_the_pins(name):
    from oracle import oracle as orc
    with tempfile.TemporaryDirectory() as tmp:
        with orc.use_library(_build_hex(tmp, name)):
            assert hex_pin_failures(orc) != [], name
