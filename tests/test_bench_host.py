"""Host-side pieces of bench.py that need no GPU: the point location of the
discretization check maps points of the fine mesh to the half-resolution
mesh's element and reference coordinates for every mesh kind (Cartesian,
masked step grid, jittered triangles, disk), checked by mapping back."""
import numpy as np
import pytest

import bench
import synth


def corners(wc, e):
    """The coarse element's vertex coordinates (Cartesian: lower-left and
    upper-right; triangles: the three vertices)."""
    if wc["kind"] in ("quad", "step"):
        x0, x1, y0, y1 = wc.get("box", (0.0, 1.0, 0.0, 1.0))
        nx, ny = (wc["nx"], wc["ny"]) if wc["kind"] == "step" else (wc["n"], wc["n"])
        if wc["kind"] == "step":
            cells = np.flatnonzero(synth.diffraction_mask(nx, ny).ravel())[e]
        else:
            cells = e
        iy, ix = np.divmod(cells, nx)
        hx, hy = (x1 - x0) / nx, (y1 - y0) / ny
        return x0 + ix * hx, y0 + iy * hy, hx, hy
    if wc["kind"] == "disk":
        xy, tv = synth.disk_triangles(wc["n"])
    else:
        xy, tv = synth.structured_triangles(wc["n"], jitter=0.2, seed=20160129, box=wc.get("box", (0.0, 1.0, 0.0, 1.0)))
    return xy[tv[e]]


@pytest.mark.parametrize("name", ["blast", "diffraction", "rarefy", "sedov"])
def test_locate_maps_points_back(name):
    w = dict(bench.WORKLOADS[name])
    # small versions of each kind
    if w["kind"] == "quad":
        w["n"] = 64
    elif w["kind"] == "step":
        w["nx"], w["ny"] = 78, 66
    elif w["kind"] == "tri":
        w["n"] = 32
    else:
        w["n"] = 4000
    wc = bench.half_resolution(w)
    rng = np.random.default_rng(7)
    if w["kind"] == "step":
        m = synth.diffraction_mask(w["nx"], w["ny"])
        iy, ix = np.nonzero(m)
        x0, x1, y0, y1 = w["box"]
        pts = np.stack([x0 + (ix + rng.uniform(0.05, 0.95, ix.size)) * (x1 - x0) / w["nx"],
                        y0 + (iy + rng.uniform(0.05, 0.95, iy.size)) * (y1 - y0) / w["ny"]], axis=1)
    elif w["kind"] == "quad":
        x0, x1, y0, y1 = w["box"]
        pts = np.stack([rng.uniform(x0, x1, 3000), rng.uniform(y0, y1, 3000)], axis=1)
    else:
        xy, tv = (synth.disk_triangles(w["n"]) if w["kind"] == "disk"
                  else synth.structured_triangles(w["n"], jitter=0.2, seed=20160129))
        b = rng.dirichlet([1, 1, 1], size=len(tv))
        pts = np.einsum("tk,tkd->td", b, xy[tv])
    e, ref = bench.locate(wc, pts)
    if wc["kind"] in ("quad", "step"):
        xl, yl, hx, hy = corners(wc, e)
        assert np.all(np.abs(ref) <= 1.0 + 1e-12)
        back = np.stack([xl + 0.5 * (ref[:, 0] + 1.0) * hx, yl + 0.5 * (ref[:, 1] + 1.0) * hy], axis=1)
        assert np.abs(back - pts).max() < 1e-12
    else:
        v = corners(wc, e)
        assert np.all(ref >= -1e-9) and np.all(ref.sum(axis=1) <= 1.0 + 1e-9)
        back = v[:, 0] + ref[:, :1] * (v[:, 1] - v[:, 0]) + ref[:, 1:] * (v[:, 2] - v[:, 0])
        moved = np.linalg.norm(back - pts, axis=1)
        # points between the fine and the coarse rim move inside the coarse polygon
        tol = 1e-12 if wc["kind"] == "tri" else 2e-3
        assert moved.max() < tol, moved.max()
        if wc["kind"] == "disk":
            assert np.mean(moved < 1e-12) > 0.99
