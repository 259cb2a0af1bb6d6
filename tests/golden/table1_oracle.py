"""The oracle on the paper's convergence problem (Sec. 4, Table 1).

rho = 1 - 0.9999 sin(2 pi x) sin(2 pi y), u = (1, 0), p = 1 on the periodic
unit square, P2 on n x n squares, CFL 0.08, all limiters on, run to
t = 0.02 (the last step shortened to land on it), compared with the exact
advected density.  Calls only the oracle.

Run as ``python tests/golden/table1_oracle.py`` to rewrite
``table1_oracle.txt`` (both readings of the point flux's dissipation speed,
28^2 .. 212^2; about half an hour on 8 cores).  The tests import
:func:`run` for the grids they check live.
"""
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import synth  # noqa: E402
from oracle import oracle as orc  # noqa: E402

T_END, CFL, GAMMA = 0.02, 0.08, 1.4
OUT = os.path.join(HERE, "table1_oracle.txt")


def run(n, llf_global=False):
    """Errors of the oracle's density at t = T_END on n x n cells:
    ``l2`` the L2 norm of rho_h - rho over the square (projection rule,
    exact for the P2 part); ``floor`` the same norm for the L2 projection
    of the exact solution at T_END (the best any P2 state can do);
    ``g2`` the root mean square over 2 x 2 Gauss points per cell;
    ``avg`` the L2 norm of the cell-average errors."""
    sol = orc.Solver(orc.Mesh.cartesian(n, n), 2, gamma=GAMMA, llf_global=llf_global)
    Q = sol.project_fn(synth.ic_paper_smooth)
    t, steps, lim = 0.0, 0, [0, 0, 0]
    while True:
        # a step with dt from the CFL rule (Sec. 4.1); if it would pass T_END,
        # step the saved state again with the remainder instead
        Qc = Q.copy()
        d = sol.step(Qc, cfl=CFL)
        last = t + d["dt"] >= T_END * (1 - 1e-15)
        if last:
            d = sol.step(Q, dt=T_END - t)
        else:
            Q[...] = Qc
        assert d["status"] == 0 and d["min_rho"] > 0 and d["min_p"] > 0
        steps += 1
        lim[0] += int(d["n_mom"]); lim[1] += int(d["n_edge"]); lim[2] += int(d["n_sc"])
        if last:
            break
        t += d["dt"]
    exact = lambda x, y: synth.exact_paper_smooth_density(x, y, T_END)  # noqa: E731
    xy = sol.projection_points(); w = sol.projection_weights()
    area, _, cx, cy = sol.mesh.geometry()
    q = sol.eval_projection_points(Q)[..., 0]
    l2 = np.sqrt(np.sum(area[:, None] * w[None, :] * (q - exact(xy[..., 0], xy[..., 1])) ** 2))
    Pe = sol.project_fn(lambda x, y: (exact(x, y), 1.0 + 0 * x, 0 * x, 1.0 + 0 * x))
    qe = sol.eval_projection_points(Pe)[..., 0]
    floor = np.sqrt(np.sum(area[:, None] * w[None, :] * (qe - exact(xy[..., 0], xy[..., 1])) ** 2))
    g = np.array([-1.0, 1.0]) / np.sqrt(3.0)
    xi, eta = [a.ravel() for a in np.meshgrid(g, g)]
    phi = orc.basis_eval(orc.QUAD, 2, xi, eta)[0]            # [4 points][ML]
    h = 1.0 / n
    qg = Q[:, 0, :] @ phi.T
    eg = qg - exact(cx[:, None] + 0.5 * h * xi[None, :], cy[:, None] + 0.5 * h * eta[None, :])
    g2 = np.sqrt(np.sum(area[:, None] * eg ** 2) / 4.0)
    avg = np.sqrt(np.sum(area * (Q[:, 0, 0] - Pe[:, 0, 0]) ** 2))
    return {"n": n, "steps": steps, "l2": l2, "floor": floor, "g2": g2, "avg": avg,
            "n_mom": lim[0], "n_edge": lim[1], "n_sc": lim[2], "s": d["s"]}


def main():
    rows = []
    for llf_global in (False, True):
        for n in (28, 42, 63, 94, 141, 212):
            r = run(n, llf_global)
            rows.append(("global" if llf_global else "local",) + tuple(
                r[k] for k in ("n", "steps", "l2", "floor", "g2", "avg", "n_mom", "n_edge", "n_sc")))
            print(rows[-1], flush=True)
            write(rows)


def write(rows):
    with open(OUT, "w") as f:
        f.write("# The oracle on the Table 1 problem (Sec. 4), written by table1_oracle.py.\n")
        f.write("# speed: dissipation speed of the LLF point flux (local: max |u|+c of the two\n")
        f.write("# traces, bounded by the global s; global: the global s).  Errors of the density\n")
        f.write("# at t = 0.02: l2 over the square, floor = l2 of the exact solution's L2\n")
        f.write("# projection, g2 = RMS over 2x2 Gauss points per cell, avg = L2 of the cell\n")
        f.write("# averages; then limiter activations summed over the steps (moment, edge, shock).\n")
        f.write("# speed n steps l2 floor g2 avg n_mom n_edge n_sc\n")
        for r in rows:
            f.write("%s %d %d %.6e %.6e %.6e %.6e %d %d %d\n" % r)


if __name__ == "__main__":
    main()
