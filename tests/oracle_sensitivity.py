"""How far the oracle's own scattered field moves under rounding-level changes
of its inputs, for the geometries of the GPU-built-S parity tests.

Each point set (collocation, MFS, proxy) of every shape is multiplied by
(1 + 1e-15 g) with g standard normal (three seeds), the whole oracle pipeline
is rerun (S build, right-hand side, dense solve, far ring and near targets),
and the largest relative change of the field (max |du| / max |u|) is printed;
also the change for the least-squares cutoffs 1e-13 and 1e-15 instead of 1e-14.
Two FP64 evaluations that differ only in rounding order differ by about the
first figure, which is what the GPU parity tolerances are set against.

Usage: python tests/oracle_sensitivity.py [teardrops cshapes_rods spheres ellipsoids]
(runs on the CPU only; calls nothing but the oracle).
"""
import copy
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, HERE)
sys.path.insert(0, os.path.dirname(HERE))

import geometries as geo  # noqa: E402
import mbs_inputs as mi  # noqa: E402
import oracle as orc  # noqa: E402
from oracle import mbs_oracle as om  # noqa: E402

NEAR = {"teardrops": geo.panel_near_targets, "cshapes_rods": geo.panel_near_targets,
        "spheres": geo.spheres_near_targets, "ellipsoids": None}


def _rel(a, b):
    return float(np.max(np.abs(a - b)) / np.max(np.abs(b)))


def fields(wl, near_fn, rcond=om.LS_RCOND):
    sd = [om.build_shape(wl.dim, wl.kappa, sh.x, sh.y, sh.z, k=sh.k, eps=sh.eps, rcond=rcond)
          for sh in wl.shapes]
    lay = orc.layout(wl, sd)
    v = wl.boundary_data()
    q = orc.solve_dense(wl, sd, lay, orc.rhs(wl, sd, lay, v))
    uf = orc.field(wl.dim, wl.kappa, mi.far_targets(wl, 96, mode="ring"), lay["xhat"], q)
    un = None
    if near_fn is not None:
        qm = orc.reconstruct_mfs(wl, sd, lay, q, v)
        un = orc.field_near(wl, sd, lay, q, qm, near_fn(wl))
    return uf, un


def perturbed(wl, seed):
    w2 = copy.deepcopy(wl)
    rng = np.random.default_rng(seed)
    for sh in w2.shapes:
        for a in ("x", "y", "z"):
            arr = getattr(sh, a)
            setattr(sh, a, arr * (1.0 + 1e-15 * rng.standard_normal(arr.shape)))
    return w2


def main(names):
    for name in names:
        wl = getattr(geo, name)()
        near = NEAR[name]
        uf0, un0 = fields(wl, near)
        far_p, near_p = [], []
        for seed in (1, 2, 3):
            uf, un = fields(perturbed(wl, seed), near)
            far_p.append(_rel(uf, uf0))
            if un is not None:
                near_p.append(_rel(un, un0))
        line = f"{name}: perturbed far {max(far_p):.2e}"
        if near_p:
            line += f" near {max(near_p):.2e}"
        for rc in (1e-13, 1e-15):
            uf, un = fields(wl, near, rc)
            line += f" | cutoff {rc:.0e}: far {_rel(uf, uf0):.2e}"
            if un is not None:
                line += f" near {_rel(un, un0):.2e}"
        print(line, flush=True)


if __name__ == "__main__":
    main(sys.argv[1:] or ["teardrops", "cshapes_rods", "spheres", "ellipsoids"])
