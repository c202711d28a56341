"""The rigid-plane Hertz benchmark of Sec. 4.2 with the oracle's
unilateral contact (a gap-aware Signorini condition on the plane nodes'
normal motion, oracle.contact): the cylinder r < 0.5 (E 200 kPa, nu 0.3)
on one grid at each dx, 16 particles per cell, its flat face pushed down
0.03 over 10 kinetically damped steps and then held until the particles
are at rest.  Prints, per dx, the transmitted load F, the Hertz half-width
b and peak p_max for that load, the outermost loaded node, the computed
pressure at x = 0 and the relative L2 error of the pressure (plane
multipliers per node column / dx) against the Hertz semi-ellipse over
|x| <= 1.5 b, raw and after a 1-2-1 filter over neighbouring columns
applied to both (the nodal multipliers alternate between neighbouring
columns at the finer spacing).  CPU only (the oracle); minutes per resolution.

  python tests/study_hertz_rigid_contact.py [--dx 0.03125,0.015625]
"""
from __future__ import annotations

import argparse
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

from oracle import analytic as A  # noqa: E402
from tests.test_oracle_validation import _settled_hertz_contact  # noqa: E402


def run(dx: float, ppc: int = 4, indent: float = 0.03) -> dict:
    t0 = time.time()
    spec, plane, gf, gap, act, lam, u, ds = _settled_hertz_contact(dx, ppc, indent)
    g = spec.grid
    ix = np.arange(g.res[0] * g.res[1]) % g.res[0]
    p = np.bincount(ix, weights=np.where(plane, lam, 0.0), minlength=g.res[0]) / dx
    xc = g.origin[0] + np.arange(g.res[0]) * dx
    F = p.sum() * dx
    b, pmax = A.hertz_line_contact(F, 0.5, 2e5, 0.3)
    ph = pmax * np.sqrt(np.clip(1.0 - (xc / b) ** 2, 0.0, None))
    sel = np.abs(xc) <= 1.5 * b

    def smooth(q):  # 1-2-1 over neighbouring node columns
        return np.convolve(q, [0.25, 0.5, 0.25], mode="same")

    ps, phs = smooth(p), smooth(ph)
    return {"dx": dx, "particles": spec.particles.n, "F": F, "b": b,
            "edge": float(np.abs(xc[p > 0]).max()), "p_max": pmax,
            "p0": float(p[np.argmin(np.abs(xc))]),
            "rel_l2": float(np.linalg.norm(p[sel] - ph[sel]) / np.linalg.norm(ph[sel])),
            "rel_l2_smoothed": float(np.linalg.norm(ps[sel] - phs[sel]) / np.linalg.norm(phs[sel])),
            "seconds": time.time() - t0}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--dx", default="0.03125,0.015625")
    args = ap.parse_args()
    print("| dx | particles | F (N/m) | b | loaded edge | p_max | p(0) | rel L2 | rel L2, 1-2-1 smoothed |")
    print("|---|---|---|---|---|---|---|---|---|")
    for dx in [float(v) for v in args.dx.split(",")]:
        r = run(dx)
        print(f"| {r['dx']:g} | {r['particles']} | {r['F']:.0f} | {r['b']:.4f} | {r['edge']:.4f} | "
              f"{r['p_max']:.0f} | {r['p0']:.0f} | {r['rel_l2']:.3f} | {r['rel_l2_smoothed']:.3f} |",
              flush=True)


if __name__ == "__main__":
    main()
