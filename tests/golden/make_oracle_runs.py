"""Writes the stored FP64 oracle results that the long GPU parity tests
compare against (tests/golden/oracle_runs/*.txt).

Every value in those files comes from ``oracle.osmpm_oracle`` alone, run
here on the CPU; nothing is read from the CUDA library.  The runs are too
long to repeat inside each GPU test session (minutes of sparse-LU Newton
solves), so they are stored once.  Regenerate with

    python tests/golden/make_oracle_runs.py [name ...]

Files: a comment header naming the workload and the number of global steps,
then one line per particle, ``<domain> <id> <x_0> ... <x_{d-1}>`` with
domain c (coarse) or f (fine), positions in id order, 17 significant digits;
the gradient run's lines carry dJ/dE before the position.
"""
from __future__ import annotations

import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from oracle import osmpm_oracle as O  # noqa: E402
from paper_2605_09097_gb300 import workloads as W  # noqa: E402

OUT = os.path.join(HERE, "oracle_runs")

# name -> (description, workload builder, global steps)
RUNS = {
    "inclusion_dxS0.02_M2_80steps": (
        "2D elastic inclusion OS-MPM (coarse dx 0.05, fine dx 0.02, M = 2), top edge moved "
        "1e-3 per step, FP64 oracle",
        lambda: W.inclusion(dx_S=0.02, M=2), 80),
    "inclusion_dxS0.02_M2_top3e-4_100steps": (
        "2D elastic inclusion OS-MPM (coarse dx 0.05, fine dx 0.02, M = 2), top edge moved "
        "3e-4 per step (3 % compression after 100 steps), FP64 oracle",
        lambda: W.inclusion(dx_S=0.02, M=2, top_disp=3e-4), 100),
    "fold3d_small_M2_2steps": (
        "3D folding plate, reduced (plate 0.48 x 0.12 x 0.04, coarse dx 0.04, fine band "
        "[0.12, 0.36) at dx 0.02, M = 2, 90 degrees over 20 steps), FP64 oracle",
        lambda: W.fold3d_small(), 2),
}


def write(name: str) -> str:
    desc, build, steps = RUNS[name]
    cB, cS, sch, dT = build()
    B, S = O.DomainState.create(cB), O.DomainState.create(cS)
    t0 = time.time()
    iters = []
    for _ in range(steps):
        st = O.SchwarzStats()
        O.schwarz_step(B, S, dT, sch, st)
        if not st.converged:
            raise RuntimeError(f"{name}: the oracle's Schwarz loop did not converge")
        iters.append(st.iters)
    path = os.path.join(OUT, name + ".txt")
    with open(path, "w") as f:
        f.write(f"# {desc}\n")
        f.write(f"# global steps: {steps} of dT = {dT!r}; Schwarz iterations per step: "
                f"{' '.join(map(str, iters))}\n")
        f.write("# written by tests/golden/make_oracle_runs.py (oracle only)\n")
        f.write("# domain id x_0 .. x_{d-1} (final positions, id order)\n")
        for tag, st_ in (("c", B), ("f", S)):
            for i, row in enumerate(st_.p.x):
                f.write(tag + " " + str(i) + " " + " ".join(f"{v:.17g}" for v in row) + "\n")
    print(f"{name}: {steps} steps in {time.time() - t0:.0f} s -> {path}")
    return path


# ---------------------------------------------------------------------------
# the batched family's gradient: instance 0 (fine dx 0.01), 50 coupled steps,
# every step exactly ADJ_ITERS Schwarz iterations (so that a run elsewhere can
# unroll the same ones), J = mean y of the inclusion's top-cap particles
# ---------------------------------------------------------------------------
ADJ_NAME = "cfg4_instance0_adjoint_50steps"
ADJ_STEPS, ADJ_ITERS, ADJ_NEWTON_TOL = 50, 4, 1e-10


def adjoint_case():
    """(coarse, fine, schwarz, dT, dJ_dx) of the stored gradient run: batched
    instance 0 with tight solver tolerances, Schwarz iterations fixed at
    ADJ_ITERS (eps_conv too small to stop earlier, k_max = ADJ_ITERS - 1)."""
    import dataclasses
    import numpy as np
    cB, cS, sch, dT = W.inclusion_instance(0)
    tight = dict(newton_tol=ADJ_NEWTON_TOL, cg_rtol=1e-12, cg_max=100000)
    cB = dataclasses.replace(cB, **tight)
    cS = dataclasses.replace(cS, **tight)
    sch = dataclasses.replace(sch, k_max=ADJ_ITERS - 1, eps_conv=1e-300)
    r_inc, _, _ = W.instance_params(0)
    cap = W.top_cap(cS.particles.x, r_inc)
    c = np.zeros((cB.particles.n + cS.particles.n, 2))
    c[cB.particles.n:][cap, 1] = 1.0 / cap.sum()
    return cB, cS, sch, dT, c


def write_adjoint() -> str:
    import numpy as np
    from oracle import adjoint as AD
    cB, cS, sch, dT, c = adjoint_case()
    nB = cB.particles.n
    B, S = O.DomainState.create(cB), O.DomainState.create(cS)
    t0 = time.time()
    recs = [AD.record_schwarz_step(B, S, dT, sch, ADJ_NEWTON_TOL, ADJ_ITERS) for _ in range(ADJ_STEPS)]
    barB, barS = AD.StateBar.zeros_like(B.p), AD.StateBar.zeros_like(S.p)
    barB.x = c[:nB].copy()
    barS.x = c[nB:].copy()
    EB, ES = np.zeros(nB), np.zeros(cS.particles.n)
    for rec in reversed(recs):
        barB, barS, eb, es = AD.schwarz_adjoint(rec, barB, barS)
        EB += eb
        ES += es
    J = float(np.sum(c[nB:] * (S.p.x - cS.particles.x)))
    path = os.path.join(OUT, ADJ_NAME + ".txt")
    with open(path, "w") as f:
        f.write("# batched inclusion instance 0 (fine dx 0.01, M = 2), FP64 oracle: 50 coupled steps "
                f"of exactly {ADJ_ITERS} Schwarz iterations, Newton tol {ADJ_NEWTON_TOL:g}\n")
        f.write(f"# J = mean y-displacement of the inclusion top-cap particles = {J!r}\n")
        f.write("# written by tests/golden/make_oracle_runs.py (oracle only)\n")
        f.write("# domain id dJ/dE x_0 x_1 (final positions, id order)\n")
        for tag, EE, st_ in (("c", EB, B), ("f", ES, S)):
            for i in range(len(EE)):
                f.write(f"{tag} {i} {EE[i]:.17g} " + " ".join(f"{v:.17g}" for v in st_.p.x[i]) + "\n")
    print(f"{ADJ_NAME}: {ADJ_STEPS} steps and the adjoint in {time.time() - t0:.0f} s -> {path}")
    return path


# ---------------------------------------------------------------------------
# the rigid-plane Hertz contact (Sec. 4.2) settled with the oracle's
# unilateral contact at dx = 1/32, 16 particles per cell, indent 0.03
# ---------------------------------------------------------------------------
HERTZ_NAME = "hertz_rigid_dx1_32_settled"
HERTZ_ARGS = dict(dx=1.0 / 32, ppc_1d=4, indent=0.03)
HERTZ_EVERY = 4   # stored particles: ids that are multiples of this


def write_hertz() -> str:
    import numpy as np
    from oracle import contact as C
    t0 = time.time()
    spec, plane, gf, gap, act, lam, u, ds, k = C.settle_hertz(**HERTZ_ARGS)
    g = spec.grid
    dx = g.dx
    ix = np.arange(g.res[0] * g.res[1]) % g.res[0]
    p = np.bincount(ix, weights=np.where(plane, lam, 0.0), minlength=g.res[0]) / dx
    held = np.bincount(ix, weights=act.astype(float), minlength=g.res[0])
    path = os.path.join(OUT, HERTZ_NAME + ".txt")
    with open(path, "w") as f:
        f.write("# rigid-plane Hertz contact of Sec. 4.2 (workloads.hertz_rigid_single), FP64 oracle "
                "with the unilateral contact of oracle.contact: settle_hertz(dx=1/32, ppc_1d=4, "
                f"indent=0.03), {k} settle steps\n")
        f.write("# written by tests/golden/make_oracle_runs.py (oracle only)\n")
        f.write("# 'p' lines: column ix, pressure (plane multipliers summed over the column / dx), "
                "held nodes in the column\n")
        f.write(f"# 'x' lines: particle id (every {HERTZ_EVERY}th), settled position\n")
        f.write(f"settle_steps {k}\n")
        for i in range(g.res[0]):
            f.write(f"p {i} {p[i]:.17g} {int(held[i])}\n")
        for i in range(0, ds.p.n, HERTZ_EVERY):
            f.write(f"x {i} {ds.p.x[i, 0]:.17g} {ds.p.x[i, 1]:.17g}\n")
    print(f"{HERTZ_NAME}: settled in {k} steps, {time.time() - t0:.0f} s -> {path}")
    return path


def load(name: str):
    """(coarse x, fine x) of a stored run, id order."""
    import numpy as np
    rows = {"c": [], "f": []}
    with open(os.path.join(OUT, name + ".txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            parts = line.split()
            rows[parts[0]].append([float(v) for v in parts[2:]])
    return np.asarray(rows["c"]), np.asarray(rows["f"])


if __name__ == "__main__":
    os.makedirs(OUT, exist_ok=True)
    for n in (sys.argv[1:] or list(RUNS) + [ADJ_NAME, HERTZ_NAME]):
        if n == ADJ_NAME:
            write_adjoint()
        elif n == HERTZ_NAME:
            write_hertz()
        else:
            write(n)
