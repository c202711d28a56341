"""Accuracy against cost of OS-MPM and of the single fine domain on the
eigenstrain inclusion of Sec. 4.3 (the paper's accuracy-efficiency study,
on the GPU).

For each stiffness ratio and fine spacing h: the single-domain reference
runs the traction-free matrix [0.1,0.9]^2 on one grid at h with dt = h
(dt / h constant, 0.01 s at h = 0.01); OS-MPM runs the fine disk r < 0.15
at h and the coarse matrix at 2h with M = 2 and dT = 2 dt.  Both relax until
the largest particle speed of every domain is below 1e-6.  Recorded per
run: steps, summed GPU time of the steps (CUDA events on the domains'
stream; the settle checks run outside the events), and the relative L2
error of sigma_yy against the Eshelby solution over the particles with
r < 0.15 (the fine region both methods resolve at h).

Asserted: OS-MPM reproduces the single domain's accuracy (its error within
6 % of the single domain's, relative) and both errors fall from h to h/2.
The default sweep is h = 0.01, 0.005 (seconds of GPU time); the environment
variable OSMPM_STUDY_H selects others, e.g. the full table:

  OSMPM_STUDY_H=0.01,0.005,0.0025 python -m pytest -s tests/test_gpu_study_eshelby.py

which prints one JSON line per run and the summary table.
"""
from __future__ import annotations

import json
import os

import numpy as np
import pytest

from oracle import analytic as A
from oracle import osmpm_oracle as O
from paper_2605_09097_gb300 import workloads as W

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

DELTA, R_INC, E_OUT, NU = 0.01, 0.05, 1e6, 0.3
MAX_STEPS, V_STOP = 400, 1e-6
RATIOS = (1.0, 2.0, 5.0)
H = tuple(float(v) for v in os.environ.get("OSMPM_STUDY_H", "0.01,0.005").split(","))


def sigma_yy_error(x, F, E, nu, ratio):
    mu, lam = O.lame(E, nu)
    sig = O.cauchy_stress(F, mu, lam)
    d = x - 0.5
    r = np.hypot(d[:, 0], d[:, 1])
    sel = r < 0.15
    P = A.eshelby_pressure(DELTA, ratio * E_OUT, NU, E_OUT, NU)
    srr, stt = A.eshelby_stress(r[sel], R_INC, P)
    c2 = (d[sel, 0] / np.maximum(r[sel], 1e-300)) ** 2
    syy = srr * (1.0 - c2) + stt * c2
    return float(np.linalg.norm(sig[sel, 1, 1] - syy) / np.linalg.norm(syy))


def timed_steps(torch, stream, step, speeds):
    """Runs step() until every speed is below V_STOP; returns (steps, ms)."""
    ms = 0.0
    for n in range(1, MAX_STEPS + 1):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        step()
        b.record(stream)
        torch.cuda.synchronize()
        ms += a.elapsed_time(b)
        if max(speeds()) < V_STOP:
            return n, ms
    raise RuntimeError("no equilibrium within %d steps" % MAX_STEPS)


def run(ratio, h, osmpm, torch, stream):
    dt = h  # 0.01 s at h = 0.01, dt / h constant
    # single fine domain
    spec = W.inclusion_single(h, E_inc=ratio * E_OUT, eigenstrain=DELTA)
    dom = osmpm.Domain(spec, stream=stream.cuda_stream)
    n1, ms1 = timed_steps(torch, stream, lambda: dom.step(dt),
                          lambda: [np.abs(dom.get_particles()[1]).max()])
    x, _, _, F = dom.get_particles()
    e1 = sigma_yy_error(x, F, spec.particles.E, spec.particles.nu, ratio)
    n_single = spec.particles.n
    dom.close()
    # OS-MPM: fine h, coarse 2h, M = 2
    cB, cS, sch, dT = W.inclusion(dx_S=h, dx_B=2 * h, M=2, dT=2 * dt, E_inc=ratio * E_OUT,
                                  top_disp=0.0, eigenstrain=DELTA, free_edges=True)
    B = osmpm.Domain(cB, stream=stream.cuda_stream)
    S = osmpm.Domain(cS, stream=stream.cuda_stream)
    its = []
    n2, ms2 = timed_steps(torch, stream,
                          lambda: its.append(osmpm.osmpm_schwarz_couple(B, S, dT, sch)["schwarz_iters"]),
                          lambda: [np.abs(B.get_particles()[1]).max(), np.abs(S.get_particles()[1]).max()])
    x, _, _, F = S.get_particles()
    e2 = sigma_yy_error(x, F, cS.particles.E, cS.particles.nu, ratio)
    row = {"ratio": ratio, "h": h,
           "single": {"particles": n_single, "steps": n1, "gpu_s": ms1 / 1e3, "err_syy": e1},
           "osmpm": {"particles": cB.particles.n + cS.particles.n, "steps": n2, "gpu_s": ms2 / 1e3,
                     "err_syy": e2, "schwarz_iters_mean": float(np.mean(its))},
           "speedup": ms1 / ms2}
    B.close()
    S.close()
    return row


@pytest.fixture(scope="module")
def env():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2605_09097_gb300 import build
    build.build()
    from paper_2605_09097_gb300 import osmpm
    return torch, osmpm


def test_osmpm_matches_single_fine_domain_accuracy(env):
    torch, osmpm = env
    stream = torch.cuda.Stream()
    rows = []
    with torch.cuda.stream(stream):
        for ratio in RATIOS:
            for h in H:
                row = run(ratio, h, osmpm, torch, stream)
                rows.append(row)
                print(json.dumps(row), flush=True)
    print("\n| E_in/E_out | h | single: particles, steps, GPU s, err | OS-MPM: particles, steps, "
          "GPU s, err | speedup |")
    print("|---|---|---|---|---|")
    for r in rows:
        s, o = r["single"], r["osmpm"]
        print(f"| {r['ratio']:g} | {r['h']:g} | {s['particles']}, {s['steps']}, {s['gpu_s']:.3f}, "
              f"{s['err_syy']:.4f} | {o['particles']}, {o['steps']}, {o['gpu_s']:.3f}, "
              f"{o['err_syy']:.4f} | {r['speedup']:.2f} |")
    for r in rows:
        assert abs(r["osmpm"]["err_syy"] - r["single"]["err_syy"]) <= 0.06 * r["single"]["err_syy"], r
    for ratio in RATIOS:
        seq = [r for r in rows if r["ratio"] == ratio]
        for a, b in zip(seq, seq[1:]):
            assert b["single"]["err_syy"] < a["single"]["err_syy"]
            assert b["osmpm"]["err_syy"] < a["osmpm"]["err_syy"]
