"""3D OS-MPM.  A small clamped bar split into an overlapping coarse and fine
subdomain is compared with the FP64 oracle particle by particle; a reduced
folding plate (the rotation rule, M = 2) is compared with the FP64 oracle's
stored run in mixed precision and in FP64, with both PCG engines; the 3D
folding-plate configuration (coarse dx 0.02, fine band dx 0.005, M = 4,
~137k particles, mixed precision) runs two global steps and is checked
through properties that hold at any size."""
import dataclasses
import os

import numpy as np
import pytest

from oracle import osmpm_oracle as O
from paper_2605_09097_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def osmpm():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2605_09097_gb300 import build
    build.build()
    from paper_2605_09097_gb300 import osmpm as m
    return m


def rel_disp(x_gpu, x_ref, x0):
    return np.linalg.norm(x_gpu - x_ref) / max(np.linalg.norm(x_ref - x0), 1e-300)


def test_overlap3d_matches_oracle(osmpm):
    cB, cS, sch, dT = W.overlap3d()
    B, S = osmpm.Domain(cB), osmpm.Domain(cS)
    oB, oS = O.DomainState.create(cB), O.DomainState.create(cS)
    st = osmpm.osmpm_schwarz_couple(B, S, dT, sch)
    so = {}
    ost = O.SchwarzStats()
    O.schwarz_step(oB, oS, dT, sch, ost, so)
    assert st["converged"] == 1 and ost.converged
    assert abs(st["schwarz_iters"] - ost.iters) <= 1
    np.testing.assert_array_equal(B.get_grid(osmpm.OSMPM_FIELD_RECEIVER) > 0, so["sets"].recvB)
    np.testing.assert_array_equal(S.get_grid(osmpm.OSMPM_FIELD_RECEIVER) > 0, so["sets"].recvS)
    assert rel_disp(B.get_particles()[0], oB.p.x, cB.particles.x) <= 1e-6
    assert rel_disp(S.get_particles()[0], oS.p.x, cS.particles.x) <= 1e-6


def test_fold3d_full_size_two_steps(osmpm):
    cB, cS, sch, dT = W.fold3d()
    assert cB.particles.n + cS.particles.n > 130_000
    B, S = osmpm.Domain(cB), osmpm.Domain(cS)
    for _ in range(2):
        st = osmpm.osmpm_schwarz_couple(B, S, dT, sch)
        assert st["converged"] == 1
    xB, vB, _, FB = B.get_particles()
    xS, vS, _, FS = S.get_particles()
    for a in (xB, vB, FB, xS, vS, FS):
        assert np.all(np.isfinite(a))
    assert np.linalg.det(FB).min() > 0 and np.linalg.det(FS).min() > 0
    # edge nodes carry the rigid rotation increment exactly (about the fold axis)
    g = cB.grid
    u = B.get_grid(osmpm.OSMPM_FIELD_U)
    m = B.get_grid(osmpm.OSMPM_FIELD_MASS)
    idx = np.arange(g.n_nodes)
    xi = np.stack([g.origin[0] + g.dx * (idx % g.res[0]),
                   g.origin[1] + g.dx * ((idx // g.res[0]) % g.res[1]),
                   g.origin[2] + g.dx * (idx // (g.res[0] * g.res[1]))], axis=1)
    edge = (xi[:, 0] >= 1.0 - 1.5 * g.dx) & (m > cB.mass_eps)
    assert edge.sum() > 10
    r = cB.dirichlet[1]
    th = r.omega * dT
    Rm = np.array([[np.cos(th), 0, np.sin(th)], [0, 1, 0], [-np.sin(th), 0, np.cos(th)]])
    rel = xi[edge] - np.asarray(r.center)
    np.testing.assert_allclose(u[edge], rel @ Rm.T - rel, atol=1e-12)
    # the clamped end does not move; the fine band moved with the plate
    clamp = cB.particles.x[:, 0] < 0.5 * g.dx
    assert np.abs(xB[clamp] - cB.particles.x[clamp]).max() < 1e-3 * g.dx
    assert np.abs(xS - cS.particles.x).max() > 0


def _stored_oracle_run(name):
    """(coarse x, fine x) of a stored FP64 oracle run (written by
    tests/golden/make_oracle_runs.py, oracle only), id order."""
    rows = {"c": [], "f": []}
    path = os.path.join(os.path.dirname(__file__), "golden", "oracle_runs", name + ".txt")
    with open(path) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                parts = line.split()
                rows[parts[0]].append([float(v) for v in parts[2:]])
    return np.asarray(rows["c"]), np.asarray(rows["f"])


@pytest.mark.parametrize("precision,pcg_mode,tol", [(1, 1, 1e-4), (1, 2, 1e-4), (0, 1, 1e-6),
                                                     (0, 2, 1e-6)])
def test_fold3d_small_matches_oracle(osmpm, precision, pcg_mode, tol):
    """Reduced folding plate (3D, the kind-1 rotation rule on the coarse
    edge, M = 2), two global steps: mixed precision (Kernels<3, float>, the
    arithmetic of the full fold) within rel-L2 1e-4 and FP64 within 1e-6 of
    the FP64 oracle, with the persistent (1) and the streaming (2) PCG."""
    cB, cS, sch, dT = W.fold3d_small(precision=precision)
    cB = dataclasses.replace(cB, pcg_mode=pcg_mode)
    cS = dataclasses.replace(cS, pcg_mode=pcg_mode)
    B, S = osmpm.Domain(cB), osmpm.Domain(cS)
    for _ in range(2):
        st = osmpm.osmpm_schwarz_couple(B, S, dT, sch)
        assert st["converged"] == 1
    xB_ref, xS_ref = _stored_oracle_run("fold3d_small_M2_2steps")
    assert xB_ref.shape == cB.particles.x.shape and xS_ref.shape == cS.particles.x.shape
    assert rel_disp(B.get_particles()[0], xB_ref, cB.particles.x) <= tol
    assert rel_disp(S.get_particles()[0], xS_ref, cS.particles.x) <= tol
