"""Batched OS-MPM with the batched PCG service (osmpm_schwarz_couple_multi,
mixed precision): host threads drive the pairs of the batched inclusion
family, every Newton system is solved in one batched streaming PCG over a
work list of (instance, tile) with the systems of the other pairs.  Each
pair must get its own result: the same pair stepped alone (mixed precision)
within the solver tolerances, and the FP64 oracle within the mixed-precision
bound."""
import dataclasses

import numpy as np
import pytest

from oracle import osmpm_oracle as O
from paper_2605_09097_gb300 import workloads as W

pytestmark = pytest.mark.gpu

MIXED_TOL = 1e-4


@pytest.fixture(scope="module")
def env():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2605_09097_gb300 import build
    build.build()
    from paper_2605_09097_gb300 import osmpm
    return torch, osmpm


def _pairs(osmpm, specs, precision=1):
    B, S, streams = [], [], []
    for cB, cS, sch, dT in specs:
        st = osmpm.create_stream()
        streams.append(st)
        B.append(osmpm.Domain(dataclasses.replace(cB, precision=precision), stream=st))
        S.append(osmpm.Domain(dataclasses.replace(cS, precision=precision), stream=st))
    return B, S, streams


def rel_disp(x_gpu, x_ref, x0):
    return np.linalg.norm(x_gpu - x_ref) / max(np.linalg.norm(x_ref - x0), 1e-300)


@pytest.mark.parametrize("threads,dof_tile,chunk,slot_tiles",
                         [(4, 0, 0, 0), (8, 512, 4, 1), (4, 65536, 16, 3)])
def test_multi_matches_pairs_stepped_alone(env, threads, dof_tile, chunk, slot_tiles):
    """Eight instances of uneven sizes, two global steps: every pair's
    displacement within 1e-6 of the same pair stepped alone (both mixed
    precision; the batched PCG differs in its form and the order of its
    sums), the Schwarz iteration counts within one.  Launch shapes: the
    defaults; small DOF tiles and chunks; one DOF tile per system (its sums
    skip the cross-block arrival count) with product work items of three
    slot tiles."""
    torch, osmpm = env
    specs = [W.inclusion_instance(i) for i in range(8)]
    assert len({s[1].grid.dx for s in specs}) == 2
    B, S, _ = _pairs(osmpm, specs)
    B1, S1, _ = _pairs(osmpm, specs)
    dT = specs[0][3]
    for _ in range(2):
        stats, status, ms = osmpm.osmpm_schwarz_couple_multi(
            B, S, dT, [s[2] for s in specs], n_threads=threads, dof_tile=dof_tile, chunk=chunk,
            slot_tiles=slot_tiles)
        assert all(s == osmpm.OSMPM_OK for s in status)
        assert ms["batches"] > 0 and ms["chunks"] >= ms["batches"] and ms["instances"] > 0
        assert 1 <= ms["max_batch"] <= len(specs)
        assert ms["iterations"] > 0 and ms["particle_iterations"] >= ms["iterations"]
        # the timed sample of product launches (every 8th chunk)
        assert ms["hvp_launches"] > 0 and ms["hvp_ms"] > 0.0
        assert 0 < ms["hvp_particle_iterations"] <= ms["particle_iterations"]
        for i in range(len(specs)):
            st1 = osmpm.osmpm_schwarz_couple(B1[i], S1[i], dT, specs[i][2])
            assert abs(stats[i]["schwarz_iters"] - st1["schwarz_iters"]) <= 1
    for i in range(len(specs)):
        x0 = specs[i][1].particles.x
        assert rel_disp(S[i].get_particles()[0], S1[i].get_particles()[0], x0) <= 1e-6
        x0 = specs[i][0].particles.x
        assert rel_disp(B[i].get_particles()[0], B1[i].get_particles()[0], x0) <= 1e-6


def test_multi_small_instances_match_oracle(env):
    """Two small instances (fine dx 0.01) in a batch of four: two global
    steps against the FP64 oracle within the mixed-precision bound."""
    torch, osmpm = env
    small = [k for k in range(64) if W.inclusion_instance(k)[1].grid.dx == 0.01][:4]
    specs = [W.inclusion_instance(k) for k in small]
    B, S, _ = _pairs(osmpm, specs)
    dT = specs[0][3]
    refs = [(O.DomainState.create(s[0]), O.DomainState.create(s[1])) for s in specs[:2]]
    for _ in range(2):
        stats, status, _ = osmpm.osmpm_schwarz_couple_multi(B, S, dT, [s[2] for s in specs],
                                                             n_threads=4)
        assert all(s == osmpm.OSMPM_OK for s in status)
        for (oB, oS), s in zip(refs, specs[:2]):
            O.schwarz_step(oB, oS, dT, s[2])
    for i, (oB, oS) in enumerate(refs):
        cB, cS = specs[i][0], specs[i][1]
        assert rel_disp(S[i].get_particles()[0], oS.p.x, cS.particles.x) <= MIXED_TOL
        assert rel_disp(B[i].get_particles()[0], oB.p.x, cB.particles.x) <= MIXED_TOL


def test_multi_rejects_fp64_domains(env):
    torch, osmpm = env
    specs = [W.inclusion_instance(0)]
    B, S, _ = _pairs(osmpm, specs, precision=0)
    with pytest.raises(osmpm.OsmpmError) as e:
        osmpm.osmpm_schwarz_couple_multi(B, S, specs[0][3], [specs[0][2]])
    assert e.value.status == osmpm.OSMPM_E_UNSUPPORTED
