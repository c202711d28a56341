"""Batched OS-MPM: many independent inclusion instances of uneven sizes
(the batched family: per-instance inclusion radius, inclusion modulus and
fine resolution from SplitMix64) advanced together by
osmpm_schwarz_couple_batch, each pair on its own stream.  The batch must
give each instance's own result (vs the same pair stepped alone, and vs
the oracle for the smaller instances)."""
import dataclasses

import numpy as np
import pytest

from oracle import osmpm_oracle as O
from paper_2605_09097_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2605_09097_gb300 import build
    build.build()
    from paper_2605_09097_gb300 import osmpm
    return torch, osmpm


def _pairs(torch, osmpm, specs, precision=0):
    B, S, streams = [], [], []
    for cB, cS, sch, dT in specs:
        st = torch.cuda.Stream()
        streams.append(st)
        B.append(osmpm.Domain(dataclasses.replace(cB, precision=precision), stream=st.cuda_stream))
        S.append(osmpm.Domain(dataclasses.replace(cS, precision=precision), stream=st.cuda_stream))
    return B, S, streams


def rel_disp(x_gpu, x_ref, x0):
    return np.linalg.norm(x_gpu - x_ref) / max(np.linalg.norm(x_ref - x0), 1e-300)


def test_batch_matches_individual_steps(env):
    torch, osmpm = env
    specs = [W.inclusion_instance(i) for i in range(6)]
    dxs = sorted({s[1].grid.dx for s in specs})
    assert len(dxs) == 2                      # uneven sizes in the batch
    B, S, _ = _pairs(torch, osmpm, specs)
    B1, S1, _ = _pairs(torch, osmpm, specs)
    dT = specs[0][3]
    for _ in range(2):
        stats, status = osmpm.osmpm_schwarz_couple_batch(B, S, dT, [s[2] for s in specs], n_threads=4)
        assert all(s == osmpm.OSMPM_OK for s in status)
        for i in range(len(specs)):
            osmpm.osmpm_schwarz_couple(B1[i], S1[i], dT, specs[i][2])
    for i in range(len(specs)):
        x0 = specs[i][1].particles.x
        assert rel_disp(S[i].get_particles()[0], S1[i].get_particles()[0], x0) <= 1e-9
        x0 = specs[i][0].particles.x
        assert rel_disp(B[i].get_particles()[0], B1[i].get_particles()[0], x0) <= 1e-9


def test_batch_small_instance_matches_oracle(env):
    torch, osmpm = env
    i = next(k for k in range(64) if W.inclusion_instance(k)[1].grid.dx == 0.01)
    specs = [W.inclusion_instance(i), W.inclusion_instance(i + 1)]
    B, S, _ = _pairs(torch, osmpm, specs)
    cB, cS, sch, dT = specs[0]
    oB, oS = O.DomainState.create(cB), O.DomainState.create(cS)
    osmpm.osmpm_schwarz_couple_batch(B, S, dT, [s[2] for s in specs], n_threads=2)
    O.schwarz_step(oB, oS, dT, sch)
    assert rel_disp(S[0].get_particles()[0], oS.p.x, cS.particles.x) <= 1e-6
    assert rel_disp(B[0].get_particles()[0], oB.p.x, cB.particles.x) <= 1e-6


def test_batch_rejects_shared_domains(env):
    torch, osmpm = env
    specs = [W.inclusion_instance(0)]
    B, S, _ = _pairs(torch, osmpm, specs)
    with pytest.raises(osmpm.OsmpmError) as e:
        osmpm.osmpm_schwarz_couple_batch([B[0], B[0]], [S[0], S[0]], 0.01, [specs[0][2]] * 2)
    assert e.value.status == osmpm.OSMPM_E_INVALID


def test_batch_many_concurrent_pairs_complete(env):
    """32 pairs on 16 host threads: the concurrent persistent PCG grids are
    sized so that all of them can be resident at once; every pair must
    finish (no grid barrier may give up) and converge."""
    torch, osmpm = env
    specs = [W.inclusion_instance(i) for i in range(32)]
    B, S, _ = _pairs(torch, osmpm, specs)
    stats, status = osmpm.osmpm_schwarz_couple_batch(B, S, specs[0][3], [s[2] for s in specs],
                                                     n_threads=16)
    assert all(s == osmpm.OSMPM_OK for s in status), status
    assert all(st["converged"] == 1 for st in stats)


def test_autotune_picks_a_candidate_and_steps_like_the_batch(env):
    """The autotuner's steps are ordinary batched steps: after it, each pair
    is where len(candidates) + 1 batched steps put it (any thread count
    gives each pair its own result), and the pick is the fastest candidate
    per PCG iteration."""
    torch, osmpm = env
    specs = [W.inclusion_instance(i) for i in range(4)]
    B, S, _ = _pairs(torch, osmpm, specs)
    B1, S1, _ = _pairs(torch, osmpm, specs)
    dT = specs[0][3]
    schs = [s[2] for s in specs]
    cands = [1, 2, 4]
    best, score = osmpm.osmpm_autotune_batch(B, S, dT, schs, cands)
    assert best in cands and sorted(score) == cands
    assert all(np.isfinite(v) and v > 0 for v in score.values())
    assert score[best] == min(score.values())
    for _ in range(len(cands) + 1):
        osmpm.osmpm_schwarz_couple_batch(B1, S1, dT, schs, n_threads=2)
    for i in range(len(specs)):
        x0 = specs[i][1].particles.x
        assert rel_disp(S[i].get_particles()[0], S1[i].get_particles()[0], x0) <= 1e-9


def test_autotune_rejects_bad_candidates(env):
    torch, osmpm = env
    specs = [W.inclusion_instance(0)]
    B, S, _ = _pairs(torch, osmpm, specs)
    with pytest.raises(osmpm.OsmpmError):
        osmpm.osmpm_autotune_batch(B, S, specs[0][3], [specs[0][2]], [2, 0])


def test_batch_pairs_sharing_a_stream_launch_directly(env):
    """Two pairs on one stream and two on streams of their own: the batch's
    worker threads launch directly (no graph capture from concurrent host
    threads), and every pair gets its own result."""
    torch, osmpm = env
    specs = [W.inclusion_instance(i) for i in range(4)]
    s0, s1, s2 = osmpm.create_stream(), osmpm.create_stream(), osmpm.create_stream()
    streams = [s0, s0, s1, s2]
    B = [osmpm.Domain(s[0], stream=st) for s, st in zip(specs, streams)]
    S = [osmpm.Domain(s[1], stream=st) for s, st in zip(specs, streams)]
    B1, S1, _ = _pairs(torch, osmpm, specs)
    dT = specs[0][3]
    schs = [s[2] for s in specs]
    for _ in range(2):
        _, status = osmpm.osmpm_schwarz_couple_batch(B, S, dT, schs, n_threads=4)
        assert all(s == osmpm.OSMPM_OK for s in status)
        for i in range(len(specs)):
            osmpm.osmpm_schwarz_couple(B1[i], S1[i], dT, schs[i])
    for i in range(len(specs)):
        x0 = specs[i][1].particles.x
        assert rel_disp(S[i].get_particles()[0], S1[i].get_particles()[0], x0) <= 1e-9
        c = S[i].counters()
        assert c["graph_error"] == 0 and c["graph_replays"] == 0 and c["graphs"] == 0, (i, c)
    for d in B + S:
        d.close()
    for st in (s0, s1, s2):
        osmpm.destroy_stream(st)
