"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle on
the same seeded inputs.  Integer work (Morton order, active nodes, Schwarz
receiver sets) must match bit for bit; floating point within the stated
tolerances (FP64 mode: particle displacement rel-L2 <= 1e-6)."""
import dataclasses

import numpy as np
import pytest

from oracle import osmpm_oracle as O
from paper_2605_09097_gb300 import workloads as W

pytestmark = pytest.mark.gpu

DISP_TOL = 1e-6  # FP64 mode: rel-L2 of particle displacement vs the oracle


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


def _perturbed(dim=2, seed=0, **kw):
    return W.perturb(W.jitter_positions(W.block(dim, **kw), seed), seed + 1)


# ----------------------------------------------------------------------------
# integer work: sort order and node sets
# ----------------------------------------------------------------------------
@pytest.mark.parametrize("case", ["cantilever", "inclusion_fine", "block3d"])
def test_morton_order_bit_exact(osmpm, case):
    if case == "cantilever":
        spec = W.cantilever()
    elif case == "inclusion_fine":
        spec = W.inclusion(dx_S=0.01)[1]
    else:
        spec = _perturbed(3, 2, n_cells=(5, 4, 3), dx=0.1)
    dom = osmpm.Domain(spec)
    np.testing.assert_array_equal(dom.get_order(), O.sort_order(spec.particles.x, spec.grid))


@pytest.mark.parametrize("dim", [2, 3])
def test_p2g_and_active_set(osmpm, dim):
    spec = _perturbed(dim, 3, n_cells=(7, 5, 4), dx=0.1)
    dom = osmpm.Domain(spec)
    nn = spec.grid.n_nodes
    dom.probe_gradient(0.01, np.zeros((nn, dim)))      # runs one P2G
    gf = O.p2g(spec.particles, spec.grid, mass_eps=spec.mass_eps)
    m = dom.get_grid(osmpm.OSMPM_FIELD_MASS)
    np.testing.assert_array_equal(m > 0, gf.active)
    np.testing.assert_allclose(m, gf.m, rtol=1e-13, atol=1e-15 * gf.m.max())
    vn = dom.get_grid(osmpm.OSMPM_FIELD_VN)
    np.testing.assert_allclose(vn, gf.vn, rtol=1e-11, atol=1e-13)


# ----------------------------------------------------------------------------
# discrete operators at a random iterate
# ----------------------------------------------------------------------------
def _problem(spec, dt, seed):
    gf = O.p2g(spec.particles, spec.grid, mass_eps=spec.mass_eps)
    mask, vel = O.dirichlet_nodes(spec.grid, [], dt)
    pr = O.make_problem(spec.particles, spec.grid, gf, dt, spec.gravity, mask, vel)
    rng = np.random.default_rng(seed)
    u = O.initial_guess(pr) + 1e-3 * spec.grid.dx * rng.standard_normal(pr.gf.vn.shape) * gf.active[:, None]
    d = rng.standard_normal(u.shape) * gf.active[:, None]
    return pr, u, d


@pytest.mark.parametrize("dim", [2, 3])
def test_gradient_hvp_energy_change(osmpm, dim):
    spec = _perturbed(dim, 5, n_cells=(8, 6, 4), dx=0.1, E=1e5, gravity=(0.2, -9.8, 0.1)[:dim])
    dt = 0.01
    pr, u, d = _problem(spec, dt, 7)
    dom = osmpm.Domain(spec)
    g_ref = O.gradient(pr, u)
    g = dom.probe_gradient(dt, u)
    scale = np.abs(g_ref).max()
    np.testing.assert_allclose(g, g_ref, rtol=0, atol=1e-11 * scale)
    H = O.hessian(pr, u)
    hd_ref = (H @ d.reshape(-1)).reshape(u.shape) * pr.gf.active[:, None]
    hd = dom.probe_hvp(dt, u, d)
    np.testing.assert_allclose(hd, hd_ref, rtol=0, atol=1e-11 * np.abs(hd_ref).max())
    s = 1e-2 * spec.grid.dx * d
    for alpha in (1.0, 0.5):
        dE_ref = O.energy_change(pr, u, s, alpha)
        dE = dom.probe_energy_change(dt, u, s, alpha)
        np.testing.assert_allclose(dE, dE_ref, rtol=1e-9)


def test_energy_change_reports_inversion(osmpm):
    spec = _perturbed(2, 5, n_cells=(4, 4), dx=0.1)
    dt = 0.01
    pr, u, d = _problem(spec, dt, 9)
    dom = osmpm.Domain(spec)
    big = 50.0 * spec.grid.dx * d
    assert np.isinf(O.energy_change(pr, u, big, 1.0))
    assert np.isinf(dom.probe_energy_change(dt, u, big, 1.0))


# ----------------------------------------------------------------------------
# whole steps
# ----------------------------------------------------------------------------
def test_free_flight(osmpm):
    spec = W.block(2, n_cells=(4, 3), dx=0.1)
    spec.particles.v[:] = np.array([0.3, -0.2])
    dom = osmpm.Domain(spec)
    st = dom.step(0.01)
    x, v, B, F = dom.get_particles()
    assert st["newton_iters"] == 1
    np.testing.assert_allclose(x, spec.particles.x + 0.01 * np.array([0.3, -0.2]), atol=1e-15)
    np.testing.assert_allclose(F, np.broadcast_to(np.eye(2), F.shape), atol=1e-14)


@pytest.mark.parametrize("pcg_mode", [0, 2])
def test_cantilever_20_steps_matches_oracle(osmpm, pcg_mode):
    """Small configuration: 2D cantilever, 2560 particles, dt = 1e-3, 20 steps
    (the persistent PCG, and the streaming PCG forced)."""
    spec = dataclasses.replace(W.cantilever(), pcg_mode=pcg_mode)
    dom = osmpm.Domain(spec)
    ref = O.DomainState.create(spec)
    x0 = spec.particles.x.copy()
    for _ in range(20):
        dom.step(1e-3)
        O.step(ref, 1e-3)
    x, v, B, F = dom.get_particles()
    assert rel_disp(x, ref.p.x, x0) <= DISP_TOL
    np.testing.assert_allclose(F, ref.p.F, atol=1e-9)
    np.testing.assert_allclose(v, ref.p.v, atol=1e-6 * np.abs(ref.p.v).max())


def test_cantilever_graph_replay_matches_plain_launches(osmpm):
    """launch_mode 0 replays a CUDA graph per Newton iteration (built once
    per iteration kind) on a created stream; launch_mode 1, and any domain
    on the legacy default stream, launch the same work directly.  All match
    the oracle; only the first replays graphs."""
    import torch
    ref = O.DomainState.create(W.cantilever())
    x0 = ref.p.x.copy()
    for _ in range(20):
        O.step(ref, 1e-3)
    stream = torch.cuda.Stream()
    for mode, st in ((0, stream.cuda_stream), (1, stream.cuda_stream), (0, 0)):
        dom = osmpm.Domain(dataclasses.replace(W.cantilever(), pcg_mode=1, launch_mode=mode), stream=st)
        newton = 0
        for _ in range(20):
            newton += dom.step(1e-3)["newton_iters"]
        x, v, B, F = dom.get_particles()
        assert rel_disp(x, ref.p.x, x0) <= DISP_TOL
        np.testing.assert_allclose(F, ref.p.F, atol=1e-9)
        c = dom.counters()
        assert c["graph_error"] == 0, f"graph build failed: cudaError {c['graph_error']}"
        if mode == 0 and st != 0:
            assert c["graph_replays"] == newton
            assert 1 <= c["graphs"] <= 8
        else:
            assert c["graph_replays"] == 0 and c["graphs"] == 0


def test_launch_mode_validated(osmpm):
    with pytest.raises(osmpm.OsmpmError):
        osmpm.Domain(dataclasses.replace(W.cantilever(), launch_mode=2))


@pytest.mark.parametrize("dim,pcg_mode", [(2, 0), (3, 0), (2, 2), (3, 2)])
def test_random_state_steps_match_oracle(osmpm, dim, pcg_mode):
    spec = _perturbed(dim, 11, n_cells=(6, 5, 4), dx=0.1, E=1e5, gravity=(0.0, -9.8, 0.0)[:dim])
    spec.pcg_mode = pcg_mode
    spec.dirichlet = [W.Dirichlet(lo=(-1e30,) * dim, hi=(0.05,) + (1e30,) * (dim - 1),
                                  comp_mask=(1 << dim) - 1)]
    dom = osmpm.Domain(spec)
    ref = O.DomainState.create(spec)
    x0 = spec.particles.x.copy()
    for _ in range(3):
        dom.step(5e-3)
        O.step(ref, 5e-3)
    x, v, B, F = dom.get_particles()
    assert rel_disp(x, ref.p.x, x0) <= DISP_TOL
    np.testing.assert_allclose(B, ref.p.B, atol=1e-8 * max(np.abs(ref.p.B).max(), 1e-12))


def test_set_particles_round_trip_and_resort(osmpm):
    spec = W.cantilever()
    dom = osmpm.Domain(spec)
    x, v, B, F = dom.get_particles()
    np.testing.assert_array_equal(x, spec.particles.x)
    rng = np.random.default_rng(1)
    x2 = x + 0.3 * spec.grid.dx * rng.uniform(-1, 1, x.shape)
    dom.set_particles(x2, v, B, F)
    got = dom.get_particles()
    np.testing.assert_array_equal(got[0], x2)
    np.testing.assert_array_equal(dom.get_order(), O.sort_order(x2, spec.grid))


# ----------------------------------------------------------------------------
# Schwarz coupling
# ----------------------------------------------------------------------------
def _run_schwarz(osmpm, cB, cS, sch, dT, steps, stream=None):
    B, S = osmpm.Domain(cB, stream=stream), osmpm.Domain(cS, stream=stream)
    rB, rS = O.DomainState.create(cB), O.DomainState.create(cS)
    out = []
    for _ in range(steps):
        st = osmpm.osmpm_schwarz_couple(B, S, dT, sch)
        ost = O.SchwarzStats()
        so = {}
        O.schwarz_step(rB, rS, dT, sch, ost, so)
        out.append((st, ost, so))
    return B, S, rB, rS, out


def test_schwarz_inclusion_small_matches_oracle(osmpm):
    cB, cS, sch, dT = W.inclusion(dx_S=0.02, M=2)
    B, S, rB, rS, out = _run_schwarz(osmpm, cB, cS, sch, dT, 2)
    st, ost, so = out[-1]
    # receiver sets of the last frame, bit for bit
    recvB = B.get_grid(osmpm.OSMPM_FIELD_RECEIVER) > 0
    recvS = S.get_grid(osmpm.OSMPM_FIELD_RECEIVER) > 0
    np.testing.assert_array_equal(recvB, so["sets"].recvB)
    np.testing.assert_array_equal(recvS, so["sets"].recvS)
    for st, ost, _ in out:
        assert st["converged"] == 1 and ost.converged
        assert abs(st["schwarz_iters"] - ost.iters) <= 1
    xB, _, _, FB = B.get_particles()
    xS, _, _, FS = S.get_particles()
    assert rel_disp(xB, rB.p.x, cB.particles.x) <= DISP_TOL
    assert rel_disp(xS, rS.p.x, cS.particles.x) <= DISP_TOL


def test_schwarz_inclusion_graph_replay_matches_oracle(osmpm):
    """The coupled step on a created stream, so every Newton iteration of
    both domains replays a captured graph while the Schwarz receiver values
    change in place between iterations; it matches the oracle like the
    plain launches."""
    import torch
    stream = torch.cuda.Stream()
    cB, cS, sch, dT = W.inclusion(dx_S=0.02, M=2)
    B, S, rB, rS, out = _run_schwarz(osmpm, cB, cS, sch, dT, 2, stream=stream.cuda_stream)
    for st, ost, _ in out:
        assert st["converged"] == 1 and ost.converged
        assert abs(st["schwarz_iters"] - ost.iters) <= 1
    xB, _, _, _ = B.get_particles()
    xS, _, _, _ = S.get_particles()
    assert rel_disp(xB, rB.p.x, cB.particles.x) <= DISP_TOL
    assert rel_disp(xS, rS.p.x, cS.particles.x) <= DISP_TOL
    for dom in (B, S):
        c = dom.counters()
        assert c["graph_error"] == 0 and c["graph_replays"] > 0 and c["graphs"] >= 1, c


@pytest.mark.parametrize("M", [1, 4])
def test_schwarz_subcycling_ratio(osmpm, M):
    cB, cS, sch, dT = W.inclusion(dx_S=0.02, M=M)
    B, S, rB, rS, out = _run_schwarz(osmpm, cB, cS, sch, dT, 1)
    xS, _, _, _ = S.get_particles()
    xB, _, _, _ = B.get_particles()
    assert rel_disp(xS, rS.p.x, cS.particles.x) <= DISP_TOL
    assert rel_disp(xB, rB.p.x, cB.particles.x) <= DISP_TOL


def test_schwarz_streaming_pcg_matches_oracle(osmpm):
    """The coupled step with the streaming PCG forced on both domains."""
    cB, cS, sch, dT = W.inclusion(dx_S=0.02, M=2)
    cB = dataclasses.replace(cB, pcg_mode=2)
    cS = dataclasses.replace(cS, pcg_mode=2)
    B, S, rB, rS, out = _run_schwarz(osmpm, cB, cS, sch, dT, 1)
    st, ost, _ = out[-1]
    assert st["converged"] == 1 and abs(st["schwarz_iters"] - ost.iters) <= 1
    assert rel_disp(S.get_particles()[0], rS.p.x, cS.particles.x) <= DISP_TOL
    assert rel_disp(B.get_particles()[0], rB.p.x, cB.particles.x) <= DISP_TOL


def test_pcg_mode_validated(osmpm):
    with pytest.raises(osmpm.OsmpmError) as e:
        osmpm.Domain(dataclasses.replace(W.cantilever(), pcg_mode=3))
    assert e.value.status == osmpm.OSMPM_E_INVALID


def test_schwarz_last_substep_projection_matches_oracle(osmpm):
    """The alternative Pi source (the fine P2G grid that ends sub-step M)."""
    cB, cS, sch, dT = W.inclusion(dx_S=0.02, M=2)
    sch = dataclasses.replace(sch, pi_source=osmpm.OSMPM_PI_LAST_SUBSTEP)
    B, S, rB, rS, out = _run_schwarz(osmpm, cB, cS, sch, dT, 1)
    st, ost, _ = out[-1]
    assert st["converged"] == 1 and ost.converged
    assert abs(st["schwarz_iters"] - ost.iters) <= 1
    assert rel_disp(S.get_particles()[0], rS.p.x, cS.particles.x) <= DISP_TOL
    assert rel_disp(B.get_particles()[0], rB.p.x, cB.particles.x) <= DISP_TOL


def test_schwarz_rejects_unknown_pi_source(osmpm):
    cB, cS, sch, dT = W.inclusion(dx_S=0.02, M=2)
    B, S = osmpm.Domain(cB), osmpm.Domain(cS)
    with pytest.raises(osmpm.OsmpmError) as e:
        osmpm.osmpm_schwarz_couple(B, S, dT, dataclasses.replace(sch, pi_source=2))
    assert e.value.status == osmpm.OSMPM_E_INVALID


def test_schwarz_no_boundary_nodes_decouples(osmpm):
    cB, cS, sch, dT = W.inclusion(dx_S=0.02, M=2)
    sch = dataclasses.replace(sch, tau_B=np.inf, tau_S=np.inf)
    B, S = osmpm.Domain(cB), osmpm.Domain(cS)
    st = osmpm.osmpm_schwarz_couple(B, S, dT, sch)
    B1, S1 = osmpm.Domain(cB), osmpm.Domain(cS)
    B1.step(dT)
    for _ in range(sch.M):
        S1.step(dT / sch.M)
    assert st["schwarz_iters"] == 2 and st["converged"] == 1
    assert (B.get_grid(osmpm.OSMPM_FIELD_RECEIVER) == 0).all()
    np.testing.assert_allclose(B.get_particles()[0], B1.get_particles()[0], atol=1e-13)
    np.testing.assert_allclose(S.get_particles()[0], S1.get_particles()[0], atol=1e-13)


def test_schwarz_identical_domains(osmpm):
    spec = W.perturb(W.block(2, n_cells=(6, 4), dx=0.1, E=1e5, gravity=(0.0, -9.81)), 4)
    Bs, Ss, sch = W.identical_pair(spec, M=1)
    B, S = osmpm.Domain(Bs), osmpm.Domain(Ss)
    st = osmpm.osmpm_schwarz_couple(B, S, 0.01, sch)
    assert (B.get_grid(osmpm.OSMPM_FIELD_RECEIVER) == 0).all()
    assert st["schwarz_iters"] == 2 and st["converged"] == 1
    ref = O.DomainState.create(spec)
    O.step(ref, 0.01)
    assert rel_disp(B.get_particles()[0], ref.p.x, spec.particles.x) <= DISP_TOL


# ----------------------------------------------------------------------------
# errors and edge cases
# ----------------------------------------------------------------------------
def test_out_of_grid_at_create(osmpm):
    spec = W.block(2, n_cells=(3, 3), dx=0.1, margin=0)
    with pytest.raises(osmpm.OsmpmError) as e:
        osmpm.Domain(spec)
    assert e.value.status == osmpm.OSMPM_E_OUT_OF_GRID


def test_out_of_grid_during_step_leaves_state(osmpm):
    spec = W.block(2, n_cells=(3, 3), dx=0.1, margin=2)
    spec.particles.v[:] = np.array([40.0, 0.0])
    dom = osmpm.Domain(spec)
    dom.step(0.01)                 # particles move one cell: support now leaves the box
    before = dom.get_particles()[0]
    with pytest.raises(osmpm.OsmpmError) as e:
        dom.step(0.01)
    assert e.value.status == osmpm.OSMPM_E_OUT_OF_GRID
    np.testing.assert_array_equal(dom.get_particles()[0], before)


def test_newton_cap_reports_and_keeps_state(osmpm):
    spec = dataclasses.replace(_perturbed(2, 1, n_cells=(3, 3), dx=0.1), newton_max=1,
                               newton_tol=1e-30)
    dom = osmpm.Domain(spec)
    with pytest.raises(osmpm.OsmpmError) as e:
        dom.step(0.01)
    assert e.value.status == osmpm.OSMPM_E_NEWTON_MAXITER
    np.testing.assert_array_equal(dom.get_particles()[0], spec.particles.x)


def test_nonfinite_input_rejected(osmpm):
    spec = W.block(2, n_cells=(3, 3), dx=0.1)
    spec.particles.v[0, 0] = np.nan
    with pytest.raises(osmpm.OsmpmError) as e:
        osmpm.Domain(spec)
    assert e.value.status == osmpm.OSMPM_E_NONFINITE


def test_schwarz_kmax_zero_warns_and_commits(osmpm):
    cB, cS, sch, dT = W.inclusion(dx_S=0.02, M=2)
    sch = dataclasses.replace(sch, k_max=0)
    B, S = osmpm.Domain(cB), osmpm.Domain(cS)
    st = osmpm.osmpm_schwarz_couple(B, S, dT, sch)
    assert st["converged"] == 0 and st["schwarz_iters"] == 1
    assert not np.array_equal(B.get_particles()[0], cB.particles.x)


def test_single_particle(osmpm):
    spec = W.block(2, n_cells=(1, 1), dx=0.1, ppc_1d=1, gravity=(0.0, -9.81))
    dom = osmpm.Domain(spec)
    ref = O.DomainState.create(spec)
    dom.step(0.01)
    O.step(ref, 0.01)
    np.testing.assert_allclose(dom.get_particles()[0], ref.p.x, atol=1e-15)


def _subset(spec, keep):
    p = spec.particles
    q = W.Particles(*(np.array(getattr(p, f.name)[keep], copy=True)
                      for f in dataclasses.fields(p)))
    return dataclasses.replace(spec, particles=q)


@pytest.mark.parametrize("dim,n_keep,pcg_mode", [(2, 67, 0), (2, 67, 2), (3, 61, 0), (3, 61, 2)])
def test_ragged_particle_counts_match_oracle(osmpm, dim, n_keep, pcg_mode):
    """Particle counts that fill neither lane groups (3 per particle in 2D,
    9 in 3D), warps nor blocks, in both PCG engines: a random subset of a
    perturbed block with gravity and a clamped face."""
    spec = _perturbed(dim, 13, n_cells=(5, 4, 3), dx=0.1, E=1e5, gravity=(0.0, -9.8, 0.0)[:dim])
    keep = np.sort(np.random.default_rng(5).choice(spec.particles.n, n_keep, replace=False))
    spec = _subset(spec, keep)
    spec.dirichlet = [W.Dirichlet(lo=(-1e30,) * dim, hi=(0.05,) + (1e30,) * (dim - 1),
                                  comp_mask=(1 << dim) - 1)]
    spec.pcg_mode = pcg_mode
    dom = osmpm.Domain(spec)
    ref = O.DomainState.create(spec)
    x0 = spec.particles.x.copy()
    for _ in range(3):
        dom.step(5e-3)
        O.step(ref, 5e-3)
    assert rel_disp(dom.get_particles()[0], ref.p.x, x0) <= DISP_TOL


@pytest.mark.parametrize("pcg_mode", [0, 2])
def test_domain_at_rest_stays_at_rest(osmpm, pcg_mode):
    """No load, no velocity, F = I: the residual is zero, Newton stops at its
    first test without a PCG iteration, and the state does not move."""
    spec = dataclasses.replace(W.block(2, n_cells=(4, 3), dx=0.1), pcg_mode=pcg_mode)
    dom = osmpm.Domain(spec)
    st = dom.step(0.01)
    x, v, B, F = dom.get_particles()
    np.testing.assert_array_equal(x, spec.particles.x)
    np.testing.assert_array_equal(v, 0.0)
    assert st["newton_iters"] == 1 and st["cg_iters"] == 0


def test_empty_domain_is_rejected(osmpm):
    spec = _subset(W.block(2, n_cells=(2, 2), dx=0.1), np.zeros(0, dtype=np.int64))
    with pytest.raises(osmpm.OsmpmError) as e:
        osmpm.Domain(spec)
    assert e.value.status == osmpm.OSMPM_E_INVALID


def test_bench_workload_full_size_one_global_step(osmpm):
    """The configuration bench.py times (inclusion, coarse dx 0.05, fine dx
    0.005, M = 2, FP64), one global Schwarz step, every particle compared
    with the oracle (rel-L2 of displacement <= 1e-6), receiver sets bit for
    bit."""
    cB, cS, sch, dT = W.inclusion(dx_S=0.005, M=2)
    B, S, rB, rS, out = _run_schwarz(osmpm, cB, cS, sch, dT, 1)
    st, ost, so = out[0]
    np.testing.assert_array_equal(B.get_grid(osmpm.OSMPM_FIELD_RECEIVER) > 0, so["sets"].recvB)
    np.testing.assert_array_equal(S.get_grid(osmpm.OSMPM_FIELD_RECEIVER) > 0, so["sets"].recvS)
    assert st["converged"] == 1 and ost.converged
    assert abs(st["schwarz_iters"] - ost.iters) <= 1
    xB, _, _, _ = B.get_particles()
    xS, _, _, FS = S.get_particles()
    assert rel_disp(xB, rB.p.x, cB.particles.x) <= DISP_TOL
    assert rel_disp(xS, rS.p.x, cS.particles.x) <= DISP_TOL
    np.testing.assert_allclose(FS, rS.p.F, atol=1e-8)


@pytest.mark.slow
def test_bench_workload_full_size_five_global_steps(osmpm):
    """The configuration bench.py times as its FP64 single-instance line
    (inclusion, coarse dx 0.05, fine dx 0.005, M = 2), five global steps,
    every particle compared with the oracle after every step (rel-L2 of
    displacement <= 1e-6: no drift over the steps whose Newton and PCG
    counts grow), receiver sets of the last step bit for bit."""
    cB, cS, sch, dT = W.inclusion(dx_S=0.005, M=2)
    B, S = osmpm.Domain(cB), osmpm.Domain(cS)
    rB, rS = O.DomainState.create(cB), O.DomainState.create(cS)
    for k in range(5):
        st = osmpm.osmpm_schwarz_couple(B, S, dT, sch)
        ost, so = O.SchwarzStats(), {}
        O.schwarz_step(rB, rS, dT, sch, ost, so)
        assert st["converged"] == 1 and ost.converged
        assert abs(st["schwarz_iters"] - ost.iters) <= 1
        assert rel_disp(B.get_particles()[0], rB.p.x, cB.particles.x) <= DISP_TOL, k
        assert rel_disp(S.get_particles()[0], rS.p.x, cS.particles.x) <= DISP_TOL, k
    np.testing.assert_array_equal(B.get_grid(osmpm.OSMPM_FIELD_RECEIVER) > 0, so["sets"].recvB)
    np.testing.assert_array_equal(S.get_grid(osmpm.OSMPM_FIELD_RECEIVER) > 0, so["sets"].recvS)
