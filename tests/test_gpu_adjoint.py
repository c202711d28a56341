"""The CUDA reverse mode (osmpm_record / osmpm_adjoint) against the oracle's
adjoint and against central differences of the CUDA forward steps."""
import dataclasses

import numpy as np
import pytest

from oracle import adjoint as AD
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


def _spec(dim, seed, tight=True):
    """A perturbed block with varying moduli, gravity and a clamped face."""
    rng = np.random.default_rng(seed)
    n_cells = (6, 4, 3)[:dim]
    g = (0.0, -9.81, 0.0)[:dim]
    spec = W.perturb(W.block(dim, n_cells=n_cells, dx=0.1, E=1e5, gravity=g), seed,
                     v_scale=0.2, B_scale=0.01, F_scale=0.02)
    spec.particles.E = spec.particles.E * (1.0 + 0.5 * rng.random(spec.particles.E.shape))
    clamp = W.Dirichlet(lo=(-W.BIG,) * dim, hi=(0.05,) + (W.BIG,) * (dim - 1),
                        comp_mask=(1 << dim) - 1)
    spec = dataclasses.replace(spec, dirichlet=[clamp])
    if tight:
        spec = dataclasses.replace(spec, newton_tol=1e-12, cg_rtol=1e-12, cg_max=100000)
    return spec, rng


def _gpu_gradient(osmpm, spec, dt, n_steps, c, initial_state=False):
    import torch
    dom = osmpm.Domain(spec)
    dom.record(True)
    for _ in range(n_steps):
        dom.step(dt)
    x = dom.get_particles()[0]
    g = torch.from_numpy(np.ascontiguousarray(c)).cuda()
    dE, state, st = dom.adjoint(g, initial_state)
    out = {k: v.cpu().numpy() for k, v in state.items()}
    return x, dE.cpu().numpy(), out, st, dom


def _rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


@pytest.mark.parametrize("dim", [2, 3])
def test_adjoint_matches_oracle(osmpm, dim):
    spec, rng = _spec(dim, 21 + dim)
    dt, n_steps = 0.01, 3
    n = spec.particles.x.shape[0]
    c = rng.standard_normal((n, dim))
    x, dE, st0, st, _ = _gpu_gradient(osmpm, spec, dt, n_steps, c, initial_state=True)
    op, oE, obar = AD.trajectory_gradient(spec, dt, n_steps, c, newton_tol=1e-13)
    assert _rel(x, op.x) <= 1e-10
    assert st["solves"] == n_steps and st["cg_iters"] > 0
    assert _rel(dE, oE) <= 1e-7
    assert _rel(st0["x"], obar.x) <= 1e-7
    assert _rel(st0["v"], obar.v) <= 1e-7
    assert _rel(st0["B"], obar.B) <= 1e-7
    assert _rel(st0["F"], obar.F) <= 1e-7


def test_adjoint_matches_central_differences_of_the_cuda_path(osmpm):
    spec, rng = _spec(2, 5)
    dt, n_steps = 0.01, 2
    n = spec.particles.x.shape[0]
    c = rng.standard_normal((n, 2))
    _, dE, _, _, _ = _gpu_gradient(osmpm, spec, dt, n_steps, c)

    def J(E):
        p = spec.particles.copy()
        p.E = E
        dom = osmpm.Domain(dataclasses.replace(spec, particles=p))
        for _ in range(n_steps):
            dom.step(dt)
        return float(np.sum(c * dom.get_particles()[0]))

    for p in rng.choice(n, 4, replace=False):
        h = 1e-4 * spec.particles.E[p]
        Ep, Em = spec.particles.E.copy(), spec.particles.E.copy()
        Ep[p] += h
        Em[p] -= h
        fd = (J(Ep) - J(Em)) / (2 * h)
        np.testing.assert_allclose(dE[p], fd, rtol=1e-5, atol=1e-6 * np.abs(dE).max())


def test_recording_leaves_the_forward_unchanged(osmpm):
    """Recording copies state only.  (Two runs of the forward agree to
    round-off, not bit for bit: the scatters sum with atomics.)"""
    spec, _ = _spec(2, 9, tight=False)
    a, b = osmpm.Domain(spec), osmpm.Domain(spec)
    b.record(True)
    for _ in range(3):
        sa = a.step(0.01)
        sb = b.step(0.01)
        assert sa["newton_iters"] == sb["newton_iters"]
    np.testing.assert_allclose(a.get_particles()[0], b.get_particles()[0], rtol=1e-13, atol=1e-15)
    np.testing.assert_allclose(a.get_particles()[3], b.get_particles()[3], rtol=1e-12, atol=1e-14)


def test_adjoint_keeps_the_state_and_the_record(osmpm):
    """Two objectives in a row from one record; the state is untouched."""
    import torch
    spec, rng = _spec(2, 13)
    n = spec.particles.x.shape[0]
    dom = osmpm.Domain(spec)
    dom.record(True)
    dom.step(0.01)
    dom.step(0.01)
    before = dom.get_particles()
    c1 = torch.from_numpy(rng.standard_normal((n, 2))).cuda()
    c2 = torch.from_numpy(rng.standard_normal((n, 2))).cuda()
    g1 = dom.adjoint(c1)[0].cpu().numpy()
    g2 = dom.adjoint(c2)[0].cpu().numpy()
    g12 = dom.adjoint(c1 + c2)[0].cpu().numpy()
    after = dom.get_particles()
    for u, v in zip(before, after):
        np.testing.assert_array_equal(u, v)
    # linear in dJ/dx
    np.testing.assert_allclose(g12, g1 + g2, rtol=1e-7, atol=1e-9 * np.abs(g12).max())


def test_autograd_function_gives_the_adjoint(osmpm):
    import torch
    spec, rng = _spec(2, 17)
    n = spec.particles.x.shape[0]
    dt, n_steps = 0.01, 2
    c = rng.standard_normal((n, 2))
    E = torch.tensor(spec.particles.E, dtype=torch.float64, device="cuda", requires_grad=True)
    x = osmpm.trajectory(E, spec, n_steps, dt)
    J = (x * torch.from_numpy(c).cuda()).sum()
    J.backward()
    _, dE, _, _, _ = _gpu_gradient(osmpm, spec, dt, n_steps, c)
    # two forward runs agree to round-off (atomic scatters), not bit for bit
    np.testing.assert_allclose(E.grad.cpu().numpy(), dE, rtol=1e-9, atol=1e-12 * np.abs(dE).max())


def test_cantilever_tip_gradient_matches_oracle(osmpm):
    """The 2560-particle cantilever under gravity, 6 steps of 0.05 s (inside
    the first swing, period about 1.9 s): gradient of the mean tip deflection
    with respect to every particle's modulus."""
    spec = dataclasses.replace(W.cantilever(), newton_tol=1e-10, cg_rtol=1e-12, cg_max=100000)
    x0 = spec.particles.x
    n = x0.shape[0]
    tip = x0[:, 0] > 0.98
    c = np.zeros((n, 2))
    c[tip, 1] = -1.0 / tip.sum()
    dt, n_steps = 0.05, 6
    _, dE, _, st, _ = _gpu_gradient(osmpm, spec, dt, n_steps, c)
    _, oE, _ = AD.trajectory_gradient(spec, dt, n_steps, c, newton_tol=1e-11)
    assert _rel(dE, oE) <= 1e-6
    # a stiffer beam deflects less: the total sensitivity is negative
    assert np.sum(dE * spec.particles.E) < 0


def test_adjoint_errors(osmpm):
    import torch
    spec, _ = _spec(2, 3, tight=False)
    n = spec.particles.x.shape[0]
    g = torch.zeros((n, 2), dtype=torch.float64, device="cuda")
    dom = osmpm.Domain(spec)
    with pytest.raises(osmpm.OsmpmError) as e:
        dom.adjoint(g)                                  # nothing recorded
    assert e.value.status == osmpm.OSMPM_E_INVALID
    dom.record(True)
    dom.step(0.01)
    x, v, B, F = dom.get_particles()
    dom.set_particles(x, v, B, F)                       # interrupts the record
    with pytest.raises(osmpm.OsmpmError) as e:
        dom.adjoint(g)
    assert e.value.status == osmpm.OSMPM_E_INVALID
    dom.record(True)                                    # a fresh record works again
    dom.step(0.01)
    dom.adjoint(g)
    other = osmpm.Domain(spec)
    g2 = torch.zeros((2 * n, 2), dtype=torch.float64, device="cuda")
    with pytest.raises(osmpm.OsmpmError) as e:
        osmpm.osmpm_adjoint(dom, other, g2)             # no coupled steps of this pair
    assert e.value.status == osmpm.OSMPM_E_INVALID
    mixed = osmpm.Domain(dataclasses.replace(spec, precision=1))
    with pytest.raises(osmpm.OsmpmError) as e:
        mixed.record(True)
    assert e.value.status == osmpm.OSMPM_E_UNSUPPORTED


# ----------------------------------------------------------------------------
# coupled steps (Alg. 1) in reverse
# ----------------------------------------------------------------------------
def _coupled(tight=True):
    """The small coupled inclusion (coarse 0.1, fine 0.05, M = 2) with seeded
    velocities and moduli, as in the oracle's coupled-adjoint pins."""
    cB, cS, sch, dT = W.inclusion(dx_S=0.05, dx_B=0.1, M=2, E_inc=4e6)
    rng = np.random.default_rng(3)
    out = []
    for spec in (cB, cS):
        p = spec.particles.copy()
        p.v = 0.01 * rng.standard_normal(p.v.shape)
        p.E = p.E * (1.0 + 0.2 * rng.random(p.E.shape))
        spec = dataclasses.replace(spec, particles=p)
        if tight:
            spec = dataclasses.replace(spec, newton_tol=1e-11, cg_rtol=1e-12, cg_max=100000)
        out.append(spec)
    return out[0], out[1], sch, dT, rng


def _coupled_gpu(osmpm, cB, cS, sch, dT, c, n_steps, initial_state=False):
    import torch
    B, S = osmpm.Domain(cB), osmpm.Domain(cS)
    B.record(True)
    S.record(True)
    iters = []
    for _ in range(n_steps):
        iters.append(osmpm.osmpm_schwarz_couple(B, S, dT, sch)["schwarz_iters"])
    g = torch.from_numpy(np.ascontiguousarray(c)).cuda()
    dE, state, st = osmpm.osmpm_adjoint(B, S, g, initial_state)
    return iters, dE.cpu().numpy(), {k: v.cpu().numpy() for k, v in state.items()}, st, (B, S)


def _coupled_oracle(cB, cS, sch, dT, c, iters):
    nB = cB.particles.n
    B, S = O.DomainState.create(cB), O.DomainState.create(cS)
    recs = [AD.record_schwarz_step(B, S, dT, sch, 1e-12, k) for k in iters]
    z = lambda p: AD.StateBar.zeros_like(p)
    barB, barS = z(B.p), z(S.p)
    barB.x = c[:nB].copy()
    barS.x = c[nB:].copy()
    EB = np.zeros(nB)
    ES = np.zeros(cS.particles.n)
    for rec in reversed(recs):
        barB, barS, eb, es = AD.schwarz_adjoint(rec, barB, barS)
        EB += eb
        ES += es
    return np.concatenate([EB, ES]), barB, barS, (B, S)


@pytest.mark.parametrize("n_steps", [1, 2])
def test_coupled_adjoint_matches_oracle(osmpm, n_steps):
    cB, cS, sch, dT, rng = _coupled()
    n = cB.particles.n + cS.particles.n
    c = rng.standard_normal((n, 2))
    iters, dE, st0, st, (B, S) = _coupled_gpu(osmpm, cB, cS, sch, dT, c, n_steps, True)
    oE, barB, barS, (oB, oS) = _coupled_oracle(cB, cS, sch, dT, c, iters)
    # the same unrolled iterations give the same forward ...
    assert _rel(B.get_particles()[0], oB.p.x) <= 1e-9
    assert _rel(S.get_particles()[0], oS.p.x) <= 1e-9
    assert st["solves"] == sum(k * (1 + sch.M) for k in iters)
    # ... and the same gradients
    assert _rel(dE, oE) <= 1e-6
    assert _rel(st0["x"], np.concatenate([barB.x, barS.x])) <= 1e-6
    assert _rel(st0["v"], np.concatenate([barB.v, barS.v])) <= 1e-6
    assert _rel(st0["B"], np.concatenate([barB.B, barS.B])) <= 1e-6
    assert _rel(st0["F"], np.concatenate([barB.F, barS.F])) <= 1e-6


def test_coupled_adjoint_matches_central_differences_of_the_cuda_path(osmpm):
    cB, cS, sch, dT, rng = _coupled()
    nB, nS = cB.particles.n, cS.particles.n
    c = rng.standard_normal((nB + nS, 2))
    iters, dE, _, _, _ = _coupled_gpu(osmpm, cB, cS, sch, dT, c, 1)

    def J(specB, specS):
        B, S = osmpm.Domain(specB), osmpm.Domain(specS)
        it = osmpm.osmpm_schwarz_couple(B, S, dT, sch)["schwarz_iters"]
        x = np.concatenate([B.get_particles()[0], S.get_particles()[0]])
        return float(np.sum(c * x)), it

    for which, spec, off in (("B", cB, 0), ("S", cS, nB)):
        for p in rng.choice(spec.particles.n, 2, replace=False):
            h = 1e-4 * spec.particles.E[p]
            vals = []
            for sgn in (1.0, -1.0):
                q = spec.particles.copy()
                q.E[p] += sgn * h
                s2 = dataclasses.replace(spec, particles=q)
                vals.append(J(s2, cS) if which == "B" else J(cB, s2))
            assert vals[0][1] == vals[1][1] == iters[0]
            fd = (vals[0][0] - vals[1][0]) / (2 * h)
            np.testing.assert_allclose(dE[off + p], fd, rtol=1e-4, atol=1e-5 * np.abs(dE).max())


def test_coupled_record_is_interrupted_by_a_single_step(osmpm):
    import torch
    cB, cS, sch, dT, _ = _coupled(tight=False)
    B, S = osmpm.Domain(cB), osmpm.Domain(cS)
    B.record(True)
    S.record(True)
    osmpm.osmpm_schwarz_couple(B, S, dT, sch)
    B.step(dT)                                          # not part of a coupled record
    g = torch.zeros((cB.particles.n + cS.particles.n, 2), dtype=torch.float64, device="cuda")
    with pytest.raises(osmpm.OsmpmError) as e:
        osmpm.osmpm_adjoint(B, S, g)
    assert e.value.status == osmpm.OSMPM_E_INVALID


# ----------------------------------------------------------------------------
# step checkpointing (osmpm_record with every >= 2)
# ----------------------------------------------------------------------------
def test_checkpointed_record_matches_full_record(osmpm):
    """Single-domain steps recorded with a checkpoint every 3 steps (7 steps:
    segments of 3, 3, 1) give the full record's gradients; the forward and
    the state after the adjoint are unchanged."""
    import torch
    spec, rng = _spec(2, 31)
    dt, n_steps = 0.01, 7
    n = spec.particles.n
    g = torch.from_numpy(rng.standard_normal((n, 2))).cuda()
    res = {}
    for every in (1, 3):
        dom = osmpm.Domain(spec)
        dom.record(True, every=every)
        for _ in range(n_steps):
            dom.step(dt)
        x = dom.get_particles()
        dE, st0, st = dom.adjoint(g, True)
        after = dom.get_particles()
        for a, b in zip(x, after):
            np.testing.assert_array_equal(a, b)
        res[every] = (x[0], dE.cpu().numpy(), {k: v.cpu().numpy() for k, v in st0.items()}, st)
    # two runs of the same steps (FP64 atomics: equal to the last bits)
    assert _rel(res[3][0], res[1][0]) <= 1e-12
    assert res[3][3]["solves"] == res[1][3]["solves"] == n_steps
    assert _rel(res[3][1], res[1][1]) <= 1e-8
    for k in ("x", "v", "B", "F"):
        assert _rel(res[3][2][k], res[1][2][k]) <= 1e-8, k


def test_checkpointed_coupled_record_matches_full_record_and_oracle(osmpm):
    """Three coupled steps recorded with a checkpoint every 2 steps: the
    gradients of the full record (1e-8) and of the oracle unrolled over the
    same iterations (1e-6)."""
    import torch
    cB, cS, sch, dT, rng = _coupled()
    n = cB.particles.n + cS.particles.n
    c = rng.standard_normal((n, 2))
    g = torch.from_numpy(np.ascontiguousarray(c)).cuda()
    res = {}
    for every in (1, 2):
        B, S = osmpm.Domain(cB), osmpm.Domain(cS)
        B.record(True, every=every)
        S.record(True, every=every)
        iters = [osmpm.osmpm_schwarz_couple(B, S, dT, sch)["schwarz_iters"] for _ in range(3)]
        dE, st0, st = osmpm.osmpm_adjoint(B, S, g, True)
        res[every] = (iters, dE.cpu().numpy(), {k: v.cpu().numpy() for k, v in st0.items()}, st)
    assert res[1][0] == res[2][0]
    assert res[2][3]["solves"] == res[1][3]["solves"]
    assert _rel(res[2][1], res[1][1]) <= 1e-8
    for k in ("x", "v", "B", "F"):
        assert _rel(res[2][2][k], res[1][2][k]) <= 1e-8, k
    oE, barB, barS, _ = _coupled_oracle(cB, cS, sch, dT, c, res[2][0])
    assert _rel(res[2][1], oE) <= 1e-6
    assert _rel(res[2][2]["x"], np.concatenate([barB.x, barS.x])) <= 1e-6


def _golden_module():
    import importlib.util
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", "make_oracle_runs.py")
    spec = importlib.util.spec_from_file_location("make_oracle_runs", path)
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def _stored_gradient(mod):
    import os
    rows = {"c": [], "f": []}
    with open(os.path.join(mod.OUT, mod.ADJ_NAME + ".txt")) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                parts = line.split()
                rows[parts[0]].append([float(v) for v in parts[2:]])
    c, f = np.asarray(rows["c"]), np.asarray(rows["f"])
    return np.concatenate([c[:, 0], f[:, 0]]), c[:, 1:], f[:, 1:]


@pytest.mark.slow
def test_batched_instance_gradient_over_50_checkpointed_steps(osmpm):
    """Instance 0 of the batched inclusion family, 50 coupled steps of four
    Schwarz iterations each, recorded with a checkpoint every 10 steps;
    J = mean y-displacement of the inclusion's top-cap particles.  dJ/dE
    against the FP64 oracle's adjoint unrolled over the same iterations
    (stored run, 1e-6) and against the full record (1e-8); over the first
    20 steps also against a central difference of the CUDA forward along a
    random direction of the moduli (1e-5)."""
    import torch
    mod = _golden_module()
    cB, cS, sch, dT, c = mod.adjoint_case()
    nB = cB.particles.n
    oE, oxB, oxS = _stored_gradient(mod)
    g = torch.from_numpy(np.ascontiguousarray(c)).cuda()

    def forward(specB, specS, every=0, steps=mod.ADJ_STEPS):
        B, S = osmpm.Domain(specB), osmpm.Domain(specS)
        if every:
            B.record(True, every=every)
            S.record(True, every=every)
        for _ in range(steps):
            st = osmpm.osmpm_schwarz_couple(B, S, dT, sch)
            assert st["schwarz_iters"] == mod.ADJ_ITERS
        return B, S

    res = {}
    for every in (10, 1):
        B, S = forward(cB, cS, every)
        xB, xS = B.get_particles()[0], S.get_particles()[0]
        dE, _, _ = osmpm.osmpm_adjoint(B, S, g)
        res[every] = dE.cpu().numpy()
        assert _rel(xB - cB.particles.x, oxB - cB.particles.x) <= 1e-8
        assert _rel(xS - cS.particles.x, oxS - cS.particles.x) <= 1e-8
        B.close()
        S.close()
    assert _rel(res[10], oE) <= 1e-6
    assert _rel(res[10], res[1]) <= 1e-8
    # directional central difference E_p (1 + eps w_p), w_p = +-1, over the
    # first 20 steps (checkpoints every 7: segments of 7, 7, 6).  Later in
    # this run the unrolled map stops being smooth (central differences at
    # eps 1e-3, 1e-4, 1e-5 disagree after 50 steps while they agree to seven
    # digits up to 25), as node and receiver sets change along it.
    n20 = 20
    B, S = forward(cB, cS, 7, steps=n20)
    dE20 = osmpm.osmpm_adjoint(B, S, g)[0].cpu().numpy()
    B.close()
    S.close()
    rng = np.random.default_rng(50)
    w = rng.choice([-1.0, 1.0], nB + cS.particles.n)
    eps = 1e-4

    def J(sign):
        specs = []
        for spec, ww in ((cB, w[:nB]), (cS, w[nB:])):
            q = spec.particles.copy()
            q.E = q.E * (1.0 + sign * eps * ww)
            specs.append(dataclasses.replace(spec, particles=q))
        B, S = forward(*specs, steps=n20)
        val = float(np.sum(c[nB:] * (S.get_particles()[0] - cS.particles.x)))
        B.close()
        S.close()
        return val

    fd = (J(1.0) - J(-1.0)) / (2 * eps)
    E = np.concatenate([cB.particles.E, cS.particles.E])
    ad = float(np.sum(dE20 * E * w))
    np.testing.assert_allclose(ad, fd, rtol=1e-5)
