"""Batched sampling: one CUDA-graph launch for many independent systems."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu
SEED = 31337


@pytest.fixture(scope="module")
def torch():
    import torch as t
    if not t.cuda.is_available():
        pytest.fail("GPU test run without a CUDA device")
    from paper_1611_09322_gb300 import build
    build.build_all()
    return t


def _systems():
    from paper_1611_09322_gb300 import workloads
    spec = [("hs", 1000, 0.1, 0.5), ("gel", 3000, 0.05, 0.6), ("hs", 777, 0.35, 0.5), ("hs", 5000, 0.2, 0.4),
            ("gel", 1500, 0.15, 0.5)]
    out = []
    for k, (kind, N, phi, xi) in enumerate(spec):
        pos, L, _ = workloads.make(kind, N, phi, 500 + k)
        out.append((pos, L, xi))
    return out


def test_batch_equals_lone_contexts(torch):
    """Each system of a batch (fused multi-system kernels, pooled FFTs) gives the
    sample a lone context on the same grid gives with the same Philox streams: same Lanczos J,
    same values to float rounding (the fused kernels are other compilations
    of the same arithmetic), and repeated launches are bitwise reproducible."""
    from paper_1611_09322_gb300 import BatchSampler, Sampler
    systems = _systems()
    Ls = [L for _, L, _ in systems]
    params = [dict(xi=xi, tol=1e-3) for _, _, xi in systems]
    b = BatchSampler(Ls, 1.0, params=params)
    offsets = np.cumsum([0] + [p.shape[0] for p, _, _ in systems])
    pos_all = torch.from_numpy(np.concatenate([p for p, _, _ in systems])).cuda()
    for sample in (3, 4):  # two launches of the same graph
        out = b.sample(pos_all, offsets, SEED, sample).cpu().numpy()
        again = b.sample(pos_all, offsets, SEED, sample).cpu().numpy()
        assert np.array_equal(out, again)
        for k, (pos, L, xi) in enumerate(systems):
            s = Sampler(L, 1.0, xi=xi, tol=1e-3, system=k, grid_M=b.plan(k)["M"])
            ref = s.sample(torch.from_numpy(pos).cuda(), SEED, sample).cpu().numpy()
            got = out[offsets[k]:offsets[k + 1]]
            assert np.abs(got - ref).max() <= 1e-5 * np.abs(ref).max(), k
            assert b.stats(k)["lanczos_iters"] == s.stats()["lanczos_iters"]
            assert b.stats(k)["converged"] == 1
            s.close()
    b.close()


def test_batch_systems_draw_independent_noise(torch):
    from paper_1611_09322_gb300 import BatchSampler, workloads
    pos, L, _ = workloads.hard_spheres(2000, 0.1, 9)
    b = BatchSampler([L, L], 1.0, xi=0.5, tol=1e-3)
    pos_all = torch.from_numpy(np.concatenate([pos, pos])).cuda()
    out = b.sample(pos_all, [0, 2000, 4000], SEED, 0).cpu().numpy()
    a, c = out[:2000], out[2000:]
    assert abs(np.corrcoef(a.ravel(), c.ravel())[0, 1]) < 0.1
    b.close()


def test_batch_rebuilds_when_sizes_change(torch):
    from paper_1611_09322_gb300 import BatchSampler, Sampler, workloads
    p1, L1, _ = workloads.hard_spheres(1200, 0.1, 1)
    p2, L2, _ = workloads.hard_spheres(900, 0.1, 2)
    b = BatchSampler([L1, L2], 1.0, xi=0.5, tol=1e-3)
    b.sample(torch.from_numpy(np.concatenate([p1, p2])).cuda(), [0, 1200, 2100], SEED, 0)
    q2 = p2[:700]
    out = b.sample(torch.from_numpy(np.concatenate([p1, q2])).cuda(), [0, 1200, 1900], SEED, 1).cpu().numpy()
    s = Sampler(L2, 1.0, xi=0.5, tol=1e-3, system=1, grid_M=b.plan(1)["M"])
    ref = s.sample(torch.from_numpy(q2).cuda(), SEED, 1).cpu().numpy()
    assert np.abs(out[1200:] - ref).max() <= 1e-5 * np.abs(ref).max()
    s.close()
    b.close()


def test_batch_grids_are_size_classes_at_least_the_plan(torch):
    from oracle import ewald
    from paper_1611_09322_gb300 import BatchSampler
    systems = _systems()
    Ls = [L for _, L, _ in systems]
    params = [dict(xi=xi, tol=1e-3) for _, _, xi in systems]
    b = BatchSampler(Ls, 1.0, params=params)
    classes = {16, 20, 24, 28, 32, 40, 48, 56, 64, 72, 80, 96, 112, 128, 144, 160, 192, 224, 256}
    for k, (_, L, xi) in enumerate(systems):
        M = b.plan(k)["M"]
        assert M in classes and M >= ewald.plan(L, 1.0, xi, 1e-3).M
    b.close()


def test_tuned_grid_step(torch):
    """tune_batch_grid_step times the batch at grids 0 and 1 size classes
    finer than planned and returns per-system parameters whose grids are
    pse_batch_grid's for the chosen step; a batch built from them samples
    (every system converged, finite output) on exactly those grids, and a
    finer grid gives each system a larger xi (autotune bit 3)."""
    from paper_1611_09322_gb300 import BatchSampler, pse_batch_grid, tune_batch_grid_step
    systems = _systems()
    Ls = [L for _, L, _ in systems]
    offsets = np.cumsum([0] + [p.shape[0] for p, _, _ in systems])
    pa = torch.from_numpy(np.concatenate([p for p, _, _ in systems])).cuda()
    r = tune_batch_grid_step(Ls, pa, offsets, steps=(0, 1), reps=2, xi=0.5, tol=1e-3, autotune=8)
    assert r["step"] in (0, 1) and set(r["ms"]) == {0, 1} and all(v > 0 for v in r["ms"].values())
    xis = {}
    for st in (0, 1):
        params = [dict(xi=0.5, tol=1e-3, autotune=8, grid_M=pse_batch_grid(L, 1.0, st, xi=0.5, tol=1e-3, autotune=8))
                  for L in Ls]
        if st == r["step"]:
            assert [pk["grid_M"] for pk in params] == [pk["grid_M"] for pk in r["params"]]
        b = BatchSampler(Ls, 1.0, params=params)
        out = b.sample(pa, offsets, SEED, 3)
        assert torch.isfinite(out).all()
        for k in range(len(Ls)):
            assert b.plan(k)["M"] == params[k]["grid_M"]
            assert b.stats(k)["converged"] == 1
        xis[st] = [b.plan(k)["xi"] for k in range(len(Ls))]
        b.close()
    assert all(x1 > x0 for x0, x1 in zip(xis[0], xis[1]))


def test_batch_grid_fit_xi(torch):
    """autotune bit 3 in a batch: each system keeps its size-class grid and
    takes the largest xi that grid admits (checked against the host plan);
    its sample equals a lone context at that (xi, grid).  The oracle
    comparison at those settings is test_batch_matches_oracle."""
    from paper_1611_09322_gb300 import BatchSampler, Sampler, pse_plan
    systems = _systems()
    Ls = [L for _, L, _ in systems]
    b = BatchSampler(Ls, 1.0, params=[dict(xi=xi, tol=1e-3, autotune=8) for _, _, xi in systems])
    offsets = np.cumsum([0] + [p.shape[0] for p, _, _ in systems])
    pos_all = torch.from_numpy(np.concatenate([p for p, _, _ in systems])).cuda()
    out = b.sample(pos_all, offsets, SEED, 6).cpu().numpy()
    for k, (pos, L, xi) in enumerate(systems):
        pl = b.plan(k)
        assert pl["xi"] >= xi and np.ceil(pl["k_cut"] * L / np.pi - 1e-9) <= pl["M"]
        bigger = pse_plan(L, 1.0, xi=pl["xi"] * 1.001, tol=1e-3, grid_M=pl["M"])
        assert np.ceil(bigger["k_cut"] * L / np.pi - 1e-9) > pl["M"] or bigger["eta"] > 1
        s = Sampler(L, 1.0, xi=pl["xi"], tol=1e-3, system=k, grid_M=pl["M"])
        ref = s.sample(torch.from_numpy(pos).cuda(), SEED, 6).cpu().numpy()
        got = out[offsets[k]:offsets[k + 1]]
        assert np.abs(got - ref).max() <= 1e-5 * np.abs(ref).max(), k
        s.close()
    b.close()


def _oracle_system(pos, plan_k, k, sample, J, precond=None):
    """The FP64 oracle's sample of system k (Philox streams 2k, 2k + 1) on the
    grid, support and xi the batch planned for it: the Lanczos real part after
    exactly J steps (Sec. II B 1) plus the gridded wave part (Sec. II B 2)."""
    from oracle import ewald, pse
    p = pos.astype(np.float64)
    plan = ewald.plan(plan_k["L"], 1.0, plan_k["xi"], plan_k["tol"], M=plan_k["M"], P=plan_k["P"])
    ur, j, _ = pse.real_sample(p, plan, SEED, sample, n_iter=J, precond=precond, system=k)
    uw = pse.wave_sample_grid(p, plan, SEED, sample, system=k)
    return ur + uw, plan


def _check(got, ref, tol=1e-4):
    assert np.abs(got - ref).max() <= tol * np.abs(ref).max()
    assert np.linalg.norm(got - ref) <= tol * np.linalg.norm(ref)


@pytest.mark.parametrize("autotune", [0, 8])
def test_batch_matches_oracle(torch, autotune):
    """Every system of a batch (mixed hard spheres and gels, uneven N, own xi
    and size-class grid, all at P = 5 so the pooled node-major interpolation
    runs) equals the FP64 oracle element by element at a fixed Lanczos J;
    with autotune bit 3 each system runs at the largest xi its grid admits,
    the setting the benchmark uses."""
    from paper_1611_09322_gb300 import BatchSampler
    systems = _systems()
    J = 6
    b = BatchSampler([L for _, L, _ in systems], 1.0,
                     params=[dict(xi=xi, tol=1e-3, fixed_iter=J, autotune=autotune) for _, _, xi in systems])
    offsets = np.cumsum([0] + [p.shape[0] for p, _, _ in systems])
    pos_all = torch.from_numpy(np.concatenate([p for p, _, _ in systems])).cuda()
    out = b.sample(pos_all, offsets, SEED, 11).cpu().numpy()
    assert len({b.plan(k)["P"] for k in range(len(systems))}) == 1
    for k, (pos, L, xi) in enumerate(systems):
        assert b.stats(k)["lanczos_iters"] == J
        ref, _ = _oracle_system(pos, b.plan(k), k, 11, J)
        _check(out[offsets[k]:offsets[k + 1]], ref)
    b.close()


def test_batch_stop_rule_matches_oracle(torch):
    """Without a fixed J every system stops by the Lanczos test on its own;
    the J it reports is the oracle's (skipped where the oracle's statistic is
    within 5% of tol) and the sample equals the oracle's at that J."""
    from oracle import ewald, pse
    from paper_1611_09322_gb300 import BatchSampler
    systems = _systems()
    b = BatchSampler([L for _, L, _ in systems], 1.0, params=[dict(xi=xi, tol=1e-3) for _, _, xi in systems])
    offsets = np.cumsum([0] + [p.shape[0] for p, _, _ in systems])
    pos_all = torch.from_numpy(np.concatenate([p for p, _, _ in systems])).cuda()
    out = b.sample(pos_all, offsets, SEED, 12).cpu().numpy()
    for k, (pos, L, xi) in enumerate(systems):
        pk = b.plan(k)
        plan = ewald.plan(pk["L"], 1.0, pk["xi"], pk["tol"], M=pk["M"], P=pk["P"])
        _, j_or, hist = pse.real_sample(pos.astype(np.float64), plan, SEED, 12, system=k)
        J = b.stats(k)["lanczos_iters"]
        assert b.stats(k)["converged"] == 1
        if J != j_or:
            assert min(abs(h / 1e-3 - 1.0) for h in hist) < 0.05, (k, J, j_or)
        ref, _ = _oracle_system(pos, pk, k, 12, J)
        _check(out[offsets[k]:offsets[k + 1]], ref)
    b.close()


def test_batch_learned_matches_oracle(torch):
    """The learned + batched form: the network installed in some systems of
    the batch (pse_batch_set_precond, fused inference kernel) gives, per
    system, the oracle's S^-1 (S M_r S)^{1/2} z1 + wave part after J steps,
    S from the oracle network with the same weights; the other systems stay
    the plain sample."""
    from oracle import precond
    from paper_1611_09322_gb300 import BatchSampler
    from paper_1611_09322_gb300.precond_train import init_theta
    systems = _systems()
    J = 7
    theta = (init_theta(5) + 0.2 * np.random.default_rng(9).standard_normal(precond.NPARAM)).astype(np.float32)
    b = BatchSampler([L for _, L, _ in systems], 1.0,
                     params=[dict(xi=xi, tol=1e-3, fixed_iter=J, autotune=8) for _, _, xi in systems])
    learned = {0, 2, 3}
    for k in learned:
        b.set_precond(k, theta)
    offsets = np.cumsum([0] + [p.shape[0] for p, _, _ in systems])
    pos_all = torch.from_numpy(np.concatenate([p for p, _, _ in systems])).cuda()
    out = b.sample(pos_all, offsets, SEED, 13).cpu().numpy()
    for k, (pos, L, xi) in enumerate(systems):
        pk = b.plan(k)
        S = None
        if k in learned:
            from oracle import ewald
            plan = ewald.plan(pk["L"], 1.0, pk["xi"], pk["tol"], M=pk["M"], P=pk["P"])
            fo, To = precond.features(pos.astype(np.float64), plan)
            S, _ = precond.forward(theta.astype(np.float64), fo, To, pk["self_mobility"] ** -0.5)
        ref, _ = _oracle_system(pos, pk, k, 13, J, precond=S)
        _check(out[offsets[k]:offsets[k + 1]], ref)
    b.close()
