"""The timed choice of xi (pse_tune_xi): the trials it reports, the model's
xi* from the start context's stage times, and a sampler created at the
chosen xi against the FP64 oracle at that xi."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

SEED = 11235


@pytest.fixture(scope="module")
def torch():
    import torch as t
    if not t.cuda.is_available():
        pytest.fail("GPU test run without a CUDA device")
    from paper_1611_09322_gb300 import build
    build.build_all()
    return t


def _maxrel(a, b):
    return np.abs(a - b).max() / np.abs(b).max()


def _rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def _grid_fits(L, xi, M, tol=1e-3):
    from paper_1611_09322_gb300 import PseError, pse_plan
    try:
        p = pse_plan(L, 1.0, xi=xi, tol=tol, grid_M=M)
    except PseError:
        return False
    return np.ceil(p["k_cut"] * L / np.pi - 1e-9) <= M


def test_tune_xi_hard_spheres(torch):
    from oracle import ewald, pse
    from paper_1611_09322_gb300 import Sampler, pse_tune_xi, pse_xi_model, workloads
    N = 100_000
    pos, L, _ = workloads.hard_spheres(N, 0.2, 6)
    d = torch.from_numpy(pos).cuda()
    r = pse_tune_xi(L, d, xi=0.5, tol=1e-3, reps=3)
    assert r["xi_start"] == 0.5 and r["t_real"] > 0 and r["t_wave"] > 0 and r["n_grids"] >= 3
    assert r["xi_model"] == pytest.approx(pse_xi_model(0.5, r["t_real"], r["t_wave"], 3.0), rel=1e-12)
    trials = r["trials"]
    assert 4 <= len(trials) <= 8 and trials[0]["xi"] == 0.5
    ok = [t for t in trials if t["ms"] > 0]
    assert min(t["ms"] for t in ok) == r["ms_best"] and r["ms_best"] <= r["ms_start"]
    assert any(t["xi"] == r["xi_best"] and t["M"] == r["M_best"] for t in ok)
    for t in trials[1:]:  # each grid at the largest xi it admits
        assert _grid_fits(L, t["xi"], t["M"]) and not _grid_fits(L, t["xi"] * 1.001, t["M"])
        assert 1 <= t["lanczos_iters"] <= 64 and t["ms_pred"] > 0
    xs = sorted(trials[1:], key=lambda t: t["xi"])
    assert all(a["M"] < b["M"] for a, b in zip(xs, xs[1:]))
    xi, M = r["xi_best"], r["M_best"]
    s = Sampler(L, 1.0, xi=xi, tol=1e-3, grid_M=M)
    plan = ewald.plan(L, 1.0, xi, 1e-3, M=M)
    assert s.plan["M"] == plan.M and s.plan["r_cut"] == pytest.approx(plan.r_cut, rel=1e-12)
    u, ur, uw = s.sample(d, SEED, 3, parts=True)
    st = s.stats()
    assert st["converged"] == 1
    p64 = pos.astype(np.float64)
    ref_r, _, _ = pse.real_sample(p64, plan, SEED, 3, n_iter=st["lanczos_iters"])
    ref_w = pse.wave_sample_grid(p64, plan, SEED, 3)
    assert _maxrel(ur.cpu().numpy(), ref_r) < 1e-4 and _maxrel(uw.cpu().numpy(), ref_w) < 1e-4
    s.close()


def test_tune_xi_small_box_and_errors(torch):
    """A box where small splittings are impossible (r_cut >= L/2): every trial
    keeps r_cut < L/2; FP64 and preconditioned parameters are refused."""
    from paper_1611_09322_gb300 import PSE_FP64, PseError, pse_tune_xi, workloads
    pos, L, _ = workloads.hard_spheres(300, 0.2, 7)
    d = torch.from_numpy(pos).cuda()
    xi_min = np.sqrt(np.log(1e3)) / (L / 2)
    r = pse_tune_xi(L, d, xi=1.2 * xi_min, tol=1e-3, reps=2, d_f=3.0)
    assert r["ms_start"] > 0 and r["ms_best"] > 0
    assert any(t["xi"] == r["xi_best"] and t["ms"] > 0 for t in r["trials"])
    assert all(t["xi"] > xi_min for t in r["trials"])
    with pytest.raises(PseError):
        pse_tune_xi(L, d, xi=0.5, tol=1e-3, precision=PSE_FP64)
    with pytest.raises(PseError):
        pse_tune_xi(L, d, xi=0.5, tol=1e-3, use_precond=1)


def test_tuned_headline_workload_full_size(torch, record_error):
    """N = 1e6 hard spheres at phi = 0.1, tol 1e-3, in the launch configuration
    the benchmark times (xi and grid from pse_tune_xi, one CUDA graph per
    sample): the Lanczos test converges; near-field rows at sampled particles
    match the oracle; the real part after the J steps the test took and the
    wave part match the oracle's at that xi, grid and J on all 3N values."""
    from oracle import ewald, pse
    from paper_1611_09322_gb300 import Sampler, pse_tune_xi, workloads
    N = 1_000_000
    pos, L, _ = workloads.hard_spheres(N, 0.1, 1)
    d = torch.from_numpy(pos).cuda()
    r = pse_tune_xi(L, d, xi=0.5, tol=1e-3, reps=5, autotune=1)
    xi, M = r["xi_best"], r["M_best"]
    s = Sampler(L, 1.0, xi=xi, tol=1e-3, grid_M=M)
    plan = ewald.plan(L, 1.0, xi, 1e-3, M=M)
    u, ur, uw = s.sample(d, SEED, 5, parts=True)
    st = s.stats()
    assert st["converged"] == 1 and st["overflow"] == 0 and torch.isfinite(u).all()
    v = np.random.default_rng(8).standard_normal((N, 3)).astype(np.float32)
    got = s.real_matvec(d, torch.from_numpy(v).cuda()).cpu().numpy()
    rows = np.random.default_rng(9).choice(N, 200, replace=False)
    ref = pse.real_rows(pos.astype(np.float64), plan, rows, v.astype(np.float64))
    assert _maxrel(got[rows], ref) < 1e-5
    J = st["lanczos_iters"]
    u, ur, uw = u.cpu().numpy(), ur.cpu().numpy(), uw.cpu().numpy()
    s.close()
    p64 = pos.astype(np.float64)
    ref_r, _, _ = pse.real_sample(p64, plan, SEED, 5, n_iter=J)
    ref_w = pse.wave_sample_grid(p64, plan, SEED, 5)
    record_error(f"headline FP32 N=1e6 phi=0.1 tol=1e-3 xi={xi:.4f} M={M} vs FP64 oracle", J=J,
                 rel=_rel(u, ref_r + ref_w), maxrel=_maxrel(u, ref_r + ref_w), maxrel_real=_maxrel(ur, ref_r),
                 maxrel_wave=_maxrel(uw, ref_w), rel_real=_rel(ur, ref_r), rel_wave=_rel(uw, ref_w))
    assert _maxrel(ur, ref_r) < 1e-4 and _rel(ur, ref_r) < 1e-4
    assert _maxrel(uw, ref_w) < 1e-4 and _rel(uw, ref_w) < 1e-4
    assert _maxrel(u, ref_r + ref_w) < 1e-4


def test_grid_fit_xi_lone_context(torch):
    """autotune bit 3: the planned (or FFT-tuned) grid is kept and xi raised to
    the largest value it admits; the sample matches the oracle at that xi."""
    from oracle import ewald, pse
    from paper_1611_09322_gb300 import Sampler, workloads
    pos, L, _ = workloads.hard_spheres(3000, 0.2, 12)
    M0 = ewald.plan(L, 1.0, 0.5, 1e-3).M
    for at in (8, 9):
        s = Sampler(L, 1.0, xi=0.5, tol=1e-3, autotune=at)
        pl = s.plan
        assert pl["xi"] >= 0.5 and (at == 9 or pl["M"] == M0) and pl["M"] >= M0
        assert _grid_fits(L, pl["xi"], pl["M"]) and not _grid_fits(L, pl["xi"] * 1.001, pl["M"])
        plan = ewald.plan(L, 1.0, pl["xi"], 1e-3, M=pl["M"])
        _, ur, uw = s.sample(torch.from_numpy(pos).cuda(), SEED, 4, parts=True)
        J = s.stats()["lanczos_iters"]
        ref_r, _, _ = pse.real_sample(pos.astype(np.float64), plan, SEED, 4, n_iter=J)
        ref_w = pse.wave_sample_grid(pos.astype(np.float64), plan, SEED, 4)
        assert _maxrel(ur.cpu().numpy(), ref_r) < 1e-4 and _maxrel(uw.cpu().numpy(), ref_w) < 1e-4
        s.close()
