"""Parity of the forces path (spreading, deterministic M F, the fused
c_det M F + c_noise M^{1/2} z step) and of the grid-noise wave sample with
the FP64 oracle, through the C ABI.

Tolerances as in test_gpu_parity: 1e-4 of the oracle's scale for FP32
contexts (float atomics in the spreading change only the last bits), 1e-9
for FP64 contexts.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

SEED = 24680


@pytest.fixture(scope="module")
def torch():
    import torch as t
    if not t.cuda.is_available():
        pytest.fail("GPU test run without a CUDA device")
    from paper_1611_09322_gb300 import build
    build.build_all()
    return t


def _hs(N, phi, seed):
    from paper_1611_09322_gb300 import workloads
    return workloads.hard_spheres(N, phi, seed)


def _maxrel(a, b):
    return np.abs(a - b).max() / np.abs(b).max()


def _rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def _sampler(L, **kw):
    from paper_1611_09322_gb300 import Sampler
    return Sampler(L, 1.0, **kw)


def _forces(N, seed=3):
    return np.random.default_rng(seed).standard_normal((N, 3)).astype(np.float32)


@pytest.mark.parametrize("N,phi,xi,tol,G", [(1000, 0.1, 0.5, 1e-3, 0), (3001, 0.2, 0.5, 1e-3, 4),
                                            (3001, 0.2, 0.5, 1e-3, 2), (3001, 0.2, 0.5, 1e-3, 1),
                                            (6000, 0.4, 0.5, 1e-3, 0), (64, 0.1, 0.5, 1e-3, 0),
                                            (2000, 0.3, 0.6, 1e-4, 0), (500, 0.05, 0.8, 1e-5, 0)])
def test_mobility_apply(torch, N, phi, xi, tol, G):
    """M F (real sparse product + spread/FFT/mode factor/FFT/interpolate) = the
    oracle's mobility_apply on the same grid, for every tile size (G = 1, 2, 4
    cells per side), dense tiles (phi = 0.4) and a box smaller than a tile;
    grids odd (25) and even (Nyquist planes)."""
    from oracle import ewald, pse
    pos, L, _ = _hs(N, phi, 21)
    plan = ewald.plan(L, 1.0, xi, tol)
    s = _sampler(L, xi=xi, tol=tol, spread_tile=G)
    assert s.plan["M"] == plan.M and s.plan["P"] == plan.P
    F = _forces(N)
    got = s.mobility_apply(torch.from_numpy(pos).cuda(), torch.from_numpy(F).cuda()).cpu().numpy()
    ref = pse.mobility_apply(F.astype(np.float64), pos.astype(np.float64), plan)
    assert _rel(got, ref) < 1e-4 and _maxrel(got, ref) < 1e-4, (_rel(got, ref), _maxrel(got, ref))
    s.close()


def test_wave_apply_part(torch):
    """The wave part alone: M F - M_r F on the GPU = the oracle's gridded M_w F."""
    from oracle import ewald, pse
    N = 1500
    pos, L, _ = _hs(N, 0.2, 22)
    plan = ewald.plan(L, 1.0, 0.5, 1e-3)
    s = _sampler(L, xi=0.5, tol=1e-3)
    F = _forces(N, 4)
    dp, dF = torch.from_numpy(pos).cuda(), torch.from_numpy(F).cuda()
    got = (s.mobility_apply(dp, dF) - s.real_matvec(dp, dF)).cpu().numpy()
    ref = pse.wave_apply_grid(F.astype(np.float64), pos.astype(np.float64), plan)
    assert _maxrel(got, ref) < 1e-4, _maxrel(got, ref)
    s.close()


@pytest.mark.parametrize("c_det,c_noise,J", [(0.7, 1.3, 5), (1.0, 1.0, 1), (0.0, 2.0, 4), (-2.0, 0.5, 3)])
def test_forces_with_noise(torch, c_det, c_noise, J):
    """c_det M F + c_noise M^{1/2} z (one CUDA graph, wave parts fused into one
    inverse FFT) = the oracle's sample_with_forces at the same J and noise."""
    from oracle import ewald, pse
    N = 1200
    pos, L, _ = _hs(N, 0.15, 23)
    plan = ewald.plan(L, 1.0, 0.5, 1e-3)
    s = _sampler(L, xi=0.5, tol=1e-3, fixed_iter=J)
    F = _forces(N, 5)
    got = s.sample_with_forces(torch.from_numpy(pos).cuda(), torch.from_numpy(F).cuda(), SEED, 9, c_det,
                               c_noise).cpu().numpy()
    ref, j = pse.sample_with_forces(pos.astype(np.float64), F.astype(np.float64), plan, SEED, 9, c_det, c_noise,
                                    n_iter=J)
    assert j == J
    assert _rel(got, ref) < 1e-4 and _maxrel(got, ref) < 1e-4, (_rel(got, ref), _maxrel(got, ref))
    s.close()


def test_forces_noise_matches_plain_sample(torch):
    """With F = 0 the forces path is c_noise times pse_sample's output (same noise)."""
    N = 2000
    pos, L, _ = _hs(N, 0.1, 24)
    s = _sampler(L, xi=0.5, tol=1e-3)
    dp = torch.from_numpy(pos).cuda()
    u = s.sample(dp, SEED, 3).cpu().numpy()
    z = torch.zeros_like(dp)
    v = s.sample_with_forces(dp, z, SEED, 3, 1.0, 2.0).cpu().numpy()
    assert _maxrel(v, 2.0 * u) < 1e-5
    s.close()


def test_forces_graph_equals_host_loop(torch):
    from oracle import ewald, pse  # noqa: F401  (oracle importable alongside)
    N = 900
    pos, L, _ = _hs(N, 0.2, 25)
    F = _forces(N, 6)
    outs = []
    for g in (True, False):
        s = _sampler(L, xi=0.5, tol=1e-3, use_graph=g)
        outs.append(s.sample_with_forces(torch.from_numpy(pos).cuda(), torch.from_numpy(F).cuda(), SEED, 1, 0.3,
                                         1.1).cpu().numpy())
        s.close()
    assert _maxrel(outs[0], outs[1]) < 1e-5


def test_forces_fp64(torch):
    from oracle import ewald, pse
    from paper_1611_09322_gb300 import PSE_FP64
    N = 700
    pos, L, _ = _hs(N, 0.2, 26)
    plan = ewald.plan(L, 1.0, 0.5, 1e-3)
    s = _sampler(L, xi=0.5, tol=1e-3, precision=PSE_FP64, fixed_iter=4)
    F = np.random.default_rng(7).standard_normal((N, 3))
    got = s.sample_with_forces(torch.from_numpy(pos.astype(np.float64)).cuda(), torch.from_numpy(F).cuda(), SEED, 2,
                               0.9, 1.1).cpu().numpy()
    ref, _ = pse.sample_with_forces(pos.astype(np.float64), F, plan, SEED, 2, 0.9, 1.1, n_iter=4)
    assert _maxrel(got, ref) < 1e-9, _maxrel(got, ref)
    det = s.mobility_apply(torch.from_numpy(pos.astype(np.float64)).cuda(), torch.from_numpy(F).cuda()).cpu().numpy()
    assert _maxrel(det, pse.mobility_apply(F, pos.astype(np.float64), plan)) < 1e-9
    s.close()


@pytest.mark.parametrize("N,phi,xi,tol,prec", [(1000, 0.1, 0.5, 1e-3, 0), (2000, 0.2, 0.6, 1e-4, 0),
                                               (64, 0.1, 0.5, 1e-3, 0), (600, 0.1, 0.5, 1e-3, 1)])
def test_grid_noise_wave_part(torch, N, phi, xi, tol, prec):
    """wave_noise = 1: white grid noise -> R2C -> mode factor -> C2R ->
    interpolation = the oracle's wave_sample_gridnoise with the same Philox
    grid noise (FP32 and FP64 contexts; odd and even grids)."""
    from oracle import ewald, pse
    pos, L, _ = _hs(N, phi, 27)
    plan = ewald.plan(L, 1.0, xi, tol)
    dt = np.float64 if prec else np.float32
    s = _sampler(L, xi=xi, tol=tol, fixed_iter=2, wave_noise=1, precision=prec)
    _, _, w = s.sample(torch.from_numpy(pos.astype(dt)).cuda(), SEED, 8, parts=True)
    got = w.cpu().numpy()
    ref = pse.wave_sample_gridnoise(pos.astype(np.float64), plan, SEED, 8)
    bound = 1e-9 if prec else 1e-4
    assert _rel(got, ref) < bound and _maxrel(got, ref) < bound, (_rel(got, ref), _maxrel(got, ref))
    s.close()


def test_grid_noise_forces_with_noise_unsupported(torch):
    from paper_1611_09322_gb300 import PseError
    N = 300
    pos, L, _ = _hs(N, 0.1, 28)
    s = _sampler(L, xi=0.5, tol=1e-3, wave_noise=1)
    dp = torch.from_numpy(pos).cuda()
    with pytest.raises(PseError):
        s.sample_with_forces(dp, torch.zeros_like(dp), 1, 1, 1.0, 1.0)
    out = s.mobility_apply(dp, torch.ones_like(dp))  # deterministic product still available
    assert torch.isfinite(out).all()
    s.close()


def test_spread_autotune_and_edge_cases(torch):
    """Timed tile choice gives the same product; N = 1; positions outside the box wrap."""
    from oracle import ewald, pse
    N = 2500
    pos, L, _ = _hs(N, 0.25, 29)
    plan = ewald.plan(L, 1.0, 0.5, 1e-3)
    F = _forces(N, 8)
    ref = pse.mobility_apply(F.astype(np.float64), pos.astype(np.float64), plan)
    s = _sampler(L, xi=0.5, tol=1e-3, autotune=2)
    shifted = pos + L * np.random.default_rng(9).integers(-2, 3, size=pos.shape).astype(np.float32)
    got = s.mobility_apply(torch.from_numpy(shifted).cuda(), torch.from_numpy(F).cuda()).cpu().numpy()
    assert _maxrel(got, ref) < 1e-4
    one = s.mobility_apply(torch.from_numpy(pos[:1].copy()).cuda(), torch.from_numpy(F[:1].copy()).cuda())
    ref1 = pse.mobility_apply(F[:1].astype(np.float64), pos[:1].astype(np.float64), plan)
    assert _maxrel(one.cpu().numpy(), ref1) < 1e-4
    s.close()


def test_mobility_apply_symmetric_positive_at_full_size(torch):
    """N = 1e6, phi = 0.1 (the sampling workload): M is symmetric positive
    definite, so <G, M F> = <F, M G> and <F, M F> > 0 for any F, G (to float
    rounding of ~1e6-term sums)."""
    pos, L, _ = _hs(1_000_000, 0.1, 1)
    s = _sampler(L, xi=0.5, tol=1e-3)
    dp = torch.from_numpy(pos).cuda()
    g = torch.Generator(device="cuda").manual_seed(5)
    F = torch.randn(dp.shape, device="cuda", generator=g)
    Gv = torch.randn(dp.shape, device="cuda", generator=g)
    MF = s.mobility_apply(dp, F).double()
    MG = s.mobility_apply(dp, Gv).double()
    a = float((Gv.double() * MF).sum())
    b = float((F.double() * MG).sum())
    assert abs(a - b) < 1e-4 * abs(float((F.double() * MF).sum()))
    assert float((F.double() * MF).sum()) > 0 and float((Gv.double() * MG).sum()) > 0
    s.close()
