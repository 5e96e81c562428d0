"""Polydisperse sampling (the size-dependent shape factor of Sec. V) through
the C ABI against the FP64 polydisperse oracle (oracle/poly.py).

Tolerances as the monodisperse parity tests: FP32 near-field product 1e-5,
samples 1e-4 (max-relative and relative 2-norm)."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu
SEED = 97531


@pytest.fixture(scope="module")
def torch():
    import torch as t
    if not t.cuda.is_available():
        pytest.fail("GPU test run without a CUDA device")
    from paper_1611_09322_gb300 import build
    build.build_all()
    return t


def _rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def _maxrel(a, b):
    return np.abs(a - b).max() / np.abs(b).max()


def _setup(torch, N, phi, radii, seed, **kw):
    from oracle import poly
    from paper_1611_09322_gb300 import PolySampler, workloads
    pos, species, L, _ = workloads.polydisperse(N, phi, seed, radii)
    s = PolySampler(L, radii, **kw)
    plan = poly.plan(L, radii, s.plan["xi"], s.plan["tol"], M=s.plan["M"], P=s.plan["P"])
    d = torch.from_numpy(pos).cuda()
    sp = torch.from_numpy(species.astype(np.int32)).cuda()
    return pos, species, np.asarray(radii)[species], L, s, plan, d, sp


@pytest.mark.parametrize("radii,phi", [((1.0, 0.5), 0.1), ((1.0, 0.6, 1.4), 0.2)])
def test_near_field_product(torch, radii, phi):
    from oracle import poly
    pos, species, rad, L, s, plan, d, sp = _setup(torch, 3000, phi, radii, 1, xi=0.5, tol=1e-3)
    v = np.random.default_rng(2).standard_normal((3000, 3)).astype(np.float32)
    got = s.real_matvec(d, sp, torch.from_numpy(v).cuda()).cpu().numpy()
    ref = poly.RealOperator(pos.astype(np.float64), rad, plan)(v.astype(np.float64))
    assert _rel(got, ref) < 1e-5 and _maxrel(got, ref) < 1e-5, (_rel(got, ref), _maxrel(got, ref))
    s.close()


@pytest.mark.parametrize("radii,phi,J", [((1.0, 0.5), 0.1, 5), ((1.0, 0.6, 1.4), 0.2, 7), ((0.8, 1.6), 0.3, 6)])
def test_fixed_iterations_real_and_wave_parts(torch, radii, phi, J, record_error):
    """J Lanczos steps on the polydisperse M_r and the species-gridded wave part
    against the oracle, element by element."""
    from oracle import poly
    pos, species, rad, L, s, plan, d, sp = _setup(torch, 2500, phi, radii, 3, xi=0.5, tol=1e-3, fixed_iter=J)
    u, ur, uw = s.sample(d, sp, SEED, 4, parts=True)
    assert s.stats()["lanczos_iters"] == J
    p64 = pos.astype(np.float64)
    ref_r, _, _ = poly.real_sample(p64, rad, plan, SEED, 4, n_iter=J)
    ref_w = poly.wave_sample_grid(p64, species, radii, plan, SEED, 4)
    ur, uw, u = ur.cpu().numpy(), uw.cpu().numpy(), u.cpu().numpy()
    record_error(f"polydisperse FP32 N=2500 radii={radii} phi={phi}", J=J, maxrel_real=_maxrel(ur, ref_r),
                 maxrel_wave=_maxrel(uw, ref_w), rel=_rel(u, ref_r + ref_w))
    assert _maxrel(ur, ref_r) < 1e-4 and _rel(ur, ref_r) < 1e-4
    assert _maxrel(uw, ref_w) < 1e-4 and _rel(uw, ref_w) < 1e-4
    s.close()


def test_stop_rule_matches_oracle(torch):
    from oracle import poly
    pos, species, rad, L, s, plan, d, sp = _setup(torch, 4000, 0.15, (1.0, 0.5), 5, xi=0.5, tol=1e-3)
    u = s.sample(d, sp, SEED, 6).cpu().numpy()
    st = s.stats()
    assert st["converged"] == 1
    p64 = pos.astype(np.float64)
    ref_r, j, hist = poly.real_sample(p64, rad, plan, SEED, 6)
    J = st["lanczos_iters"]
    if J != j:
        assert min(abs(h / 1e-3 - 1.0) for h in hist) < 0.05, (J, j, hist)
        ref_r, _, _ = poly.real_sample(p64, rad, plan, SEED, 6, n_iter=J)
    ref = ref_r + poly.wave_sample_grid(p64, species, (1.0, 0.5), plan, SEED, 6)
    assert _maxrel(u, ref) < 1e-4 and _rel(u, ref) < 1e-4
    s.close()


def test_equal_radii_reduce_to_the_monodisperse_sampler(torch):
    """Two species of the same radius (species tables, per-species grids) and
    one species (the monodisperse path) give the monodisperse sample."""
    from paper_1611_09322_gb300 import PolySampler, Sampler, workloads
    pos, L, _ = workloads.hard_spheres(3000, 0.15, 7)
    d = torch.from_numpy(pos).cuda()
    mono = Sampler(L, 1.0, xi=0.5, tol=1e-3, fixed_iter=6)
    ref = mono.sample(d, SEED, 8).cpu().numpy()
    sp = torch.from_numpy((np.arange(3000) % 2).astype(np.int32)).cuda()
    two = PolySampler(L, (1.0, 1.0), xi=0.5, tol=1e-3, fixed_iter=6)
    one = PolySampler(L, (1.0,), xi=0.5, tol=1e-3, fixed_iter=6)
    for s, species in ((two, sp), (one, torch.zeros_like(sp))):
        got = s.sample(d, species, SEED, 8).cpu().numpy()
        assert _maxrel(got, ref) < 1e-5, _maxrel(got, ref)
        s.close()
    mono.close()


def test_monodisperse_calls_refused(torch):
    from paper_1611_09322_gb300 import PseError
    pos, species, rad, L, s, plan, d, sp = _setup(torch, 500, 0.1, (1.0, 0.5), 9, xi=0.5, tol=1e-3)
    for call in (lambda: Sampler_sample(s, d), lambda: s.mobility_apply(d, d), lambda: s.sample_full_lanczos(d, 1)):
        with pytest.raises(PseError) as e:
            call()
        assert "ENOTSUPPORTED" in str(e.value)
    s.sample(d, sp, SEED, 1)  # still usable
    assert s.stats()["converged"] == 1
    s.close()


def Sampler_sample(s, d):
    from paper_1611_09322_gb300 import Sampler
    return Sampler.sample(s, d, 1)
