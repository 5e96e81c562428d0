"""Lanczos on the whole mobility (Sec. IV's comparison method) through the C
ABI against the FP64 oracle's full_sample: every iteration applies M = M_r +
gridded M_w to the Lanczos vector (the M F product of Sec. III).

Tolerances: FP32 1e-4 (relative 2-norm and max-relative), FP64 1e-9, as in
the other parity tests; the spreading's float atomics change the last bits
from call to call, far inside these bounds."""
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


def _rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def _maxrel(a, b):
    return np.abs(a - b).max() / np.abs(b).max()


@pytest.mark.parametrize("N,phi,xi,tol,J", [(1000, 0.1, 0.5, 1e-3, 6), (2000, 0.3, 0.6, 1e-3, 10),
                                            (1500, 0.2, 0.4, 1e-4, 14), (700, 0.1, 0.5, 1e-3, 1)])
def test_fixed_iterations_match_oracle(torch, N, phi, xi, tol, J):
    from oracle import ewald, pse
    from paper_1611_09322_gb300 import Sampler, workloads
    pos, L, _ = workloads.hard_spheres(N, phi, 41)
    s = Sampler(L, 1.0, xi=xi, tol=tol, fixed_iter=J)
    got = s.sample_full_lanczos(torch.from_numpy(pos).cuda(), SEED, 3).cpu().numpy()
    assert s.stats()["lanczos_iters"] == J
    plan = ewald.plan(L, 1.0, xi, tol, M=s.plan["M"], P=s.plan["P"])
    ref, j, _ = pse.full_sample(pos.astype(np.float64), plan, SEED, 3, n_iter=J)
    assert j == J
    assert _rel(got, ref) < 1e-4 and _maxrel(got, ref) < 1e-4, (_rel(got, ref), _maxrel(got, ref))
    s.close()


@pytest.mark.parametrize("N,phi", [(1000, 0.1), (3000, 0.2)])
def test_stop_rule_matches_oracle(torch, N, phi, record_error):
    """With the stop test the GPU takes the oracle's iteration count (unless
    the oracle's statistic sits within 5% of tol) and its sample equals the
    oracle's; the full-mobility count exceeds the real-space count of the
    PSE sample on the same configuration (the paper's point: M_r is better
    conditioned than M)."""
    from oracle import ewald, pse
    from paper_1611_09322_gb300 import Sampler, workloads
    pos, L, _ = workloads.hard_spheres(N, phi, 42)
    s = Sampler(L, 1.0, xi=0.5, tol=1e-3)
    d = torch.from_numpy(pos).cuda()
    got = s.sample_full_lanczos(d, SEED, 4).cpu().numpy()
    st = s.stats()
    assert st["converged"] == 1
    plan = ewald.plan(L, 1.0, 0.5, 1e-3, M=s.plan["M"], P=s.plan["P"])
    ref, j, hist = pse.full_sample(pos.astype(np.float64), plan, SEED, 4)
    J = st["lanczos_iters"]
    if J != j:
        assert min(abs(h / 1e-3 - 1.0) for h in hist) < 0.05, (J, j, hist)
        ref, _, _ = pse.full_sample(pos.astype(np.float64), plan, SEED, 4, n_iter=J)
    record_error(f"full-mobility Lanczos FP32 N={N} phi={phi} vs FP64 oracle", J=J, rel=_rel(got, ref),
                 maxrel=_maxrel(got, ref))
    assert _rel(got, ref) < 1e-4 and _maxrel(got, ref) < 1e-4
    s.sample(d, SEED, 4)
    assert s.stats()["lanczos_iters"] < J
    s.close()


def test_fp64_context(torch):
    from oracle import ewald, pse
    from paper_1611_09322_gb300 import PSE_FP64, Sampler, workloads
    pos, L, _ = workloads.hard_spheres(1200, 0.2, 43)
    s = Sampler(L, 1.0, xi=0.5, tol=1e-3, precision=PSE_FP64)
    got = s.sample_full_lanczos(torch.from_numpy(pos.astype(np.float64)).cuda(), SEED, 5).cpu().numpy()
    J = s.stats()["lanczos_iters"]
    plan = ewald.plan(L, 1.0, 0.5, 1e-3, M=s.plan["M"], P=s.plan["P"])
    ref, j, _ = pse.full_sample(pos.astype(np.float64), plan, SEED, 5)
    assert J == j
    assert _rel(got, ref) < 1e-9
    s.close()


def test_graph_and_host_loop_agree(torch):
    """The device-side loop in one CUDA graph and the host-driven loop run the
    same kernels: the same J and the same sample up to the spreading's
    atomic-order rounding."""
    from paper_1611_09322_gb300 import Sampler, workloads
    pos, L, _ = workloads.hard_spheres(2000, 0.1, 44)
    d = torch.from_numpy(pos).cuda()
    a = Sampler(L, 1.0, xi=0.5, tol=1e-3)
    b = Sampler(L, 1.0, xi=0.5, tol=1e-3, use_graph=False)
    ua = a.sample_full_lanczos(d, SEED, 6).cpu().numpy()
    ub = b.sample_full_lanczos(d, SEED, 6).cpu().numpy()
    assert a.stats()["lanczos_iters"] == b.stats()["lanczos_iters"]
    assert _maxrel(ua, ub) < 1e-5
    a.close()
    b.close()


def test_refused_with_the_learned_preconditioner(torch):
    from paper_1611_09322_gb300 import PseError, Sampler, workloads
    from paper_1611_09322_gb300.precond_train import init_theta
    pos, L, _ = workloads.hard_spheres(500, 0.1, 45)
    s = Sampler(L, 1.0, xi=0.5, tol=1e-3)
    s.precond_set_weights(init_theta(0))
    with pytest.raises(PseError) as e:
        s.sample_full_lanczos(torch.from_numpy(pos).cuda(), SEED, 7)
    assert "ENOTSUPPORTED" in str(e.value)
    s.precond_set_weights(None)
    s.sample_full_lanczos(torch.from_numpy(pos).cuda(), SEED, 7)
    assert s.stats()["converged"] == 1
    s.close()
