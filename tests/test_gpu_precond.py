"""Learned preconditioner on the GPU vs the FP64 oracle network."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu
SEED = 4242


@pytest.fixture(scope="module")
def torch():
    import torch as t
    if not t.cuda.is_available():
        pytest.fail("GPU test run without a CUDA device")
    from paper_1611_09322_gb300 import build
    build.build_all()
    return t


def _setup(torch, N=1500, phi=0.3, seed=7):
    from oracle import ewald
    from paper_1611_09322_gb300 import Sampler, workloads
    pos, L, _ = workloads.hard_spheres(N, phi, seed)
    plan = ewald.plan(L, 1.0, 0.5, 1e-3)
    s = Sampler(L, 1.0, xi=0.5, tol=1e-3)
    return pos, plan, s, torch.from_numpy(pos).cuda()


def _sym(m):
    out = np.empty(m.shape[:-2] + (6,))
    out[..., 0], out[..., 1], out[..., 2] = m[..., 0, 0], m[..., 1, 1], m[..., 2, 2]
    out[..., 3], out[..., 4], out[..., 5] = m[..., 0, 1], m[..., 0, 2], m[..., 1, 2]
    return out


def _full(v):
    v = np.asarray(v, dtype=np.float64)
    m = np.zeros(v.shape[:-1] + (3, 3))
    m[..., 0, 0], m[..., 1, 1], m[..., 2, 2] = v[..., 0], v[..., 1], v[..., 2]
    m[..., 0, 1] = m[..., 1, 0] = v[..., 3]
    m[..., 0, 2] = m[..., 2, 0] = v[..., 4]
    m[..., 1, 2] = m[..., 2, 1] = v[..., 5]
    return m


def test_features_match_oracle(torch):
    from oracle import precond
    pos, plan, s, d = _setup(torch)
    f, t = s.precond_features(d)
    fo, To = precond.features(pos.astype(np.float64), plan)
    assert np.abs(f.cpu().numpy() - fo).max() < 2e-5 * max(1.0, np.abs(fo).max())
    assert np.abs(t.cpu().numpy() - _sym(To)).max() < 2e-5
    s.close()


def test_targets_match_oracle(torch):
    """Newton-Schulz (float32) = eigendecomposition (float64) of the same local M_r."""
    from oracle import precond
    pos, plan, s, d = _setup(torch, N=800, phi=0.35)
    g = s.precond_targets(d).cpu().numpy()
    idx = np.arange(0, 800, 7)
    go = precond.local_targets(pos.astype(np.float64), plan, idx=idx)
    assert np.abs(g[idx] - _sym(go)).max() < 2e-4 * np.abs(go).max()
    s.close()


def test_gradient_matches_oracle(torch):
    from oracle import precond
    from paper_1611_09322_gb300 import pse_precond_loss_grad
    pos, plan, s, d = _setup(torch, N=600)
    fo, To = precond.features(pos.astype(np.float64), plan)
    go = precond.local_targets(pos.astype(np.float64), plan)
    th = precond.init_params(1) + 0.05 * np.random.default_rng(3).standard_normal(precond.NPARAM)
    s0 = s.precond_s0
    Lo, Go = precond.loss_grad(th, fo, To, go, s0)
    c = lambda a: torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()
    loss, grad = pse_precond_loss_grad(c(fo), c(_sym(To)), c(_sym(go)), c(th), s0)
    g = grad.cpu().numpy().astype(np.float64)
    assert abs(loss.item() - Lo) < 1e-4 * abs(Lo) + 1e-9
    assert np.linalg.norm(g - Go) < 1e-3 * np.linalg.norm(Go)
    s.close()


def test_training_and_preconditioned_sample(torch):
    """GPU Adam lowers the loss below the analytic self block's; the sample with
    the trained S equals the oracle's S^{-1} (S M_r S)^{1/2} z1 after J steps."""
    from oracle import ewald, precond, pse
    from paper_1611_09322_gb300 import Sampler, precond_train, workloads
    theta, info = precond_train.train(sets=[("hs", 4000, 0.3, 11), ("hs", 3000, 0.1, 12)], steps=400, lr=3e-3)
    assert info["loss_final"] < 0.5 * info["loss_init"]
    assert info["loss_final"] < info["loss_self_block"]
    N = 1200
    pos, L, _ = workloads.hard_spheres(N, 0.3, 13)
    plan = ewald.plan(L, 1.0, 0.5, 1e-3)
    J = 8
    s = Sampler(L, 1.0, xi=0.5, tol=1e-3, fixed_iter=J)
    s.precond_set_weights(theta)
    d = torch.from_numpy(pos).cuda()
    S_gpu = _full(s.precond_blocks(d).cpu().numpy())
    fo, To = precond.features(pos.astype(np.float64), plan)
    S_or, _ = precond.forward(theta.astype(np.float64), fo, To, s.precond_s0)
    assert np.abs(S_gpu - S_or).max() < 1e-4 * np.abs(S_or).max()
    _, r, _ = s.sample(d, SEED, 3, parts=True)
    ref, _, _ = pse.real_sample(pos.astype(np.float64), plan, SEED, 3, n_iter=J, precond=S_or)
    got = r.cpu().numpy()
    assert np.linalg.norm(got - ref) / np.linalg.norm(ref) < 1e-4
    s.close()


def test_iteration_counts_with_and_without(torch):
    """What the trained network changes: Lanczos iterations to reach tol (same
    stop rule), plain vs learned, over several samples; both samples are
    converged to the same tolerance.  The gain is recorded, not assumed."""
    from paper_1611_09322_gb300 import Sampler, precond_train, workloads
    theta, _ = precond_train.train(sets=[("hs", 4000, 0.3, 21), ("hs", 3000, 0.4, 22)], steps=400, lr=3e-3)
    pos, L, _ = workloads.hard_spheres(5000, 0.3, 23)
    d = torch.from_numpy(pos).cuda()
    plain = Sampler(L, 1.0, xi=0.5, tol=1e-3)
    learned = Sampler(L, 1.0, xi=0.5, tol=1e-3)
    learned.precond_set_weights(theta)
    jp, jl = [], []
    for k in range(5):
        plain.sample(d, SEED, k)
        learned.sample(d, SEED, k)
        sp, sl = plain.stats(), learned.stats()
        assert sp["converged"] == 1 and sl["converged"] == 1
        jp.append(sp["lanczos_iters"])
        jl.append(sl["lanczos_iters"])
    print(f"\nLanczos iterations at tol 1e-3, phi 0.3: plain {np.mean(jp):.2f}, learned {np.mean(jl):.2f}")
    assert np.mean(jl) <= np.mean(jp) + 1.0
    plain.close()
    learned.close()
