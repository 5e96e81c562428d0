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


def test_learned_form_never_costs_time_without_a_gain(torch):
    """What the trained network changes, and the fallback that keeps it
    honest: the mean Lanczos count over held-out configurations without and
    with the network decides.  If the network cuts it by at least one
    iteration it is kept and must do so on a fresh configuration too;
    otherwise the preconditioner falls back to P = I, and the learned form
    then runs exactly the plain sampler's kernels: the same J, the same
    sample bit for bit, and no more time (within 10% timing noise)."""
    from paper_1611_09322_gb300 import Sampler, precond_train, workloads
    theta, info = precond_train.train_or_fallback(xi=0.5, tol=1e-3, sets=[("hs", 4000, 0.3, 21),
                                                                           ("hs", 3000, 0.4, 22)],
                                                  steps=400, lr=3e-3)
    print(f"\nheld-out Lanczos iterations at tol 1e-3: plain {info['iters_plain']:.2f}, "
          f"learned {info['iters_learned']:.2f}, fallback {info['fallback']}")
    assert info["fallback"] == (info["gain"] < 1.0)
    pos, L, _ = workloads.hard_spheres(20000, 0.3, 23)
    d = torch.from_numpy(pos).cuda()
    plain = Sampler(L, 1.0, xi=0.5, tol=1e-3)
    learned = Sampler(L, 1.0, xi=0.5, tol=1e-3)
    learned.precond_set_weights(theta)
    jp, jl = [], []
    for k in range(5):
        up = plain.sample(d, SEED, k).clone()
        ul = learned.sample(d, SEED, k)
        sp, sl = plain.stats(), learned.stats()
        assert sp["converged"] == 1 and sl["converged"] == 1
        jp.append(sp["lanczos_iters"])
        jl.append(sl["lanczos_iters"])
        if theta is None:
            assert torch.equal(up, ul)
    if theta is not None:
        assert np.mean(jl) <= np.mean(jp) - 1.0
        return

    def t(s):
        out = torch.empty_like(d)
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
        for i in range(5):
            s.sample(d, SEED, 100 + i, out=out)
        ev[0].record()
        for i in range(40):
            s.sample(d, SEED, 200 + i, out=out)
        ev[1].record()
        torch.cuda.synchronize()
        return ev[0].elapsed_time(ev[1])
    tp, tl = min(t(plain) for _ in range(3)), min(t(learned) for _ in range(3))
    print(f"plain {tp / 40:.4f} ms, learned (fallback P = I) {tl / 40:.4f} ms per sample")
    assert jl == jp and tl <= 1.10 * tp
    plain.close()
    learned.close()
