"""Pins of the oracle's preconditioner network (CPU)."""
import numpy as np

from oracle import ewald, precond


def _data(N=120, phi=0.3, seed=1):
    from paper_1611_09322_gb300 import workloads
    pos, L, _ = workloads.hard_spheres(N, phi, seed)
    p = pos.astype(np.float64)
    plan = ewald.plan(L, 1.0, 0.5, 1e-3)
    f, T = precond.features(p, plan)
    tg = precond.local_targets(p, plan)
    s0 = (ewald.rpy.self_real(0.5) / (6 * np.pi)) ** -0.5
    return p, plan, f, T, tg, s0


def test_backprop_matches_finite_differences():
    _, _, f, T, tg, s0 = _data()
    th = precond.init_params(3)
    th = th + 0.05 * np.random.default_rng(0).standard_normal(th.size)
    _, g = precond.loss_grad(th, f, T, tg, s0)
    eps = 1e-6
    for k in [0, 17, 127, 140, 200, 300, 417, 430, 448, 449]:
        tp, tm = th.copy(), th.copy()
        tp[k] += eps
        tm[k] -= eps
        fd = (precond.loss(tp, f, T, tg, s0) - precond.loss(tm, f, T, tg, s0)) / (2 * eps)
        assert abs(fd - g[k]) <= 1e-6 * max(1e-3, abs(fd)) + 1e-10, (k, fd, g[k])


def test_blocks_spd_equivariant_and_self_fallback():
    p, plan, f, T, tg, s0 = _data()
    th = precond.init_params(5) * 3.0
    S, _ = precond.forward(th, f, T, s0)
    assert np.linalg.eigvalsh(S).min() > 0
    # zero network output -> the analytic self block s0 I
    z = np.zeros_like(th)
    S0, _ = precond.forward(z, f, T, s0)
    assert np.allclose(S0, s0 * np.eye(3)[None])
    # rotating the configuration rotates S and leaves the features unchanged
    rng = np.random.default_rng(2)
    Q, _ = np.linalg.qr(rng.standard_normal((3, 3)))
    c = p.mean(axis=0)
    big = ewald.plan(1e4, 1.0, 0.5, 1e-3)
    f1, T1 = precond.features(p - c + 5000.0, big)
    f2, T2 = precond.features((p - c) @ Q.T + 5000.0, big)
    assert np.allclose(f1, f2, atol=1e-9)
    S1, _ = precond.forward(th, f1, T1, s0)
    S2, _ = precond.forward(th, f2, T2, s0)
    assert np.allclose(np.einsum("ab,nbc,dc->nad", Q, S1, Q), S2, atol=1e-9)


def test_targets_are_inverse_square_roots():
    """For an isolated particle the local matrix is the self block: target = s0 I."""
    plan = ewald.plan(200.0, 1.0, 0.5, 1e-3)
    p = np.array([[10.0, 10.0, 10.0], [50.0, 50.0, 50.0]])
    tg = precond.local_targets(p, plan)
    s0 = (ewald.rpy.self_real(0.5) / (6 * np.pi)) ** -0.5
    assert np.allclose(tg, s0 * np.eye(3)[None], rtol=1e-12)
    # a contact pair: block of (M_2)^{-1/2} differs from s0 I
    p = np.array([[10.0, 10.0, 10.0], [12.0, 10.0, 10.0]])
    tg = precond.local_targets(p, plan)
    M = precond._real_block_matrix(p, plan)
    lam, Q = np.linalg.eigh(M)
    assert np.allclose(tg[0], ((Q * lam ** -0.5) @ Q.T)[:3, :3])
    assert abs(tg[0][0, 0] - s0) > 1e-3
