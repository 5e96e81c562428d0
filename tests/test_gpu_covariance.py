"""The covariance of the GPU sampler over 10^4 draws (N = 64 hard spheres,
phi = 0.1, FP32 context): whitened statistics and fixed projections against
the covariance the method samples -- M_r (all images within r_cut) plus the
exact covariance of the gridded wave operator -- at 4 sigma, and against the
fully converged Ewald-summed RPY mobility M within 2%."""
import math

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

SEED = 8642


@pytest.fixture(scope="module")
def torch():
    import torch as t
    if not t.cuda.is_available():
        pytest.fail("GPU test run without a CUDA device")
    from paper_1611_09322_gb300 import build
    build.build_all()
    return t


def test_sample_covariance_over_ten_thousand_draws(torch):
    from oracle import ewald, pse
    from paper_1611_09322_gb300 import Sampler, workloads
    N, n = 64, 10_000
    pos, L, _ = workloads.hard_spheres(N, 0.1, 5)
    p64 = pos.astype(np.float64)
    plan = ewald.plan(L, 1.0, 0.5, 1e-3)
    # Lanczos run to 1e-8 so that the real part is M_r^{1/2} z1 to rounding
    s = Sampler(L, 1.0, xi=0.5, tol=1e-3, lanczos_tol=1e-8)
    assert s.plan["M"] == plan.M
    d = torch.from_numpy(pos).cuda()
    U = torch.empty((n, N, 3), dtype=torch.float32, device="cuda")
    for i in range(n):
        s.sample(d, SEED, i, out=U[i])
    assert s.stats()["converged"] == 1
    U = U.reshape(n, 3 * N).double().cpu().numpy()
    s.close()
    assert np.isfinite(U).all() and abs(U.mean()) < 5 * U.std() / math.sqrt(U.size)
    Mr = ewald.mobility_real_dense(p64, L, 1.0, 0.5, plan.r_cut)
    C = Mr + pse.wave_covariance_grid(p64, plan)
    q = np.random.default_rng(1).standard_normal((20, 3 * N))
    for cov, slack in ((C, 0.0), (ewald.mobility_dense(p64, L, 1.0, 0.5, tol=1e-12)[0], 0.02)):
        Lc = np.linalg.cholesky(cov)
        white = np.sum(np.linalg.solve(Lc, U.T) ** 2, axis=0) / (3 * N)
        assert abs(white.mean() - 1) < 4 * math.sqrt(2 / (3 * N * n)) + slack, white.mean()
        ratio = (U @ q.T).var(axis=0) / np.einsum("ki,ij,kj->k", q, cov, q)
        assert np.all(np.abs(ratio - 1) < 4 * math.sqrt(2 / n) + slack), ratio
