"""The Euler-Maruyama Brownian step (pse_bd_step): overlap repulsion from the
neighbour list, the fused dt M F + sqrt(2 kT dt) M^{1/2} z displacement and
the in-place position update, against the FP64 oracle's bd_step."""
import math

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


def _compressed(N, phi, seed, squeeze=0.97):
    """Hard spheres with overlaps: the packing and its box scaled by `squeeze`."""
    from paper_1611_09322_gb300 import workloads
    pos, L, _ = workloads.hard_spheres(N, phi, seed)
    return (pos * np.float32(squeeze)).astype(np.float32), L * squeeze


def _wrapdiff(a, b, L):
    d = a - b
    return d - L * np.round(d / L)


def _maxrel(a, b):
    return np.abs(a - b).max() / np.abs(b).max()


def _close(got, ref, rel, L, dtype):
    """|got - ref| within rel of ref's scale plus one ulp of a stored position
    (the new position is rounded to the context's type before it is read back)."""
    err = np.abs(got - ref).max()
    bound = rel * np.abs(ref).max() + float(np.spacing(dtype(L)))
    assert err <= bound, (err, bound)


@pytest.mark.parametrize("kT,J", [(1.0, 5), (0.0, 0), (0.5, 3)])
def test_bd_step_matches_oracle(torch, kT, J):
    from oracle import ewald, pse
    from paper_1611_09322_gb300 import Sampler
    N = 1500
    pos, L = _compressed(N, 0.3, 41)
    plan = ewald.plan(L, 1.0, 0.5, 1e-3)
    s = Sampler(L, 1.0, xi=0.5, tol=1e-3, fixed_iter=J if J else 0)
    d = torch.from_numpy(pos.copy()).cuda()
    dt, k_rep = 1e-3, 100.0
    s.bd_step(d, SEED, 4, dt, kT, k_rep)
    got = _wrapdiff(d.cpu().numpy().astype(np.float64), pos.astype(np.float64), L)
    _, dx, _ = pse.bd_step(pos.astype(np.float64), plan, SEED, 4, dt, kT, k_rep, n_iter=J if J else None)
    _close(got, dx, 1e-4, L, np.float32)
    assert np.all(d.cpu().numpy() >= 0) and np.all(d.cpu().numpy() < L)
    s.close()


def test_bd_step_external_force_and_fp64(torch):
    from oracle import ewald, pse
    from paper_1611_09322_gb300 import PSE_FP64, Sampler
    N = 800
    pos, L = _compressed(N, 0.25, 42)
    plan = ewald.plan(L, 1.0, 0.5, 1e-3)
    fext = np.zeros((N, 3))
    fext[:, 2] = -2.0  # uniform body force
    s = Sampler(L, 1.0, xi=0.5, tol=1e-3, precision=PSE_FP64, fixed_iter=4)
    d = torch.from_numpy(pos.astype(np.float64)).cuda()
    s.bd_step(d, SEED, 7, 2e-3, 1.0, 50.0, f_ext=torch.from_numpy(fext).cuda())
    got = _wrapdiff(d.cpu().numpy(), pos.astype(np.float64), L)
    _, dx, _ = pse.bd_step(pos.astype(np.float64), plan, SEED, 7, 2e-3, 1.0, 50.0, f_ext=fext, n_iter=4)
    _close(got, dx, 1e-9, L, np.float64)
    s.close()


def test_bd_trajectory_diffuses(torch):
    """50 steps of a dilute suspension: positions stay in the box, the mean
    square displacement per particle is positive and below that of free
    diffusion with the self-mobility, 6 D0 t (hydrodynamic interactions and
    contacts slow particles down), and above a third of it at phi = 0.1."""
    from paper_1611_09322_gb300 import Sampler, workloads
    N = 4000
    pos, L, _ = workloads.hard_spheres(N, 0.1, 43)
    s = Sampler(L, 1.0, xi=0.5, tol=1e-3)
    d = torch.from_numpy(pos.copy()).cuda()
    dt, steps = 1e-2, 50
    unwrapped = pos.astype(np.float64).copy()
    prev = pos.astype(np.float64).copy()
    for k in range(steps):
        s.bd_step(d, SEED, 1000 + k, dt, 1.0, 100.0)
        cur = d.cpu().numpy().astype(np.float64)
        unwrapped += _wrapdiff(cur, prev, L)
        prev = cur
    assert np.all(np.isfinite(prev)) and np.all(prev >= 0) and np.all(prev < L)
    msd = np.mean(np.sum((unwrapped - pos) ** 2, axis=1))
    free = 6 * (1.0 / (6 * math.pi)) * dt * steps
    assert free / 3 < msd < 1.05 * free, (msd, free)
    s.close()
