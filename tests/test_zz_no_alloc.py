"""The allocation-free near-field product, for callers that may not allocate
device memory (their memory belongs to an application pool or a fixed
budget).  It must give the same M_r v as the context-based pse_real_matvec,
call after call, although every call reuses one static scratch array."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


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


@pytest.mark.parametrize("N,phi,xi,tol", [(5000, 0.1, 0.5, 1e-3), (16384, 0.3, 0.6, 1e-4)])
def test_noalloc_matches_context_matvec_twice(torch, N, phi, xi, tol):
    from paper_1611_09322_gb300 import Sampler, pse_real_matvec_noalloc, workloads
    pos, L, _ = workloads.hard_spheres(N, phi, 31)
    d = torch.from_numpy(pos).cuda()
    s = Sampler(L, 1.0, xi=xi, tol=tol)
    for call in range(2):  # two calls in a row, different vectors each time
        v = torch.from_numpy(np.random.default_rng(call).standard_normal((N, 3)).astype(np.float32)).cuda()
        ref = s.real_matvec(d, v).cpu().numpy()
        out = torch.empty_like(v)
        pse_real_matvec_noalloc(L, 1.0, xi, tol, d, v, out)
        got = out.cpu().numpy()
        assert _rel(got, ref) < 1e-5
        assert np.abs(got - ref).max() <= 1e-5 * np.abs(ref).max()
    s.close()


def test_noalloc_alternating_configurations(torch):
    """Back-to-back calls with different boxes and parameters: the shared scratch
    (cell counts, table, neighbour list) is re-initialised each time."""
    from paper_1611_09322_gb300 import Sampler, pse_real_matvec_noalloc, workloads
    cases = [(3000, 0.2, 0.5, 1e-3), (2000, 0.1, 0.7, 1e-5), (3000, 0.2, 0.5, 1e-3)]
    for N, phi, xi, tol in cases:
        pos, L, _ = workloads.hard_spheres(N, phi, 32)
        d = torch.from_numpy(pos).cuda()
        v = torch.from_numpy(np.random.default_rng(N).standard_normal((N, 3)).astype(np.float32)).cuda()
        s = Sampler(L, 1.0, xi=xi, tol=tol)
        ref = s.real_matvec(d, v).cpu().numpy()
        out = torch.empty_like(v)
        pse_real_matvec_noalloc(L, 1.0, xi, tol, d, v, out)
        assert _rel(out.cpu().numpy(), ref) < 1e-5
        s.close()


def test_noalloc_rejects_oversize(torch):
    from paper_1611_09322_gb300 import PseError, pse_real_matvec_noalloc, workloads
    N = 16385
    pos, L, _ = workloads.hard_spheres(N, 0.1, 33)
    d = torch.from_numpy(pos).cuda()
    out = torch.empty_like(d)
    with pytest.raises(PseError) as e:
        pse_real_matvec_noalloc(L, 1.0, 0.5, 1e-3, d, d, out)
    assert "EINVAL" in str(e.value)
