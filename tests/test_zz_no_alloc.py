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


def test_noalloc_matches_oracle(torch):
    """The same product against the FP64 oracle's sparse M_r (eq. Mreal with
    the App. A scalars and the eq. self diagonal)."""
    from oracle import ewald, pse
    from paper_1611_09322_gb300 import pse_real_matvec_noalloc, workloads
    N, phi, xi, tol = 4000, 0.2, 0.5, 1e-3
    pos, L, _ = workloads.hard_spheres(N, phi, 34)
    v = np.random.default_rng(5).standard_normal((N, 3)).astype(np.float32)
    ref = pse.RealOperator(pos.astype(np.float64), ewald.plan(L, 1.0, xi, tol))(v.astype(np.float64))
    out = torch.empty((N, 3), dtype=torch.float32, device="cuda")
    pse_real_matvec_noalloc(L, 1.0, xi, tol, torch.from_numpy(pos).cuda(), torch.from_numpy(v).cuda(), out)
    got = out.cpu().numpy()
    assert np.abs(got - ref).max() <= 1e-5 * np.abs(ref).max()


def test_noalloc_allocates_nothing(torch):
    """Free device memory is the same before and after further calls: the
    scratch is the static array reserved at the first call."""
    from paper_1611_09322_gb300 import pse_real_matvec_noalloc, workloads
    N = 8000
    pos, L, _ = workloads.hard_spheres(N, 0.1, 35)
    d = torch.from_numpy(pos).cuda()
    v = torch.randn((N, 3), dtype=torch.float32, device="cuda")
    out = torch.empty_like(v)
    pse_real_matvec_noalloc(L, 1.0, 0.5, 1e-3, d, v, out)
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    for _ in range(3):
        pse_real_matvec_noalloc(L, 1.0, 0.5, 1e-3, d, v, out)
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0


def test_noalloc_neighbour_overflow_is_reported(torch):
    """More neighbours within r_cut than the static list holds (160 per
    particle at N = 16384): the list is cut, nothing is written out of
    bounds, and the call returns PSE_ENOMEM."""
    from paper_1611_09322_gb300 import PseError, pse_real_matvec_noalloc, workloads
    N = 16384
    pos, L, _ = workloads.hard_spheres(N, 0.3, 36)
    d = torch.from_numpy(pos).cuda()
    out = torch.empty_like(d)
    with pytest.raises(PseError) as e:  # xi a = 0.25, tol 1e-6: r_cut = 14.9, ~990 neighbours each
        pse_real_matvec_noalloc(L, 1.0, 0.25, 1e-6, d, d, out)
    assert "ENOMEM" in str(e.value)


def test_noalloc_rejects_too_many_cells(torch):
    """A box with more cells than the static cell arrays hold is refused
    before anything is launched."""
    from paper_1611_09322_gb300 import PseError, pse_real_matvec_noalloc
    N, L = 100, 400.0  # r_cut 5.26: 76 cells per side
    pos = torch.from_numpy(np.random.default_rng(7).uniform(0, L, (N, 3)).astype(np.float32)).cuda()
    out = torch.empty_like(pos)
    with pytest.raises(PseError) as e:
        pse_real_matvec_noalloc(L, 1.0, 0.5, 1e-3, pos, pos, out)
    assert "EINVAL" in str(e.value)


def test_noalloc_rejects_bad_tensors(torch):
    from paper_1611_09322_gb300 import pse_real_matvec_noalloc
    pos = torch.rand((50, 3), dtype=torch.float32, device="cuda") * 30
    with pytest.raises(ValueError):
        pse_real_matvec_noalloc(30.0, 1.0, 0.5, 1e-3, pos, pos.double(), torch.empty_like(pos))
    with pytest.raises(ValueError):
        pse_real_matvec_noalloc(30.0, 1.0, 0.5, 1e-3, pos, pos, torch.empty((40, 3), device="cuda"))


def test_noalloc_rejects_oversize(torch):
    from paper_1611_09322_gb300 import PseError, pse_real_matvec_noalloc, workloads
    N = 16385
    pos, L, _ = workloads.hard_spheres(N, 0.1, 33)
    d = torch.from_numpy(pos).cuda()
    out = torch.empty_like(d)
    with pytest.raises(PseError) as e:
        pse_real_matvec_noalloc(L, 1.0, 0.5, 1e-3, d, d, out)
    assert "EINVAL" in str(e.value)
