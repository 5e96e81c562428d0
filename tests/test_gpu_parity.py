"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Tolerances (FP32 context, PSE tol 1e-3): relative 2-norm and element-wise
max error <= 1e-4 of the oracle's scale.  The FP32 path's own error budget
is ~1e-6 (float32 grid, FFT, table interpolation with 4096 knots, float32
Lanczos vectors with FP64 scalars), so 1e-4 leaves two decades of margin.
FP64 context: 1e-9.
"""
import math

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

SEED = 987654321


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


def _rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def _maxrel(a, b):
    return np.abs(a - b).max() / np.abs(b).max()


def _sampler(L, **kw):
    from paper_1611_09322_gb300 import Sampler
    return Sampler(L, 1.0, **kw)


@pytest.mark.parametrize("N,phi", [(1000, 0.1), (777, 0.3), (3001, 0.2)])
def test_real_matvec(torch, N, phi):
    """pse_real_matvec = the oracle's sparse M_r (eq. Mreal, App. A, eq. self)."""
    from oracle import ewald, pse
    pos, L, _ = _hs(N, phi, 11)
    s = _sampler(L, xi=0.5, tol=1e-3)
    v = np.random.default_rng(1).standard_normal((N, 3)).astype(np.float32)
    got = s.real_matvec(torch.from_numpy(pos).cuda(), torch.from_numpy(v).cuda()).cpu().numpy()
    ref = pse.RealOperator(pos.astype(np.float64), ewald.plan(L, 1.0, 0.5, 1e-3))(v.astype(np.float64))
    assert _rel(got, ref) < 1e-5 and _maxrel(got, ref) < 1e-5
    s.close()


@pytest.mark.parametrize("N,phi,xi,tol", [(1000, 0.1, 0.5, 1e-3), (64, 0.1, 0.5, 1e-3), (2000, 0.2, 0.6, 1e-4),
                                          (500, 0.05, 0.8, 1e-5)])
def test_wave_part(torch, N, phi, xi, tol):
    """Wave sample: same Philox noise, same grid and Gaussian -> same NUFFT result.
    Cases cover odd M (25), even M with Nyquist planes (10), P = 6 and P = 8."""
    from oracle import ewald, pse
    pos, L, _ = _hs(N, phi, 12)
    plan = ewald.plan(L, 1.0, xi, tol)
    s = _sampler(L, xi=xi, tol=tol, fixed_iter=2)
    assert s.plan["M"] == plan.M and s.plan["P"] == plan.P
    _, _, w = s.sample(torch.from_numpy(pos).cuda(), SEED, 5, parts=True)
    got = w.cpu().numpy()
    ref = pse.wave_sample_grid(pos.astype(np.float64), plan, SEED, 5)
    assert _rel(got, ref) < 1e-4 and _maxrel(got, ref) < 1e-4, (_rel(got, ref), _maxrel(got, ref))
    s.close()


@pytest.mark.parametrize("N,phi,form", [(3001, 0.2, 0), (6000, 0.4, 0), (64, 0.1, 0), (3001, 0.2, 1),
                                        (64, 0.1, 1)])
def test_interpolation_dense_and_tiny(torch, N, phi, form):
    """The wave sample for a dense packing and a box of a few grid nodes, with
    the node-major grid copy (form 0) and from the planar grids (form 1)."""
    from oracle import ewald, pse
    pos, L, _ = _hs(N, phi, 16)
    plan = ewald.plan(L, 1.0, 0.5, 1e-3)
    s = _sampler(L, xi=0.5, tol=1e-3, fixed_iter=2, interp_form=form)
    _, _, w = s.sample(torch.from_numpy(pos).cuda(), SEED, 6, parts=True)
    got = w.cpu().numpy()
    ref = pse.wave_sample_grid(pos.astype(np.float64), plan, SEED, 6)
    assert _rel(got, ref) < 1e-4 and _maxrel(got, ref) < 1e-4, (_rel(got, ref), _maxrel(got, ref))
    s.close()


@pytest.mark.parametrize("tol,xi", [(1e-2, 0.5), (5e-3, 0.5), (1e-4, 0.5), (3e-5, 0.5), (1e-5, 0.6), (1e-6, 0.5),
                                    (3e-7, 0.5), (1e-7, 0.5)])
def test_interpolation_support_sizes(torch, tol, xi):
    """Node-major interpolation for every compiled support P = 3 .. 10 (tol
    1e-2 .. 3e-7) and the planar fallback beyond it (P = 11 at 1e-7) against
    the oracle's wave sample, and equal to the planar form."""
    from oracle import ewald, pse
    N = 1200
    pos, L, _ = _hs(N, 0.15, 17)
    plan = ewald.plan(L, 1.0, xi, tol)
    outs = []
    for form in (0, 1):
        s = _sampler(L, xi=xi, tol=tol, fixed_iter=1, interp_form=form)
        assert s.plan["P"] == plan.P
        _, _, w = s.sample(torch.from_numpy(pos).cuda(), SEED, 2, parts=True)
        outs.append(w.cpu().numpy())
        s.close()
    ref = pse.wave_sample_grid(pos.astype(np.float64), plan, SEED, 2)
    assert _maxrel(outs[0], ref) < 1e-4 and _maxrel(outs[0], outs[1]) < 1e-5, plan.P


@pytest.mark.parametrize("N,phi,J", [(1000, 0.1, 6), (1000, 0.1, 1), (1500, 0.3, 12), (130, 0.2, 30)])
def test_real_part_fixed_iterations(torch, N, phi, J):
    """Real sample after exactly J Lanczos steps = the oracle's J-step Lanczos."""
    from oracle import ewald, pse
    pos, L, _ = _hs(N, phi, 13)
    plan = ewald.plan(L, 1.0, 0.5, 1e-3)
    s = _sampler(L, xi=0.5, tol=1e-3, fixed_iter=J)
    _, r, _ = s.sample(torch.from_numpy(pos).cuda(), SEED, 9, parts=True)
    got = r.cpu().numpy()
    st = s.stats()
    assert st["lanczos_iters"] == J
    ref, j, _ = pse.real_sample(pos.astype(np.float64), plan, SEED, 9, n_iter=J)
    assert _rel(got, ref) < 1e-4 and _maxrel(got, ref) < 1e-4, (_rel(got, ref), _maxrel(got, ref))
    s.close()


@pytest.mark.parametrize("shape", [11, 12])
@pytest.mark.parametrize("kind,N,phi", [("hs", 20000, 0.2), ("hs", 30000, 0.1), ("gel", 30000, 0.1)])
def test_brick_tiled_and_list_free_matvec(torch, kind, N, phi, shape):
    """Shape 11 (each brick's neighbourhood staged in shared memory) and
    shape 12 (no neighbour list: every product walks the 27 stencil cells) on
    boxes large enough for many bricks, hard spheres and a clustered gel
    (whose densest bricks overflow the staging and gather from global
    memory): the J-step real part equals the oracle's and the default
    shape's."""
    from oracle import ewald, pse
    from paper_1611_09322_gb300 import workloads
    pos, L, _ = workloads.make(kind, N, phi, 16)
    J = 5
    plan = ewald.plan(L, 1.0, 0.5, 1e-3)
    d = torch.from_numpy(pos).cuda()
    outs = []
    for sh in (shape, 5):
        s = _sampler(L, xi=0.5, tol=1e-3, fixed_iter=J, matvec_shape=sh)
        _, r, _ = s.sample(d, SEED, 10, parts=True)
        assert s.stats()["matvec_shape"] == sh
        outs.append(r.cpu().numpy())
        s.close()
    ref, _, _ = pse.real_sample(pos.astype(np.float64), plan, SEED, 10, n_iter=J)
    assert _rel(outs[0], ref) < 1e-4 and _maxrel(outs[0], ref) < 1e-4
    assert _maxrel(outs[0], outs[1]) < 1e-5


@pytest.mark.parametrize("shape", [1, 2, 3, 4, 5, 6, 7, 8, 9, 10, 11, 12, 0])
def test_matvec_launch_shapes(torch, shape):
    """Every near-field matvec launch shape (threads x gathers per particle,
    threads per block), and the timed choice (shape 0 with autotune bit 2),
    gives the oracle's J-step real part; dense packing so that some lists
    exceed one gather round."""
    from oracle import ewald, pse
    N, J = 1500, 6
    pos, L, _ = _hs(N, 0.35, 15)
    plan = ewald.plan(L, 1.0, 0.5, 1e-3)
    s = _sampler(L, xi=0.5, tol=1e-3, fixed_iter=J, matvec_shape=shape, autotune=4 if shape == 0 else 0)
    _, r, _ = s.sample(torch.from_numpy(pos).cuda(), SEED, 9, parts=True)
    got = r.cpu().numpy()
    st = s.stats()
    assert st["lanczos_iters"] == J
    assert st["matvec_shape"] == shape if shape else 1 <= st["matvec_shape"] <= 11
    ref, _, _ = pse.real_sample(pos.astype(np.float64), plan, SEED, 9, n_iter=J)
    assert _rel(got, ref) < 1e-4 and _maxrel(got, ref) < 1e-4, (_rel(got, ref), _maxrel(got, ref))
    s.close()


@pytest.mark.parametrize("N,phi,xi,tol", [(1000, 0.1, 0.5, 1e-3), (2000, 0.3, 0.5, 1e-3), (1200, 0.2, 0.4, 1e-4)])
def test_full_sample_with_convergence_test(torch, N, phi, xi, tol):
    """Default path (device-side Lanczos loop with the stop test): the GPU stops
    at the oracle's j, and u = u_real + u_wave matches the oracle's sample."""
    from oracle import ewald, pse
    pos, L, _ = _hs(N, phi, 14)
    plan = ewald.plan(L, 1.0, xi, tol)
    s = _sampler(L, xi=xi, tol=tol)
    u = s.sample(torch.from_numpy(pos).cuda(), SEED, 21).cpu().numpy()
    st = s.stats()
    ur, jo, hist = pse.real_sample(pos.astype(np.float64), plan, SEED, 21)
    assert st["converged"] == 1
    if st["lanczos_iters"] != jo:
        # only acceptable when the oracle's stop statistic sits at the threshold
        k = min(st["lanczos_iters"], jo)
        assert abs(hist[k - 2] - tol) < 0.05 * tol, (st, jo, hist)
        pytest.skip("stop statistic within 5% of tol: iteration counts legitimately differ")
    ref = ur + pse.wave_sample_grid(pos.astype(np.float64), plan, SEED, 21)
    assert _rel(u, ref) < 1e-4 and _maxrel(u, ref) < 1e-4
    s.close()


def test_fp64_context(torch, record_error):
    """precision = FP64 (N = 1000 hard spheres at phi = 0.1, tol 1e-3): the
    whole path in float64 matches the oracle to 1e-9."""
    from oracle import ewald, pse
    from paper_1611_09322_gb300 import PSE_FP64
    N, phi = 1000, 0.1
    pos, L, _ = _hs(N, phi, 15)
    plan = ewald.plan(L, 1.0, 0.5, 1e-3)
    s = _sampler(L, xi=0.5, tol=1e-3, precision=PSE_FP64)
    p64 = torch.from_numpy(pos.astype(np.float64)).cuda()
    u, r, w = s.sample(p64, SEED, 3, parts=True)
    st = s.stats()
    ur, jo, _ = pse.real_sample(pos.astype(np.float64), plan, SEED, 3)
    uw = pse.wave_sample_grid(pos.astype(np.float64), plan, SEED, 3)
    assert st["lanczos_iters"] == jo
    u = u.cpu().numpy()
    record_error("config1 FP64 N=1000 phi=0.1 vs oracle (same algorithm)", J=jo, rel=_rel(u, ur + uw),
                 maxrel=_maxrel(u, ur + uw))
    assert _rel(w.cpu().numpy(), uw) < 1e-9
    assert _rel(r.cpu().numpy(), ur) < 1e-9
    assert _rel(u, ur + uw) < 1e-9
    s.close()


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_against_exact_split_sample_N64(torch, prec, record_error):
    """N = 64 hard spheres at phi = 0.1 (the dense cross-check of the FP64
    configuration): the sample at tol 1e-3 against the exact split sample
    M_r^{1/2} z1 (dense eigendecomposition of the all-image M_r at tol 1e-3's
    r_cut) + the exact non-uniform wave sum with the same noise.  The
    difference is the method's own truncation (Lanczos stop, NUFFT
    quadrature).  The oracle itself sits at ~6e-5 (real) and ~0.019 (wave,
    relative 2-norm) from this exact sample on this configuration, the wave
    error constant of the tolerance rule; the bounds are 3 tol and 30 tol."""
    from oracle import ewald, pse
    from paper_1611_09322_gb300 import PSE_FP32, PSE_FP64
    N, phi, xi, tol = 64, 0.1, 0.5, 1e-3
    pos, L, _ = _hs(N, phi, 17)
    p64 = pos.astype(np.float64)
    plan = ewald.plan(L, 1.0, xi, tol)
    s = _sampler(L, xi=xi, tol=tol, precision=PSE_FP64 if prec == "fp64" else PSE_FP32)
    d = torch.from_numpy(p64 if prec == "fp64" else pos).cuda()
    u, r, w = s.sample(d, SEED, 5, parts=True)
    r, w = r.cpu().numpy().astype(np.float64), w.cpu().numpy().astype(np.float64)
    Mr = ewald.mobility_real_dense(p64, L, 1.0, xi, plan.r_cut)
    lam, Q = np.linalg.eigh(Mr)
    assert lam.min() > 0
    z1 = pse.real_noise(N, SEED, 5).ravel()
    ur_exact = (Q @ (np.sqrt(lam) * (Q.T @ z1))).reshape(N, 3)
    uw_exact = pse.wave_sample_direct(p64, plan, SEED, 5)
    er, ew = _rel(r, ur_exact), _rel(w, uw_exact)
    eu = _rel(r + w, ur_exact + uw_exact)
    record_error(f"config1 {prec} N=64 vs exact split sample (dense M_r^1/2, direct wave sum)",
                 J=s.stats()["lanczos_iters"], rel_real=er, rel_wave=ew, rel=eu)
    assert er < 3 * tol and ew < 30 * tol
    s.close()


def test_graph_and_host_loop_identical(torch):
    """The CUDA-graph path (device-side loop) and the host-driven loop run the
    same kernels in the same order: bitwise-equal output."""
    pos, L, _ = _hs(1000, 0.1, 16)
    d = torch.from_numpy(pos).cuda()
    a = _sampler(L, xi=0.5, tol=1e-3)
    b = _sampler(L, xi=0.5, tol=1e-3, use_graph=False)
    ua = a.sample(d, SEED, 4)
    ub = b.sample(d, SEED, 4)
    assert torch.equal(ua, ub)
    assert a.stats()["lanczos_iters"] == b.stats()["lanczos_iters"]
    a.close()
    b.close()


def test_reproducible_and_host_buffers(torch):
    pos, L, _ = _hs(700, 0.1, 17)
    d = torch.from_numpy(pos).cuda()
    s = _sampler(L, xi=0.5, tol=1e-3)
    u1 = s.sample(d, SEED, 8).clone()
    u2 = s.sample(d, SEED, 8).clone()
    u3 = s.sample(d, SEED, 9).clone()
    assert torch.equal(u1, u2)
    assert not torch.equal(u1, u3)
    h = s.sample_host(pos, SEED, 8)
    assert np.array_equal(h, u1.cpu().numpy())
    s.close()


def test_single_particle(torch):
    """N = 1: M_r = self term * I, so the real part is sqrt(self) z1 exactly."""
    from oracle import ewald, pse, rpy
    L = 20.0
    pos = np.array([[3.0, 4.0, 5.0]], dtype=np.float32)
    s = _sampler(L, xi=0.5, tol=1e-3)
    u, r, w = s.sample(torch.from_numpy(pos).cuda(), SEED, 1, parts=True)
    z = pse.real_noise(1, SEED, 1)
    expect = math.sqrt(rpy.self_real(0.5) / (6 * math.pi)) * z
    assert _rel(r.cpu().numpy(), expect) < 1e-5
    plan = ewald.plan(L, 1.0, 0.5, 1e-3)
    assert _rel(w.cpu().numpy(), pse.wave_sample_grid(pos.astype(np.float64), plan, SEED, 1)) < 1e-4
    s.close()


def test_positions_outside_box_are_wrapped(torch):
    pos, L, _ = _hs(400, 0.1, 18)
    shift = pos.astype(np.float64).copy()
    shift[::3] += 2 * L
    shift[1::3] -= L
    s = _sampler(L, xi=0.5, tol=1e-3)
    a = s.sample(torch.from_numpy(pos).cuda(), SEED, 2).cpu().numpy()
    b = s.sample(torch.from_numpy(shift.astype(np.float32)).cuda(), SEED, 2).cpu().numpy()
    assert _rel(b, a) < 1e-4
    s.close()


def test_invalid_calls(torch):
    from paper_1611_09322_gb300 import PseError, Sampler
    with pytest.raises(PseError):
        Sampler(5.0, 1.0, xi=0.5, tol=1e-3)  # r_cut > L/2
    pos, L, _ = _hs(100, 0.1, 19)
    s = _sampler(L, xi=0.5, tol=1e-3)
    with pytest.raises(ValueError):
        s.sample(torch.from_numpy(pos.astype(np.float64)).cuda(), 1, 0)
    s.close()


@pytest.mark.parametrize("prec", [0, 1])
def test_coincident_and_overlapping_particles(torch, prec):
    """Degenerate configurations: pairs of distinct particles at exactly the
    same position (block F(0) I, one zero mode each) and pairs a small
    fraction of a radius apart, inside a random suspension: the near-field
    product and the J-step real sample match the oracle, the full sample is
    finite and the Lanczos test converges."""
    from oracle import ewald, pse
    pos, L, _ = _hs(600, 0.1, 31)
    pos = pos.astype(np.float64)
    pos[1] = pos[0]
    pos[3] = pos[2]
    pos[5] = pos[4] + np.array([0.05, 0.0, 0.0])
    pos[7] = pos[6] + np.array([0.0, 0.3, -0.2])
    dt = np.float64 if prec else np.float32
    p = pos.astype(dt)
    plan = ewald.plan(L, 1.0, 0.5, 1e-3)
    p64 = p.astype(np.float64)
    op = pse.RealOperator(p64, plan)
    v = np.random.default_rng(4).standard_normal((600, 3)).astype(dt)
    s = _sampler(L, xi=0.5, tol=1e-3, precision=prec)
    if prec == 0:  # the caller-vector product is an FP32 entry point
        got = s.real_matvec(torch.from_numpy(p).cuda(), torch.from_numpy(v).cuda()).cpu().numpy()
        assert _maxrel(got, op(v.astype(np.float64))) < 1e-5
    u = s.sample(torch.from_numpy(p).cuda(), SEED, 3)
    st = s.stats()
    assert torch.isfinite(u).all() and st["converged"] == 1
    s.close()
    J = 5
    s = _sampler(L, xi=0.5, tol=1e-3, precision=prec, fixed_iter=J)
    _, r, _ = s.sample(torch.from_numpy(p).cuda(), SEED, 4, parts=True)
    ref, _, _ = pse.real_sample(p64, plan, SEED, 4, n_iter=J)
    # each coincident pair gives M_r an exact zero eigenvalue, where the square
    # root's derivative is unbounded: rounding differences of size eps reach
    # the result as ~sqrt(eps), so FP64 agrees to 1e-7 here, not to 1e-9
    assert _maxrel(r.cpu().numpy(), ref) < (1e-7 if prec else 1e-4)
    s.close()


def test_empty_inputs_are_rejected_and_leave_the_context_usable(torch):
    """N = 0 (a single context, or one system of a batch) is refused with
    PSE_EINVAL before anything is launched; the next valid call works."""
    from paper_1611_09322_gb300 import BatchSampler, PseError
    pos, L, _ = _hs(300, 0.1, 32)
    s = _sampler(L, xi=0.5, tol=1e-3)
    empty = torch.empty((0, 3), dtype=torch.float32, device="cuda")
    with pytest.raises(PseError):
        s.sample(empty, SEED, 0)
    with pytest.raises(PseError):
        s.real_matvec(empty, empty)
    u = s.sample(torch.from_numpy(pos).cuda(), SEED, 0)
    assert torch.isfinite(u).all() and s.stats()["converged"] == 1
    s.close()
    b = BatchSampler([L, L], 1.0, xi=0.5, tol=1e-3)
    d = torch.from_numpy(pos).cuda()
    with pytest.raises(PseError):
        b.sample(d, [0, 300, 300], SEED, 0)
    out = b.sample(torch.cat([d, d]), [0, 300, 600], SEED, 0)
    assert torch.isfinite(out).all()
    b.close()


@pytest.mark.parametrize("M,N", [(64, 2000), (256, 2000), (32, 2000), (16, 250)])
def test_fused_noise_fft_matches_cufft_and_oracle(torch, M, N):
    """Grids M = 64 and 256: the sample path's own noise + three-pass C2R
    (wave_fft = 1) gives the wave part of the oracle's gridded sample and of
    the cuFFT path (wave_fft = 0) to float rounding; the real part is the
    same bit for bit (same kernels).  Other grids keep cuFFT either way."""
    from oracle import ewald, pse
    pos, L, _ = _hs(N, 0.1, 33)
    assert ewald.plan(L, 1.0, 0.5, 1e-3).M <= M
    plan = ewald.plan(L, 1.0, 0.5, 1e-3, M=M)
    outs = []
    for f in (1, 0):
        s = _sampler(L, xi=0.5, tol=1e-3, grid_M=M, fixed_iter=3, wave_fft=f)
        _, r, w = s.sample(torch.from_numpy(pos).cuda(), SEED, 11, parts=True)
        outs.append((r.cpu().numpy(), w.cpu().numpy()))
        # the fused path launches our y and z passes, the cuFFT path none
        fused = f == 1 and M in (64, 256)
        assert s.profile_stages(torch.from_numpy(pos).cuda(), SEED, 11)["fft"][1] == (2 if fused else 0)
        s.close()
    ref = pse.wave_sample_grid(pos.astype(np.float64), plan, SEED, 11)
    assert _maxrel(outs[0][1], ref) < 1e-4 and _maxrel(outs[0][1], outs[1][1]) < 1e-5
    assert np.array_equal(outs[0][0], outs[1][0])


def test_pipelined_host_buffers(torch):
    """pse_sample_host_async: consecutive calls with pinned host buffers (two
    staging pairs alternating, copies on the context's copy stream) give, after
    pse_host_sync, exactly the samples of the device-buffer call; a change of
    N in between re-allocates safely."""
    pos, L, _ = _hs(3000, 0.1, 34)
    s = _sampler(L, xi=0.5, tol=1e-3)
    hp = torch.from_numpy(pos).pin_memory()
    outs = [torch.empty_like(hp).pin_memory() for _ in range(5)]
    for i, o in enumerate(outs):
        s.sample_host_async_ptr(3000, hp.data_ptr(), o.data_ptr(), SEED, 40 + i)
    s.host_sync()
    d = torch.from_numpy(pos).cuda()
    for i, o in enumerate(outs):
        assert torch.equal(o, s.sample(d, SEED, 40 + i).cpu())
    small = torch.from_numpy(pos[:1000].copy()).pin_memory()
    o2 = torch.empty_like(small).pin_memory()
    s.sample_host_async_ptr(1000, small.data_ptr(), o2.data_ptr(), SEED, 3)
    s.host_sync()
    assert torch.equal(o2, s.sample(torch.from_numpy(pos[:1000].copy()).cuda(), SEED, 3).cpu())
    s.close()
