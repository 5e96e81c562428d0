"""GB300-native Positively Split Ewald (PSE) Brownian displacement sampler.

Python side of the C ABI in ``include/pse.h`` (arXiv:1611.09322).  The
functions ``pse_*`` below carry the names of the C entry points and only
marshal arguments; all arithmetic runs in the CUDA kernels of libpse.so.
PyTorch supplies device memory and the current stream.
"""
from __future__ import annotations

import ctypes

import numpy as np

from . import _lib
from ._lib import PSE_FP32, PSE_FP64, PseError, pse_params, pse_plan_info, pse_stats

__all__ = ["Sampler", "PolySampler", "BatchSampler", "pse_plan", "pse_batch_grid", "tune_batch_grid_step", "pse_real_scalars", "pse_real_scalars_poly", "pse_real_matvec_noalloc", "pse_precond_loss_grad",
           "pse_precond_train", "pse_xi_model", "pse_tune_xi", "PseError", "PSE_FP32", "PSE_FP64", "make_params"]


def make_params(tol=1e-3, xi=0.5, precision=PSE_FP32, max_iter=0, fixed_iter=0, grid_M=0, support_P=0,
                use_precond=0, lanczos_tol=0.0, use_graph=True, autotune=0, system=0, wave_noise=0,
                spread_tile=0, matvec_shape=0, interp_form=0, wave_fft=0):
    p = pse_params()
    p.tol = tol
    p.xi = xi
    p.precision = precision
    p.max_iter = max_iter
    p.fixed_iter = fixed_iter
    p.grid_M = grid_M
    p.support_P = support_P
    p.use_precond = use_precond
    p.lanczos_tol = lanczos_tol
    p.use_graph = 0 if use_graph else -1
    p.autotune = autotune
    p.system = system
    p.wave_noise = wave_noise
    p.spread_tile = spread_tile
    p.matvec_shape = matvec_shape
    p.interp_form = interp_form
    p.wave_fft = wave_fft
    return p


def pse_plan(L, a=1.0, **kw):
    """Host-only Sec. II C parameter planning (no GPU needed); returns a dict."""
    lib = _lib.load()
    p = make_params(**kw)
    out = pse_plan_info()
    _lib.check(lib.pse_plan(L, a, ctypes.byref(p), ctypes.byref(out)), "pse_plan")
    return out.as_dict()


def pse_real_scalars(r, xi, a=1.0):
    """Host-only Appendix A scalars F(r), G(r) (float64 numpy arrays)."""
    lib = _lib.load()
    r = np.ascontiguousarray(r, dtype=np.float64)
    F = np.empty_like(r)
    G = np.empty_like(r)
    vp = lambda x: x.ctypes.data_as(ctypes.c_void_p)
    _lib.check(lib.pse_real_scalars(xi, a, r.size, vp(r), vp(F), vp(G)), "pse_real_scalars")
    return F, G


def pse_real_scalars_poly(r, xi, ai, aj):
    """Host-only real-space scalars (F, G) of a pair of spheres of radii ai, aj (mobility units)."""
    lib = _lib.load()
    r = np.ascontiguousarray(r, dtype=np.float64)
    F = np.empty_like(r)
    G = np.empty_like(r)
    vp = lambda x: x.ctypes.data_as(ctypes.c_void_p)
    _lib.check(lib.pse_real_scalars_poly(xi, ai, aj, r.size, vp(r), vp(F), vp(G)), "pse_real_scalars_poly")
    return F, G


def pse_xi_model(xi0, t_real, t_wave, d_f=3.0):
    """Host-only eq. xistar with constants calibrated by times at xi0 (no GPU needed)."""
    lib = _lib.load()
    out = ctypes.c_double()
    _lib.check(lib.pse_xi_model(xi0, t_real, t_wave, d_f, ctypes.byref(out)), "pse_xi_model")
    return out.value


def pse_tune_xi(L, pos, a=1.0, d_f=3.0, reps=5, **kw):
    """Timed choice of xi around the model's xi* for positions `pos` (CUDA float32); returns a dict."""
    lib = _lib.load()
    p = make_params(**kw)
    out = _lib.pse_xi_tuning()
    _lib.check(lib.pse_tune_xi(L, a, ctypes.byref(p), pos.shape[0], _ptr(pos), d_f, reps, ctypes.byref(out),
                               _stream()), "pse_tune_xi")
    return out.as_dict()


def pse_batch_grid(L, a=1.0, step=0, **kw):
    """Grid side the system (L, a) gets in a batch, `step` size classes finer (pse_batch_grid)."""
    lib = _lib.load()
    p = make_params(**kw)
    m = ctypes.c_int(0)
    _lib.check(lib.pse_batch_grid(L, a, ctypes.byref(p), int(step), ctypes.byref(m)), "pse_batch_grid")
    return m.value


def tune_batch_grid_step(Ls, pos_all, offsets, a=1.0, steps=(0, 1, 2), reps=5, seed=1, **kw):
    """Timed choice, for a whole batch, of how many size classes finer than
    its planned grids the systems' FFT grids are (with autotune bit 3 each
    then takes the largest xi its grid admits: a finer grid buys a shorter
    r_cut).  Builds one batch per candidate step, times `reps` samples each
    (CUDA events, after two untimed ones) and returns a dict: "step" (the
    fastest), "ms" per step and "params" (per-system keyword dicts with the
    chosen grids, for BatchSampler(params=...))."""
    import torch
    ms = {}
    chosen = None
    for st in steps:
        params = [dict(kw, grid_M=pse_batch_grid(L, a, st, **kw)) for L in Ls]
        b = BatchSampler(Ls, a, params=params)
        out = torch.empty_like(pos_all)
        for i in range(2):
            b.sample(pos_all, offsets, seed, 90_000 + i, out=out)
        stream = torch.cuda.current_stream()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for i in range(reps):
            b.sample(pos_all, offsets, seed, 90_100 + i, out=out)
        e1.record(stream)
        e1.synchronize()
        ms[st] = e0.elapsed_time(e1) / reps
        b.close()
        if chosen is None or ms[st] < ms[chosen[0]]:
            chosen = (st, params)
    return {"step": chosen[0], "ms": ms, "params": chosen[1]}


def pse_real_matvec_noalloc(L, a, xi, tol, pos, v, out):
    """M_r v through the allocation-free entry point (static device scratch, N <= 16384).

    For callers that may not allocate device memory: `out` must be
    preallocated by the caller; nothing is allocated by the library.
    """
    import torch
    lib = _lib.load()
    dev = torch.cuda.current_device()
    for name, t in (("pos", pos), ("v", v), ("out", out)):
        if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == torch.float32 and t.is_contiguous()
                and t.dim() == 2 and t.shape[1] == 3 and t.shape[0] == pos.shape[0] and t.device.index == dev):
            raise ValueError(f"{name} must be a contiguous (N, 3) float32 CUDA tensor on the current device, "
                             f"shaped like pos")
    _lib.check(lib.pse_real_matvec_noalloc(L, a, xi, tol, pos.shape[0], _ptr(pos), _ptr(v), _ptr(out), _stream()),
               "pse_real_matvec_noalloc")
    return out


def pse_precond_loss_grad(feat, tens, target, theta, s0):
    """Loss and gradient of the preconditioner network on the GPU (torch CUDA tensors)."""
    import torch
    lib = _lib.load()
    grad = torch.empty(_lib.PSE_PRECOND_NPARAM, dtype=torch.float32, device=feat.device)
    loss = torch.empty(1, dtype=torch.float64, device=feat.device)
    _lib.check(lib.pse_precond_loss_grad(feat.shape[0], _ptr(feat), _ptr(tens), _ptr(target), _ptr(theta), s0,
                                         _ptr(grad), _ptr(loss), _stream()), "pse_precond_loss_grad")
    return loss, grad


def pse_precond_train(feat, tens, target, theta, s0, steps, lr):
    """Full-batch Adam on the GPU; theta (CUDA float32) is updated in place. Returns the loss history."""
    import torch
    lib = _lib.load()
    work = torch.zeros(3 * _lib.PSE_PRECOND_NPARAM + 4, dtype=torch.float32, device=feat.device)
    hist = torch.zeros(steps, dtype=torch.float64, device=feat.device)
    _lib.check(lib.pse_precond_train(feat.shape[0], _ptr(feat), _ptr(tens), _ptr(target), _ptr(theta), s0, steps,
                                     lr, _ptr(work), _ptr(hist), _stream()), "pse_precond_train")
    return hist


def _stream():
    import torch
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else ctypes.c_void_p(0)


class Sampler:
    """One PSE sampler for a periodic cube of side L (a context of libpse)."""

    def __init__(self, L, a=1.0, **kw):
        self.lib = _lib.load()
        self.params = make_params(**kw)
        self.L, self.a = L, a
        h = ctypes.c_void_p()
        _lib.check(self.lib.pse_create_ex(ctypes.byref(h), L, a, ctypes.byref(self.params)), "pse_create_ex")
        self.ctx = h
        info = pse_plan_info()
        _lib.check(self.lib.pse_get_plan(self.ctx, ctypes.byref(info)), "pse_get_plan")
        self.plan = info.as_dict()
        self.fp64 = self.params.precision == PSE_FP64

    def close(self):
        if getattr(self, "ctx", None):
            self.lib.pse_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check_pos(self, pos):
        import torch
        want = torch.float64 if self.fp64 else torch.float32
        if not (pos.is_cuda and pos.dtype == want and pos.is_contiguous() and pos.dim() == 2 and pos.shape[1] == 3):
            raise ValueError(f"positions must be a contiguous (N, 3) {want} CUDA tensor")

    def sample(self, pos, seed, sample_index=0, out=None, parts=False):
        """u = M_r^{1/2} z1 + M_w^{1/2} dW2 at `pos`; with parts=True returns (u, u_real, u_wave)."""
        import torch
        self._check_pos(pos)
        N = pos.shape[0]
        if out is None:
            out = torch.empty_like(pos)
        real = torch.empty_like(pos) if parts else None
        wave = torch.empty_like(pos) if parts else None
        if self.fp64:
            st = self.lib.pse_sample_f64(self.ctx, N, _ptr(pos), seed, sample_index, _ptr(out), _ptr(real),
                                         _ptr(wave), _stream())
        elif parts:
            st = self.lib.pse_sample_parts(self.ctx, N, _ptr(pos), seed, sample_index, _ptr(out), _ptr(real),
                                           _ptr(wave), _stream())
        else:
            st = self.lib.pse_sample(self.ctx, N, _ptr(pos), seed, sample_index, _ptr(out), _stream())
        _lib.check(st, "pse_sample")
        return (out, real, wave) if parts else out

    def sample_host(self, pos_host, seed, sample_index=0, out_host=None):
        """Host buffers in and out (the copies happen inside libpse); numpy float32 (N, 3)."""
        pos_host = np.ascontiguousarray(pos_host, dtype=np.float32)
        if out_host is None:
            out_host = np.empty_like(pos_host)
        st = self.lib.pse_sample_host(self.ctx, pos_host.shape[0], pos_host.ctypes.data_as(ctypes.c_void_p), seed,
                                      sample_index, out_host.ctypes.data_as(ctypes.c_void_p), _stream())
        _lib.check(st, "pse_sample_host")
        return out_host

    def sample_host_ptr(self, N, h_pos_ptr, h_out_ptr, seed, sample_index=0):
        """As sample_host with raw host pointers (e.g. pinned torch tensors)."""
        _lib.check(self.lib.pse_sample_host(self.ctx, N, ctypes.c_void_p(h_pos_ptr), seed, sample_index,
                                            ctypes.c_void_p(h_out_ptr), _stream()), "pse_sample_host")

    def sample_host_async_ptr(self, N, h_pos_ptr, h_out_ptr, seed, sample_index=0):
        """Pipelined host-buffer sample (pse_sample_host_async); the result is in h_out after host_sync()."""
        _lib.check(self.lib.pse_sample_host_async(self.ctx, N, ctypes.c_void_p(h_pos_ptr), seed, sample_index,
                                                  ctypes.c_void_p(h_out_ptr), _stream()), "pse_sample_host_async")

    def host_sync(self):
        _lib.check(self.lib.pse_host_sync(self.ctx), "pse_host_sync")

    def real_matvec(self, pos, v, out=None):
        """M_r v (near-field product, eq. Mreal) for (N, 3) CUDA float32 tensors."""
        import torch
        self._check_pos(pos)
        if out is None:
            out = torch.empty_like(v)
        _lib.check(self.lib.pse_real_matvec(self.ctx, pos.shape[0], _ptr(pos), _ptr(v), _ptr(out), _stream()),
                   "pse_real_matvec")
        return out

    def sample_with_forces(self, pos, force, seed, sample_index=0, c_det=1.0, c_noise=1.0, out=None):
        """c_det M F + c_noise M^{1/2} z at `pos` (pse_sample_with_forces); (N, 3) CUDA tensors."""
        import torch
        self._check_pos(pos)
        if force.dtype != pos.dtype or force.shape != pos.shape or not force.is_contiguous() or not force.is_cuda:
            raise ValueError("force must be a contiguous CUDA tensor shaped and typed like pos")
        if out is None:
            out = torch.empty_like(pos)
        fn = self.lib.pse_sample_with_forces_f64 if self.fp64 else self.lib.pse_sample_with_forces
        _lib.check(fn(self.ctx, pos.shape[0], _ptr(pos), _ptr(force), seed, sample_index, float(c_det),
                      float(c_noise), _ptr(out), _stream()), "pse_sample_with_forces")
        return out

    def bd_step(self, pos, seed, step, dt, kT=1.0, k_rep=0.0, f_ext=None):
        """One Euler-Maruyama step in place: pos += dt M F + sqrt(2 kT dt) M^{1/2} z (pse_bd_step)."""
        self._check_pos(pos)
        if f_ext is not None and (f_ext.dtype != pos.dtype or f_ext.shape != pos.shape or not f_ext.is_cuda):
            raise ValueError("f_ext must be a CUDA tensor shaped and typed like pos")
        fn = self.lib.pse_bd_step_f64 if self.fp64 else self.lib.pse_bd_step
        _lib.check(fn(self.ctx, pos.shape[0], _ptr(pos), _ptr(f_ext), float(dt), float(kT), float(k_rep), seed, step,
                      _stream()), "pse_bd_step")
        return pos

    def sample_full_lanczos(self, pos, seed, sample_index=0, out=None):
        """M^{1/2} z by Lanczos on the whole mobility (pse_sample_full_lanczos: Sec. IV's comparison method)."""
        import torch
        self._check_pos(pos)
        if out is None:
            out = torch.empty_like(pos)
        fn = self.lib.pse_sample_full_lanczos_f64 if self.fp64 else self.lib.pse_sample_full_lanczos
        _lib.check(fn(self.ctx, pos.shape[0], _ptr(pos), seed, sample_index, _ptr(out), _stream()),
                   "pse_sample_full_lanczos")
        return out

    def mobility_apply(self, pos, force, out=None):
        """The deterministic product M F (c_det = 1, c_noise = 0)."""
        return self.sample_with_forces(pos, force, 0, 0, 1.0, 0.0, out=out)

    def profile_stages(self, pos, seed, sample_index=0, out=None):
        """Per-stage device times (ms) and launch counts of one sample (pse_profile_stages)."""
        import torch
        self._check_pos(pos)
        if out is None:
            out = torch.empty_like(pos)
        n = len(_lib.STAGES)
        ms = (ctypes.c_double * n)()
        nl = (ctypes.c_int * n)()
        _lib.check(self.lib.pse_profile_stages(self.ctx, pos.shape[0], _ptr(pos), seed, sample_index, _ptr(out),
                                               ms, nl, _stream()), "pse_profile_stages")
        return {name: (ms[i], nl[i]) for i, name in enumerate(_lib.STAGES)}

    # ---------------------------------------------------------- learned preconditioner
    def precond_features(self, pos):
        """(N, 8) features and (N, 6) structure tensors (xx, yy, zz, xy, xz, yz), caller order."""
        import torch
        self._check_pos(pos)
        N = pos.shape[0]
        feat = torch.empty((N, 8), dtype=torch.float32, device=pos.device)
        tens = torch.empty((N, 6), dtype=torch.float32, device=pos.device)
        _lib.check(self.lib.pse_precond_features(self.ctx, N, _ptr(pos), _ptr(feat), _ptr(tens), _stream()),
                   "pse_precond_features")
        return feat, tens

    def precond_targets(self, pos):
        """(N, 6) local inverse-square-root blocks [(M_loc)^{-1/2}]_ii, caller order."""
        import torch
        self._check_pos(pos)
        N = pos.shape[0]
        tgt = torch.empty((N, 6), dtype=torch.float32, device=pos.device)
        _lib.check(self.lib.pse_precond_targets(self.ctx, N, _ptr(pos), _ptr(tgt), _stream()), "pse_precond_targets")
        return tgt

    def precond_set_weights(self, theta):
        """Install network weights (PSE_PRECOND_NPARAM floats) or None to switch it off."""
        if theta is None:
            _lib.check(self.lib.pse_precond_set_weights(self.ctx, None, 0), "pse_precond_set_weights")
            return
        th = np.ascontiguousarray(np.asarray(theta, dtype=np.float32).ravel())
        _lib.check(self.lib.pse_precond_set_weights(self.ctx, th.ctypes.data_as(ctypes.c_void_p), th.size),
                   "pse_precond_set_weights")

    def precond_blocks(self, pos):
        """(N, 6) blocks S_i of the installed network, caller order."""
        import torch
        self._check_pos(pos)
        N = pos.shape[0]
        S = torch.empty((N, 6), dtype=torch.float32, device=pos.device)
        _lib.check(self.lib.pse_precond_blocks(self.ctx, N, _ptr(pos), _ptr(S), _stream()), "pse_precond_blocks")
        return S

    @property
    def precond_s0(self):
        return float(self.plan["self_mobility"] ** -0.5)

    def stats(self, strict=False):
        s = pse_stats()
        st = self.lib.pse_get_stats(self.ctx, ctypes.byref(s))
        if strict:
            _lib.check(st, "pse_get_stats")
        d = s.as_dict()
        d["status"] = _lib.STATUS.get(st, st)
        return d


class PolySampler(Sampler):
    """PSE sampler for spheres of several radii (species; pse_create_poly, pse_sample_poly)."""

    def __init__(self, L, radii, **kw):
        self.lib = _lib.load()
        self.params = make_params(**kw)
        self.L = L
        self.radii = np.ascontiguousarray(radii, dtype=np.float64)
        h = ctypes.c_void_p()
        _lib.check(self.lib.pse_create_poly(ctypes.byref(h), L, self.radii.size,
                                            self.radii.ctypes.data_as(ctypes.c_void_p), ctypes.byref(self.params)),
                   "pse_create_poly")
        self.ctx = h
        info = pse_plan_info()
        _lib.check(self.lib.pse_get_plan(self.ctx, ctypes.byref(info)), "pse_get_plan")
        self.plan = info.as_dict()
        self.a = self.plan["a"]
        self.fp64 = False

    def _check_species(self, pos, species):
        import torch
        if not (species.is_cuda and species.dtype == torch.int32 and species.is_contiguous()
                and species.shape == (pos.shape[0],)):
            raise ValueError("species must be a contiguous (N,) int32 CUDA tensor")

    def sample(self, pos, species, seed, sample_index=0, out=None, parts=False):
        """u at `pos` for particles of the given species; with parts=True (u, u_real, u_wave)."""
        import torch
        self._check_pos(pos)
        self._check_species(pos, species)
        if out is None:
            out = torch.empty_like(pos)
        real = torch.empty_like(pos) if parts else None
        wave = torch.empty_like(pos) if parts else None
        _lib.check(self.lib.pse_sample_poly(self.ctx, pos.shape[0], _ptr(pos), _ptr(species), seed, sample_index,
                                            _ptr(out), _ptr(real), _ptr(wave), _stream()), "pse_sample_poly")
        return (out, real, wave) if parts else out

    def real_matvec(self, pos, species, v, out=None):
        import torch
        self._check_pos(pos)
        self._check_species(pos, species)
        if out is None:
            out = torch.empty_like(v)
        _lib.check(self.lib.pse_real_matvec_poly(self.ctx, pos.shape[0], _ptr(pos), _ptr(species), _ptr(v),
                                                 _ptr(out), _stream()), "pse_real_matvec_poly")
        return out


class BatchSampler:
    """Many independent systems sampled by one CUDA-graph launch (pse_batch_*)."""

    def __init__(self, Ls, a=1.0, params=None, **kw):
        self.lib = _lib.load()
        n = len(Ls)
        a_arr = np.full(n, a, dtype=np.float64) if np.isscalar(a) else np.asarray(a, dtype=np.float64)
        L_arr = np.asarray(Ls, dtype=np.float64)
        if params is None:
            params = [dict(kw) for _ in range(n)]
        arr = (pse_params * n)(*[make_params(**pk) for pk in params])
        h = ctypes.c_void_p()
        _lib.check(self.lib.pse_batch_create(ctypes.byref(h), n, L_arr.ctypes.data_as(ctypes.c_void_p),
                                             a_arr.ctypes.data_as(ctypes.c_void_p), ctypes.cast(arr, ctypes.c_void_p)),
                   "pse_batch_create")
        self.h = h
        self.n = n
        self._keep = (L_arr, a_arr, arr)

    def plan(self, k):
        info = pse_plan_info()
        _lib.check(self.lib.pse_batch_get_plan(self.h, k, ctypes.byref(info)), "pse_batch_get_plan")
        return info.as_dict()

    def sample(self, pos_all, offsets, seed, sample_index=0, out=None):
        """pos_all: (sum N, 3) float32 CUDA, systems concatenated; offsets: n+1 ints."""
        import torch
        off = np.ascontiguousarray(offsets, dtype=np.int64)
        if not (pos_all.is_cuda and pos_all.dtype == torch.float32 and pos_all.is_contiguous()
                and pos_all.dim() == 2 and pos_all.shape[1] == 3):
            raise ValueError("positions must be a contiguous (N, 3) float32 CUDA tensor")
        if off.shape != (self.n + 1,) or off[-1] != pos_all.shape[0]:
            raise ValueError("offsets must hold n_systems + 1 entries ending at the number of particles")
        if out is None:
            out = torch.empty_like(pos_all)
        elif out.shape != pos_all.shape or out.dtype != pos_all.dtype or not out.is_contiguous() or not out.is_cuda:
            raise ValueError("out must be a contiguous CUDA tensor shaped and typed like the positions")
        _lib.check(self.lib.pse_batch_sample(self.h, off.ctypes.data_as(ctypes.c_void_p), _ptr(pos_all), seed,
                                             sample_index, _ptr(out), _stream()), "pse_batch_sample")
        return out

    def set_precond(self, k, theta):
        """Install learned-preconditioner weights in system k (None removes them)."""
        if theta is None:
            _lib.check(self.lib.pse_batch_set_precond(self.h, k, None, 0), "pse_batch_set_precond")
            return
        th = np.ascontiguousarray(np.asarray(theta, dtype=np.float32).ravel())
        _lib.check(self.lib.pse_batch_set_precond(self.h, k, th.ctypes.data_as(ctypes.c_void_p), th.size),
                   "pse_batch_set_precond")

    def stats(self, k):
        s = pse_stats()
        st = self.lib.pse_batch_get_stats(self.h, k, ctypes.byref(s))
        d = s.as_dict()
        d["status"] = _lib.STATUS.get(st, st)
        return d

    def close(self):
        if getattr(self, "h", None):
            self.lib.pse_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
