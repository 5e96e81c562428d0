"""Seeded synthetic particle configurations (hard spheres, relaxed packings, fractal gels).

Shared by the CUDA path's benchmark and by the test oracle; holds none of
the sampler's arithmetic.  The heavy lifting is plain C
(``csrc/workloads.c``) built into ``_build/libpse_workloads.so`` by
:func:`paper_1611_09322_gb300.build.build_workloads`.

Every generator returns float32 positions wrapped into [0, L): float32 is
the sampler's input type, and the oracle upcasts exactly those values.
"""
from __future__ import annotations

import ctypes
import math
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB = None


def _lib():
    global _LIB
    if _LIB is None:
        from . import build
        path = build.build_workloads()
        lib = ctypes.CDLL(path)
        dp = ctypes.POINTER(ctypes.c_double)
        lib.wl_rsa.restype = ctypes.c_int64
        lib.wl_rsa.argtypes = [ctypes.c_int64, ctypes.c_double, ctypes.c_double, ctypes.c_uint64,
                               ctypes.c_int64, dp]
        lib.wl_rsa_poly.restype = ctypes.c_int64
        lib.wl_rsa_poly.argtypes = [ctypes.c_int64, ctypes.c_double, dp, ctypes.c_double, ctypes.c_uint64,
                                    ctypes.c_int64, dp]
        lib.wl_relax.restype = ctypes.c_double
        lib.wl_relax.argtypes = [ctypes.c_int64, ctypes.c_double, ctypes.c_double, ctypes.c_int64,
                                 ctypes.c_double, ctypes.c_double, dp]
        lib.wl_cca_gel.restype = ctypes.c_int64
        lib.wl_cca_gel.argtypes = [ctypes.c_int64, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                   ctypes.c_double, ctypes.c_int64, ctypes.c_uint64, dp]
        _LIB = lib
    return _LIB


def box_length(N, phi, a=1.0):
    """Side of the periodic cube holding N spheres of radius a at volume fraction phi."""
    return (N * 4.0 / 3.0 * math.pi * a ** 3 / phi) ** (1.0 / 3.0)


def _f32(pos, L):
    p = np.mod(np.asarray(pos, dtype=np.float64), L).astype(np.float32)
    p[p >= np.float32(L)] = 0.0
    return p


def hard_spheres(N, phi, seed, a=1.0, relax_steps=10000, rsa_phi_max=0.3):
    """Random hard spheres at volume fraction phi.

    phi <= rsa_phi_max: random sequential addition (RSA) at diameter 2a.
    Above it (RSA jams near 0.38): RSA at the diameter that fills
    rsa_phi_max, inflated to 2a and relaxed by harmonic overlap descent for
    up to relax_steps steps.  Returns (float32 (N, 3) positions, L, info).
    """
    L = box_length(N, phi, a)
    out = np.zeros((N, 3), dtype=np.float64)
    lib = _lib()
    dp = out.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    d_rsa = 2 * a if phi <= rsa_phi_max else 2 * a * (rsa_phi_max / phi) ** (1.0 / 3.0)
    n = lib.wl_rsa(N, L, d_rsa, seed, 200 * N + 1000, dp)
    if n != N:
        raise RuntimeError(f"RSA placed {n} of {N} spheres (phi={phi})")
    worst = 0.0
    if d_rsa < 2 * a:
        worst = lib.wl_relax(N, L, 2 * a, relax_steps, 0.25, 1e-4 * a, dp)
    return _f32(out, L), L, {"max_overlap": worst, "rsa_diameter": d_rsa}


def polydisperse(N, phi, seed, radii=(1.0, 0.5), fractions=None):
    """Random non-overlapping spheres of several radii (species) at total volume fraction phi.

    Species s holds round(fractions[s] N) spheres (equal numbers by default);
    they are placed by RSA largest first.  Returns (float32 (N, 3) positions,
    int32 (N,) species indices, L, info)."""
    radii = np.asarray(radii, dtype=np.float64)
    S = radii.size
    fr = np.full(S, 1.0 / S) if fractions is None else np.asarray(fractions, dtype=np.float64)
    counts = np.floor(fr / fr.sum() * N).astype(np.int64)
    counts[np.argmax(radii)] += N - counts.sum()
    order = np.argsort(-radii, kind="stable")
    species = np.concatenate([np.full(counts[s], s, dtype=np.int32) for s in order])
    rad = radii[species]
    L = (np.sum(4.0 / 3.0 * math.pi * rad ** 3) / phi) ** (1.0 / 3.0)
    out = np.zeros((N, 3), dtype=np.float64)
    dp = out.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    rp = np.ascontiguousarray(rad).ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    n = _lib().wl_rsa_poly(N, L, rp, float(radii.max()), seed, 400 * N + 1000, dp)
    if n != N:
        raise RuntimeError(f"polydisperse RSA placed {n} of {N} spheres (phi={phi})")
    return _f32(out, L), species, L, {"radii": radii.tolist(), "counts": counts.tolist()}


def gel(N, phi, seed, a=1.0, df=1.9, kf=1.3, csize=256):
    """Fractal-gel stand-in: tunable-dimension CCA clusters (df, kf) packed at phi.

    Returns (float32 (N, 3) positions, L, info).
    """
    L = box_length(N, phi, a)
    out = np.zeros((N, 3), dtype=np.float64)
    dp = out.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    n = _lib().wl_cca_gel(N, L, a, df, kf, csize, seed, dp)
    if n != N:
        raise RuntimeError(f"gel placed {n} of {N} spheres (phi={phi})")
    return _f32(out, L), L, {"df_target": df, "cluster_size": csize}


def cluster(n, seed, a=1.0, df=1.9, kf=1.3):
    """One isolated CCA cluster of n monomers (float64, centred), for d_f checks."""
    L = 1e6
    out = np.zeros((n, 3), dtype=np.float64)
    dp = out.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    got = _lib().wl_cca_gel(n, L, a, df, kf, n, seed, dp)
    if got != n:
        raise RuntimeError("cluster generation failed")
    c = out - out.mean(axis=0)
    c -= L * np.round(c / L)
    return c


def batch_spec(nsys=64, seed=1000, n_lo=1000, n_hi=50000, phi_lo=0.05, phi_hi=0.4, gel_phi_max=0.2):
    """The batched workload: nsys systems, N log-uniform in [n_lo, n_hi], phi uniform.

    Half the systems are gels (only where phi <= gel_phi_max, else hard
    spheres).  Returns a list of dicts (N, phi, kind, seed).
    """
    rng = np.random.default_rng(seed)
    Ns = np.exp(rng.uniform(math.log(n_lo), math.log(n_hi), nsys)).astype(np.int64)
    phis = rng.uniform(phi_lo, phi_hi, nsys)
    kinds = ["gel" if (s % 2 == 1 and phis[s] <= gel_phi_max) else "hs" for s in range(nsys)]
    return [dict(N=int(Ns[s]), phi=float(phis[s]), kind=kinds[s], seed=seed + s) for s in range(nsys)]


def make(kind, N, phi, seed, a=1.0):
    if kind == "gel":
        return gel(N, phi, seed, a)
    return hard_spheres(N, phi, seed, a)
