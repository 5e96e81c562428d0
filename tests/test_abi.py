"""The C ABI library (no GPU needed): it loads, exports every declared entry
point, and its host-only parameter planning agrees with the oracle's."""
import ctypes
import os
import re

import pytest

from paper_1611_09322_gb300 import _lib, build, pse_plan

ROOT = os.path.abspath(os.path.join(os.path.dirname(__file__), ".."))


@pytest.fixture(scope="module")
def lib():
    build.build_cuda()
    return _lib.load()


def _declared():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", fn)).read()
            names |= set(re.findall(r"^\S[^;(]*?\b(pse_\w+)\s*\(", txt, flags=re.M))
    return names


def test_every_declared_symbol_is_exported(lib):
    names = _declared()
    assert {"pse_create", "pse_sample", "pse_destroy", "pse_plan"} <= names
    for n in names:
        assert hasattr(lib, n), n
    assert names <= set(_lib.SIGNATURES), names - set(_lib.SIGNATURES)


def test_strerror(lib):
    assert lib.pse_strerror(0) == b"ok"
    assert b"Lanczos" in lib.pse_strerror(5)


@pytest.mark.parametrize("L,xi,tol", [(34.7293, 0.5, 1e-3), (347.293, 0.5, 1e-3), (382.3, 0.5, 1e-5),
                                      (127.9, 0.7, 1e-4), (13.89, 0.5, 1e-3)])
def test_plan_matches_oracle(lib, L, xi, tol):
    from oracle import ewald
    p = pse_plan(L, 1.0, xi=xi, tol=tol)
    o = ewald.plan(L, 1.0, xi, tol)
    assert p["M"] == o.M and p["P"] == o.P
    for k in ("r_cut", "k_cut", "m", "eta", "h"):
        assert abs(p[k] - getattr(o, k)) <= 1e-12 * max(1.0, abs(getattr(o, k))), k
    from oracle import rpy
    import math
    assert abs(p["self_mobility"] - rpy.self_real(xi) / (6 * math.pi)) < 1e-15
    assert p["ncell"] * p["r_cut"] <= L and p["ncell"] >= 2


def test_plan_rejects_bad_input(lib):
    for L, a, tol, xi in [(0.0, 1.0, 1e-3, 0.5), (30.0, -1.0, 1e-3, 0.5), (30.0, 1.0, 0.5, 0.5),
                          (30.0, 1.0, 0.0, 0.5), (8.0, 1.0, 1e-3, 0.5)]:  # last: r_cut > L/2
        with pytest.raises(_lib.PseError):
            pse_plan(L, a, xi=xi, tol=tol)


@pytest.mark.parametrize("xi,a", [(0.5, 1.0), (0.3, 1.0), (0.6, 1.3)])
def test_host_scalars_match_oracle(lib, xi, a):
    """The library's FP64 Appendix A evaluation (the device table's source)
    equals the oracle's on both branches, the small-r region and r = 0."""
    import numpy as np
    from oracle import rpy
    from paper_1611_09322_gb300 import pse_real_scalars
    r = np.concatenate([[0.0, 1e-4, 0.01, 0.1, 0.199 * a, 0.2 * a], np.linspace(0.21, 3 * a, 200), [2 * a, 8.0]])
    F, G = pse_real_scalars(r, xi, a)
    Fo, Go = rpy.fg(r, xi, a)
    assert np.abs(F - Fo).max() < 1e-12 and np.abs(G - Go).max() < 1e-12
    with pytest.raises(_lib.PseError):
        pse_real_scalars(np.array([-1.0]), xi, a)


def test_batch_grid_classes():
    """pse_batch_grid: step 0 is the smallest size class at or above the
    plan's grid, a class maps to itself, and each step is the next class."""
    from paper_1611_09322_gb300 import PseError, pse_batch_grid, pse_plan
    for L in (20.0, 50.0, 100.0, 347.3):
        M0 = pse_plan(L, 1.0, xi=0.5, tol=1e-3)["M"]
        g = [pse_batch_grid(L, 1.0, s, xi=0.5, tol=1e-3) for s in range(4)]
        assert g[0] >= M0 and g[0] < g[1] < g[2] < g[3]
        assert pse_batch_grid(L, 1.0, 0, xi=0.5, tol=1e-3, grid_M=g[0]) == g[0]
        assert pse_batch_grid(L, 1.0, 1, xi=0.5, tol=1e-3, grid_M=g[0]) == g[1]
        assert pse_batch_grid(L, 1.0, 0, xi=0.5, tol=1e-3, grid_M=g[1]) == g[1]
        # no class lies strictly between the plan's grid and step 0's
        assert pse_batch_grid(L, 1.0, 0, xi=0.5, tol=1e-3, grid_M=M0) == g[0]
    with pytest.raises(PseError):
        pse_batch_grid(50.0, 1.0, -1, xi=0.5, tol=1e-3)
