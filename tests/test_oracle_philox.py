"""Pins of the oracle's Philox4x32-10 and Box-Muller normals."""
import os

import numpy as np

from oracle import philox

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def test_known_answer_vectors():
    with open(os.path.join(GOLDEN, "philox_kat.txt")) as f:
        rows = [l.split() for l in f if not l.startswith("#") and l.strip()]
    assert len(rows) == 3
    for row in rows:
        v = [int(x, 16) for x in row]
        out = philox.philox4x32_10(*v[:6])
        assert [int(o) for o in out] == v[6:]


def test_uniforms_exact_and_open():
    x = np.array([0, 511, 512, 0xFFFFFFFF], dtype=np.uint64)
    u = philox.uniform23(x)
    assert u[0] == u[1] == 0.5 * 2 ** -23
    assert u[2] == 1.5 * 2 ** -23
    assert u[3] == 1 - 0.5 * 2 ** -23
    allk = philox.uniform23(np.arange(0, 2 ** 32, 4099, dtype=np.uint64))
    assert np.all(allk.astype(np.float32).astype(np.float64) == allk)


def test_normals_moments_and_independence():
    z = philox.normals4(np.arange(200000, dtype=np.uint64), 0, 12345, 7).ravel()
    n = z.size
    assert abs(z.mean()) < 4 / np.sqrt(n)
    assert abs(z.var() - 1) < 4 * np.sqrt(2 / n)
    zz = philox.normals4(np.arange(200000, dtype=np.uint64), 1, 12345, 7).ravel()
    assert abs(np.mean(z * zz)) < 4 / np.sqrt(n)
    z2 = philox.normals4(np.arange(10, dtype=np.uint64), 0, 12345, 8)
    assert not np.allclose(z2, philox.normals4(np.arange(10, dtype=np.uint64), 0, 12345, 7))
