"""The seeded configuration generators (shared inputs; no PSE arithmetic)."""
import numpy as np
import pytest

from paper_1611_09322_gb300 import workloads


def _min_dist(p, L):
    d = p[:, None, :] - p[None, :, :]
    d -= L * np.round(d / L)
    r = np.linalg.norm(d, axis=2)
    np.fill_diagonal(r, np.inf)
    return r.min()


def test_rsa_non_overlapping_and_seeded():
    p, L, _ = workloads.hard_spheres(1000, 0.1, 1)
    assert p.dtype == np.float32 and p.shape == (1000, 3)
    assert np.all((p >= 0) & (p < L))
    assert _min_dist(p.astype(np.float64), L) >= 2.0 - 1e-4
    assert abs(1000 * 4 / 3 * np.pi / L ** 3 - 0.1) < 1e-12
    p2, _, _ = workloads.hard_spheres(1000, 0.1, 1)
    assert np.array_equal(p, p2)
    p3, _, _ = workloads.hard_spheres(1000, 0.1, 2)
    assert not np.array_equal(p, p3)


def test_dense_packing_relaxed():
    p, L, info = workloads.hard_spheres(2000, 0.4, 3)
    assert info["rsa_diameter"] < 2.0
    assert _min_dist(p.astype(np.float64), L) > 2.0 - 2e-3


def test_gel_clusters_fractal():
    ns = [32, 64, 128, 256, 512]
    rg = [np.sqrt((np.linalg.norm(workloads.cluster(n, 11), axis=1) ** 2).mean()) for n in ns]
    df = 1 / np.polyfit(np.log(ns), np.log(rg), 1)[0]
    assert abs(df - 1.9) < 0.15
    c = workloads.cluster(256, 5)
    d = np.linalg.norm(c[:, None] - c[None], axis=2)
    np.fill_diagonal(d, np.inf)
    assert abs(d.min() - 2.0) < 1e-6
    # every monomer touches another (aggregation by contact)
    assert np.all(d.min(axis=1) < 2.0 + 1e-6)


def test_gel_box():
    p, L, _ = workloads.gel(3000, 0.05, 4, csize=128)
    assert _min_dist(p.astype(np.float64), L) > 2.0 - 1e-4


def test_batch_spec():
    spec = workloads.batch_spec()
    assert len(spec) == 64
    Ns = np.array([s["N"] for s in spec])
    assert Ns.min() >= 1000 and Ns.max() <= 50000
    assert all(s["kind"] == "hs" or s["phi"] <= 0.2 for s in spec)
