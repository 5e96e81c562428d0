"""The xi* model (Sec. II C, eqs. work and xistar) in the host library: its
value is the minimiser of the calibrated work, found here by brute force, and
it reduces to eq. xistar when the measured times are the terms of eq. work."""
import math

import numpy as np
import pytest

from paper_1611_09322_gb300 import PseError, pse_xi_model


def _work(xi, xi0, t_real, t_wave, d_f):
    return t_real * (xi0 / xi) ** d_f + t_wave * (xi / xi0) ** 3


@pytest.mark.parametrize("xi0,t_real,t_wave,d_f", [(0.5, 0.71, 0.40, 3.0), (0.5, 0.2, 1.5, 2.0),
                                                   (0.8, 3.0, 0.1, 1.0), (0.3, 1.0, 1.0, 2.5)])
def test_model_is_the_minimiser_of_the_calibrated_work(xi0, t_real, t_wave, d_f):
    xs = np.exp(np.linspace(math.log(0.1 * xi0), math.log(10 * xi0), 200001))
    best = xs[np.argmin(_work(xs, xi0, t_real, t_wave, d_f))]
    got = pse_xi_model(xi0, t_real, t_wave, d_f)
    assert abs(got - best) <= 2e-4 * best
    # a stationary point: the work rises on both sides
    assert _work(got, xi0, t_real, t_wave, d_f) < _work(got * 1.01, xi0, t_real, t_wave, d_f)
    assert _work(got, xi0, t_real, t_wave, d_f) < _work(got * 0.99, xi0, t_real, t_wave, d_f)


def test_model_balanced_costs_keep_xi():
    """d_f t_real = 3 t_wave: the derivative of the work vanishes at xi0."""
    assert pse_xi_model(0.5, 3.0, 2.0, 2.0) == pytest.approx(0.5, rel=1e-15)
    assert pse_xi_model(0.7, 1.0, 1.0, 3.0) == pytest.approx(0.7, rel=1e-15)


@pytest.mark.parametrize("d_f", [1.0, 2.0, 3.0])
def test_model_reduces_to_eq_xistar(d_f):
    """With t_real = C_R n_iter N phi xi0^-d_f and t_wave = C_W (xi0^3 N / phi) log N
    (eq. work, the FFT's logarithm taken at large N), the model's xi* equals
    eq. xistar, (3 C_W log N / (C_R d_f n_iter phi^2))^(-1/(d_f + 3)), for any xi0."""
    C_R, C_W, n_iter, N, phi = 2.3e-9, 4.1e-9, 7, 1e6, 0.1
    ref = (3 * C_W * math.log(N) / (C_R * d_f * n_iter * phi ** 2)) ** (-1 / (d_f + 3))
    for xi0 in (0.2, 0.5, 1.3):
        t_real = C_R * n_iter * N * phi * xi0 ** (-d_f)
        t_wave = C_W * xi0 ** 3 * N / phi * math.log(N)
        assert pse_xi_model(xi0, t_real, t_wave, d_f) == pytest.approx(ref, rel=1e-12)


def test_model_rejects_bad_arguments():
    for args in ((0.0, 1.0, 1.0, 3.0), (0.5, 0.0, 1.0, 3.0), (0.5, 1.0, -1.0, 3.0), (0.5, 1.0, 1.0, 0.5),
                 (0.5, 1.0, 1.0, 3.5), (0.5, float("nan"), 1.0, 3.0), (float("inf"), 1.0, 1.0, 3.0)):
        with pytest.raises(PseError):
            pse_xi_model(*args)
