"""Pins of the learned-correction oracle (oracle/correction.py) against closed forms,
an independent FFT route, finite differences and the C oracle's own CIC."""
import math

import numpy as np
import pytest

from oracle import correction as NC
from oracle import oracle as O


def rel(a, b):
    return float(np.linalg.norm((np.asarray(a) - np.asarray(b)).ravel()) / np.linalg.norm(np.asarray(b).ravel()))


def test_conv_matches_fft_circular_correlation():
    """y(c) = sum_d K(d) x(c + d) is the circular convolution of x with K placed at -d."""
    rng = np.random.default_rng(1)
    n, ci, co = 6, 3, 2
    x = rng.standard_normal((ci, n, n, n))
    W = rng.standard_normal((27, co, ci))
    b = rng.standard_normal(co)
    y = NC.conv(x, W, b)
    X = np.fft.fftn(x, axes=(1, 2, 3))
    for o in range(co):
        acc = np.zeros((n, n, n), complex)
        for i in range(ci):
            K = np.zeros((n, n, n))
            for k, (dz, dy, dx) in enumerate(NC.OFFSETS):
                K[(-dz) % n, (-dy) % n, (-dx) % n] = W[k, o, i]
            acc += X[i] * np.fft.fftn(K)
        assert rel(y[o], np.fft.ifftn(acc).real + b[o]) < 1e-13


def test_identity_kernel_reproduces_input():
    rng = np.random.default_rng(2)
    x = rng.standard_normal((4, 5, 5, 5))
    W = np.zeros((27, 4, 4))
    W[13] = np.eye(4)
    assert NC.OFFSETS[13] == (0, 0, 0)
    assert np.array_equal(NC.conv(x, W, np.zeros(4)), x)


def test_network_gradients_match_finite_differences():
    rng = np.random.default_rng(3)
    n = 4
    params = [(0.4 * rng.standard_normal((27, co, ci)), 0.1 * rng.standard_normal(co)) for ci, co, _ in NC.LAYERS]
    x = rng.standard_normal((2, n, n, n))
    t = rng.standard_normal((3, n, n, n))
    loss, grads = NC.loss_and_grads(params, x, t)
    h = 1e-6
    for layer, idx in [(0, (5, 3, 1)), (1, (13, 7, 2)), (2, (26, 0, 15)), (3, (0, 2, 9)), (3, (17, 1, 4))]:
        W, b = params[layer]
        Wp = W.copy(); Wp[idx] += h
        Wm = W.copy(); Wm[idx] -= h
        pp = list(params); pp[layer] = (Wp, b)
        pm_ = list(params); pm_[layer] = (Wm, b)
        fd = (NC.loss_and_grads(pp, x, t)[0] - NC.loss_and_grads(pm_, x, t)[0]) / (2 * h)
        assert abs(fd - grads[layer][0][idx]) <= 1e-6 * max(1.0, abs(fd)), (layer, idx, fd, grads[layer][0][idx])
    for layer in range(4):
        W, b = params[layer]
        bp = b.copy(); bp[1] += h
        bm = b.copy(); bm[1] -= h
        pp = list(params); pp[layer] = (W, bp)
        pm_ = list(params); pm_[layer] = (W, bm)
        fd = (NC.loss_and_grads(pp, x, t)[0] - NC.loss_and_grads(pm_, x, t)[0]) / (2 * h)
        assert abs(fd - grads[layer][1][1]) <= 1e-6 * max(1.0, abs(fd))


def test_input_gradient_is_the_adjoint_of_conv():
    """<conv(x) - b, g> = <x, dx(g)> for any x, g (the transpose of a linear map)."""
    rng = np.random.default_rng(4)
    x = rng.standard_normal((3, 5, 5, 5))
    g = rng.standard_normal((2, 5, 5, 5))
    W = rng.standard_normal((27, 2, 3))
    y = NC.conv(x, W, np.zeros(2))
    _, _, dx = NC.conv_backward(x, W, g)
    assert abs(np.sum(y * g) - np.sum(x * dx)) < 1e-11 * abs(np.sum(y * g))


def test_force_of_single_mode():
    n = 16
    z, y, x = np.meshgrid(*(np.arange(n) / n,) * 3, indexing="ij")
    phi = np.cos(2 * np.pi * (x + 2 * y))
    F = NC.force(phi)
    assert np.max(np.abs(F[0] - n * math.sin(2 * math.pi / n) * np.sin(2 * np.pi * (x + 2 * y)))) < 1e-12
    assert np.max(np.abs(F[1] - n * math.sin(4 * math.pi / n) * np.sin(2 * np.pi * (x + 2 * y)))) < 1e-12
    assert np.max(np.abs(F[2])) < 1e-12


def test_restriction_of_separable_mode():
    n = 8
    z, y, x = np.meshgrid(*(np.arange(2 * n) / (2 * n),) * 3, indexing="ij")
    k = (1, 3, 2)
    f = np.cos(2 * np.pi * k[0] * x) * np.cos(2 * np.pi * k[1] * y) * np.cos(2 * np.pi * k[2] * z)
    r = NC.restrict(f)
    zc, yc, xc = np.meshgrid(*(np.arange(n) / n,) * 3, indexing="ij")
    fac = np.prod([0.5 + 0.5 * math.cos(2 * math.pi * kk / (2 * n)) for kk in k])
    expect = fac * np.cos(2 * np.pi * k[0] * xc) * np.cos(2 * np.pi * k[1] * yc) * np.cos(2 * np.pi * k[2] * zc)
    assert np.max(np.abs(r - expect)) < 1e-13
    assert np.allclose(NC.restrict(np.full((2 * n,) * 3, 2.5)), 2.5, rtol=0, atol=1e-14)


def test_cic_interp_matches_c_oracle():
    rng = np.random.default_rng(5)
    n = 8
    f = rng.standard_normal((n, n, n))
    pos = rng.random((50, 3))
    assert rel(NC.cic_interp(f, pos), O.cic_interp(f, pos)) < 1e-14


def test_adam_first_step_is_signed_lr():
    g = np.array([0.3, -2.0, 1e-3])
    th, m, v = NC.adam(np.zeros(3), g, np.zeros(3), np.zeros(3), 1, 0.01)
    assert np.allclose(th, -0.01 * np.sign(g), rtol=1e-4)


def test_correction_kick_of_uniform_field():
    """A uniform correction c0 adds dtau_kick * a_n * c0 to every momentum (Newtonian kick is u-independent)."""
    from paper_2607_17929_gb300 import ics
    n = 8
    out = []
    for corr in (None, np.array([0.3, -0.2, 0.05])):
        s = O.OracleSim(n, n ** 3, 0.31, 160.0, 100.0, 0.0, 100, newtonian=True)
        a_m = O.a_after(s.a_n[0], -0.5 * s.dtau[0], 0.31, s.h0)
        pos, mom = ics.zeldovich_ics(n, 160.0, 0.31, 0.67, s.a_n[0], a_m, 2)
        s.set_particles(pos, mom)
        s.step()
        s.solve()
        s.update(None if corr is None else np.broadcast_to(corr[:, None, None, None], (3, n, n, n)))
        out.append((s.particles()[1], s.a_n[1], 0.5 * (s.dtau[0] + s.dtau[1])))
    (u0, a1, dtk), (u1, _, _) = out
    assert np.max(np.abs(u1 - u0 - dtk * a1 * np.array([0.3, -0.2, 0.05]))) < 1e-15
