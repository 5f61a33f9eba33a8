"""Seeded synthetic initial conditions shared by the oracle and the CUDA path.

This module is input preparation only: it holds none of the particle-mesh
step's arithmetic (no deposit, no field solve, no kick or drift, no time
schedule).  Both sides of every parity test receive the arrays it returns.

Recipe (the paper's own comparison runs use external 3LPT initial conditions,
Sec. 4.4; these are a textbook stand-in with the same structure):

* white noise: one standard normal deviate per lattice site from a
  counter-based generator, SplitMix64 (Steele, Lea & Flood 2014) keyed by
  (seed, site, draw) and turned into normals by the Box-Muller transform;
* power spectrum P(k) = A k^ns T_BBKS(k)^2 with the BBKS transfer function
  (Bardeen, Bond, Kaiser & Szalay 1986), shape parameter Gamma = Omega_m h,
  normalised to sigma_8 with a top-hat window of radius 8 Mpc/h;
* linear growth D(a) of flat LCDM from the Heath (1977) integral
  D ~ E(a) * int_0^a da' / (a' E(a'))^3, growth rate f = dlnD/dlna;
* Zel'dovich displacement Psi_k = i k delta_k / k^2 (continuous k, Nyquist
  planes and k = 0 zeroed), particles on a lattice offset by half a spacing,
  x = q + D(a_pos)/D(1) Psi(q) and per-mass momentum
  u = a dx/dtau = a_vel * Hc(a_vel) * f(a_vel) * D(a_vel)/D(1) * Psi(q),
  where Hc = a H0 sqrt(Omega_m a^-3 + Omega_L) is the conformal Hubble rate.

Units: comoving box length 1, c = 1, H0 = box[Mpc/h] / 2997.92458.
"""
from __future__ import annotations

import math

import numpy as np

C_OVER_H0_MPCH = 2997.92458

_M64 = np.uint64(0xFFFFFFFFFFFFFFFF)


def splitmix64(x: np.ndarray) -> np.ndarray:
    """SplitMix64 output function applied to a uint64 counter array."""
    with np.errstate(over="ignore"):
        z = (x + np.uint64(0x9E3779B97F4A7C15)) & _M64
        z = ((z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)) & _M64
        z = ((z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)) & _M64
        return z ^ (z >> np.uint64(31))


def white_noise(n: int, seed: int) -> np.ndarray:
    """Unit-variance Gaussian white noise on an n^3 lattice, [z][y][x] order.

    Site s draws counters 2s and 2s+1 of stream `seed`; Box-Muller maps the
    two uniforms (53-bit, in (0,1]) to one normal deviate.
    """
    s = np.arange(n ** 3, dtype=np.uint64)
    key = np.uint64(seed & 0xFFFFFF) << np.uint64(40)
    r1 = splitmix64(key ^ (s << np.uint64(1)))
    r2 = splitmix64(key ^ ((s << np.uint64(1)) | np.uint64(1)))
    inv = 1.0 / 9007199254740992.0  # 2^-53
    u1 = ((r1 >> np.uint64(11)).astype(np.float64) + 1.0) * inv
    u2 = (r2 >> np.uint64(11)).astype(np.float64) * inv
    return (np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * np.pi * u2)).reshape(n, n, n)


def t_bbks(k_hmpc: np.ndarray, gamma: float) -> np.ndarray:
    """BBKS transfer function, k in h/Mpc."""
    q = np.maximum(k_hmpc, 1e-30) / gamma
    return (np.log1p(2.34 * q) / (2.34 * q)) * (
        1.0 + 3.89 * q + (16.1 * q) ** 2 + (5.46 * q) ** 3 + (6.71 * q) ** 4
    ) ** -0.25


def _tophat(x: np.ndarray) -> np.ndarray:
    return 3.0 * (np.sin(x) - x * np.cos(x)) / x ** 3


def spectrum_amplitude(omega_m: float, h: float, ns: float, sigma8: float) -> float:
    """A such that A k^ns T^2 has the given sigma_8 (k in h/Mpc, P in (Mpc/h)^3)."""
    lk = np.linspace(math.log(1e-5), math.log(1e3), 200001)
    k = np.exp(lk)
    integrand = k ** 3 * k ** ns * t_bbks(k, omega_m * h) ** 2 * _tophat(8.0 * k) ** 2
    s2 = np.trapezoid(integrand, lk) / (2.0 * math.pi ** 2)
    return sigma8 ** 2 / s2


def _efun(a, omega_m):
    return np.sqrt(omega_m / a ** 3 + (1.0 - omega_m))


def growth(a: float, omega_m: float) -> tuple[float, float]:
    """Unnormalised linear growth D(a) and f = dlnD/dlna for flat LCDM."""
    x = np.linspace(0.0, a, 20001)[1:]
    xi = np.concatenate([[0.0], x])
    yi = np.concatenate([[0.0], 1.0 / (x * _efun(x, omega_m)) ** 3])
    integral = np.trapezoid(yi, xi)
    e = float(_efun(a, omega_m))
    d = 2.5 * omega_m * e * integral
    de_da = -1.5 * omega_m / a ** 4 / e
    dd_da = 2.5 * omega_m * (de_da * integral + e / (a * e) ** 3)
    return d, a * dd_da / d


def _rfft3(x):
    try:
        import scipy.fft as sf
        return sf.rfftn(x, workers=-1)
    except ImportError:  # pragma: no cover
        return np.fft.rfftn(x)


def _irfft3(x, n):
    try:
        import scipy.fft as sf
        return sf.irfftn(x, s=(n, n, n), workers=-1)
    except ImportError:  # pragma: no cover
        return np.fft.irfftn(x, s=(n, n, n))


def zeldovich_ics(n_side: int, box_mpch: float, omega_m: float, h: float,
                  a_pos: float, a_vel: float, seed: int,
                  sigma8: float = 0.8, ns: float = 0.96,
                  amplitude_scale: float = 1.0):
    """Positions (box units, [0,1)) and per-mass momenta u for n_side^3 particles.

    Returns (pos, mom), each float64 [n_side^3, 3] in (x, y, z) order, rows in
    lattice order id = (iz * n + iy) * n + ix.
    """
    n = int(n_side)
    A = spectrum_amplitude(omega_m, h, ns, sigma8) * amplitude_scale ** 2
    w = white_noise(n, seed)
    wk = _rfft3(w)
    kz = np.fft.fftfreq(n, 1.0 / n)[:, None, None]
    ky = np.fft.fftfreq(n, 1.0 / n)[None, :, None]
    kx = np.arange(n // 2 + 1, dtype=np.float64)[None, None, :]
    k2n = kx ** 2 + ky ** 2 + kz ** 2
    kbox = 2.0 * math.pi * np.sqrt(k2n)
    k_hmpc = kbox / box_mpch
    p_box = A * k_hmpc ** ns * t_bbks(k_hmpc, omega_m * h) ** 2 / box_mpch ** 3
    p_box[0, 0, 0] = 0.0
    dk = wk * np.sqrt(n ** 3 * p_box)
    nyq = (np.abs(kx) == n // 2) | (np.abs(ky) == n // 2) | (np.abs(kz) == n // 2)
    dk = np.where(nyq, 0.0, dk)
    dk[0, 0, 0] = 0.0
    d1, _ = growth(1.0, omega_m)
    dp, _ = growth(a_pos, omega_m)
    dv, fv = growth(a_vel, omega_m)
    h0 = box_mpch / C_OVER_H0_MPCH
    hc_v = a_vel * h0 * math.sqrt(omega_m / a_vel ** 3 + (1.0 - omega_m))
    k2 = np.where(k2n == 0, 1.0, (2.0 * math.pi) ** 2 * k2n)
    psi = []
    for kc in (kx, ky, kz):
        psi.append(_irfft3(1j * (2.0 * math.pi * kc) * dk / k2, n).reshape(-1))
    psi = np.stack(psi, axis=1)
    iz, iy, ix = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
    q = (np.stack([ix.reshape(-1), iy.reshape(-1), iz.reshape(-1)], axis=1) + 0.5) / n
    pos = q + (dp / d1) * psi
    pos = pos - np.floor(pos)
    pos[pos >= 1.0] = 0.0
    mom = (a_vel * hc_v * fv * dv / d1) * psi
    return np.ascontiguousarray(pos), np.ascontiguousarray(mom)


def plane_wave_ics(n_side: int, amplitude: float, mode: int, a_pos: float,
                   a_vel: float, omega_m: float, box_mpch: float):
    """One Zel'dovich plane wave along x: delta(q) = amplitude*D(a)/D(a_pos)*cos(2 pi mode q_x).

    The displacement Psi_x = -amplitude/(2 pi mode) sin(2 pi mode q_x) gives
    delta = -dPsi/dq = amplitude cos(...) at a_pos; velocities follow the
    growing mode.  Used for the linear-growth check.
    """
    n = int(n_side)
    iz, iy, ix = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
    q = (np.stack([ix.reshape(-1), iy.reshape(-1), iz.reshape(-1)], axis=1) + 0.5) / n
    kq = 2.0 * math.pi * mode
    psi = np.zeros_like(q)
    psi[:, 0] = -amplitude / kq * np.sin(kq * q[:, 0])
    dp, _ = growth(a_pos, omega_m)
    dv, fv = growth(a_vel, omega_m)
    h0 = box_mpch / C_OVER_H0_MPCH
    hc_v = a_vel * h0 * math.sqrt(omega_m / a_vel ** 3 + (1.0 - omega_m))
    pos = q + psi
    pos = pos - np.floor(pos)
    mom = (a_vel * hc_v * fv * dv / dp) * psi
    return np.ascontiguousarray(pos), np.ascontiguousarray(mom)


def a_half_step_before(a0: float, dtau0: float, omega_m: float, box_mpch: float) -> float:
    """Scale factor at tau_0 - dtau_0 / 2, where the initial momenta live (leap-frog staggering): Newton's
    method on the conformal-time integral int da / (a Hc), Hc = a H0 sqrt(Omega_m / a^3 + 1 - Omega_m),
    with 16-point Gauss-Legendre quadrature over the half step."""
    h0 = box_mpch / 2997.92458

    def hc(a):
        return a * h0 * math.sqrt(omega_m / a ** 3 + 1 - omega_m)

    x, w = np.polynomial.legendre.leggauss(16)

    def tau(a_lo, a_hi):
        m, r = 0.5 * (a_lo + a_hi), 0.5 * (a_hi - a_lo)
        return r * sum(wi / ((m + r * xi) * hc(m + r * xi)) for xi, wi in zip(x, w))

    a = a0 * math.exp(-0.5 * dtau0 * hc(a0))
    for _ in range(50):
        g = tau(a, a0) - 0.5 * dtau0
        a += g * a * hc(a)
    return a

