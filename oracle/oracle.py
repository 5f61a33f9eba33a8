"""ctypes binding of the plain FP64 C oracle (pm_oracle.c).

Test infrastructure only: the library product never imports this module.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "pm_oracle.c")
_SO = os.path.join(_HERE, "liboracle.so")

_dp = np.ctypeslib.ndpointer(dtype=np.float64, flags="C_CONTIGUOUS")
_i64p = np.ctypeslib.ndpointer(dtype=np.int64, flags="C_CONTIGUOUS")


def build_oracle(force: bool = False) -> str:
    """Compile pm_oracle.c with gcc into liboracle.so next to it (with OpenMP where gcc has it)."""
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + f".tmp{os.getpid()}"
        base = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"]
        if subprocess.call(base + ["-fopenmp"], stderr=subprocess.DEVNULL) != 0:
            subprocess.check_call(base)
        os.replace(tmp, _SO)
    return _SO


def set_threads(n: int = 0) -> int:
    """Threads of the oracle's OpenMP loops (0: all cores); returns the count in use (1 without OpenMP).
    Results do not depend on it: the parallel loops have independent iterations and no reductions."""
    return int(lib().or_set_threads(int(n)))


_lib = None


def lib():
    global _lib
    if _lib is None:
        L = C.CDLL(build_oracle())
        L.or_set_threads.restype = C.c_int
        L.or_set_threads.argtypes = [C.c_int]
        L.or_conformal_hubble.restype = C.c_double
        L.or_conformal_hubble.argtypes = [C.c_double, C.c_double, C.c_double]
        L.or_tau_between.restype = C.c_double
        L.or_tau_between.argtypes = [C.c_double] * 4
        L.or_a_after.restype = C.c_double
        L.or_a_after.argtypes = [C.c_double] * 4
        L.or_schedule.argtypes = [C.c_int, C.c_double, C.c_double, C.c_double, C.c_double, _dp, _dp, _dp]
        L.or_fft3d_interleaved.argtypes = [_dp, C.c_int, C.c_int]
        L.or_cic_interp.argtypes = [_dp, C.c_int, _dp, C.c_long, _dp]
        L.or_deposit_mass.argtypes = [C.c_int, _dp, C.c_long, C.c_double, _dp]
        L.or_gradient.argtypes = [_dp, C.c_int, C.c_int, _dp]
        L.or_project.argtypes = [C.c_int, _dp, _dp, C.c_long, C.c_double, C.c_double, _dp, _dp, C.c_int,
                                 _dp, _dp, _dp]
        L.or_tensor_step_ri.argtypes = [_dp, _dp, C.c_double, C.c_double, C.c_double, C.c_double, C.c_double]
        L.or_power_spectrum.argtypes = [C.c_int, _dp, C.c_double, C.c_int, _dp, _dp, _i64p]
        L.or_solve_sources_flat.argtypes = ([C.c_int] + [C.c_double] * 8 + [C.c_int, C.c_int] + [_dp] * 7 +
                                            [C.c_int, C.c_int, C.c_double, _dp])
        L.or_sources_flat.argtypes = [C.c_int] + [C.c_double] * 6 + [C.c_int, C.c_int] + [_dp] * 9 + [C.c_int]
        L.or_laplacian7.argtypes = [_dp, C.c_int, _dp]
        L.or_hc_remainder.argtypes = [C.c_int, C.c_double, C.c_double, _dp, _dp, _dp, _dp]
        L.or_kick_drift.argtypes = [C.c_int, _dp, _dp, C.c_long] + [C.c_double] * 4 + [C.c_int, _dp, _dp, _dp]
        L.or_polarisations.argtypes = [np.ctypeslib.ndpointer(dtype=np.int64, flags="C_CONTIGUOUS"), _dp, _dp, _dp]
        L.or_project_vertex.argtypes = [C.c_int, np.ctypeslib.ndpointer(dtype=np.int64, flags="C_CONTIGUOUS"), _dp,
                                        _dp, C.c_long, C.c_double, C.c_double, _dp, _dp, _dp]
        L.or_sim_create.restype = C.c_void_p
        L.or_sim_create.argtypes = [C.c_int, C.c_long, C.c_double, C.c_double, C.c_double, C.c_double, C.c_int,
                                    C.c_int]
        L.or_sim_destroy.argtypes = [C.c_void_p]
        L.or_sim_schedule.argtypes = [C.c_void_p, _dp, _dp, _dp]
        L.or_sim_set_particles.argtypes = [C.c_void_p, _dp, _dp]
        L.or_sim_step.restype = C.c_int
        L.or_sim_step.argtypes = [C.c_void_p]
        L.or_sim_solve.restype = C.c_int
        L.or_sim_solve.argtypes = [C.c_void_p]
        L.or_sim_update.restype = C.c_int
        L.or_sim_update.argtypes = [C.c_void_p, C.c_void_p]
        L.or_sim_get_field.argtypes = [C.c_void_p, C.c_int, _dp]
        L.or_sim_get_tensor.argtypes = [C.c_void_p, C.c_int, _dp]
        L.or_sim_get_particles.argtypes = [C.c_void_p, _dp, _dp]
        L.or_sim_step_index.restype = C.c_int
        L.or_sim_step_index.argtypes = [C.c_void_p]
        _lib = L
    return _lib


# ---- thin numpy helpers around the C entry points ---------------------------

def fft3d(a: np.ndarray, sign: int = -1) -> np.ndarray:
    """Unnormalised 3D DFT of an N^3 complex array with the oracle's own FFT."""
    n = a.shape[0]
    buf = np.ascontiguousarray(a, dtype=np.complex128).view(np.float64).reshape(-1).copy()
    lib().or_fft3d_interleaved(buf, n, sign)
    return buf.view(np.complex128).reshape(n, n, n)


def tau_between(a0, a1, omega_m, h0):
    return lib().or_tau_between(a0, a1, omega_m, h0)


def a_after(a0, dtau, omega_m, h0):
    return lib().or_a_after(a0, dtau, omega_m, h0)


def schedule(nsteps, a_i, a_f, omega_m, h0):
    a_n = np.zeros(nsteps + 1); dt = np.zeros(nsteps); ah = np.zeros(nsteps)
    lib().or_schedule(nsteps, a_i, a_f, omega_m, h0, a_n, dt, ah)
    return a_n, dt, ah


def deposit_mass(n, pos, mass):
    rho = np.zeros(n ** 3)
    pos = np.ascontiguousarray(pos, dtype=np.float64).reshape(-1)
    lib().or_deposit_mass(n, pos, pos.size // 3, mass, rho)
    return rho.reshape(n, n, n)


def cic_interp(field, pos):
    n = field.shape[0]
    pos = np.ascontiguousarray(pos, dtype=np.float64).reshape(-1)
    out = np.zeros(pos.size // 3)
    lib().or_cic_interp(np.ascontiguousarray(field, dtype=np.float64).reshape(-1), n, pos, pos.size // 3, out)
    return out


def gradient(field, d):
    n = field.shape[0]
    g = np.zeros(n ** 3)
    lib().or_gradient(np.ascontiguousarray(field, dtype=np.float64).reshape(-1), n, d, g)
    return g.reshape(n, n, n)


def project(n, pos, mom, mass, a, phi_prev, chi_prev, newtonian=False):
    nc = n ** 3
    s00 = np.zeros(nc); s0i = np.zeros(3 * nc); sij = np.zeros(6 * nc)
    pos = np.ascontiguousarray(pos, dtype=np.float64).reshape(-1)
    mom = np.ascontiguousarray(mom, dtype=np.float64).reshape(-1)
    lib().or_project(n, pos, mom, pos.size // 3, mass, a,
                     np.ascontiguousarray(phi_prev, dtype=np.float64).reshape(-1),
                     np.ascontiguousarray(chi_prev, dtype=np.float64).reshape(-1), int(newtonian), s00, s0i, sij)
    return s00.reshape(n, n, n), s0i.reshape(3, n, n, n), sij.reshape(6, n, n, n)


def project_vertex(n, v, pos, mom, mass, a, phi_p=None, chi_p=None):
    """Projection [S00, S0x, S0y, S0z, Sxx, Sxy, Sxz, Syy, Syz, Szz] at vertex v=(x, y, z) from the listed particles."""
    pos = _flat(pos); mom = _flat(mom)
    npart = pos.size // 3
    phi_p = np.zeros(npart) if phi_p is None else _flat(phi_p)
    chi_p = np.zeros(npart) if chi_p is None else _flat(chi_p)
    out = np.zeros(10)
    lib().or_project_vertex(n, np.asarray(v, dtype=np.int64), pos, mom, npart, mass, a, phi_p, chi_p, out)
    return out


def tensor_step(h, v, k2, hc, dt, s):
    hb = np.array([h.real, h.imag], dtype=np.float64)
    vb = np.array([v.real, v.imag], dtype=np.float64)
    lib().or_tensor_step_ri(hb, vb, k2, hc, dt, float(np.real(s)), float(np.imag(s)))
    return complex(hb[0], hb[1]), complex(vb[0], vb[1])


def power_spectrum(rho, omega_m, nbins):
    n = rho.shape[0]
    k = np.zeros(nbins); pk = np.zeros(nbins); nm = np.zeros(nbins, dtype=np.int64)
    lib().or_power_spectrum(n, np.ascontiguousarray(rho, dtype=np.float64).reshape(-1), omega_m, nbins, k, pk, nm)
    return k, pk, nm


def _flat(a):
    return np.ascontiguousarray(a, dtype=np.float64).reshape(-1)


def sources(n, a, hc, dtau_prev, dtau_prev2, four_pi_g, omega_m, s00, s0i, sij, phi_prev, chi_prev, phi_prev2,
            newtonian=False, bootstrap=False, full_hc=False):
    """Configuration-space sources R, F (3), Sig (6: xx,xy,xz,yy,yz,zz)."""
    nc = n ** 3
    R = np.zeros(nc); F = np.zeros(3 * nc); S = np.zeros(6 * nc)
    lib().or_sources_flat(n, a, hc, dtau_prev, dtau_prev2, four_pi_g, omega_m, int(newtonian), int(bootstrap),
                          _flat(s00), _flat(s0i), _flat(sij), _flat(phi_prev), _flat(chi_prev), _flat(phi_prev2),
                          R, F, S, int(full_hc))
    return R.reshape(n, n, n), F.reshape(3, n, n, n), S.reshape(6, n, n, n)


def solve_sources(n, R, F=None, Sig=None, *, a=1.0, hc=0.0, dtau_prev=1.0, dtau_prev2=1.0, dtau=1.0, hc_half=0.0,
                  four_pi_g=1.0, omega_m=1.0, newtonian=False, bootstrap=False, tensor=None, b_space=False,
                  b_seed=False, b_decay=1.0, bstate=None):
    """Run the oracle's Fourier solve on given sources; returns phi, chi, B, tensor state.  With b_space, B
    comes from Eq. spacespace and `bstate` (complex (3, n, n, n), updated in place) carries B_k."""
    nc = n ** 3
    F = np.zeros(3 * nc) if F is None else _flat(F)
    Sig = np.zeros(6 * nc) if Sig is None else _flat(Sig)
    phi = np.zeros(nc); chi = np.zeros(nc); B = np.zeros(3 * nc)
    ts = np.zeros(8 * nc) if tensor is None else np.ascontiguousarray(tensor, dtype=np.complex128).view(
        np.float64).reshape(-1).copy()
    bs = np.zeros(6 * nc) if bstate is None else bstate.view(np.float64).reshape(-1)
    assert bstate is None or (bstate.dtype == np.complex128 and bstate.flags.c_contiguous and bstate.size == 3 * nc)
    lib().or_solve_sources_flat(n, a, hc, dtau_prev, dtau_prev2, dtau, hc_half, four_pi_g, omega_m, int(newtonian),
                                int(bootstrap), _flat(R), F, Sig, phi, chi, B, ts, int(b_space), int(b_seed),
                                float(b_decay), bs)
    return (phi.reshape(n, n, n), chi.reshape(n, n, n), B.reshape(3, n, n, n),
            ts.view(np.complex128).reshape(4, n, n, n))


def laplacian7(field):
    n = field.shape[0]
    out = np.zeros(n ** 3)
    lib().or_laplacian7(_flat(field), n, out)
    return out.reshape(field.shape)


def hc_remainder(hc, dtau_prev2, phi, chi, phi_prev2):
    """Nonlinear remainder Nl of Eq. fullHc on phi_{n-1}, chi_{n-1}, phi_{n-2}."""
    n = phi.shape[0]
    out = np.zeros(n ** 3)
    lib().or_hc_remainder(n, hc, dtau_prev2, _flat(phi), _flat(chi), _flat(phi_prev2), out)
    return out.reshape(phi.shape)


def kick_drift(n, pos, mom, a_kick, a_drift, dtau_kick, dtau_drift, phi, chi, B, newtonian=False):
    """One kick + drift of the given particles in the given fields (copies in, returns new arrays)."""
    p = _flat(pos).copy(); u = _flat(mom).copy()
    lib().or_kick_drift(n, p, u, p.size // 3, a_kick, a_drift, dtau_kick, dtau_drift, int(newtonian),
                        _flat(phi), _flat(chi), _flat(B))
    return p.reshape(-1, 3), u.reshape(-1, 3)


def polarisations_kt(nv, kt):
    ep = np.zeros(9); ex = np.zeros(9)
    lib().or_polarisations(np.asarray(nv, dtype=np.int64), np.asarray(kt, dtype=np.float64), ep, ex)
    return ep.reshape(3, 3), ex.reshape(3, 3)


FIELD_IDS = {"phi": 0, "chi": 1, "Bx": 2, "By": 3, "Bz": 4, "R": 5, "Fx": 6, "Fy": 7, "Fz": 8,
             "Sxx": 9, "Sxy": 10, "Sxz": 11, "Syy": 12, "Syz": 13, "Szz": 14}
TENSOR_IDS = {"h+": 0, "hx": 1, "h+'": 2, "hx'": 3}


class OracleSim:
    """The oracle's time stepper: set_particles() bootstraps, step() runs one PM step."""

    def __init__(self, n_mesh, n_part, omega_m, box_mpch, z_init, z_final=0.0, n_steps=100, newtonian=False,
                 full_hc=False, b_space=False):
        self.n = int(n_mesh)
        self.np = int(n_part)
        self.omega_m = omega_m
        self.h0 = box_mpch / 2997.92458
        self.mass = omega_m / n_part
        flags = int(bool(newtonian)) | (2 if full_hc else 0) | (4 if b_space else 0)
        self._h = lib().or_sim_create(self.n, self.np, omega_m, box_mpch, z_init, z_final, n_steps, flags)
        self.n_steps = n_steps
        self.a_n, self.dtau, self.a_half = np.zeros(n_steps + 1), np.zeros(n_steps), np.zeros(n_steps)
        lib().or_sim_schedule(self._h, self.a_n, self.dtau, self.a_half)

    def __del__(self):
        if getattr(self, "_h", None):
            lib().or_sim_destroy(self._h)
            self._h = None

    def set_particles(self, pos, mom):
        lib().or_sim_set_particles(self._h, np.ascontiguousarray(pos, dtype=np.float64).reshape(-1),
                                   np.ascontiguousarray(mom, dtype=np.float64).reshape(-1))

    def step(self):
        return lib().or_sim_step(self._h)

    def solve(self):
        """First half of a step: project and solve (fields of step n)."""
        return lib().or_sim_solve(self._h)

    def update(self, corr=None):
        """Second half: kick (plus the extra kick of a force correction corr [3][n][n][n]) and drift."""
        if corr is None:
            return lib().or_sim_update(self._h, None)
        c = np.ascontiguousarray(corr, dtype=np.float64).reshape(-1)
        return lib().or_sim_update(self._h, c.ctypes.data_as(C.c_void_p))

    @property
    def step_index(self):
        return lib().or_sim_step_index(self._h)

    def field(self, name):
        out = np.zeros(self.n ** 3)
        lib().or_sim_get_field(self._h, FIELD_IDS[name], out)
        return out.reshape(self.n, self.n, self.n)

    def tensor(self, name):
        out = np.zeros(2 * self.n ** 3)
        lib().or_sim_get_tensor(self._h, TENSOR_IDS[name], out)
        return out.view(np.complex128).reshape(self.n, self.n, self.n)

    def particles(self):
        pos = np.zeros(3 * self.np); mom = np.zeros(3 * self.np)
        lib().or_sim_get_particles(self._h, pos, mom)
        return pos.reshape(-1, 3), mom.reshape(-1, 3)
