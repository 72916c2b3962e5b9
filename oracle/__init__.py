"""Plain FP64 CPU oracle of the D3Q19 Shan-Chen lattice Boltzmann step.

TEST INFRASTRUCTURE ONLY.  Only the tests, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package.  The product path
(``paper_1904_11792_gb300``) never imports it, and it never imports the
product path; the two share no code.

The arithmetic lives in ``lbm_oracle.c`` (plain C, one loop per equation of
the paper's "Numerical model" section, Eqs. 2-7).  This module compiles it
with gcc on first use and wraps it with ctypes and numpy.  ``np_oracle`` is a
second, independent NumPy implementation used to cross-check it on tiny grids.

Population arrays have shape (19, nz, ny, nx), float64, C order: direction a,
then z, y, x (x fastest), holding the pre-collision populations.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lbm_oracle.c")
_LIB_PATH = os.path.join(_HERE, "liblbm_oracle.so")
_lock = threading.Lock()
_lib = None

Q = 19


def build(force: bool = False) -> str:
    """Compile the oracle into ``oracle/liblbm_oracle.so`` (gcc, OpenMP)."""
    stale = (not os.path.exists(_LIB_PATH)) or (
        os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC))
    if force or stale:
        tmp = _LIB_PATH + ".tmp%d" % os.getpid()
        cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fPIC", "-shared",
               "-fopenmp", "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB_PATH)
            D, I, LL = ctypes.c_double, ctypes.c_int, ctypes.c_longlong
            P = ctypes.c_void_p
            lib.orc_num_threads.restype = I
            lib.orc_set_num_threads.argtypes = [I]
            lib.orc_lattice.argtypes = [P, P, P]
            lib.orc_psi.argtypes = [D, I, D]
            lib.orc_psi.restype = D
            lib.orc_feq.argtypes = [D, P, P]
            lib.orc_step.argtypes = [I, I, I, D, D, I, D, P, I]
            lib.orc_step.restype = I
            lib.orc_force.argtypes = [I, I, I, D, I, D, P, P]
            lib.orc_force.restype = I
            lib.orc_moments.argtypes = [I, I, I, D, I, D, P, I, P, P, P, P]
            lib.orc_moments.restype = I
            lib.orc_init_ligament.argtypes = [I, I, I, D, D, D, D, D, D, D, P]
            lib.orc_init_profile.argtypes = [I, I, I, D, D, D, D, P, I, D, D, P]
            lib.orc_ccl.argtypes = [I, I, I, P, P, P]
            lib.orc_ccl.restype = I
            lib.orc_diagnostics.argtypes = [I, I, I, P, D, D, P, P, P]
            lib.orc_droplets.argtypes = [I, I, I, P, D, D, P, I]
            lib.orc_droplets.restype = I
            lib.orc_step_nodes.argtypes = [I, I, I, D, D, I, D, P, P, I, P]
            lib.orc_coexistence.argtypes = [I, D, D, I, D, D, D, I, D, I, LL, P, P, P]
            lib.orc_coexistence_ex.argtypes = [I, D, P, D, I, D, D, D, I, D, I, LL, P, P, P]
            lib.orc_coexistence_ex.restype = I
            lib.orc_mrt_matrix.argtypes = [P]
            lib.orc_step_forcing.argtypes = [I, I, I, D, P, D, I, D, P, I]
            lib.orc_step_forcing.restype = I
            lib.orc_coexistence.restype = I
            _lib = lib
    return _lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


def num_threads() -> int:
    """OpenMP threads the oracle uses (1 without OpenMP)."""
    return _load().orc_num_threads()


def set_num_threads(n: int) -> None:
    _load().orc_set_num_threads(int(n))


def lattice():
    """(c[19,3] int, w[19] float, opp[19] int): the oracle's D3Q19 tables."""
    lib = _load()
    c = np.zeros((Q, 3), dtype=np.int32)
    w = np.zeros(Q, dtype=np.float64)
    opp = np.zeros(Q, dtype=np.int32)
    lib.orc_lattice(_ptr(c), _ptr(w), _ptr(opp))
    return c, w, opp


def psi(rho: float, form: int = 0, rho0: float = 1.0) -> float:
    """Pseudo-potential psi(rho) (functional defined after Eq. 5)."""
    return _load().orc_psi(float(rho), int(form), float(rho0))


def feq(rho: float, u) -> np.ndarray:
    """Second-order equilibrium of Eq. 2 (reading R1: with the leading 1)."""
    out = np.zeros(Q)
    uu = _f64(u)
    _load().orc_feq(float(rho), _ptr(uu), _ptr(out))
    return out


def step(f: np.ndarray, tau: float, G: float, nsteps: int = 1, psi_form: int = 0,
         rho0: float = 1.0) -> np.ndarray:
    """nsteps A-B time steps (Eqs. 4, 5, 6, 2, 3); returns a new array."""
    g = _f64(f).copy()
    _, nz, ny, nx = g.shape
    rc = _load().orc_step(nx, ny, nz, float(tau), float(G), int(psi_form), float(rho0),
                          _ptr(g), int(nsteps))
    if rc != 0:
        raise MemoryError("oracle step: allocation failed")
    return g


def force(f: np.ndarray, G: float, psi_form: int = 0, rho0: float = 1.0) -> np.ndarray:
    """Shan-Chen force field of Eq. 5, shape (3, nz, ny, nx)."""
    g = _f64(f)
    _, nz, ny, nx = g.shape
    F = np.zeros((3, nz, ny, nx))
    _load().orc_force(nx, ny, nz, float(G), int(psi_form), float(rho0), _ptr(g), _ptr(F))
    return F


def moments(f: np.ndarray, G: float, psi_form: int = 0, rho0: float = 1.0,
            bare: bool = False):
    """(rho, ux, uy, uz): Eq. 4 density and the velocity (j + F/2)/rho (R7)."""
    g = _f64(f)
    _, nz, ny, nx = g.shape
    out = [np.zeros((nz, ny, nx)) for _ in range(4)]
    _load().orc_moments(nx, ny, nz, float(G), int(psi_form), float(rho0), _ptr(g),
                        int(bool(bare)), *[_ptr(o) for o in out])
    return tuple(out)


def init_ligament(nx: int, ny: int, nz: int, R0: float, lam: float, eps: float, phase: float,
                  rho_l: float, rho_v: float, width: float = 2.0) -> np.ndarray:
    """Perturbed-cylinder initial state (set-up section; readings R9, R11-R13)."""
    f = np.zeros((Q, nz, ny, nx))
    _load().orc_init_ligament(nx, ny, nz, float(R0), float(lam), float(eps), float(phase),
                              float(rho_l), float(rho_v), float(width), _ptr(f))
    return f


def init_profile(nx: int, ny: int, nz: int, R0: float, lam: float, eps: float, phase: float,
                 prof, d0: float, dd: float) -> np.ndarray:
    """Initial state from a tabulated radial profile rho(d) (reading R15)."""
    p = _f64(prof)
    f = np.zeros((Q, nz, ny, nx))
    _load().orc_init_profile(nx, ny, nz, float(R0), float(lam), float(eps), float(phase),
                             _ptr(p), int(p.size), float(d0), float(dd), _ptr(f))
    return f


def ccl(mask: np.ndarray):
    """Periodic 6-connected components of a (nz, ny, nx) mask by flood fill.

    Returns (count, labels, sizes)."""
    m = np.ascontiguousarray(mask, dtype=np.uint8)
    nz, ny, nx = m.shape
    labels = np.zeros(m.shape, dtype=np.int32)
    sizes = np.zeros(m.size, dtype=np.int64)
    n = _load().orc_ccl(nx, ny, nz, _ptr(m), _ptr(labels), _ptr(sizes))
    if n < 0:
        raise MemoryError("oracle ccl: allocation failed")
    return n, labels, sizes[:n].copy()


DIAG_KEYS = ("mass", "mom_x", "mom_y", "mom_z", "liquid_volume_w", "liquid_count",
             "min_slice_area_w", "min_slice_count", "min_slice_x", "max_u", "rho_min",
             "rho_max", "numeric_ok")


def diagnostics(f: np.ndarray, rho_l: float, rho_v: float, slices: bool = False):
    """Sequential FP64 diagnostics (mass, momentum, liquid volume, neck area ...)."""
    g = _f64(f)
    _, nz, ny, nx = g.shape
    out = np.zeros(len(DIAG_KEYS))
    sw = np.zeros(nx)
    sn = np.zeros(nx)
    _load().orc_diagnostics(nx, ny, nz, _ptr(g), float(rho_l), float(rho_v), _ptr(out),
                            _ptr(sw), _ptr(sn))
    d = dict(zip(DIAG_KEYS, out.tolist()))
    d["neck_radius"] = float(np.sqrt(d["min_slice_area_w"] / np.pi))
    if slices:
        return d, sw, sn
    return d


DROPLET_KEYS = ("first", "nodes", "volume_w", "mass", "cx", "cy", "cz", "rx", "ry", "rz", "x_slices")


def droplets(f: np.ndarray, rho_l: float, rho_v: float, max_out: int | None = None):
    """Per-droplet statistics (connected liquid components), largest first.

    Returns (count, records): records is a (min(count, max_out), 11) array
    with the columns of DROPLET_KEYS."""
    g = _f64(f)
    _, nz, ny, nx = g.shape
    if max_out is None:
        max_out = g[0].size
    out = np.zeros((max(max_out, 1), len(DROPLET_KEYS)))
    n = _load().orc_droplets(nx, ny, nz, _ptr(g), float(rho_l), float(rho_v), _ptr(out), int(max_out))
    if n < 0:
        raise MemoryError("oracle droplets: allocation failed")
    return n, out[:min(n, max_out)].copy()


def mrt_matrix() -> np.ndarray:
    """The 19 x 19 D3Q19 moment matrix M of the MRT collision."""
    M = np.zeros((Q, Q))
    _load().orc_mrt_matrix(_ptr(M))
    return M


def mrt_rates(tau: float, s_e: float = 1.19, s_eps: float = 1.4, s_q: float = 1.2,
              s_pi: float = 1.4, s_m: float = 1.98) -> np.ndarray:
    """The 19 diagonal relaxation rates: shear moments (9, 11, 13, 14, 15)
    relax at 1/tau (nu = (tau - 1/2)/3); the conserved moments (0, 3, 5, 7)
    take 0 (their value does not matter); the others the given rates."""
    s = np.zeros(Q)
    s[1], s[2] = s_e, s_eps
    s[[4, 6, 8]] = s_q
    s[[9, 11, 13, 14, 15]] = 1.0 / tau
    s[[10, 12]] = s_pi
    s[[16, 17, 18]] = s_m
    return s


def step_forcing(f: np.ndarray, G: float, nsteps: int = 1, rates=None, tau: float = 1.0,
                 psi_form: int = 0, rho0: float = 1.0) -> np.ndarray:
    """nsteps MRT steps with Guo forcing (rates: 19 values), or, with rates
    None, SRT steps of relaxation time tau with the same Guo forcing."""
    g = _f64(f).copy()
    _, nz, ny, nx = g.shape
    r = None if rates is None else _f64(rates)
    rc = _load().orc_step_forcing(nx, ny, nz, float(tau), None if r is None else _ptr(r), float(G),
                                  int(psi_form), float(rho0), _ptr(g), int(nsteps))
    if rc != 0:
        raise MemoryError("oracle step_forcing: allocation failed")
    return g


def step_nodes(f: np.ndarray, nodes, tau: float, G: float, psi_form: int = 0,
               rho0: float = 1.0) -> np.ndarray:
    """Populations after one step at the given flat node indices, shape (k, 19)."""
    g = _f64(f)
    _, nz, ny, nx = g.shape
    idx = np.ascontiguousarray(nodes, dtype=np.int64)
    out = np.zeros((idx.size, Q))
    _load().orc_step_nodes(nx, ny, nz, float(tau), float(G), int(psi_form), float(rho0),
                           _ptr(g), _ptr(idx), int(idx.size), _ptr(out))
    return out


def coexistence(tau: float, G: float, n: int = 128, rho_l0: float = 2.5, rho_v0: float = 0.1,
                tol: float = 1e-12, check: int = 1000, max_steps: int = 400000,
                psi_form: int = 0, rho0: float = 1.0, f_init: np.ndarray | None = None,
                mrt_rates=None):
    """Flat-interface coexistence run (reading R14).

    mrt_rates (19 values) runs the MRT collision with Guo forcing instead of
    the paper's SRT step.  Returns dict(rho_l, rho_v, steps, dmax, profile,
    f) with f the final (19, 3, 3, n) state, which can seed a run at another
    tau."""
    f = np.zeros((Q, 3, 3, n)) if f_init is None else _f64(f_init).copy()
    out = np.zeros(4)
    prof = np.zeros(n)
    rates = None if mrt_rates is None else _f64(mrt_rates)
    rc = _load().orc_coexistence_ex(int(n), float(tau), None if rates is None else _ptr(rates),
                                    float(G), int(psi_form), float(rho0),
                                    float(rho_l0), float(rho_v0), int(f_init is None), float(tol),
                                    int(check), int(max_steps), _ptr(f), _ptr(out), _ptr(prof))
    if rc != 0:
        raise MemoryError("oracle coexistence: allocation failed")
    return dict(rho_l=out[0], rho_v=out[1], steps=int(out[2]), dmax=out[3], profile=prof, f=f)
