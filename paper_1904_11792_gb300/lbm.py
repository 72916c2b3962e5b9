"""Thin ctypes binding of liblbm.so (declared in include/lbm.h).

Every function here marshals arguments and calls the C ABI of the same name;
all lattice arithmetic runs in the library's CUDA kernels.  There is no CPU
fallback: the first call without a built liblbm.so raises ImportError, and
creating a lattice without a GB300 GPU fails with the library's error.

PyTorch is used only for plumbing: ``Lattice`` allocates the population and
psi buffers with torch (so they live in torch's caching allocator) and runs
the library on torch's current CUDA stream.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "liblbm.so")

Q = 19
LBM_OK, LBM_ERR_ARG, LBM_ERR_CUDA, LBM_ERR_OOM, LBM_ERR_NUMERIC, LBM_ERR_TIMEOUT, LBM_ERR_STATE = range(7)
LBM_PSI_EXP, LBM_PSI_RHO = 0, 1
LBM_F64, LBM_F32, LBM_F16DEV, LBM_BF16DEV = 0, 1, 2, 3
LBM_AB, LBM_AA = 0, 1
PRECISIONS = {"f64": LBM_F64, "f32": LBM_F32, "f16dev": LBM_F16DEV, "bf16dev": LBM_BF16DEV}
PATTERNS = {"ab": LBM_AB, "aa": LBM_AA}

# Every symbol include/lbm.h declares (checked by the tests).
EXPORTS = (
    "lbm_config_default", "lbm_required_bytes", "lbm_create", "lbm_create_ex", "lbm_destroy",
    "lbm_last_error", "lbm_strerror", "lbm_lattice", "lbm_set_stream", "lbm_set_option",
    "lbm_get_option", "lbm_init_ligament", "lbm_init_profile", "lbm_step", "lbm_diag_history",
    "lbm_sync",
    "lbm_moments", "lbm_diagnostics", "lbm_droplets", "lbm_get_populations", "lbm_set_populations",
    "lbm_state_bytes", "lbm_save_state", "lbm_load_state", "lbm_kernel_time",
    "lbm_batch_create", "lbm_batch_destroy", "lbm_batch_last_error", "lbm_batch_set_stream",
    "lbm_batch_set_option", "lbm_batch_info", "lbm_batch_init", "lbm_batch_step",
    "lbm_batch_step_sequential", "lbm_batch_sync", "lbm_batch_get_populations",
    "lbm_batch_diagnostics", "lbm_diagnostics_noalloc", "lbm_diagnostics_noalloc_max_scratch",
    "lbm_noalloc_last_error",
)


class LbmError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__("liblbm status %d: %s" % (status, message))
        self.status = status


class lbm_config(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
                ("tau", ctypes.c_double), ("G", ctypes.c_double), ("psi_form", ctypes.c_int),
                ("rho0", ctypes.c_double), ("precision", ctypes.c_int), ("pattern", ctypes.c_int),
                ("rho_ref", ctypes.c_double), ("block_x", ctypes.c_int), ("block_y", ctypes.c_int),
                ("block_z", ctypes.c_int), ("ext_state", ctypes.c_void_p),
                ("ext_state_bytes", ctypes.c_size_t), ("ext_psi", ctypes.c_void_p),
                ("ext_psi_bytes", ctypes.c_size_t), ("stream", ctypes.c_void_p)]


class lbm_diag(ctypes.Structure):
    _fields_ = [("step", ctypes.c_longlong), ("mass", ctypes.c_double),
                ("mom", ctypes.c_double * 3), ("liquid_volume_w", ctypes.c_double),
                ("liquid_count", ctypes.c_longlong), ("min_slice_area_w", ctypes.c_double),
                ("min_slice_count", ctypes.c_longlong), ("min_slice_x", ctypes.c_int),
                ("neck_radius", ctypes.c_double), ("max_u", ctypes.c_double),
                ("rho_min", ctypes.c_double), ("rho_max", ctypes.c_double),
                ("droplets", ctypes.c_int), ("droplets_min8", ctypes.c_int),
                ("largest_droplet", ctypes.c_longlong), ("numeric_ok", ctypes.c_int)]

    def as_dict(self) -> dict:
        d = {k: getattr(self, k) for k, _ in self._fields_ if k != "mom"}
        d["mom"] = tuple(self.mom)
        return d


class lbm_droplet(ctypes.Structure):
    _fields_ = [("first_node", ctypes.c_longlong), ("nodes", ctypes.c_longlong),
                ("volume_w", ctypes.c_double), ("mass", ctypes.c_double),
                ("centroid", ctypes.c_double * 3), ("resultant", ctypes.c_double * 3),
                ("x_slices", ctypes.c_int), ("reserved", ctypes.c_int)]

    def as_dict(self) -> dict:
        return dict(first_node=self.first_node, nodes=self.nodes, volume_w=self.volume_w,
                    mass=self.mass, centroid=tuple(self.centroid), resultant=tuple(self.resultant),
                    x_slices=self.x_slices)


class lbm_instance(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
                ("tau", ctypes.c_double), ("G", ctypes.c_double), ("R0", ctypes.c_double),
                ("lambda_", ctypes.c_double), ("eps", ctypes.c_double), ("phase", ctypes.c_double),
                ("rho_l", ctypes.c_double), ("rho_v", ctypes.c_double), ("width", ctypes.c_double)]


_lib = None


def load(path: Optional[str] = None) -> ctypes.CDLL:
    """Loads liblbm.so (build it first with ``paper_1904_11792_gb300.build``)."""
    global _lib
    if _lib is not None:
        return _lib
    p = path or LIB_PATH
    if not os.path.exists(p):
        raise ImportError("liblbm.so not built (%s); run paper_1904_11792_gb300.build.build()" % p)
    lib = ctypes.CDLL(p)
    H, P, I, D, LL = ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_longlong
    sig = {
        "lbm_config_default": (None, [P]),
        "lbm_required_bytes": (I, [P, P, P]),
        "lbm_create": (H, [I, I, I, D, D, I]),
        "lbm_create_ex": (H, [P]),
        "lbm_destroy": (None, [H]),
        "lbm_last_error": (ctypes.c_char_p, []),
        "lbm_strerror": (ctypes.c_char_p, [I]),
        "lbm_lattice": (I, [P, P]),
        "lbm_set_stream": (I, [H, P]),
        "lbm_set_option": (I, [H, ctypes.c_char_p, D]),
        "lbm_get_option": (I, [H, ctypes.c_char_p, P]),
        "lbm_init_ligament": (I, [H, D, D, D, D, D, D, D]),
        "lbm_init_profile": (I, [H, D, D, D, D, P, I, D, D]),
        "lbm_step": (I, [H, I]),
        "lbm_sync": (I, [H]),
        "lbm_diag_history": (I, [H, P, I, P]),
        "lbm_moments": (I, [H, P, P, P, P]),
        "lbm_diagnostics": (I, [H, P, I]),
        "lbm_droplets": (I, [H, P, I, P]),
        "lbm_get_populations": (I, [H, P]),
        "lbm_set_populations": (I, [H, P]),
        "lbm_state_bytes": (I, [H, P]),
        "lbm_save_state": (I, [H, P, ctypes.c_size_t]),
        "lbm_load_state": (I, [H, P, ctypes.c_size_t]),
        "lbm_kernel_time": (I, [H, I, P, P]),
        "lbm_batch_create": (H, [P, I, I, I, D, P]),
        "lbm_batch_destroy": (None, [H]),
        "lbm_batch_last_error": (ctypes.c_char_p, []),
        "lbm_batch_set_stream": (I, [H, P]),
        "lbm_batch_set_option": (I, [H, ctypes.c_char_p, D]),
        "lbm_batch_info": (I, [H, P, P, P]),
        "lbm_batch_init": (I, [H]),
        "lbm_batch_step": (I, [H, I]),
        "lbm_batch_step_sequential": (I, [H, I]),
        "lbm_batch_sync": (I, [H]),
        "lbm_batch_get_populations": (I, [H, I, P]),
        "lbm_batch_diagnostics": (I, [H, I, P, I]),
        "lbm_diagnostics_noalloc": (I, [P, I, I, I, I, D, D, D, P, P]),
        "lbm_diagnostics_noalloc_max_scratch": (ctypes.c_size_t, []),
        "lbm_noalloc_last_error": (ctypes.c_char_p, []),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name, None)
        if fn is None:
            continue
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def last_error() -> str:
    return load().lbm_last_error().decode()


def check(status: int) -> None:
    if status != LBM_OK:
        raise LbmError(status, last_error())


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


# ---- C ABI, one Python function per entry point -----------------------------

def lbm_config_default() -> lbm_config:
    c = lbm_config()
    load().lbm_config_default(ctypes.byref(c))
    return c


def lbm_required_bytes(cfg: lbm_config):
    s, p = ctypes.c_size_t(), ctypes.c_size_t()
    check(load().lbm_required_bytes(ctypes.byref(cfg), ctypes.byref(s), ctypes.byref(p)))
    return s.value, p.value


def lbm_create(nx, ny, nz, tau, G, psi_form=LBM_PSI_EXP):
    h = load().lbm_create(nx, ny, nz, float(tau), float(G), psi_form)
    if not h:
        raise LbmError(-1, last_error())
    return h


def lbm_create_ex(cfg: lbm_config):
    h = load().lbm_create_ex(ctypes.byref(cfg))
    if not h:
        raise LbmError(-1, last_error())
    return h


def lbm_destroy(h) -> None:
    load().lbm_destroy(h)


def lbm_strerror(status: int) -> str:
    return load().lbm_strerror(status).decode()


def lbm_lattice():
    c = np.zeros((Q, 3), dtype=np.int32)
    w = np.zeros(Q)
    check(load().lbm_lattice(_ptr(c), _ptr(w)))
    return c, w


def lbm_set_stream(h, stream: int) -> None:
    check(load().lbm_set_stream(h, ctypes.c_void_p(stream)))


def lbm_set_option(h, key: str, value: float) -> None:
    check(load().lbm_set_option(h, key.encode(), float(value)))


def lbm_get_option(h, key: str) -> float:
    v = ctypes.c_double()
    check(load().lbm_get_option(h, key.encode(), ctypes.byref(v)))
    return v.value


def lbm_init_ligament(h, R0, lam, eps, phase, rho_l, rho_v, width=2.0) -> None:
    check(load().lbm_init_ligament(h, float(R0), float(lam), float(eps), float(phase),
                                   float(rho_l), float(rho_v), float(width)))


def lbm_init_profile(h, R0, lam, eps, phase, prof, d0, dd) -> None:
    p = np.ascontiguousarray(prof, dtype=np.float64)
    check(load().lbm_init_profile(h, float(R0), float(lam), float(eps), float(phase), _ptr(p),
                                  int(p.size), float(d0), float(dd)))


def lbm_step(h, n: int) -> None:
    check(load().lbm_step(h, int(n)))


def lbm_diag_history(h, max_records: int = 1024) -> list:
    arr = (lbm_diag * max(max_records, 1))()
    n = ctypes.c_int()
    check(load().lbm_diag_history(h, arr, int(max_records), ctypes.byref(n)))
    return [arr[i].as_dict() for i in range(n.value)]


def lbm_sync(h) -> None:
    check(load().lbm_sync(h))


def lbm_moments(h, shape, want=("rho", "ux", "uy", "uz")):
    arrs = {k: np.zeros(shape) for k in want}
    ptrs = [(_ptr(arrs[k]) if k in arrs else None) for k in ("rho", "ux", "uy", "uz")]
    check(load().lbm_moments(h, *ptrs))
    return arrs


def lbm_diagnostics(h, want_ccl: bool = False) -> lbm_diag:
    d = lbm_diag()
    check(load().lbm_diagnostics(h, ctypes.byref(d), int(bool(want_ccl))))
    return d


def lbm_droplets(h, max_droplets: int = 1 << 20) -> tuple:
    """(count, [lbm_droplet, ...] largest first, at most max_droplets)."""
    n = ctypes.c_int(0)
    buf = (lbm_droplet * max(int(max_droplets), 1))()
    check(load().lbm_droplets(h, buf, int(max_droplets), ctypes.byref(n)))
    return n.value, [buf[k] for k in range(min(n.value, int(max_droplets)))]


def lbm_get_populations(h, shape) -> np.ndarray:
    out = np.zeros((Q,) + tuple(shape))
    check(load().lbm_get_populations(h, _ptr(out)))
    return out


def lbm_set_populations(h, f: np.ndarray) -> None:
    a = np.ascontiguousarray(f, dtype=np.float64)
    check(load().lbm_set_populations(h, _ptr(a)))


def lbm_state_bytes(h) -> int:
    v = ctypes.c_size_t()
    check(load().lbm_state_bytes(h, ctypes.byref(v)))
    return v.value


def lbm_save_state(h, out: Optional[np.ndarray] = None) -> np.ndarray:
    n = lbm_state_bytes(h)
    buf = np.zeros(n, dtype=np.uint8) if out is None else out
    check(load().lbm_save_state(h, _ptr(buf), n))
    return buf


def lbm_load_state(h, buf: np.ndarray) -> None:
    b = np.ascontiguousarray(buf, dtype=np.uint8)
    check(load().lbm_load_state(h, _ptr(b), b.size))


def lbm_kernel_time(h, k: int):
    n, ms = ctypes.c_longlong(), ctypes.c_double()
    check(load().lbm_kernel_time(h, int(k), ctypes.byref(n), ctypes.byref(ms)))
    return n.value, ms.value


# ---- batched form -------------------------------------------------------------

def _bcheck(status: int) -> None:
    if status != LBM_OK:
        raise LbmError(status, load().lbm_batch_last_error().decode())


class Batch:
    """Many independent ligaments of uneven size stepped together.

    ``instances``: sequence of dicts (or objects) with nx, ny, nz, tau, G,
    R0, lam, eps, phase, rho_l, rho_v, width."""

    def __init__(self, instances, precision="f32", psi_form=LBM_PSI_EXP, rho0=1.0):
        import torch
        arr = (lbm_instance * len(instances))()
        self.shapes = []
        for k, d in enumerate(instances):
            g = (lambda key: d[key]) if isinstance(d, dict) else (lambda key: getattr(d, key))
            arr[k] = lbm_instance(g("nx"), g("ny"), g("nz"), g("tau"), g("G"), g("R0"), g("lam"),
                                  g("eps"), g("phase"), g("rho_l"), g("rho_v"), g("width"))
            self.shapes.append((g("nz"), g("ny"), g("nx")))
        prec = PRECISIONS[precision] if isinstance(precision, str) else precision
        stream = torch.cuda.current_stream().cuda_stream or 1
        self.b = load().lbm_batch_create(arr, len(instances), prec, psi_form, float(rho0),
                                         ctypes.c_void_p(stream))
        if not self.b:
            raise LbmError(-1, load().lbm_batch_last_error().decode())

    def close(self):
        if getattr(self, "b", None):
            load().lbm_batch_destroy(self.b)
            self.b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def set_option(self, key, value):
        _bcheck(load().lbm_batch_set_option(self.b, key.encode(), float(value)))

    def info(self):
        n, t = ctypes.c_longlong(), ctypes.c_int()
        blk = (ctypes.c_int * 3)()
        _bcheck(load().lbm_batch_info(self.b, ctypes.byref(n), ctypes.byref(t), blk))
        return dict(total_nodes=n.value, tiles=t.value, block=tuple(blk))

    def init(self):
        _bcheck(load().lbm_batch_init(self.b))

    def step(self, n=1):
        _bcheck(load().lbm_batch_step(self.b, int(n)))

    def step_sequential(self, n=1):
        _bcheck(load().lbm_batch_step_sequential(self.b, int(n)))

    def sync(self):
        _bcheck(load().lbm_batch_sync(self.b))

    def populations(self, k) -> np.ndarray:
        out = np.zeros((Q,) + self.shapes[k])
        _bcheck(load().lbm_batch_get_populations(self.b, int(k), _ptr(out)))
        return out

    def diagnostics(self, k, ccl=False) -> dict:
        d = lbm_diag()
        _bcheck(load().lbm_batch_diagnostics(self.b, int(k), ctypes.byref(d), int(bool(ccl))))
        return d.as_dict()


# ---- convenience wrapper --------------------------------------------------

class Lattice:
    """One lattice on the current CUDA device, buffers owned by torch.

    ``Lattice(nx, ny, nz, tau, G, precision="f32", pattern="ab")`` creates
    the library handle with torch-allocated population and psi buffers and
    binds it to torch's current stream.
    """

    def __init__(self, nx, ny, nz, tau, G, precision="f32", pattern="ab", psi_form=LBM_PSI_EXP,
                 rho0=1.0, rho_ref=0.0, block=None, torch_buffers=True):
        import torch
        cfg = lbm_config_default()
        cfg.nx, cfg.ny, cfg.nz = nx, ny, nz
        cfg.tau, cfg.G, cfg.psi_form, cfg.rho0 = tau, G, psi_form, rho0
        cfg.precision = PRECISIONS[precision] if isinstance(precision, str) else precision
        cfg.pattern = PATTERNS[pattern] if isinstance(pattern, str) else pattern
        cfg.rho_ref = rho_ref
        if block is not None:
            cfg.block_x, cfg.block_y, cfg.block_z = block
        self._buffers = []
        if torch_buffers:
            sb, pb = lbm_required_bytes(cfg)
            st = torch.empty(sb, dtype=torch.uint8, device="cuda")
            ps = torch.empty(pb, dtype=torch.uint8, device="cuda")
            self._buffers = [st, ps]
            cfg.ext_state, cfg.ext_state_bytes = st.data_ptr(), sb
            cfg.ext_psi, cfg.ext_psi_bytes = ps.data_ptr(), pb
        # torch's default stream has handle 0; the library then gets the
        # legacy default stream (cudaStreamLegacy = 1) instead of its own
        cfg.stream = torch.cuda.current_stream().cuda_stream or 1
        self.shape = (nz, ny, nx)
        self.h = lbm_create_ex(cfg)

    def close(self):
        if getattr(self, "h", None):
            lbm_destroy(self.h)
            self.h = None
        self._buffers = []

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def init_ligament(self, R0, lam, eps, phase, rho_l, rho_v, width=2.0):
        lbm_init_ligament(self.h, R0, lam, eps, phase, rho_l, rho_v, width)

    def init_profile(self, R0, lam, eps, phase, prof, d0, dd):
        lbm_init_profile(self.h, R0, lam, eps, phase, prof, d0, dd)

    def step(self, n=1):
        lbm_step(self.h, n)

    def sync(self):
        lbm_sync(self.h)

    def set_option(self, key, value):
        lbm_set_option(self.h, key, value)

    def get_option(self, key):
        return lbm_get_option(self.h, key)

    @property
    def step_count(self) -> int:
        return int(lbm_get_option(self.h, "step"))

    def populations(self) -> np.ndarray:
        return lbm_get_populations(self.h, self.shape)

    def set_populations(self, f):
        lbm_set_populations(self.h, f)

    def moments(self, want=("rho", "ux", "uy", "uz")):
        return lbm_moments(self.h, self.shape, want)

    def rho(self) -> np.ndarray:
        return lbm_moments(self.h, self.shape, ("rho",))["rho"]

    def diag_history(self, max_records: int = 1024) -> list:
        return lbm_diag_history(self.h, max_records)

    def diagnostics(self, ccl=False) -> dict:
        return lbm_diagnostics(self.h, ccl).as_dict()

    def droplets(self, max_droplets: int = 1 << 20) -> tuple:
        """(count, list of droplet dicts, largest first)."""
        n, d = lbm_droplets(self.h, max_droplets)
        return n, [x.as_dict() for x in d]

    def save_state(self) -> np.ndarray:
        return lbm_save_state(self.h)

    def load_state(self, buf):
        lbm_load_state(self.h, buf)
