"""Allocation-free diagnostics entry point (lbm_diagnostics_noalloc).

Callers that cannot allocate device memory when they ask for diagnostics
(code running while another stream of the process is capturing a CUDA graph,
code inside an allocator callback, hosts that forbid the library to grow its
device memory after start-up) use this entry point: it reduces with the same
kernels as lbm_diagnostics, but into a fixed static device array.  Collected
last (file name) so that a failure here stops a -x run after everything else.
"""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

RL, RV = 2.648878066946715, 0.0731992478525716


def _lib():
    from paper_1904_11792_gb300 import build, lbm
    build.build()
    lib = lbm.load()
    lib.lbm_diagnostics_noalloc.restype = ctypes.c_int
    lib.lbm_diagnostics_noalloc.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                            ctypes.c_int, ctypes.c_double, ctypes.c_double,
                                            ctypes.c_double, ctypes.c_void_p, ctypes.c_void_p]
    lib.lbm_noalloc_last_error.restype = ctypes.c_char_p
    return lbm, lib


def _noalloc(lib, lat, shape, precision, rho_ref, out, stream):
    nx, ny, nz = shape
    rc = lib.lbm_diagnostics_noalloc(ctypes.c_void_p(lat._buffers[0].data_ptr()), nx, ny, nz,
                                     precision, rho_ref, RL, RV, ctypes.c_void_p(out.data_ptr()),
                                     ctypes.c_void_p(stream))
    assert rc == 0, lib.lbm_noalloc_last_error().decode()


# Two calls in a row on different lattices (they share the static scratch),
# for each storage precision; the *DEV forms pass the lattice's rho_ref, from
# which the entry point rebuilds the deviation shifts, and one lattice of each
# pair streams in place (AA) after an even number of steps, whose array is
# then in the canonical layout the entry point reads.
@pytest.mark.parametrize("precision", ["f32", "f64", "f16dev", "bf16dev"])
def test_noalloc_diagnostics_equal_handle_diagnostics_two_calls(precision):
    import torch
    L, lib = _lib()
    stream = torch.cuda.current_stream().cuda_stream or 1
    rho_ref = RV if precision.endswith("dev") else 0.0
    cases = []
    for shape, R0, pattern in (((64, 32, 32), 8.0, "ab"), ((40, 24, 20), 5.0, "aa")):
        lat = L.Lattice(*shape, 1.0, -6.0, precision=precision, pattern=pattern, rho_ref=rho_ref)
        lat.init_ligament(R0, float(shape[0]), 0.1, 0.0, RL, RV, 2.0)
        lat.step(12)            # even step count: the current array is the first one
        cases.append((shape, lat, lat.diagnostics()))
    outs = [torch.full((13,), float("nan"), dtype=torch.float64, device="cuda") for _ in cases]
    for (shape, lat, _), out in zip(cases, outs):
        _noalloc(lib, lat, shape, L.PRECISIONS[precision], rho_ref, out, stream)
    torch.cuda.synchronize()
    for (shape, lat, want), out in zip(cases, outs):
        r = out.cpu().numpy()
        assert abs(r[0] - want["mass"]) <= 1e-12 * want["mass"]
        np.testing.assert_allclose(r[1:4], want["mom"], rtol=0, atol=1e-12 * want["mass"])
        assert abs(r[4] - want["liquid_volume_w"]) <= 1e-12 * want["liquid_volume_w"]
        assert int(r[5]) == want["liquid_count"]
        assert abs(r[6] - want["min_slice_area_w"]) <= 1e-12 * max(1.0, want["min_slice_area_w"])
        assert int(r[7]) == want["min_slice_count"] and int(r[8]) == want["min_slice_x"]
        assert abs(r[9] - want["max_u"]) <= 1e-12 * max(want["max_u"], 1e-30)
        assert r[10] == want["rho_min"] and r[11] == want["rho_max"] and int(r[12]) == 1
        lat.close()


def test_noalloc_rejects_lattices_beyond_the_static_scratch():
    import torch
    L, lib = _lib()
    lib.lbm_diagnostics_noalloc_max_scratch.restype = ctypes.c_size_t
    assert lib.lbm_diagnostics_noalloc_max_scratch() == 524288
    out = torch.zeros(13, dtype=torch.float64, device="cuda")
    dummy = torch.zeros(16, dtype=torch.float32, device="cuda")
    # nx = 2^20 needs more slice partials than the static array holds; the
    # size check runs before any launch, so the tiny buffer is never read
    rc = lib.lbm_diagnostics_noalloc(ctypes.c_void_p(dummy.data_ptr()), 1 << 20, 4, 4, L.LBM_F32,
                                     0.0, RL, RV, ctypes.c_void_p(out.data_ptr()), None)
    assert rc == L.LBM_ERR_ARG
    assert "static maximum" in lib.lbm_noalloc_last_error().decode()
