"""CPU checks of the C ABI boundary: the library builds, loads and exports
every symbol include/*.h declares; argument validation needs no GPU."""
import os
import re

import numpy as np
import pytest

import oracle

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lbm():
    from paper_1904_11792_gb300 import build, lbm as binding
    build.build()
    binding.load()
    return binding


def declared_functions():
    names = set()
    inc = os.path.join(ROOT, "include")
    for fn in os.listdir(inc):
        if not fn.endswith(".h"):
            continue
        text = open(os.path.join(inc, fn)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"\b(lbm_\w+)\s*\(", text):
            names.add(m.group(1))
    return names


def test_every_declared_symbol_is_exported(lbm):
    lib = lbm.load()
    names = declared_functions()
    assert len(names) >= 20
    missing = [n for n in sorted(names) if not hasattr(lib, n)]
    assert not missing, missing
    # the binding names the same entry points
    assert set(lbm.EXPORTS) == names


def test_lattice_table_matches_oracle(lbm):
    c, w = lbm.lbm_lattice()
    oc, ow, _ = oracle.lattice()
    np.testing.assert_array_equal(c, oc)
    np.testing.assert_array_equal(w, ow)


def test_strerror(lbm):
    assert lbm.lbm_strerror(lbm.LBM_OK) == "ok"
    assert "argument" in lbm.lbm_strerror(lbm.LBM_ERR_ARG)
    assert lbm.lbm_strerror(99) == "unknown status"


# the last case is the smallest cube with more than 2^31 - 1 nodes (in-plane
# indices are 32-bit)
@pytest.mark.parametrize("args", [(2, 8, 8, 1.0, -6.0), (8, 8, 8, 0.5, -6.0),
                                  (8, 8, 8, float("nan"), -6.0), (8, 8, 8, 1.0, float("inf")),
                                  (1291, 1291, 1291, 1.0, -6.0)])
def test_argument_validation_without_gpu(lbm, args):
    with pytest.raises(lbm.LbmError) as ei:
        lbm.lbm_create(*args)
    msg = str(ei.value)
    assert "tau" in msg or "dimension" in msg or "G must" in msg or "2^31-1 nodes" in msg


def test_required_bytes(lbm):
    cfg = lbm.lbm_config_default()
    cfg.nx, cfg.ny, cfg.nz = 10, 6, 4
    cfg.precision, cfg.pattern = lbm.LBM_F32, lbm.LBM_AB
    assert lbm.lbm_required_bytes(cfg) == (2 * 19 * 240 * 4, 240 * 4)
    cfg.precision, cfg.pattern = lbm.LBM_F16DEV, lbm.LBM_AA
    assert lbm.lbm_required_bytes(cfg) == (19 * 240 * 2, 240 * 4)
    cfg.precision = lbm.LBM_F64
    assert lbm.lbm_required_bytes(cfg) == (19 * 240 * 8, 240 * 8)
    cfg.block_x, cfg.block_y, cfg.block_z = 64, 16, 1
    with pytest.raises(lbm.LbmError):
        lbm.lbm_required_bytes(cfg)
