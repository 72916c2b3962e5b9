"""The paper's printed results reproduced through the GPU path: Table 1
(flat-interface densities and Laplace surface tension at G = -5.3, tau from
Oh = 0.1) for every column."""
import os

import pytest

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "table1.txt")


def test_table1_on_gpu():
    from paper_1904_11792_gb300 import build, lbm, studies
    build.build()
    lbm.load()
    paper = [[float(v) for v in line.split()] for line in open(GOLDEN)
             if line.strip() and not line.startswith("#")]
    rows = studies.table1()
    assert len(rows) == len(paper) == 7
    for r, (R0, rl, rv, sg) in zip(rows, paper):
        assert r["R0"] == R0
        assert abs(r["rho_l"] - rl) <= 0.003, r
        assert abs(r["rho_v"] - rv) <= 0.002, r
        assert abs(r["sigma"] / sg - 1.0) <= 0.05, r
