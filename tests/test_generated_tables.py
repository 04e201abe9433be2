"""The committed coefficient tables are what their generator scripts write.

Each table of the CUDA path (the FP64 fixed-point Box-Muller tables, the FP64
and FP32 inverse-CDF polynomials, the FP32 Box-Muller log / sine / cosine
fits) comes from a script beside it in csrc/; re-running the script must
reproduce the committed values, so a table can neither drift from its script
nor be edited by hand.
"""

import os
import re
import subprocess
import sys

import pytest

CSRC = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                    "paper_2109_01329_gb300", "csrc")


def _run(script: str) -> str:
    return subprocess.run([sys.executable, script], cwd=CSRC, check=True, capture_output=True,
                          text=True, timeout=600).stdout


@pytest.mark.parametrize("script,header", [("gen_bm64_tables.py", "bm64_tables.h"),
                                           ("gen_icdf64_tables.py", "icdf64_tables.h"),
                                           ("gen_icdf32_tables.py", "icdf32_tables.h")])
def test_header_matches_its_generator(script, header):
    pytest.importorskip("mpmath")
    with open(os.path.join(CSRC, header)) as f:
        committed = f.read()
    assert _run(script) == committed, f"{header} differs from the output of {script}"


def test_fp32_box_muller_fits_are_the_kernel_constants():
    pytest.importorskip("mpmath")
    out = _run("gen_bm32_poly.py")
    with open(os.path.join(CSRC, "device_common.cuh")) as f:
        src = f.read()
    for name in ("S", "C", "L"):
        m = re.search(rf"^{name} = \{{(.*)\}}$", out, re.M)
        assert m, f"no {name} fit in the generator output"
        for coef in (c.strip() for c in m.group(1).split(",")):
            assert coef in src, f"{name} coefficient {coef} missing from device_common.cuh"
