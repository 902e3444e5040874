"""Parity cases against the bounds-checked build of the library (needs a
GB300).

compute-sanitizer is not available on the GPU pool, so a build compiled with
-DSPH_CHECK stands in for it on the neighbour passes: every sorted-slot
index a walk or a hit segment produces is checked against the particle
count, and an out-of-range one sets SPH_DEV_BOUNDS instead of being read.
The parity cases below run in a subprocess that loads that build
(SPH_GB300_LIB); each asserts that the step matches the oracle and that the
bit stays clear.
"""
import os
import subprocess
import sys

import pytest

from paper_2311_15088_gb300 import build

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))

CASES = ("dam_break_4096_first_step or fluid_with_boids_inside or crowded_cells or narrow_x_cells "
         "or edge_cases_small_scenes or neighbor_lists_bitwise")


def test_parity_cases_on_the_bounds_checked_build():
    lib = build.build(checked=True)
    env = dict(os.environ, SPH_GB300_LIB=lib)
    r = subprocess.run([sys.executable, "-m", "pytest", os.path.join(HERE, "test_gpu_parity.py"), "-q", "-x",
                        "-m", "gpu", "-k", CASES, "-p", "no:cacheprovider"],
                       env=env, capture_output=True, text=True, cwd=os.path.dirname(HERE), timeout=1200)
    tail = (r.stdout + r.stderr)[-3000:]
    assert r.returncode == 0, tail
    assert " passed" in r.stdout and "failed" not in r.stdout, tail
