"""The library's Marching Cubes case table (built on the host from its own statement of
the triangulation rule) equals the oracle's, case by case, including triangle order and
orientation.  Host code only: runs without a GPU."""
import numpy as np

import oracle
from paper_1709_03763_b300 import mc_case


def test_library_table_equals_oracle_rule():
    for m in range(256):
        assert np.array_equal(mc_case(m), oracle.mc_case(m)), m
