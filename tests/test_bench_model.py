"""The benchmark's evaluation model follows the library's split search (CPU
only): its anchor stride is the one the kernels are built with."""
import os
import re

import bench

HERE = os.path.dirname(os.path.abspath(__file__))


def test_search_stride_matches_the_kernels():
    src = open(os.path.join(HERE, "..", "paper_2003_02256_gb300", "csrc", "masw_internal.h")).read()
    m = re.search(r"constexpr int SEARCH_STRIDE = (\d+);", src)
    assert m and int(m.group(1)) == bench.SEARCH_STRIDE
