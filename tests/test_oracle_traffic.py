"""Pin of the memory-access model (paper Sec. 4.1) against the printed Table 1."""
import os

import numpy as np

from oracle import traffic


def test_table1_memory_accesses():
    rows = np.loadtxt(os.path.join(os.path.dirname(__file__), "golden", "table1_memory_accesses.txt"))
    assert len(rows) == 20
    for d, p, a1, a2, red, a2s, reds in rows:
        d, p = int(d), int(p)
        assert traffic.accesses_alg1(d, p) == a1
        assert traffic.accesses_alg2(d, p) == a2
        assert traffic.accesses_alg2(d, p, standalone=True) == a2s
        assert abs(round(traffic.reduction(d, p), 2) - red) < 1e-9
        assert abs(round(traffic.reduction(d, p, standalone=True), 2) - reds) < 1e-9
