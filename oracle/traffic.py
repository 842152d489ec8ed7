"""Memory-access model of paper Sec. 4.1 ("Reduction in memory traffic", Table 1).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Counts are volumetric/facet values read or written per cell and smoothing step,
assuming every local operator matrix and the residual stay in cache:
  Alg. 1 (vanilla):          (2d+5)(p+1)^d
  Alg. 2 / Alg. 4:           3(p+1)^d + 7d(p+1)^(d-1)
  Alg. 2 as a standalone solver with the exit test of Alg. 3:
                             5(p+1)^d + 7d(p+1)^(d-1)
"""


def accesses_alg1(d, p):
    """Values accessed per cell and step by Alg. 1 (Table 1, Sec. 4.1.3)."""
    q = p + 1
    return (2 * d + 5) * q ** d


def accesses_alg2(d, p, standalone=False):
    """Values accessed per cell and step by Alg. 2 / Alg. 4, or as a standalone
    solver with the exit test of Alg. 3 (Table 1, Sec. 4.1.3)."""
    q = p + 1
    return (5 if standalone else 3) * q ** d + 7 * d * q ** (d - 1)


def reduction(d, p, standalone=False):
    """Ratio of the two counts (the reduction columns of Table 1)."""
    return accesses_alg1(d, p) / accesses_alg2(d, p, standalone)
