"""The parameter set of the paper's modularity sweep (Section 7.3.4), built
on the host: mu in {2, 4, ..., 2^18} x eps in {.01, ..., .99}."""
import numpy as np

import paper_2012_11188_gb300.scan as scan


def test_paper_sigma_grid():
    mus, epss = scan.paper_sigma()
    assert mus.dtype == np.int32 and epss.dtype == np.float64
    assert mus.shape == epss.shape == (18 * 99,)
    assert sorted(set(mus.tolist())) == [2 ** k for k in range(1, 19)]
    assert sorted(set(epss.tolist())) == [float(f"0.{k:02d}") for k in range(1, 100)]
    # every pair exactly once, eps given as the correctly rounded k/100
    assert len(set(zip(mus.tolist(), epss.tolist()))) == 1782
    assert epss[6] == 0.07 and epss[98] == 0.99
