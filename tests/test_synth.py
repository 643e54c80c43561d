"""Host-side input generators: the paper's cases built by plane slabs (as the experiment script and large
grids use them) equal the whole-grid generator the parity tests use, value for value."""
import numpy as np
import pytest

import synth


@pytest.mark.parametrize("case", [1, 2, 3, 4])
def test_paper_case_slabs_equal_the_whole_grid(case):
    n = 37
    F, h, src = synth.speed_paper_case(case, n)
    assert F.shape == (n, n, n) and h == 1.0 / n
    parts = [synth.speed_paper_case_slab(case, n, z0, min(n, z0 + 5)) for z0 in range(0, n, 5)]
    assert np.array_equal(np.concatenate(parts), F)
    # the centre source, in node coordinates (grid point 0 at the origin)
    assert np.allclose(src, 0.5 * (n - 1) * h)
    if case == 4:
        assert (F == 0).any() and (F == 1).any() and set(np.unique(F)) <= {0.0, 1.0}
    if case == 3:
        assert F.min() > 0.0 and F.max() < 2.0
