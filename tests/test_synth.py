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


def test_torch_generator_matches_numpy():
    """The device-side generator (used for grids too large for the host) is the host generator: the same
    splitmix64 bits, the same normals to rounding, the same field to rounding (run here on the CPU)."""
    torch = pytest.importorskip("torch")
    z_np = synth.splitmix64(17, 5, 1000, start=12345)
    z_t = synth.splitmix64_torch(17, 5, 1000, 12345, "cpu").numpy().view(np.uint64)
    assert np.array_equal(z_np, z_t)
    a, b = synth.normal(17, 5, 2001), synth.normal_torch(17, 5, 2001, "cpu", chunk=300).numpy()
    assert np.max(np.abs(a - b)) <= 1e-13
    dims, h = (24, 17, 31), 1.0 / 30
    F = synth.speed_grf(dims, h, 1815)
    G = synth.speed_grf_torch(dims, h, 1815, "cpu", dtype=torch.float64).numpy()
    assert F.shape == G.shape == (31, 17, 24)
    assert np.max(np.abs(F - G) / F) <= 1e-12


def test_grf_field_has_the_stated_statistics():
    """C4's field: mean 0, standard deviation 0.5 over the realisation, and a Gaussian correlation of
    length 0.05 (at a lag of ell the correlation is exp(-1/2); at 4 ell it is gone)."""
    n = 96
    h = 1.0 / (n - 1)
    g = synth.grf_field((n, n, n), h, 1811 + 4)
    assert abs(g.mean()) < 1e-12 and abs(g.std() - 0.5) < 1e-12

    def corr(lag):
        return float(np.mean(g * np.roll(g, lag, axis=2)) / np.mean(g * g))

    lag = round(0.05 / h)                                    # 5 nodes = 0.0526
    want = np.exp(-(lag * h) ** 2 / (2 * 0.05 ** 2))         # 0.575
    assert abs(corr(lag) - want) < 0.08, (corr(lag), want)
    assert abs(corr(4 * lag)) < 0.1
    assert corr(1) > corr(lag) > corr(2 * lag)
