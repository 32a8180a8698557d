"""The seeded workload generators against the recipes they state: the cross sections,
sources, initial states and angular rules of each synthetic problem, checked from their
defining properties (block pattern, disc area, support of the source, sample statistics and
correlation of the log-normal field, ranges of the batched draws)."""
import numpy as np
import pytest

from paper_2603_19647_gb300 import inputs


def test_slab():
    wl = inputs.slab_1d()
    assert (wl.nx, wl.ny, wl.quadrature, wl.nv, wl.c_dt, wl.steps) == (256, 1, ("gl", 16), 16, 0.01, 100)
    assert np.all(wl.sigma_t == 1.0) and np.all(wl.sigma_s == 0.99) and not wl.source.any()
    x = (np.arange(256) + 0.5) / 256
    assert np.argmax(wl.rho0) in (127, 128) and wl.rho0[0] < 1e-20
    assert np.allclose(wl.rho0, np.exp(-(x - 0.5) ** 2 / 0.005), rtol=0, atol=0)


def test_checkerboard_blocks_and_source():
    wl = inputs.checkerboard()
    assert (wl.nx, wl.ny, wl.nv, wl.c_dt, wl.steps) == (256, 256, 128, 0.005, 200)
    ss = wl.sigma_s.reshape(256, 256)          # [row y][column x]
    for J in range(8):
        for I in range(8):
            blk = ss[32 * J:32 * (J + 1), 32 * I:32 * (I + 1)]
            assert np.all(blk == (100.0 if (I + J) % 2 == 0 else 0.01)), (I, J)
    assert np.allclose(wl.sigma_t - wl.sigma_s, 0.1, rtol=0, atol=1e-12)
    G = wl.source.reshape(256, 256)
    assert set(np.unique(G)) == {0.0, 1.0}
    rows, cols = np.nonzero(G)
    # |x - 1/2|, |y - 1/2| < 1/16: the 32 x 32 cells about the centre (centres at +-31/512)
    assert (rows.min(), rows.max(), cols.min(), cols.max()) == (112, 143, 112, 143)
    assert G.sum() == 32 * 32 and not wl.rho0.any()


def test_lognormal_field_statistics():
    """log sigma_s has sample mean 0 and sample standard deviation `std` exactly (the
    normalisation), and the squared-exponential correlation of length 0.1: averaged over
    eight seeds, about exp(-1/8) at a lag of 0.05, exp(-1/2) at 0.1 and little at 0.2 (a field
    of correlation length 0.05 or 0.2 fails these)."""
    corr = {13: [], 26: [], 51: []}
    for seed in range(8):
        wl = inputs.lognormal(n=256, seed=seed)
        z = np.log(wl.sigma_s).reshape(256, 256)
        assert abs(z.mean()) < 1e-12 and abs(z.std() - 2.0) < 1e-12
        assert np.allclose(wl.sigma_t - wl.sigma_s, 0.05, rtol=0, atol=1e-9 * wl.sigma_s.max())
        for lag in corr:
            c = 0.5 * (np.mean(z[:, :-lag] * z[:, lag:]) + np.mean(z[:-lag, :] * z[lag:, :]))
            corr[lag].append(c / z.var())
    assert abs(np.mean(corr[13]) - np.exp(-0.125)) < 0.06
    assert abs(np.mean(corr[26]) - np.exp(-0.5)) < 0.12
    assert np.mean(corr[51]) < 0.3
    wl = inputs.lognormal(n=64)
    assert (wl.nv, wl.c_dt, wl.steps, wl.meta["seed"]) == (128, 0.002, 500, 3)
    assert np.unravel_index(np.argmax(wl.rho0), (64, 64)) in {(31, 31), (31, 32), (32, 31), (32, 32)}
    assert not wl.source.any()


def test_lognormal_is_reproducible_and_seeded():
    a, b = inputs.lognormal(n=32, seed=5), inputs.lognormal(n=32, seed=5)
    c = inputs.lognormal(n=32, seed=6)
    assert np.array_equal(a.sigma_s, b.sigma_s) and not np.array_equal(a.sigma_s, c.sigma_s)


def test_batched_draws():
    wls = inputs.batched()
    assert len(wls) == 64
    sides = [w.nx for w in wls]
    assert min(sides) >= 128 and max(sides) <= 512 and all(w.nx == w.ny for w in wls)
    assert {w.nv for w in wls} == {64, 128}
    assert all(0.5 <= w.meta["std"] <= 3.0 for w in wls)
    for w in wls:
        assert (w.c_dt, w.steps) == (0.005, 100)
        z = np.log(w.sigma_s)
        assert abs(z.std() - w.meta["std"]) < 1e-9
        iy, ix = np.unravel_index(np.argmax(w.rho0), (w.ny, w.nx))
        assert 0.2 - 1.0 / w.nx <= (ix + 0.5) / w.nx <= 0.8 + 1.0 / w.nx
        assert 0.2 - 1.0 / w.ny <= (iy + 0.5) / w.ny <= 0.8 + 1.0 / w.ny
    # the draws do not depend on the test-size scale
    small = inputs.batched(scale=0.1)
    assert [w.meta["std"] for w in small] == [w.meta["std"] for w in wls]
    assert [w.nv for w in small] == [w.nv for w in wls]


def test_diffusive_disc():
    wl = inputs.diffusive_disc(n=512)
    assert (wl.nv, wl.c_dt, wl.steps) == (256, 0.001, 300)
    inside = wl.sigma_s == 1000.0
    assert set(np.unique(wl.sigma_s)) == {1.0, 1000.0}
    assert abs(inside.mean() - np.pi * 0.3 ** 2) < 2e-3       # area of the disc of radius 0.3
    assert np.allclose(wl.sigma_t - wl.sigma_s, 0.01, rtol=0, atol=1e-12)
    assert inside.reshape(512, 512)[256, 256] and not inside.reshape(512, 512)[0, 0]


@pytest.mark.parametrize("name", sorted(inputs.BY_NAME))
def test_every_workload_is_consistent(name):
    wl = inputs.BY_NAME[name]() if name not in ("lognormal", "diffusive_disc") else \
        inputs.BY_NAME[name](n=32)
    n = wl.ncell
    for a in (wl.sigma_t, wl.sigma_s, wl.rho0):
        assert a.shape == (n,) and np.all(np.isfinite(a))
    assert wl.source.shape == (n,) and np.all(wl.source >= 0)
    assert np.all(wl.sigma_s >= 0) and np.all(wl.sigma_t >= wl.sigma_s)
    assert wl.c_dt > 0 and wl.steps > 0
