"""GPU parity of each hot-path kernel against the oracle, through the C ABI.

FP64 mode: every kernel reproduces the oracle up to rounding; the bound used is a
relative L2 error of 1e-12 for single applications (sweeps, moments) and 1e-10 where
an iterative solve or an SVD sits in between (the FP64 parity bound of the method)."""
import numpy as np
import pytest

from conftest import oracle_problem, oracle_quadrature
from gpu_util import make_pair, match_directions, rel_l2
from oracle import dsa, rom
from oracle import transport as tr
from paper_2603_19647_gb300 import inputs, rte

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("desc", [("gl", 16), ("gl", 4), ("cl_hemi", 32, 8), ("cl_hemi", 32, 16),
                                  ("cl_hemi", 16, 8), ("cl_hemi", 8, 4)])
def test_quadrature_matches_oracle(desc):
    wl = inputs.slab_1d(n=8) if desc[0] == "gl" else inputs.checkerboard(n=8)
    wl.quadrature = desc
    h = rte.create_from_workload(wl)
    perm, (mu, eta, w), (omu, oeta, ow) = match_directions(h, desc)
    assert np.max(np.abs(mu - omu[perm])) < 1e-14
    assert np.max(np.abs(eta - oeta[perm])) < 1e-14
    assert np.max(np.abs(w - ow[perm])) < 1e-15
    h.destroy()


def _hetero_2d(nx, ny, quad, seed):
    rng = np.random.default_rng(seed)
    wl = inputs.checkerboard(n=8, quad=quad)
    wl.nx, wl.ny = nx, ny
    n = nx * ny
    ss = rng.uniform(0, 50, n)
    wl.sigma_s, wl.sigma_t = ss, ss + rng.uniform(0.05, 2, n)
    wl.source = rng.uniform(0, 1, n)
    wl.rho0 = rng.uniform(0, 1, n)
    wl.domain = (0.0, 1.3, 0.0, 0.7)
    return wl, rng


@pytest.mark.parametrize("quad", [(32, 8), (16, 8), (8, 4), (32, 16)])
@pytest.mark.parametrize("shape", [(37, 29), (1, 1), (5, 64), (64, 3), (129, 70)])
def test_sweep_2d(quad, shape):
    wl, rng = _hetero_2d(*shape, quad, seed=shape[0] * 7 + quad[1])
    h, p = make_pair(wl)
    for _ in range(2):   # twice: the control block resets itself between launches
        rho = rng.uniform(-1, 1, wl.ncell)
        got = h.rte_op_sweep(rho)
        ref = tr.apply_T_sigma_s(p, rho)
        assert rel_l2(got, ref) < 1e-12
    h.destroy()


@pytest.mark.parametrize("lanes,rows,warps", [(32, 1, 1), (32, 2, 4), (32, 8, 8), (16, 4, 3),
                                               (8, 2, 8), (8, 8, 2), (16, 1, 5), (4, 1, 8),
                                               (4, 4, 3), (2, 1, 8), (2, 2, 5)])
@pytest.mark.parametrize("mode", ["si", "f"])
def test_sweep_2d_tilings(lanes, rows, warps, mode):
    """Every tile shape (directions per lane group, rows per lane group, warps per CTA) gives
    the same SI sweep and fused f sweep, on a ragged grid."""
    wl, rng = _hetero_2d(45, 53, (32, 8), seed=lanes + rows + warps)
    h, p = make_pair(wl, sweep_lanes=lanes, sweep_rows=rows, sweep_warps=warps)
    if mode == "si":
        rho = rng.uniform(-1, 1, wl.ncell)
        assert rel_l2(h.rte_op_sweep(rho), tr.apply_T_sigma_s(p, rho)) < 1e-12
    else:
        perm, _, _ = match_directions(h, wl.quadrature)
        f0 = rng.uniform(0, 1, (p.nv, wl.ncell))
        h.rte_set_initial(f0=f0[perm])
        g = np.array([0.3, 0.6, 0.2, 0.9])
        h.rte_set_inflow(g)
        p.inflow = g
        rho = rng.uniform(0, 1, wl.ncell)
        bt = h.rte_op_fsweep(rho)
        f_ref, _ = tr.final_f(p, rho, f0)
        assert rel_l2(h.rte_get_angular_flux(), f_ref[perm]) < 1e-12
        assert rel_l2(bt, tr.b_tilde(p, f_ref)) < 1e-12
    h.destroy()


@pytest.mark.parametrize("lanes,th,warps", [(8, 4, 1), (8, 8, 2), (16, 4, 3), (32, 4, 4),
                                             (32, 8, 2), (8, 4, 5), (16, 8, 1)])
@pytest.mark.parametrize("shape", [(45, 53), (8, 9), (3, 130)])
def test_sweep_2d_tile_kernel(lanes, th, warps, shape):
    """The tile-sequence kernel in FP64 (each lane solves whole 8 x TH tiles, the diagonal
    from the staged inverse table): SI sweep twice, fused f sweep with inflow and b~, on
    ragged grids (partial tiles in both directions)."""
    wl, rng = _hetero_2d(*shape, (32, 8), seed=lanes * th + warps + shape[1])
    h, p = make_pair(wl, sweep_kernel=2, sweep_lanes=lanes, sweep_rows=th, sweep_warps=warps)
    st = h.rte_get_stats()
    assert st["sweep_si_kernel"] == 2 and st["sweep_f_kernel"] == 2
    for _ in range(2):
        rho = rng.uniform(-1, 1, wl.ncell)
        assert rel_l2(h.rte_op_sweep(rho), tr.apply_T_sigma_s(p, rho)) < 1e-12
    perm, _, _ = match_directions(h, wl.quadrature)
    f0 = rng.uniform(0, 1, (p.nv, wl.ncell))
    h.rte_set_initial(f0=f0[perm])
    g = np.array([0.3, 0.6, 0.2, 0.9])
    h.rte_set_inflow(g)
    p.inflow = g
    rho = rng.uniform(0, 1, wl.ncell)
    bt = h.rte_op_fsweep(rho)
    f_ref, _ = tr.final_f(p, rho, f0)
    assert rel_l2(h.rte_get_angular_flux(), f_ref[perm]) < 1e-12
    assert rel_l2(bt, tr.b_tilde(p, f_ref)) < 1e-12
    h.destroy()


@pytest.mark.parametrize("n,nd", [(1, 16), (7, 4), (256, 16), (1000, 8), (4097, 16)])
def test_sweep_1d(n, nd):
    rng = np.random.default_rng(n)
    wl = inputs.slab_1d(n=n, n_dirs=nd)
    ss = rng.uniform(0, 20, n)
    wl.sigma_s, wl.sigma_t = ss, ss + rng.uniform(0.01, 1, n)
    h, p = make_pair(wl)
    rho = rng.uniform(-1, 1, n)
    assert rel_l2(h.rte_op_sweep(rho), tr.apply_T_sigma_s(p, rho)) < 1e-12
    h.destroy()


@pytest.mark.parametrize("case", ["2d", "1d"])
def test_fused_f_sweep(case):
    """f^n = L^-1(Sigma_s rho + tau f^{n-1} + G + g^bc) and b~^n from f^n, with inflow."""
    if case == "2d":
        wl, rng = _hetero_2d(33, 21, (16, 8), seed=3)
        g = np.array([0.7, 0.2, 0.4, 1.1])
    else:
        rng = np.random.default_rng(5)
        wl = inputs.slab_1d(n=300)
        wl.source = rng.uniform(0, 1, 300)
        g = np.array([0.7, 0.2, 0.0, 0.0])
    h, p = make_pair(wl)
    perm, _, _ = match_directions(h, wl.quadrature)
    f0_oracle = rng.uniform(0, 1, (p.nv, wl.ncell))
    h.rte_set_initial(f0=f0_oracle[perm])
    h.rte_set_inflow(g)
    p.inflow = g
    rho = rng.uniform(0, 1, wl.ncell)
    bt = h.rte_op_fsweep(rho)
    f_lib = h.rte_get_angular_flux()
    f_ref, _ = tr.final_f(p, rho, f0_oracle)
    assert rel_l2(f_lib, f_ref[perm]) < 1e-12
    assert rel_l2(bt, tr.b_tilde(p, f_ref)) < 1e-12
    h.destroy()


@pytest.mark.parametrize("rtol", [1e-6, 1e-10])
@pytest.mark.parametrize("name", ["checkerboard", "slab", "large"])
def test_dsa_cg(name, rtol):
    """Both CG arrangements: grids up to 2^18 cells take the one-barrier kernel, larger ones
    (here 520^2) the two-phase kernel."""
    wl = (inputs.checkerboard(n=40) if name == "checkerboard"
          else inputs.checkerboard(n=520) if name == "large" else inputs.slab_1d(n=256))
    h, p = make_pair(wl, cg_rtol=rtol)
    rng = np.random.default_rng(9)
    res = rng.uniform(-1, 1, wl.ncell)
    got, its = h.rte_op_dsa(res)
    ref, its_ref = dsa.dsa_correction(p, dsa.dsa_matrix(p), res, rtol, 500)
    assert its == its_ref
    assert rel_l2(got, ref) < 1e-10
    h.destroy()


@pytest.mark.parametrize("precision", [rte.RTE_FP64, rte.RTE_FP32])
@pytest.mark.parametrize("rtol", [1e-6, 1e-10])
@pytest.mark.parametrize("name", ["checkerboard", "slab", "ragged", "batch_max"])
def test_dsa_cg_in_one_cluster(name, rtol, precision):
    """options.dsa_cluster: the same CG solve in one thread-block cluster, against the
    oracle's CG on grids from a 1D slab to the largest batched instance (512^2 cells); FP32
    with dsa_fp64 = 1, as batched instances take it."""
    wl = (inputs.checkerboard(n=40) if name == "checkerboard"
          else inputs.slab_1d(n=256) if name == "slab"
          else inputs.checkerboard(n=512) if name == "batch_max" else inputs.checkerboard(n=37))
    h, p = make_pair(wl, cg_rtol=rtol, dsa_cluster=1, precision=precision, dsa_fp64=1, tune=0)
    rng = np.random.default_rng(9)
    res = rng.uniform(-1, 1, wl.ncell)
    got, its = h.rte_op_dsa(res)
    ref, its_ref = dsa.dsa_correction(p, dsa.dsa_matrix(p), res, rtol, 500)
    assert its == its_ref
    assert rel_l2(got, ref) < 1e-10
    got2, its2 = h.rte_op_dsa(res)   # a second solve on the same buffers: the same bits
    assert its2 == its and np.array_equal(got2, got)
    h.destroy()


def test_rom_incremental_svd_and_apply():
    wl = inputs.checkerboard(n=24)
    h, p = make_pair(wl, r_max=12)
    n = wl.ncell
    rng = np.random.default_rng(11)
    X, Y = np.meshgrid(np.linspace(0, 1, 24), np.linspace(0, 1, 24))
    o = rom.IncrementalSVD(n, 12)
    for k in range(20):
        x = (np.exp(-((X - 0.2 - 0.03 * k) ** 2 + (Y - 0.5) ** 2) / 0.02) * (1 + 0.05 * k)).ravel()
        x = x + 1e-4 * rng.standard_normal(n)
        b = x + 0.1 * np.roll(x, 3) + 1e-3 * rng.standard_normal(n)
        te = 1e-4 if k >= 14 else -1.0
        grew = h.rte_op_rom_append(rte.RTE_ROM_IG, x, b, te)
        grew_o = o.append(x, b, trunc_eps=(te if te >= 0 else None))
        assert grew == grew_o
        S, U, Ar = h.rte_op_rom_get(rte.RTE_ROM_IG)
        assert S.size == o.rank
        assert np.max(np.abs(S - o.S) / o.S) < 1e-10
        sg = np.sign(np.sum(U * o.U.T, axis=1))
        assert np.max(np.abs(U * sg[:, None] - o.U.T)) < 1e-8
        Ao = o.operator() * sg[:, None] * sg[None, :]
        assert np.max(np.abs(Ar - Ao)) < 1e-9 * np.max(np.abs(Ao))
        rhs = b + 0.01 * rng.standard_normal(n)
        assert rel_l2(h.rte_op_rom_apply(rte.RTE_ROM_IG, rhs), o.solve_apply(rhs)) < 1e-9
    h.destroy()


def test_infinite_medium_on_gpu():
    """Closed form: uniform medium, uniform isotropic start, inflow g^n = rho0 (1 + c dt sigma_a)^-n."""
    wl = inputs.checkerboard(n=20, quad=(16, 8))
    n = wl.ncell
    st, ss, c_dt, rho0 = 2.0, 1.5, 0.3, 1.7
    wl.sigma_t, wl.sigma_s, wl.source = np.full(n, st), np.full(n, ss), np.zeros(n)
    wl.c_dt, wl.rho0 = c_dt, np.full(n, rho0)
    h = rte.create_from_workload(wl, options=rte.default_options(eps_sisa=1e-14, cg_rtol=1e-12,
                                                                  rom=rte.RTE_ROM_OFF))
    for k in range(1, 8):
        gk = rho0 * (1 + c_dt * (st - ss)) ** (-k)
        h.rte_set_inflow([gk] * 4)
        h.rte_step(1)
        assert np.max(np.abs(h.rte_get_scalar_flux() - gk)) < 1e-12 * gk
    h.destroy()


def test_enoconv_and_manual_rom_states():
    wl = inputs.checkerboard(n=16, quad=(8, 4))
    h = rte.create_from_workload(wl, options=rte.default_options(max_iter=1, eps_sisa=1e-14))
    with pytest.raises(rte.RteError) as ei:
        h.rte_step(1)
    assert ei.value.status == rte.RTE_ENOCONV
    assert np.all(np.isfinite(h.rte_get_scalar_flux()))
    h.destroy()
    h = rte.create_from_workload(wl, options=rte.default_options(rom=rte.RTE_ROM_MANUAL))
    with pytest.raises(rte.RteError) as ei:
        h.rte_rom_update()
    assert ei.value.status == rte.RTE_ESTATE
    h.rte_step(1)
    with pytest.raises(rte.RteError):
        h.rte_step(1)
    h.rte_rom_update()
    h.rte_step(1)
    assert h.rte_get_stats()["ig_rank"] >= 1
    h.destroy()

def test_caller_stream():
    """rte_set_stream puts the handle's work on the caller's stream (here a torch stream) and
    NULL returns it to its own: the march is the same bit for bit either way."""
    torch = pytest.importorskip("torch")
    wl = inputs.checkerboard(n=32)
    res = []
    for use_stream in (False, True, True):
        h = rte.create_from_workload(wl)
        s = torch.cuda.Stream() if use_stream else None
        if s is not None:
            h.rte_set_stream(s.cuda_stream)
        h.rte_step(10)
        if s is not None:
            h.rte_set_stream(None)
        h.rte_step(5)
        res.append(h.rte_get_scalar_flux())
        h.destroy()
    assert np.array_equal(res[0], res[1]) and np.array_equal(res[0], res[2])


def test_rom_at_maximum_rank():
    """r_max = 64, the largest rank the library takes: 90 appends in general position, so the
    core SVD reaches its largest size (65 x 65), the rank cap drops the smallest triple in
    each of the last 26, and the factored bases are multiplied out once they hold 24 columns
    beyond the rank (append 88); singular values, the reduced operator and the apply against
    the oracle's iSVD."""
    wl = inputs.checkerboard(n=64, quad=(8, 4))
    h, p = make_pair(wl, r_max=64)
    n = wl.ncell
    rng = np.random.default_rng(17)
    o = rom.IncrementalSVD(n, 64)
    for k in range(90):
        x = rng.standard_normal(n)
        b = x + 0.1 * np.roll(x, 5) + 0.01 * rng.standard_normal(n)
        assert h.rte_op_rom_append(rte.RTE_ROM_PC, x, b, -1.0) == o.append(x, b), k
    S, U, Ar = h.rte_op_rom_get(rte.RTE_ROM_PC)
    assert S.size == o.rank == 64
    assert np.max(np.abs(S - o.S) / o.S) < 1e-10
    sg = np.sign(np.sum(U * o.U.T, axis=1))
    Ao = o.operator() * sg[:, None] * sg[None, :]
    assert np.max(np.abs(Ar - Ao)) < 1e-9 * np.max(np.abs(Ao))
    rhs = rng.standard_normal(n)
    assert rel_l2(h.rte_op_rom_apply(rte.RTE_ROM_PC, rhs), o.solve_apply(rhs)) < 1e-9
    h.destroy()
