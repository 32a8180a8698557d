"""Checkpoint and resume (rte_save / rte_load) through the C ABI.  A march continued from a
loaded checkpoint repeats the uninterrupted march bit for bit, in every precision and with
the ROMs mid-construction; blobs of another problem, truncated or altered blobs are refused
and leave the handle unchanged."""
import numpy as np
import pytest

from paper_2603_19647_gb300 import inputs, rte

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("name,precision,levels", [("checkerboard", rte.RTE_FP64, 1),
                                                   ("checkerboard", rte.RTE_FP32, 1),
                                                   ("checkerboard", rte.RTE_FP32_BF16F, 1),
                                                   ("checkerboard", rte.RTE_FP64, 2),
                                                   ("slab", rte.RTE_FP64, 1),
                                                   ("slab", rte.RTE_FP32, 1)])
def test_resume_is_bit_identical(name, precision, levels):
    wl = inputs.checkerboard(n=32) if name == "checkerboard" else inputs.slab_1d(n=64)
    wl.inflow = np.array([0.2, 0.0, 0.1, 0.0])
    opts = rte.default_options(precision=precision, pc_levels=levels)
    a = rte.create_from_workload(wl, options=opts)
    a.rte_step(20)
    blob = a.rte_save()
    a.rte_step(15)
    b = rte.create_from_workload(wl, options=opts)
    b.rte_step(3)   # another state, replaced by the load
    b.rte_load(blob)
    b.rte_step(15)
    sa, sb = a.rte_get_stats(), b.rte_get_stats()
    assert np.array_equal(a.rte_get_scalar_flux(), b.rte_get_scalar_flux())
    assert np.array_equal(a.rte_get_angular_flux(), b.rte_get_angular_flux())
    for k in ("steps", "phase", "total_iterations", "total_sweeps", "ig_rank", "pc_rank",
              "pc_level_rank"):
        assert sa[k] == sb[k], k
    a.destroy()
    b.destroy()


def test_load_refuses_foreign_or_damaged_blobs():
    wl = inputs.checkerboard(n=32)
    a = rte.create_from_workload(wl)
    a.rte_step(5)
    blob = a.rte_save()
    a.rte_step(2)
    rho = a.rte_get_scalar_flux()
    other_dt = inputs.checkerboard(n=32)
    other_dt.c_dt *= 2
    other_sigma = inputs.checkerboard(n=32)
    other_sigma.sigma_s = other_sigma.sigma_s.copy()
    other_sigma.sigma_s[7] *= 0.5
    others = [rte.create_from_workload(inputs.checkerboard(n=16)),
              rte.create_from_workload(wl, options=rte.default_options(precision=rte.RTE_FP32)),
              rte.create_from_workload(wl, options=rte.default_options(r_max=20)),
              rte.create_from_workload(other_dt), rte.create_from_workload(other_sigma),
              rte.create_from_workload(wl, options=rte.default_options(pc_levels=2))]
    for o in others:
        with pytest.raises(rte.RteError) as e:
            o.rte_load(blob)
        assert e.value.status == rte.RTE_EINVAL
        o.destroy()
    for bad in (blob[:-8], blob[:100], b"x" * len(blob), blob + b"\0" * 8):
        with pytest.raises(rte.RteError) as e:
            a.rte_load(bad)
        assert e.value.status == rte.RTE_EINVAL
        assert np.array_equal(a.rte_get_scalar_flux(), rho)
    a.rte_load(blob)
    assert a.rte_get_stats()["steps"] == 5
    a.destroy()
    m = rte.create_from_workload(wl, options=rte.default_options(rom=rte.RTE_ROM_MANUAL))
    m.rte_step(1)
    with pytest.raises(rte.RteError) as e:
        m.rte_save()
    assert e.value.status == rte.RTE_ESTATE
    m.rte_rom_update()
    assert len(m.rte_save()) > 0
    m.destroy()
