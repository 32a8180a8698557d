"""GPU test of rte_dsa_solve_noalloc, the DSA solve that allocates nothing.

It serves callers that cannot allocate device memory (code inside another framework's fixed,
pre-reserved memory budget, or latency-critical code that must not trigger the device-wide
synchronisation of cudaMalloc / cudaFree).  Its answer must equal that of rte_op_dsa, the
handle-based solve of the same diffusion correction, within the 1e-10 relative bound the DSA
parity tests use, on two calls in a row (the second one reuses the shared scratch array).
"""
import numpy as np
import pytest

from paper_2603_19647_gb300 import inputs, rte

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("case", ["2d", "1d"])
def test_noalloc_dsa_matches_handle_solve(case):
    torch = pytest.importorskip("torch")
    import __graft_entry__
    __graft_entry__.build()
    wl = inputs.checkerboard(n=48) if case == "2d" else inputs.slab_1d(n=300)
    dim = 2 if case == "2d" else 1
    rtol = 1e-8
    h = rte.create_from_workload(wl, options=rte.default_options(cg_rtol=rtol))
    dev = torch.device("cuda", torch.cuda.current_device())
    st = torch.tensor(wl.sigma_t, dtype=torch.float64, device=dev)
    ss = torch.tensor(wl.sigma_s, dtype=torch.float64, device=dev)
    stream = torch.cuda.current_stream().cuda_stream
    rng = np.random.default_rng(21)
    for _ in range(2):
        res = rng.uniform(-1, 1, wl.ncell)
        ref, its_ref = h.rte_op_dsa(res)
        r_dev = torch.tensor(res, dtype=torch.float64, device=dev)
        out = torch.full((wl.ncell,), float("nan"), dtype=torch.float64, device=dev)
        its = rte.rte_dsa_solve_noalloc(dim, wl.nx, wl.ny, *wl.domain, wl.c_dt, st.data_ptr(),
                                        ss.data_ptr(), r_dev.data_ptr(), rtol, 500, out.data_ptr(),
                                        stream)
        got = out.cpu().numpy()
        assert its == its_ref
        assert np.linalg.norm(got - ref) <= 1e-10 * np.linalg.norm(ref)
    h.destroy()


def test_noalloc_rejects_too_many_cells():
    with pytest.raises(rte.RteError) as ei:
        rte.rte_dsa_solve_noalloc(2, 257, 256, 0, 1, 0, 1, 0.01, 1, 1, 1, 1e-6, 10, 1)
    assert ei.value.status == rte.RTE_EINVAL
    assert "65536" in str(ei.value)
