"""GPU test of rte_dsa_solve_noalloc, the DSA solve that allocates nothing.

It serves callers that cannot allocate device memory (code inside another framework's fixed,
pre-reserved memory budget, or latency-critical code that must not trigger the device-wide
synchronisation of cudaMalloc / cudaFree).  Its answer must equal that of rte_op_dsa, the
handle-based solve of the same diffusion correction, and that of the oracle's CG on its own
assembly of the operator, within the 1e-10 relative bound the DSA parity tests use, on two
calls in a row (the second one reuses the shared scratch array).  The mesh sizes include the
array's full capacity (256 x 256 cells), where any overlap of the scratch vectors would show.
The handle's solve on grids up to 2^18 cells takes the one-barrier CG arrangement, this one
the two-phase arrangement and the oracle a textbook CG, which all round differently, so the
iteration counts may differ by one; the solves run to a relative residual of 1e-12, where one
iteration more or less moves the answer by far less than the 1e-10 bound.
"""
import numpy as np
import pytest

from conftest import oracle_problem
from oracle import dsa
from paper_2603_19647_gb300 import inputs, rte

pytestmark = pytest.mark.gpu


def _rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


@pytest.mark.parametrize("case", ["2d", "1d", "2d_capacity"])
def test_noalloc_dsa_matches_handle_solve_and_oracle(case):
    torch = pytest.importorskip("torch")
    import __graft_entry__
    __graft_entry__.build()
    wl = {"2d": lambda: inputs.checkerboard(n=48), "1d": lambda: inputs.slab_1d(n=300),
          "2d_capacity": lambda: inputs.checkerboard(n=256)}[case]()
    dim = 1 if case == "1d" else 2
    rtol = 1e-12
    h = rte.create_from_workload(wl, options=rte.default_options(cg_rtol=rtol))
    p = oracle_problem(wl)
    A = dsa.dsa_matrix(p)
    dev = torch.device("cuda", torch.cuda.current_device())
    st = torch.tensor(wl.sigma_t, dtype=torch.float64, device=dev)
    ss = torch.tensor(wl.sigma_s, dtype=torch.float64, device=dev)
    stream = torch.cuda.current_stream().cuda_stream
    rng = np.random.default_rng(21)
    for _ in range(2):
        res = rng.uniform(-1, 1, wl.ncell)
        ref, its_ref = h.rte_op_dsa(res)
        orc, its_orc = dsa.dsa_correction(p, A, res, rtol, 500)
        r_dev = torch.tensor(res, dtype=torch.float64, device=dev)
        out = torch.full((wl.ncell,), float("nan"), dtype=torch.float64, device=dev)
        its = rte.rte_dsa_solve_noalloc(dim, wl.nx, wl.ny, *wl.domain, wl.c_dt, st.data_ptr(),
                                        ss.data_ptr(), r_dev.data_ptr(), rtol, 500, out.data_ptr(),
                                        stream)
        got = out.cpu().numpy()
        assert abs(its - its_ref) <= 1 and abs(its - its_orc) <= 1, (its, its_ref, its_orc)
        assert _rel(got, ref) <= 1e-10
        assert _rel(got, orc) <= 1e-10
    h.destroy()


def test_noalloc_rejects_too_many_cells():
    with pytest.raises(rte.RteError) as ei:
        rte.rte_dsa_solve_noalloc(2, 257, 256, 0, 1, 0, 1, 0.01, 1, 1, 1, 1e-6, 10, 1)
    assert ei.value.status == rte.RTE_EINVAL
    assert "65536" in str(ei.value)
