"""CPU checks of the C-ABI library: it builds, loads, exports every entry point declared in
include/rte.h, and rejects invalid problems with RTE_EINVAL before touching the GPU."""
import ctypes
import os
import re

import numpy as np
import pytest

from conftest import ROOT
from paper_2603_19647_gb300 import build as gbuild
from paper_2603_19647_gb300 import rte


@pytest.fixture(scope="module")
def lib():
    gbuild.build()
    return rte.load()


def _declared():
    names = []
    inc = os.path.join(ROOT, "include")
    for fn in sorted(os.listdir(inc)):
        if fn.endswith(".h"):
            src = open(os.path.join(inc, fn)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names += re.findall(r"\b(rte_\w+)\s*\(", src)
    return sorted(set(names))


def test_every_declared_symbol_is_exported(lib):
    names = _declared()
    assert len(names) >= 19
    for n in names:
        assert hasattr(lib, n), n
    assert set(names) <= set(rte._SIGS)


def test_default_options(lib):
    o = rte.default_options()
    assert (o.eps_sisa, o.eps_ig, o.eps_pc, o.eps_up) == (1e-8, 1e-6, 1e-6, 1e-6)
    assert (o.max_iter, o.r_max, o.cg_rtol, o.cg_max_iter) == (500, 40, 1e-6, 500)
    assert o.pc_levels == 1 and rte.MAX_PC_LEVELS == 4
    assert o.sa_kind == rte.RTE_SA_DSA and o.mh_window == 4
    assert o.degree == 0 and o.dsa_fp64 == 0 and o.graph == 0 and o.dsa_cluster == 0


def _create(**kw):
    args = dict(mesh=rte.Mesh(2, 4, 4, 0, 1, 0, 1), quad=rte.quadrature_from(("cl_hemi", 8, 4)),
                sigma_t=np.ones(16), sigma_s=np.full(16, 0.5), source=np.zeros(16), c_dt=0.1)
    args.update(kw)
    return rte.rte_create(**args)


@pytest.mark.parametrize("bad", [
    dict(sigma_s=np.full(16, 2.0)),                       # sigma_t < sigma_s
    dict(sigma_s=np.full(16, -0.1)),                      # sigma_s < 0
    dict(sigma_t=np.r_[np.ones(15), np.nan]),             # non-finite
    dict(c_dt=0.0),
    dict(c_dt=-1.0),
    dict(mesh=rte.Mesh(3, 4, 4, 0, 1, 0, 1)),
    dict(mesh=rte.Mesh(2, 4, 4, 1, 0, 0, 1)),             # empty domain
    dict(quad=rte.quadrature_from(("cl_hemi", 6, 4))),    # n_phi not a multiple of 4
    dict(quad=rte.quadrature_from(mu=[0.5, -0.5], eta=[0.5, 0.5], w=[0.5, 0.6])),  # sum w != 1
    dict(quad=rte.quadrature_from(mu=[0.5, -0.5, 0.5, -0.5], eta=[0.5, 0.5, -0.5, 0.0],
                                  w=[0.25] * 4)),         # a direction on an axis
    dict(options=rte.default_options(r_max=65)),
    dict(options=rte.default_options(precision=7)),
    dict(options=rte.default_options(pc_levels=5)),
    dict(options=rte.default_options(sa_kind=2)),
    dict(options=rte.default_options(mh_window=1)),
    dict(options=rte.default_options(mh_window=17)),
    dict(options=rte.default_options(graph=3)),
    dict(options=rte.default_options(dsa_cluster=2)),
    dict(options=rte.default_options(time_scheme=2)),
    dict(options=rte.default_options(time_scheme=rte.RTE_BDF2, precision=rte.RTE_FP32_BF16F)),
    dict(options=rte.default_options(pc_levels=-1)),
    dict(options=rte.default_options(degree=2)),
    dict(options=rte.default_options(sweep_lanes=2, precision=rte.RTE_FP32)),  # FP64 / Q1 only
    dict(options=rte.default_options(sweep_lanes=4, precision=rte.RTE_FP32_BF16F)),
    dict(options=rte.default_options(degree=1, precision=rte.RTE_FP32_BF16F)),
    dict(options=rte.default_options(degree=1), source=np.r_[np.zeros(63), np.inf]),
])
def test_invalid_problems_rejected(lib, bad):
    with pytest.raises(rte.RteError) as ei:
        _create(**bad)
    assert ei.value.status == rte.RTE_EINVAL
    assert len(str(ei.value)) > 12


def test_batch_create_rejects_bad_instance(lib):
    """Validation of every instance happens before any device work; the message names the
    failing instance."""
    from paper_2603_19647_gb300 import inputs
    wls = inputs.batched(count=3, seed=4, scale=0.05)
    wls[1].sigma_s = wls[1].sigma_t + 1.0      # sigma_s > sigma_t
    with pytest.raises(rte.RteError) as ei:
        rte.rte_batch_create(wls)
    assert ei.value.status == rte.RTE_EINVAL
    assert "instance 1" in str(ei.value)


def test_bf16_storage_is_2d_only(lib):
    from paper_2603_19647_gb300 import inputs
    wl = inputs.slab_1d(n=16)
    with pytest.raises(rte.RteError) as ei:
        rte.create_from_workload(wl, options=rte.default_options(precision=rte.RTE_FP32_BF16F))
    assert ei.value.status == rte.RTE_EINVAL


def test_q1_is_2d_only(lib):
    from paper_2603_19647_gb300 import inputs
    wl = inputs.slab_1d(n=16)
    with pytest.raises(rte.RteError) as ei:
        rte.create_from_workload(wl, options=rte.default_options(degree=1))
    assert ei.value.status == rte.RTE_EINVAL


@pytest.mark.parametrize("desc", [("gl", 2), ("gl", 16), ("gl", 32), ("cl_hemi", 32, 8),
                                  ("cl_hemi", 16, 8), ("cl_hemi", 32, 16), ("cl_hemi", 4, 2)])
def test_quadrature_rule_matches_oracle(lib, desc):
    """The library's host-side angular rules (Gauss-Legendre in 1D, the CL hemisphere rule of
    App. A in 2D) against the oracle's own, direction by direction (same order)."""
    from conftest import oracle_quadrature
    dim = 1 if desc[0] == "gl" else 2
    mu, eta, w = rte.rte_quadrature_rule(rte.quadrature_from(desc), dim)
    omu, oeta, ow = oracle_quadrature(desc)
    assert mu.size == omu.size
    for d in range(mu.size):
        k = int(np.argmin((omu - mu[d]) ** 2 + (oeta - eta[d]) ** 2))
        assert abs(mu[d] - omu[k]) < 1e-14 and abs(eta[d] - oeta[k]) < 1e-14
        assert abs(w[d] - ow[k]) < 1e-15
    assert abs(w.sum() - 1.0) < 1e-13


@pytest.mark.parametrize("desc,dim", [(("gl", 16), 2), (("cl_hemi", 32, 8), 1), (("gl", 3), 1),
                                      (("cl_hemi", 6, 4), 2), (("cl_hemi", 32, 8), 3)])
def test_quadrature_rule_rejects_bad_descriptions(lib, desc, dim):
    with pytest.raises(rte.RteError) as ei:
        rte.rte_quadrature_rule(rte.quadrature_from(desc), dim)
    assert ei.value.status == rte.RTE_EINVAL
    assert len(str(ei.value)) > 12


def test_march_cli_help():
    """The command-line march parses its options before touching the GPU."""
    import subprocess
    import sys
    r = subprocess.run([sys.executable, "-m", "paper_2603_19647_gb300.march", "--help"],
                       cwd=ROOT, capture_output=True, text=True)
    assert r.returncode == 0 and "--precision" in r.stdout


def test_struct_layouts_match_the_header(tmp_path):
    """The binding's ctypes structs have the C header's size and field offsets (a field added
    to the header but not to the binding, or in another order, would shift every field after
    it without any error)."""
    import shutil
    import subprocess
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    structs = {"rte_mesh": rte.Mesh, "rte_quadrature": rte.Quadrature, "rte_problem": rte.Problem,
               "rte_options": rte.Options, "rte_stats": rte.Stats}
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "rte.h"', "int main(void) {"]
    for cname, py in structs.items():
        lines.append(f'  printf("{cname} size %zu\\n", sizeof({cname}));')
        for field, _ in py._fields_:
            lines.append(f'  printf("{cname} {field} %zu\\n", offsetof({cname}, {field}));')
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    inc = os.path.join(ROOT, "include")
    subprocess.run([cc, "-std=c99", "-I", inc, str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    got = {}
    for line in out:
        if line:
            name, field, value = line.split()
            got[(name, field)] = int(value)
    for cname, py in structs.items():
        assert got[(cname, "size")] == ctypes.sizeof(py), cname
        for field, _ in py._fields_:
            assert got[(cname, field)] == getattr(py, field).offset, (cname, field)
