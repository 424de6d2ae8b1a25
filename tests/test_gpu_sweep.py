"""The p- and d-benchmark meshes of §4 (structured Q_p quads, p <= 8; Q1
with d <= 8 and d = 20), at full size, through every assembly mode and both
formats: the GPU pattern against the sizes the paper prints and the oracle's
arrays, the values against the oracle's sequential assembly (Listing 2)."""

import numpy as np
import pytest

import oracle
import workloads as wl
from tests import gpu_util as gu
from tests.golden import load

pytestmark = pytest.mark.gpu

PRINTED = {(r["m"], r["p"], r["d"]): r for r in load.structured_patterns()}
POINTS = wl.paper_sweep_points()


@pytest.fixture(scope="module")
def ctx():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2012_00585_gb300 import feasm
    c = feasm.fe_create(0)
    yield c
    feasm.fe_destroy(c)


@pytest.mark.parametrize("bench,m,p,d", POINTS, ids=[f"{b}-m{m}-p{p}-d{d}" for b, m, p, d in POINTS])
def test_sweep_point(ctx, bench, m, p, d):
    from paper_2012_00585_gb300 import feasm
    D, n_dofs = wl.quad_qp_grid(m, p, d)
    n_e = D.shape[0]
    g = gu.GpuAssembly(ctx, D, n_dofs)
    rp_o, ci_o = oracle.csr_pattern(D, n_dofs)
    rp, ci = g.csr_host()
    assert np.array_equal(rp, rp_o) and np.array_equal(ci, ci_o)
    if (m, p, d) in PRINTED:  # the paper's printed sizes
        assert n_dofs == PRINTED[(m, p, d)]["n_dofs"]
        assert rp[-1] == PRINTED[(m, p, d)]["nnz"]
    crp, ca = g.crac_host()
    crp_o, ca_o = oracle.crac_from_csr(rp_o, ci_o, n_dofs)
    assert np.array_equal(crp, crp_o) and np.array_equal(ca, ca_o)

    K = wl.random_matrices(n_e, D.shape[1], seed=m + 10 * p + 100 * d)
    exp = oracle.assemble_csr(D, K, rp_o, ci_o)
    tau = gu.row_tolerance(rp_o, exp, gu.contribution_abs_row_sums(D, K, n_dofs))
    for fmt in ("csr", "crac"):
        got = g.assemble(K, fmt, feasm.FE_DETERMINISTIC).cpu().numpy()
        assert np.array_equal(got.view(np.uint64), exp.view(np.uint64)), fmt
        for mode in (feasm.FE_ATOMIC, feasm.FE_ROWLOCK):
            got = g.assemble(K, fmt, mode).cpu().numpy()
            gu.assert_within_row_tol(rp_o, got, exp, tau)
    assert feasm.fe_device_status(ctx) == 0
    # lock words restored by the row-locked runs
    rp2, _ = g.csr_host()
    crp2, _ = g.crac_host()
    assert np.array_equal(rp2, rp_o) and np.array_equal(crp2, crp_o)
    # colour order: structured quads take 4 colours, and the coloured sum is
    # the sequential sum in colour order
    nc = feasm.fe_pattern_colour(ctx, g.pattern.handle)
    assert nc == 4
    _, colour = oracle.greedy_colouring(D, n_dofs)
    order = np.lexsort((np.arange(n_e), colour))
    exp_c = oracle.assemble_csr(D, K, rp_o, ci_o, order=order)
    for fmt in ("csr", "crac"):
        got = g.assemble(K, fmt, feasm.FE_COLOURED).cpu().numpy()
        assert np.array_equal(got.view(np.uint64), exp_c.view(np.uint64)), fmt
    g.free()
