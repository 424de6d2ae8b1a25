"""The consumers and alternative assemblies of the paper: SpMV through CSR
and through CRAC (the paper's outlook), and the spin_int row-locked assembly
(Listings 3-5), against the oracle."""

import numpy as np
import pytest

import oracle
import workloads as wl
from tests import gpu_util as gu

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2012_00585_gb300 import feasm
    c = feasm.fe_create(0)
    yield c
    feasm.fe_destroy(c)


def _scattered():
    """200 elements of 6 random DOFs out of 300: unused DOFs give empty rows."""
    rng = np.random.default_rng(5)
    D = np.stack([rng.choice(300, size=6, replace=False) for _ in range(200)]).astype(np.int32)
    assert len(np.unique(D)) < 300
    return D, 300


MESHES = [("hex5_d3", *wl.hex_q1_grid(5, 3)), ("tet3_d3", *wl.tet_p2_kuhn(3, d=3, seed=2)),
          ("quad9", *wl.quad_q1_grid(9, 1)), ("hex4_d1", *wl.hex_q1_grid(4, 1)), ("scattered", *_scattered())]


@pytest.mark.parametrize("lanes", [0, 2, 8, 16])
@pytest.mark.parametrize("name,D,n_dofs", MESHES, ids=[m[0] for m in MESHES])
def test_spmv_csr_and_crac(ctx, name, D, n_dofs, lanes):
    import torch
    from paper_2012_00585_gb300 import feasm
    feasm.fe_tune_set(ctx, feasm.FE_KNOB_SPMV_LANES, lanes)
    K = wl.random_matrices(D.shape[0], D.shape[1], seed=1)
    g = gu.GpuAssembly(ctx, D, n_dofs)
    v = g.assemble(K, "csr", feasm.FE_DETERMINISTIC)
    rp, ci = oracle.csr_pattern(D, n_dofs)
    x = np.random.default_rng(2).standard_normal(n_dofs)
    y_o = oracle.spmv_csr(rp, ci, v.cpu().numpy(), x)
    xd = torch.from_numpy(x).cuda()
    rows = np.repeat(np.arange(n_dofs), np.diff(rp))
    scale = np.zeros(n_dofs)
    np.add.at(scale, rows, np.abs(v.cpu().numpy() * x[ci]))
    for f in (feasm.fe_spmv_csr, feasm.fe_spmv_crac):
        y = torch.full((n_dofs,), float("nan"), dtype=torch.float64, device="cuda")
        f(ctx, g.pattern.handle, v, xd, y)
        torch.cuda.synchronize()
        got = y.cpu().numpy()
        assert np.all(np.abs(got - y_o) <= 1e-13 * scale + 1e-300), f.__name__
        y2 = torch.empty_like(y)
        f(ctx, g.pattern.handle, v, xd, y2)
        torch.cuda.synchronize()
        assert torch.equal(y, y2)  # reproducible run to run
    g.free()
    feasm.fe_tune_set(ctx, feasm.FE_KNOB_SPMV_LANES, 0)


@pytest.mark.parametrize("fmt", ["csr", "crac"])
@pytest.mark.parametrize("name,D,n_dofs", MESHES, ids=[m[0] for m in MESHES])
def test_rowlock_assembly(ctx, fmt, name, D, n_dofs):
    import torch
    from paper_2012_00585_gb300 import feasm
    g = gu.GpuAssembly(ctx, D, n_dofs)
    rp0, ci0 = g.csr_host()
    crp0, _ = g.crac_host()
    # paper's all-ones element: integer sums, exact in any order
    ones = wl.ones_matrices(D.shape[0], D.shape[1])
    rp, ci = oracle.csr_pattern(D, n_dofs)
    got = g.assemble(ones, fmt, feasm.FE_ROWLOCK).cpu().numpy()
    assert np.array_equal(got, oracle.assemble_csr(D, ones, rp, ci))
    K = wl.random_matrices(D.shape[0], D.shape[1], seed=4)
    got = g.assemble(K, fmt, feasm.FE_ROWLOCK).cpu().numpy()
    exp = oracle.assemble_csr(D, K, rp, ci)
    gu.assert_within_row_tol(rp, got, exp, gu.row_tolerance(rp, exp, gu.contribution_abs_row_sums(D, K, n_dofs)))
    assert feasm.fe_device_status(ctx) == 0
    # the lock words (row pointers) are back to their values
    rp1, _ = g.csr_host()
    crp1, _ = g.crac_host()
    assert np.array_equal(rp1, rp0) and np.array_equal(crp1, crp0)
    g.free()


@pytest.mark.parametrize("fmt", ["csr", "crac"])
def test_rowlock_timeout_is_reported(ctx, fmt):
    """Failure detection without a fault: one row's lock word is left held
    (its row pointer complemented, as a holder that never releases), the
    bounded spin runs out, the row is skipped and FE_ERR_TIMEOUT reaches the
    host through the device status word; the rest of the matrix is right and
    the context stays usable."""
    import torch
    from paper_2012_00585_gb300 import feasm
    D, n_dofs = wl.hex_q1_grid(3, 1)
    K = wl.random_matrices(D.shape[0], D.shape[1], seed=12)
    g = gu.GpuAssembly(ctx, D, n_dofs)
    rp, ci = oracle.csr_pattern(D, n_dofs)
    exp = oracle.assemble_csr(D, K, rp, ci)
    locks = (g.pattern.csr() if fmt == "csr" else g.pattern.crac())[0]
    held = 21  # an interior DOF of the 4x4x4-node grid
    saved = locks[held].item()
    feasm.fe_tune_set(ctx, feasm.FE_KNOB_LOCK_SPIN, 10)
    try:
        locks[held] = ~saved
        torch.cuda.synchronize()
        got = g.assemble(K, fmt, feasm.FE_ROWLOCK).cpu().numpy()
        assert feasm.fe_device_status(ctx) == feasm.FE_ERR_TIMEOUT
        locks[held] = saved
        torch.cuda.synchronize()
    finally:
        feasm.fe_tune_set(ctx, feasm.FE_KNOB_LOCK_SPIN, 0)
    row = np.repeat(np.arange(n_dofs), np.diff(rp))
    other = row != held
    tau = gu.row_tolerance(rp, exp, gu.contribution_abs_row_sums(D, K, n_dofs))
    assert np.all(np.abs(got[other] - exp[other]) <= tau[row[other]])
    assert np.all(got[~other] == 0.0)  # the held row received nothing
    # released: the same call is complete again and the status is clean
    got = g.assemble(K, fmt, feasm.FE_ROWLOCK).cpu().numpy()
    assert feasm.fe_device_status(ctx) == 0
    gu.assert_within_row_tol(rp, got, exp, tau)
    g.free()


def test_pattern_free_async_is_stream_ordered(ctx):
    """fe_pattern_free_async releases the arrays at the stream's current
    point: work queued before it on the stream still reads them."""
    import torch
    from paper_2012_00585_gb300 import feasm
    D, n_dofs = wl.hex_q1_grid(4, 3)
    K = wl.random_matrices(D.shape[0], D.shape[1], seed=21)
    rp, ci = oracle.csr_pattern(D, n_dofs)
    exp = oracle.assemble_csr(D, K, rp, ci)
    s = torch.cuda.Stream()
    Dd = torch.from_numpy(D).cuda()
    Kd = torch.from_numpy(K).cuda()
    for _ in range(3):
        p = feasm.fe_pattern_build(ctx, D.shape[0], D.shape[1], n_dofs, Dd, feasm.FE_PATTERN_ALL, s)
        v = torch.empty(feasm.fe_pattern_info_get(p)["nnz"], dtype=torch.float64, device="cuda")
        feasm.fe_assemble_csr(ctx, p, Kd, v, feasm.FE_DETERMINISTIC, 0, s)
        feasm.fe_pattern_free_async(p, s)
        s.synchronize()
        assert np.array_equal(v.cpu().numpy().view(np.uint64), exp.view(np.uint64))
    assert feasm.fe_device_status(ctx) == 0


def test_allocation_failure_is_reported():
    """Host-side fault injection: a context whose memory pool is bounded to
    8 MiB.  A mesh whose pattern needs more fails with FE_ERR_OOM; what the
    build had allocated is released, the context stays usable, and a small
    mesh still builds and assembles exactly."""
    import torch
    from paper_2012_00585_gb300 import feasm
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    c = feasm.fe_create_ex(0, 0, 8 << 20)
    try:
        D, n_dofs = wl.hex_q1_grid(24, 3)  # needs well over 8 MiB of pattern and workspace
        Dd = torch.from_numpy(D).cuda()
        for _ in range(2):
            with pytest.raises(feasm.FeError) as ei:
                feasm.fe_pattern_build(c, D.shape[0], D.shape[1], n_dofs, Dd, feasm.FE_PATTERN_ALL)
            assert ei.value.code == feasm.FE_ERR_OOM
        Ds, n_s = wl.hex_q1_grid(3, 3)
        K = wl.random_matrices(Ds.shape[0], Ds.shape[1], seed=31)
        p = feasm.fe_pattern_build(c, Ds.shape[0], Ds.shape[1], n_s, torch.from_numpy(Ds).cuda(), feasm.FE_PATTERN_ALL)
        v = torch.empty(feasm.fe_pattern_info_get(p)["nnz"], dtype=torch.float64, device="cuda")
        feasm.fe_assemble_csr(c, p, torch.from_numpy(K).cuda(), v, feasm.FE_DETERMINISTIC, 0)
        torch.cuda.synchronize()
        rp, ci = oracle.csr_pattern(Ds, n_s)
        assert np.array_equal(v.cpu().numpy().view(np.uint64), oracle.assemble_csr(Ds, K, rp, ci).view(np.uint64))
        feasm.fe_pattern_free(p)
        assert feasm.fe_device_status(c) == 0
    finally:
        feasm.fe_destroy(c)
