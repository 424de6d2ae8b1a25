"""The debug build (device index checks compiled in, FEASM_DEBUG=1), run in a
child process: clean inputs give the oracle's results with a clean status
word, and an invalid pattern that the kernels' own checks turn into an error
-- the last row pointer moved past the values array -- is reported as
FE_ERR_DEVICE, that row is skipped, every other row is right, and the
context stays usable."""

import os
import subprocess
import sys
import textwrap

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = textwrap.dedent("""
    import sys
    sys.path.insert(0, {root!r})
    import numpy as np
    import torch
    import oracle
    import workloads as wl
    from paper_2012_00585_gb300 import feasm
    from tests import gpu_util as gu

    # the checks below rely on the debug build: stop before any invalid input otherwise
    assert feasm.fe_debug_checks(), "not the debug build"
    ctx = feasm.fe_create(0)

    # clean inputs, every mode and both formats
    for D, n_dofs in (wl.hex_q1_grid(4, 3), wl.tet_p2_kuhn(2, d=3, seed=5), wl.hex_q1_grid(5, 1),
                      wl.quad_qp_grid(3, 3, 2)):
        K = wl.random_matrices(D.shape[0], D.shape[1], seed=7)
        g = gu.GpuAssembly(ctx, D, n_dofs)
        feasm.fe_pattern_colour(ctx, g.pattern.handle)
        rp, ci = oracle.csr_pattern(D, n_dofs)
        exp = oracle.assemble_csr(D, K, rp, ci)
        tau = gu.row_tolerance(rp, exp, gu.contribution_abs_row_sums(D, K, n_dofs))
        for fmt in ("csr", "crac"):
            got = g.assemble(K, fmt, feasm.FE_DETERMINISTIC).cpu().numpy()
            assert np.array_equal(got.view(np.uint64), exp.view(np.uint64)), fmt
            for mode in (feasm.FE_ATOMIC, feasm.FE_ROWLOCK, feasm.FE_COLOURED):
                gu.assert_within_row_tol(rp, g.assemble(K, fmt, mode).cpu().numpy(), exp, tau)
        assert feasm.fe_device_status(ctx) == 0
        g.free()

    # the planted error: the last row's end pointer past the values array
    D, n_dofs = wl.hex_q1_grid(5, 1)
    K = wl.random_matrices(D.shape[0], D.shape[1], seed=8)
    g = gu.GpuAssembly(ctx, D, n_dofs)
    rp, ci = oracle.csr_pattern(D, n_dofs)
    exp = oracle.assemble_csr(D, K, rp, ci)
    nnz = int(rp[-1])
    row_ptr = g.pattern.csr()[0]
    row_ptr[n_dofs] = nnz + 1000
    torch.cuda.synchronize()
    v = torch.zeros(nnz, dtype=torch.float64, device="cuda")
    got = g.assemble(K, "csr", feasm.FE_DETERMINISTIC, values=v).cpu().numpy()
    assert feasm.fe_device_status(ctx) == feasm.FE_ERR_DEVICE
    last = slice(int(rp[-2]), nnz)
    assert np.array_equal(got[:last.start].view(np.uint64), exp[:last.start].view(np.uint64))
    assert np.all(got[last] == 0.0)
    row_ptr[n_dofs] = nnz
    torch.cuda.synchronize()
    got = g.assemble(K, "csr", feasm.FE_DETERMINISTIC).cpu().numpy()
    assert np.array_equal(got.view(np.uint64), exp.view(np.uint64))
    assert feasm.fe_device_status(ctx) == 0
    g.free()
    feasm.fe_destroy(ctx)
    print("debug build checks ok")
""")


def test_debug_build_index_checks():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    env = dict(os.environ, FEASM_DEBUG="1")
    r = subprocess.run([sys.executable, "-c", CHILD.format(root=ROOT)], env=env, capture_output=True, text=True,
                       timeout=1200, cwd=ROOT)
    assert r.returncode == 0, r.stdout[-4000:] + r.stderr[-4000:]
    assert "debug build checks ok" in r.stdout
