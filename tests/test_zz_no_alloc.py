"""The CSR pattern build that allocates nothing, checked against the regular
pattern build through the C ABI.

Callers that cannot allocate device memory (an application that owns all of
HBM through its own allocator, or a latency-bound loop that cannot take
cudaMalloc's implicit synchronisation) use fe_pattern_csr_noalloc, whose only
working memory is a fixed array inside the library.  This file is collected
last so that a run stopping at the first failure has already run every other
test; it also passes on its own in a fresh process.
"""

import numpy as np
import pytest

import workloads as wl

pytestmark = pytest.mark.gpu


def _reference_csr(fe, ctx, Dd, n_dofs):
    p = fe.Pattern(ctx, Dd, n_dofs, fe.FE_PATTERN_CSR)
    rp, ci = p.csr()
    out = rp.cpu().numpy(), ci.cpu().numpy()
    p.free()
    return out


def _noalloc_csr(fe, Dd, n_dofs, capacity):
    import torch
    rp = torch.full((n_dofs + 1,), -1, dtype=torch.int64, device="cuda")
    ci = torch.full((max(capacity, 1),), -1, dtype=torch.int32, device="cuda")
    nnz = fe.fe_pattern_csr_noalloc(Dd.shape[0], Dd.shape[1], n_dofs, Dd, rp, ci, capacity)
    return nnz, rp.cpu().numpy(), ci.cpu().numpy()[:nnz]


def test_noalloc_pattern_matches_regular_build_twice_in_a_row():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2012_00585_gb300 import feasm as fe
    ctx = fe.fe_create(0)
    try:
        # two different meshes back to back: the second call must not see the
        # first call's leftovers in the shared scratch array
        cases = [wl.hex_q1_grid(6, 3), wl.tet_p2_kuhn(2, d=3, seed=5), wl.quad_q1_grid(16, 1)]
        for D, n_dofs in cases:
            Dd = torch.from_numpy(D).cuda()
            rp_ref, ci_ref = _reference_csr(fe, ctx, Dd, n_dofs)
            for _ in range(2):
                nnz, rp, ci = _noalloc_csr(fe, Dd, n_dofs, int(rp_ref[-1]))
                assert nnz == rp_ref[-1]
                assert np.array_equal(rp, rp_ref)
                assert np.array_equal(ci, ci_ref)
        # too little output room: a clear error that reports the size needed
        D, n_dofs = cases[0]
        Dd = torch.from_numpy(D).cuda()
        with pytest.raises(fe.FeError) as ei:
            _noalloc_csr(fe, Dd, n_dofs, 10)
        assert ei.value.code == fe.FE_ERR_INVALID_ARG and ei.value.nnz == 9 * 19 ** 3
        # a mesh that needs more than the fixed scratch is rejected, not truncated
        D, n_dofs = wl.hex_q1_grid(40, 3)
        Dd = torch.from_numpy(D).cuda()
        with pytest.raises(fe.FeError) as ei:
            _noalloc_csr(fe, Dd, n_dofs, 1)
        assert ei.value.code == fe.FE_ERR_UNSUPPORTED
    finally:
        fe.fe_destroy(ctx)
