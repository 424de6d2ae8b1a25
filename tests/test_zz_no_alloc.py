"""The CSR pattern build that allocates nothing, checked against the oracle's
pattern through the C ABI.

Callers that cannot allocate device memory (an application that owns all of
HBM through its own allocator, or a latency-bound loop that cannot take
cudaMalloc's implicit synchronisation) use fe_pattern_csr_noalloc, whose only
working memory is a fixed 16 MiB array inside the library.  This file is
collected last so that a run stopping at the first failure has already run
every other test; it also passes on its own in a fresh process (it needs no
library context).
"""

import numpy as np
import pytest

import oracle
import workloads as wl

pytestmark = pytest.mark.gpu

SCRATCH = 16 << 20


def _noalloc_csr(fe, Dd, n_dofs, capacity):
    import torch
    rp = torch.full((n_dofs + 1,), -1, dtype=torch.int64, device="cuda")
    ci = torch.full((max(capacity, 1),), -1, dtype=torch.int32, device="cuda")
    nnz = fe.fe_pattern_csr_noalloc(Dd.shape[0], Dd.shape[1], n_dofs, Dd, rp, ci, capacity)
    return nnz, rp.cpu().numpy(), ci.cpu().numpy()[:nnz]


def _check_against_oracle(fe, D, n_dofs, calls=2):
    import torch
    rp_o, ci_o = oracle.csr_pattern(D, n_dofs)
    Dd = torch.from_numpy(np.ascontiguousarray(D)).cuda()
    for _ in range(calls):
        nnz, rp, ci = _noalloc_csr(fe, Dd, n_dofs, int(rp_o[-1]))
        assert nnz == rp_o[-1]
        assert np.array_equal(rp, rp_o)
        assert np.array_equal(ci, ci_o)


def _gpu():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    torch.cuda.set_device(0)
    from paper_2012_00585_gb300 import feasm as fe
    return fe


def test_noalloc_pattern_matches_oracle_twice_in_a_row():
    fe = _gpu()
    # different meshes back to back, each twice: no call may see the previous
    # call's leftovers in the shared scratch array
    cases = [wl.hex_q1_grid(6, 3), wl.tet_p2_kuhn(2, d=3, seed=5), wl.quad_q1_grid(16, 1),
             wl.quad_qp_grid(5, 3, 2)]
    for D, n_dofs in cases:
        _check_against_oracle(fe, D, n_dofs)
    # too little output room: a clear error that reports the size needed
    import torch
    D, n_dofs = cases[0]
    Dd = torch.from_numpy(D).cuda()
    with pytest.raises(fe.FeError) as ei:
        _noalloc_csr(fe, Dd, n_dofs, 10)
    assert ei.value.code == fe.FE_ERR_INVALID_ARG and ei.value.nnz == 9 * 19 ** 3
    # bad connectivity is reported as such, whatever the mesh size
    bad = Dd.clone()
    bad[2, 5] = n_dofs
    with pytest.raises(fe.FeError) as ei:
        _noalloc_csr(fe, bad, n_dofs, 1)
    assert ei.value.code == fe.FE_ERR_DOF_RANGE
    # and the next call is exact again
    _check_against_oracle(fe, D, n_dofs, calls=1)


def test_noalloc_largest_accepted_mesh_and_next_size_rejected():
    """The first ne elements of a 36^3 elasticity hex mesh (3 DOFs per node,
    all DOFs of the full cube as rows, the unused ones empty): the largest ne
    the fixed array accepts is exact against the oracle, ne + 1 is rejected
    with FE_ERR_UNSUPPORTED, and the boundary lies where the documented
    size formula puts it (within 5 %)."""
    import torch
    fe = _gpu()
    D_full, n_dofs = wl.hex_q1_grid(36, 3)
    Dd_full = torch.from_numpy(D_full).cuda()

    def accepted(ne):
        try:
            fe.fe_pattern_csr_noalloc(ne, D_full.shape[1], n_dofs, Dd_full, rp, ci, 0)
        except fe.FeError as e:
            if e.code == fe.FE_ERR_INVALID_ARG:  # fits, but no output room given
                return True
            assert e.code == fe.FE_ERR_UNSUPPORTED, e.code
            return False
        return True

    rp = torch.empty(n_dofs + 1, dtype=torch.int64, device="cuda")
    ci = torch.empty(1, dtype=torch.int32, device="cuda")
    lo, hi = 1, D_full.shape[0]
    assert accepted(lo) and not accepted(hi)
    while hi - lo > 1:
        mid = (lo + hi) // 2
        if accepted(mid):
            lo = mid
        else:
            hi = mid
    # documented requirement: 4 ne nln^2 + 8 ne nln + 8 ne + 36 n_nodes + 8 n_dofs bytes
    nln, n_nodes = 8, n_dofs // 3
    predicted = (SCRATCH - 36 * n_nodes - 8 * n_dofs) / (4 * nln * nln + 8 * nln + 8)
    assert abs(lo - predicted) <= 0.05 * predicted, (lo, predicted)
    _check_against_oracle(fe, D_full[:lo], n_dofs)
    assert not accepted(lo + 1)
