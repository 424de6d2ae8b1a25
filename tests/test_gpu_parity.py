"""GPU parity: the CUDA path, called through the C ABI, against the CPU oracle.

Bar: the pattern (CSR, CRAC, adjacency) bit-exact; FE_DETERMINISTIC values
bit-exact (same ascending-element sum as Listing 2); FE_ATOMIC values within
|d| <= 1e-12 * sum_j |G_ij| per row, and bit-exact when every sum is an exact
integer (the paper's all-ones element).
"""

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


def _check_pattern(g, D, n_dofs):
    rp_o, ci_o = oracle.csr_pattern(D, n_dofs)
    rp, ci = g.csr_host()
    assert np.array_equal(rp, rp_o)
    assert np.array_equal(ci, ci_o)
    crp_o, ca_o = oracle.crac_from_csr(rp_o, ci_o, n_dofs)
    crp, ca = g.crac_host()
    assert np.array_equal(crp, crp_o)
    assert np.array_equal(ca, ca_o)
    B, ap, adj = g.pattern.adjacency()
    ap, adj = ap.cpu().numpy(), adj.cpu().numpy()
    n_loc = D.shape[1]
    # the block size is the largest B <= 32 for which every element lists
    # whole aligned blocks of B consecutive DOFs
    exp_B = 1
    for b in range(32, 1, -1):
        if n_loc % b == 0 and n_dofs % b == 0 and D.shape[0] > 0:
            blk = D.reshape(D.shape[0], n_loc // b, b)
            if np.all(blk[:, :, 0] % b == 0) and np.all(blk - blk[:, :, :1] == np.arange(b)):
                exp_B = b
                break
    assert B == exp_B
    Nn = D[:, ::B] // B
    deg = np.bincount(Nn.ravel(), minlength=n_dofs // B)
    assert np.array_equal(np.diff(ap), deg)
    inc = np.arange(Nn.size, dtype=np.int64)
    order = np.argsort(Nn.ravel(), kind="stable")  # stable: ascending incidence id per block
    assert np.array_equal(adj.astype(np.int64), inc[order])
    info = g.pattern.info
    assert info["block"] == B
    assert info["nnz"] == rp_o[-1] and info["n_ca"] == ca_o.shape[0]
    assert info["max_row_len"] == int(np.max(np.diff(rp_o))) if n_dofs else True
    # runs of consecutive blocks per element (the compressed DOF array of §2.1, at block level)
    assert info["n_elem_runs"] == sum(len(oracle.compress_dofs(row)) // 2 for row in Nn)
    return rp_o, ci_o, crp_o, ca_o


def _run_all_modes(g, D, K, n_dofs, rp_o, ci_o, crp_o, ca_o, exact_atomic=False):
    from paper_2012_00585_gb300 import feasm
    v_o = oracle.assemble_csr(D, K, rp_o, ci_o)
    v_oc = oracle.assemble_crac(D, K, crp_o, ca_o, ci_o.shape[0])
    assert np.array_equal(v_o, v_oc)
    tau = gu.row_tolerance(rp_o, v_o, gu.contribution_abs_row_sums(D, K, n_dofs))
    out = {}
    for fmt in ("csr", "crac"):
        det = g.assemble(K, fmt, feasm.FE_DETERMINISTIC).cpu().numpy()
        assert np.array_equal(det.view(np.uint64), v_o.view(np.uint64)), f"{fmt} deterministic not bit-exact"
        at = g.assemble(K, fmt, feasm.FE_ATOMIC).cpu().numpy()
        if exact_atomic:
            assert np.array_equal(at, v_o)
        else:
            gu.assert_within_row_tol(rp_o, at, v_o, tau)
        out[fmt] = (det, at)
    return v_o, out


# ------------------------------------------------------------ configs ---

def test_c1_quad_laplace_16x16(ctx):
    """Config 1: 16x16 Q1 quads, 1 DOF/node, 4x4 Laplace by 2x2 Gauss."""
    D, n_dofs = wl.quad_q1_grid(16, 1)
    K = wl.broadcast_matrices(wl.laplace_q1_quad(), D.shape[0])
    g = gu.GpuAssembly(ctx, D, n_dofs)
    pat = _check_pattern(g, D, n_dofs)
    assert g.pattern.info["nnz"] == 2401 and g.pattern.info["n_ca"] == 1668
    v_o, _ = _run_all_modes(g, D, K, n_dofs, *pat)
    g.free()


@pytest.mark.parametrize("n", [4, 9])
def test_c2_hex_elasticity_small(ctx, n):
    """Config 2's mesh family at reduced size (several tiles, ragged tail)."""
    D, n_dofs = wl.hex_q1_grid(n, 3)
    K = wl.broadcast_matrices(wl.elasticity_q1_hex(1.0 / n), D.shape[0])
    K[3, 5, 7] += 0.125  # one perturbed element: no kernel may assume K is uniform
    K[3, 7, 5] += 0.125
    g = gu.GpuAssembly(ctx, D, n_dofs)
    pat = _check_pattern(g, D, n_dofs)
    assert g.pattern.info["nnz"] == 9 * (3 * n + 1) ** 3
    _run_all_modes(g, D, K, n_dofs, *pat)
    g.free()


@pytest.mark.parametrize("n", [2, 4])
def test_c3_p2_tets_permuted_spd(ctx, n):
    """Config 3's generator at reduced size: permuted P2 tets, random SPD 30x30."""
    D, n_dofs = wl.tet_p2_kuhn(n, d=3, seed=n)
    K = wl.random_spd_matrices(D.shape[0], 30, seed=n)
    g = gu.GpuAssembly(ctx, D, n_dofs)
    pat = _check_pattern(g, D, n_dofs)
    assert not g.pattern.info["uniform_runs"]  # run structure varies per element
    assert g.pattern.info["block"] == 3
    _run_all_modes(g, D, K, n_dofs, *pat)
    g.free()


@pytest.mark.parametrize("case", ["tets_permuted", "hex_d3", "quads_q3", "scattered"])
def test_atomic_locality_order(ctx, case):
    """FE_ATOMIC through the locality order of the elements (forced on with
    FE_KNOB_ATOMIC_ORDER = 2; the automatic choice takes it only for large
    meshes with scattered numbering): within the row tolerance of the oracle
    in both formats, and the deterministic modes unchanged.  Several seeds
    (clusters) per mesh: the tet mesh has more than 16,384 blocks."""
    from paper_2012_00585_gb300 import feasm
    if case == "tets_permuted":
        D, n_dofs = wl.tet_p2_kuhn(14, d=3, seed=21)  # 24,389 blocks: two clusters and a ragged one
        K = wl.random_spd_matrices(D.shape[0], 30, seed=2)
    elif case == "hex_d3":
        D, n_dofs = wl.hex_q1_grid(7, 3)
        K = wl.random_matrices(D.shape[0], 24, seed=3)
    elif case == "quads_q3":
        D, n_dofs = wl.quad_qp_grid(6, 3, 1)
        K = wl.random_matrices(D.shape[0], 16, seed=4)
    else:
        rng = np.random.default_rng(9)
        n_dofs = 700
        D = np.stack([rng.choice(n_dofs - 50, 7, replace=False) for _ in range(300)]).astype(np.int32)
        K = wl.random_matrices(D.shape[0], 7, seed=5)
    feasm.fe_tune_set(ctx, feasm.FE_KNOB_ATOMIC_ORDER, 2)
    try:
        g = gu.GpuAssembly(ctx, D, n_dofs)
    finally:
        feasm.fe_tune_set(ctx, feasm.FE_KNOB_ATOMIC_ORDER, 0)
    assert g.pattern.info["atomic_order"] == 1
    pat = _check_pattern(g, D, n_dofs)
    _run_all_modes(g, D, K, n_dofs, *pat)
    # all-ones K: integer sums, exact whatever the order of the adds
    ones = np.ones_like(K)
    v_o = oracle.assemble_csr(D, ones, pat[0], pat[1])
    for fmt in ("csr", "crac"):
        assert np.array_equal(g.assemble(ones, fmt, feasm.FE_ATOMIC).cpu().numpy(), v_o)
    g.free()
    feasm.fe_tune_set(ctx, feasm.FE_KNOB_ATOMIC_ORDER, 1)
    try:
        g = gu.GpuAssembly(ctx, D, n_dofs)
        assert g.pattern.info["atomic_order"] == 0
        g.free()
    finally:
        feasm.fe_tune_set(ctx, feasm.FE_KNOB_ATOMIC_ORDER, 0)


def test_c4_mixed_sizes_one_by_one(ctx):
    """Config 4's two element kinds: Q1 Laplace (8x8, d=1) and elasticity (24x24)."""
    for n, d in [(5, 1), (7, 1), (5, 3), (6, 3)]:
        D, n_dofs = wl.hex_q1_grid(n, d)
        Kr = wl.laplace_q1_hex(1.0 / n) if d == 1 else wl.elasticity_q1_hex(1.0 / n)
        K = wl.scaled_matrices(Kr, D.shape[0], seed=n)
        g = gu.GpuAssembly(ctx, D, n_dofs)
        pat = _check_pattern(g, D, n_dofs)
        _run_all_modes(g, D, K, n_dofs, *pat)
        g.free()


@pytest.mark.slow
def test_c2_full_size_64cubed(ctx):
    """Config 2 at full size (262,144 hexes, 823,875 DOFs), every entry."""
    import torch
    from paper_2012_00585_gb300 import feasm
    n = 64
    D, n_dofs = wl.hex_q1_grid(n, 3)
    assert n_dofs == 823_875
    Kr = wl.elasticity_q1_hex(1.0 / n)
    g = gu.GpuAssembly(ctx, D, n_dofs)
    info = g.pattern.info
    assert info["nnz"] == 64_701_513 and info["n_ca"] == 14_527_112
    assert info["atomic_order"] == 0  # natural numbering: elements stay in ascending order
    rp_o, ci_o = oracle.csr_pattern(D, n_dofs)
    rp, ci = g.csr_host()
    assert np.array_equal(rp, rp_o) and np.array_equal(ci, ci_o)
    crp_o, ca_o = oracle.crac_from_csr(rp_o, ci_o, n_dofs)
    crp, ca = g.crac_host()
    assert np.array_equal(crp, crp_o) and np.array_equal(ca, ca_o)
    Kd = wl.broadcast_matrices(Kr, D.shape[0], device="cuda")
    K = Kd.cpu().numpy()
    v_o = oracle.assemble_csr(D, K, rp_o, ci_o)
    tau = gu.row_tolerance(rp_o, v_o, gu.contribution_abs_row_sums(D, K, n_dofs))
    for fmt in ("csr", "crac"):
        det = g.assemble(Kd, fmt, feasm.FE_DETERMINISTIC).cpu().numpy()
        assert np.array_equal(det.view(np.uint64), v_o.view(np.uint64))
        at = g.assemble(Kd, fmt, feasm.FE_ATOMIC).cpu().numpy()
        gu.assert_within_row_tol(rp_o, at, v_o, tau)
    del Kd
    torch.cuda.empty_cache()
    g.free()


# --------------------------------------------------------- edge cases ---

def test_all_ones_atomic_is_exact(ctx):
    """Paper's dummy element: integer sums, so atomic order cannot matter."""
    D, n_dofs = wl.tet_p2_kuhn(3, d=2, seed=1)
    K = wl.ones_matrices(*D.shape[:1], D.shape[1])
    g = gu.GpuAssembly(ctx, D, n_dofs)
    pat = _check_pattern(g, D, n_dofs)
    _run_all_modes(g, D, K, n_dofs, *pat, exact_atomic=True)
    g.free()


@pytest.mark.parametrize("case", ["qp3_d1", "qp2_d4", "hex_d2", "q8_rows_over_256", "d20_quad",
                                  "scattered", "single", "unused_dofs"])
def test_generic_sizes_and_layouts(ctx, case):
    """Element sizes and layouts beyond the specialised shapes (36, 16 with
    2 DOFs per node, 81, 80, ...), rows longer than 256 (16-bit slot maps),
    scattered DOFs, empty rows."""
    rng = np.random.default_rng(0)
    if case == "qp3_d1":
        D, n_dofs = wl.quad_qp_grid(5, 3, 1)          # n_loc 16
    elif case == "qp2_d4":
        D, n_dofs = wl.quad_qp_grid(4, 2, 4)          # n_loc 36
    elif case == "hex_d2":
        D, n_dofs = wl.hex_q1_grid(4, 2)              # n_loc 16
    elif case == "q8_rows_over_256":
        D, n_dofs = wl.quad_qp_grid(3, 8, 1)          # n_loc 81, rows up to 289
    elif case == "d20_quad":
        D, n_dofs = wl.quad_q1_grid(3, 20)            # n_loc 80
    elif case == "scattered":
        D = np.stack([rng.choice(500, size=9, replace=False) for _ in range(300)]).astype(np.int32)
        n_dofs = 520
    elif case == "single":
        D, n_dofs = np.array([[3, 1, 2]], dtype=np.int32), 4
    else:
        D = np.array([[0, 1, 5, 6], [5, 6, 9, 10], [0, 1, 9, 10]], dtype=np.int32)
        n_dofs = 14
    K = wl.random_matrices(D.shape[0], D.shape[1], seed=3)
    g = gu.GpuAssembly(ctx, D, n_dofs)
    if case == "q8_rows_over_256":
        assert g.pattern.info["map_bytes"] == 2
    pat = _check_pattern(g, D, n_dofs)
    _run_all_modes(g, D, K, n_dofs, *pat)
    g.free()


@pytest.mark.parametrize("p,d", [(2, 1), (3, 1), (4, 1), (5, 1), (8, 1), (1, 2), (1, 3), (1, 4), (1, 5), (1, 6),
                                 (1, 7), (1, 8), (2, 4), (4, 4)])
def test_quad_shapes_permuted_nodes(ctx, p, d):
    """The quad shapes with their own row kernels (Q2..Q8 scalar, Q1 with
    2..8 DOFs per node, Q2..Q4 with 4) on a mesh whose node numbers are
    shuffled: irregular rows and CRAC runs that differ from element to
    element (Q8: rows over 256 nodes, 16-bit slot maps)."""
    D, n_dofs = wl.quad_qp_grid(6, p, d)
    perm = np.random.default_rng(100 * p + d).permutation(n_dofs // d)
    D = (perm[D // d] * d + D % d).astype(np.int32)
    K = wl.random_matrices(D.shape[0], D.shape[1], seed=p + 10 * d)
    g = gu.GpuAssembly(ctx, D, n_dofs)
    assert g.pattern.adjacency()[0] == d
    pat = _check_pattern(g, D, n_dofs)
    _run_all_modes(g, D, K, n_dofs, *pat)
    g.free()


@pytest.mark.parametrize("case", ["hex_d16", "quad_d32", "scattered_128"])
def test_largest_elements(ctx, case):
    """Elements of FE_MAX_NLOC = 128 DOFs, the largest the library takes: 16
    DOFs per hex node (the generic row kernel), 32 per quad node (the largest
    DOF block), and unblocked elements of 128 scattered DOFs (run-start masks
    of four words, rows over 256 entries: 16-bit slot maps).  Every mode
    against the oracle: deterministic and coloured bit-exact (the coloured
    sum in colour order), atomic and row-locked within the row tolerance."""
    from paper_2012_00585_gb300 import feasm
    if case == "hex_d16":
        D, n_dofs = wl.hex_q1_grid(3, 16)
    elif case == "quad_d32":
        D, n_dofs = wl.quad_q1_grid(4, 32)
    else:
        rng = np.random.default_rng(11)
        D = np.stack([rng.choice(600, size=128, replace=False) for _ in range(40)]).astype(np.int32)
        n_dofs = 600
    assert D.shape[1] == feasm.FE_MAX_NLOC
    K = wl.random_matrices(D.shape[0], D.shape[1], seed=12)
    g = gu.GpuAssembly(ctx, D, n_dofs)
    if case == "scattered_128":
        assert g.pattern.info["map_bytes"] == 2
    pat = _check_pattern(g, D, n_dofs)
    v_o, _ = _run_all_modes(g, D, K, n_dofs, *pat)
    rp_o, ci_o = pat[0], pat[1]
    tau = gu.row_tolerance(rp_o, v_o, gu.contribution_abs_row_sums(D, K, n_dofs))
    for fmt in ("csr", "crac"):
        gu.assert_within_row_tol(rp_o, g.assemble(K, fmt, feasm.FE_ROWLOCK).cpu().numpy(), v_o, tau)
    feasm.fe_pattern_colour(ctx, g.pattern.handle)
    _, colour = oracle.greedy_colouring(D, n_dofs)
    order = np.lexsort((np.arange(D.shape[0]), colour))
    exp_c = oracle.assemble_csr(D, K, rp_o, ci_o, order=order)
    for fmt in ("csr", "crac"):
        got = g.assemble(K, fmt, feasm.FE_COLOURED).cpu().numpy()
        assert np.array_equal(got.view(np.uint64), exp_c.view(np.uint64)), fmt
    assert feasm.fe_device_status(ctx) == 0
    g.free()


def test_accumulate_both_modes(ctx):
    from paper_2012_00585_gb300 import feasm
    D, n_dofs = wl.tet_p2_kuhn(2, d=3, seed=9)
    K1 = wl.random_spd_matrices(D.shape[0], 30, seed=1)
    K2 = wl.random_spd_matrices(D.shape[0], 30, seed=2)
    g = gu.GpuAssembly(ctx, D, n_dofs)
    rp, ci = oracle.csr_pattern(D, n_dofs)
    v1 = oracle.assemble_csr(D, K1, rp, ci)
    v12 = oracle.assemble_csr(D, K2, rp, ci, values=v1)
    for fmt in ("csr", "crac"):
        base = g.assemble(K1, fmt, feasm.FE_DETERMINISTIC)
        got = g.assemble(K2, fmt, feasm.FE_DETERMINISTIC, accumulate=1, values=base).cpu().numpy()
        assert np.array_equal(got, v12)
        base = g.assemble(K1, fmt, feasm.FE_ATOMIC)
        got = g.assemble(K2, fmt, feasm.FE_ATOMIC, accumulate=1, values=base).cpu().numpy()
        tau = gu.row_tolerance(rp, v12)
        gu.assert_within_row_tol(rp, got, v12, 2 * tau)
    g.free()


def test_deterministic_is_reproducible_and_formats_agree(ctx):
    from paper_2012_00585_gb300 import feasm
    D, n_dofs = wl.tet_p2_kuhn(3, d=3, seed=4)
    K = wl.random_spd_matrices(D.shape[0], 30, seed=4)
    g = gu.GpuAssembly(ctx, D, n_dofs)
    a = g.assemble(K, "csr", feasm.FE_DETERMINISTIC).cpu().numpy()
    b = g.assemble(K, "csr", feasm.FE_DETERMINISTIC).cpu().numpy()
    c = g.assemble(K, "crac", feasm.FE_DETERMINISTIC).cpu().numpy()
    assert a.tobytes() == b.tobytes() == c.tobytes()
    g.free()


def test_empty_mesh(ctx):
    import torch
    from paper_2012_00585_gb300 import feasm
    Dd = torch.empty((0, 4), dtype=torch.int32, device="cuda")
    p = feasm.Pattern(ctx, Dd, 5)
    assert p.info["nnz"] == 0 and p.info["n_ca"] == 2
    rp, ci = p.csr()
    assert rp.cpu().tolist() == [0] * 6
    crp, ca = p.crac()
    assert ca.cpu().tolist() == [5, 0]
    v = torch.empty(0, dtype=torch.float64, device="cuda")
    K = torch.empty(0, dtype=torch.float64, device="cuda")
    for f in (feasm.fe_assemble_csr, feasm.fe_assemble_crac):
        for mode in (feasm.FE_ATOMIC, feasm.FE_DETERMINISTIC):
            f(ctx, p.handle, K, v, mode, 0)
    torch.cuda.synchronize()
    p.free()


def test_invalid_connectivity_reports_errors(ctx):
    import torch
    from paper_2012_00585_gb300 import feasm
    bad_range = torch.tensor([[0, 1, 7]], dtype=torch.int32, device="cuda")
    with pytest.raises(feasm.FeError) as ei:
        feasm.fe_pattern_build(ctx, 1, 3, 5, bad_range)
    assert ei.value.code == feasm.FE_ERR_DOF_RANGE
    neg = torch.tensor([[0, -1, 2]], dtype=torch.int32, device="cuda")
    with pytest.raises(feasm.FeError) as ei:
        feasm.fe_pattern_build(ctx, 1, 3, 5, neg)
    assert ei.value.code == feasm.FE_ERR_DOF_RANGE
    dup = torch.tensor([[0, 2, 4], [1, 3, 1]], dtype=torch.int32, device="cuda")
    with pytest.raises(feasm.FeError) as ei:
        feasm.fe_pattern_build(ctx, 2, 3, 5, dup)
    assert ei.value.code == feasm.FE_ERR_DUP_DOF
    ok = torch.tensor([[0, 2, 4]], dtype=torch.int32, device="cuda")
    with pytest.raises(feasm.FeError) as ei:
        feasm.fe_pattern_build(ctx, 1, 3, 5, ok, flags=0x100)
    assert ei.value.code == feasm.FE_ERR_INVALID_ARG
    with pytest.raises(feasm.FeError) as ei:
        feasm.fe_pattern_build(ctx, 1, 200, 5, ok)
    assert ei.value.code == feasm.FE_ERR_UNSUPPORTED
    # the context stays usable after rejected inputs
    p = feasm.Pattern(ctx, ok, 5)
    assert p.info["nnz"] == 9
    # parts that were not built are reported, not used
    p2 = feasm.Pattern(ctx, ok, 5, flags=feasm.FE_PATTERN_CSR | feasm.FE_PATTERN_MAP_CSR)
    K = torch.ones(9, dtype=torch.float64, device="cuda")
    v = torch.zeros(9, dtype=torch.float64, device="cuda")
    with pytest.raises(feasm.FeError) as ei:
        feasm.fe_assemble_crac(ctx, p2.handle, K, v)
    assert ei.value.code == feasm.FE_ERR_NOT_BUILT
    with pytest.raises(feasm.FeError) as ei:
        feasm.fe_pattern_crac(p2.handle)
    assert ei.value.code == feasm.FE_ERR_NOT_BUILT
    feasm.fe_assemble_csr(ctx, p2.handle, K, v, feasm.FE_ATOMIC)
    torch.cuda.synchronize()
    assert v.cpu().tolist() == [1.0] * 9
    p.free()
    p2.free()


@pytest.mark.slow
def test_c3_full_size_sampled_rows(ctx):
    """Config 3 at full size: 96^3 hexes -> 5,308,416 permuted P2 tets,
    21,567,171 DOFs, random SPD 30x30 K drawn on the device (38 GB).  The
    whole pattern is checked by properties that hold at any size (nnz is
    permutation invariant and equals the natural-numbering count); sampled
    rows are checked entry by entry against the oracle run on the sub-mesh of
    the elements that touch them (in ascending element order, which leaves
    those rows' sums unchanged)."""
    import torch
    from paper_2012_00585_gb300 import feasm
    n = 96
    D, n_dofs = wl.tet_p2_kuhn(n, d=3, seed=2012)
    assert D.shape == (5_308_416, 30) and n_dofs == 21_567_171
    g = gu.GpuAssembly(ctx, D, n_dofs)
    info = g.pattern.info
    assert info["nnz"] == 1_842_870_537 and info["block"] == 3
    assert info["atomic_order"] == 1  # scattered numbering, 14.7 GB of values: the locality order is built
    rp_d, ci_d = g.pattern.csr()
    crp_d, ca_d = g.pattern.crac()
    Kd = wl.random_spd_matrices(D.shape[0], 30, seed=7, device="cuda", chunk=1 << 18)
    rng = np.random.default_rng(0)
    rows = np.unique(np.concatenate([rng.choice(n_dofs, 60, replace=False), [0, n_dofs - 1]]))
    # elements touching the sampled rows, ascending
    hit = np.isin(D, rows).any(axis=1)
    els = np.nonzero(hit)[0]
    Dsub = D[els]
    Ksub = Kd[torch.from_numpy(els).cuda()].cpu().numpy()
    rp_o, ci_o = oracle.csr_pattern(Dsub, n_dofs)
    v_o = oracle.assemble_csr(Dsub, Ksub, rp_o, ci_o)
    crp_o, ca_o = oracle.crac_from_csr(rp_o, ci_o, n_dofs)
    rp_h = rp_d.cpu().numpy()
    crp_h = crp_d.cpu().numpy()
    assert np.all(np.diff(rp_h) >= 0) and rp_h[-1] == info["nnz"]
    for fmt in ("csr", "crac"):
        for mode in (feasm.FE_DETERMINISTIC, feasm.FE_ATOMIC):
            v = g.assemble(Kd, fmt, mode)
            for i in rows:
                a, b = int(rp_h[i]), int(rp_h[i + 1])
                ao, bo = int(rp_o[i]), int(rp_o[i + 1])
                assert np.array_equal(ci_d[a:b].cpu().numpy(), ci_o[ao:bo])
                ca_row = ca_d[int(crp_h[i]):int(crp_h[i + 1])].cpu().numpy()
                ca_row_o = ca_o[int(crp_o[i]):int(crp_o[i + 1])].copy()
                ca_row_o[1::2] += a - ao  # value positions are relative to the row's start
                assert np.array_equal(ca_row, ca_row_o)
                got = v[a:b].cpu().numpy()
                exp = v_o[ao:bo]
                if mode == feasm.FE_DETERMINISTIC:
                    assert np.array_equal(got.view(np.uint64), exp.view(np.uint64))
                else:
                    assert np.all(np.abs(got - exp) <= 1e-12 * np.abs(exp).sum())
            del v
    assert feasm.fe_device_status(ctx) == 0
    del Kd
    torch.cuda.empty_cache()
    g.free()


@pytest.mark.parametrize("gkind", [1, 2])
@pytest.mark.parametrize("akind", [1, 2])
def test_every_kernel_variant(ctx, gkind, akind):
    """Each schedule knob value gives the same results: deterministic
    variants bit-exact, atomic variants within the row tolerance (gather
    kernel 2 applies to the shapes with slices of at most 16 entries; the
    others take kernel 1)."""
    from paper_2012_00585_gb300 import feasm
    feasm.fe_tune_set(ctx, feasm.FE_KNOB_GATHER_KERNEL, gkind)
    feasm.fe_tune_set(ctx, feasm.FE_KNOB_ATOMIC_KERNEL, akind)
    try:
        for D, n_dofs, K in [
            (*wl.hex_q1_grid(5, 3), None),
            (*wl.tet_p2_kuhn(3, d=3, seed=8), None),
            (*wl.hex_q1_grid(6, 1), None),
            (*wl.quad_q1_grid(9, 2), None),
            (*wl.quad_q1_grid(11, 1), None),
            (*wl.quad_qp_grid(3, 3, 1), None),
        ]:
            K = wl.random_matrices(D.shape[0], D.shape[1], seed=gkind * 10 + akind)
            g = gu.GpuAssembly(ctx, D, n_dofs)
            pat = _check_pattern(g, D, n_dofs)
            _run_all_modes(g, D, K, n_dofs, *pat)
            g.free()
    finally:
        feasm.fe_tune_set(ctx, feasm.FE_KNOB_GATHER_KERNEL, 0)
        feasm.fe_tune_set(ctx, feasm.FE_KNOB_ATOMIC_KERNEL, 0)


@pytest.mark.parametrize("fmt", ["csr", "crac"])
def test_signed_zero_contributions(ctx, fmt):
    """Listing 2 starts every slot at +0.0: a slot whose contributions are all
    -0.0 sums to +0.0, and a -0.0 first term does not leave a -0.0 behind.
    The deterministic path must give the same bits."""
    from paper_2012_00585_gb300 import feasm
    for D, n_dofs in (wl.hex_q1_grid(4, 3), wl.tet_p2_kuhn(2, d=3, seed=3)):
        n_e, n_loc = D.shape
        K = np.full((n_e, n_loc, n_loc), -0.0)
        K[1::3] = wl.random_matrices((n_e + 1) // 3, n_loc, seed=9)[: K[1::3].shape[0]]
        g = gu.GpuAssembly(ctx, D, n_dofs)
        rp, ci = oracle.csr_pattern(D, n_dofs)
        exp = oracle.assemble_csr(D, K, rp, ci)
        assert np.any(np.signbit(K)) and not np.any(np.signbit(exp[exp == 0]))
        got = g.assemble(K, fmt, feasm.FE_DETERMINISTIC).cpu().numpy()
        assert np.array_equal(got.view(np.uint64), exp.view(np.uint64))
        g.free()


@pytest.mark.parametrize("case", ["hex_d3", "tets_permuted", "quads_q3"])
def test_crac_only_pattern(ctx, case):
    """A pattern built for CRAC alone (no CSR slot map): the CRAC gather then
    reads the run map expanded per column block in the symbolic phase (with
    both maps built it shares the CSR map instead), bit-exact against the
    oracle; the atomic CRAC path within the row tolerance; the CSR assembly
    reports that its map was not built."""
    from paper_2012_00585_gb300 import feasm
    if case == "hex_d3":
        D, n_dofs = wl.hex_q1_grid(6, 3)
    elif case == "tets_permuted":
        D, n_dofs = wl.tet_p2_kuhn(3, d=3, seed=4)
    else:
        D, n_dofs = wl.quad_qp_grid(5, 3, 1)
    K = wl.random_matrices(D.shape[0], D.shape[1], seed=11)
    g = gu.GpuAssembly(ctx, D, n_dofs, flags=feasm.FE_PATTERN_CRAC | feasm.FE_PATTERN_MAP_CRAC)
    rp_o, ci_o = oracle.csr_pattern(D, n_dofs)
    v_o = oracle.assemble_csr(D, K, rp_o, ci_o)
    det = g.assemble(K, "crac", feasm.FE_DETERMINISTIC).cpu().numpy()
    assert np.array_equal(det.view(np.uint64), v_o.view(np.uint64))
    at = g.assemble(K, "crac", feasm.FE_ATOMIC).cpu().numpy()
    gu.assert_within_row_tol(rp_o, at, v_o, gu.row_tolerance(rp_o, v_o, gu.contribution_abs_row_sums(D, K, n_dofs)))
    with pytest.raises(feasm.FeError) as ei:
        g.assemble(K, "csr", feasm.FE_DETERMINISTIC)
    assert ei.value.code == feasm.FE_ERR_NOT_BUILT
    g.free()
