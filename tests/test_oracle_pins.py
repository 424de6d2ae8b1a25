"""Pins of the CPU oracle against facts that do not come from the oracle itself.

* values printed in the paper (Fig. 1 arrays and look-ups, the compressed
  DOF example of §2.1, nnz and n_ca of the structured benchmark meshes, §4);
* closed forms (nnz of tensor-product meshes, n_ca under natural numbering);
* brute force on tiny meshes (dense assembly by pure Python loops);
* invariants (symmetry, zero row sums, rigid-body null space, sum of all
  entries, integer incidence counts for the paper's all-ones element).

Each test is chosen so that a plausible slip in the oracle (a dropped
contribution, a wrong index, a transposed K, an off-by-one in CRAC) fails.
"""

import math

import numpy as np
import pytest

import oracle
import workloads as wl
from tests.golden import load as golden


# ---------------------------------------------------------------- Fig. 1 ---

def _fig1_zero_based():
    f = golden.fig1()
    row_ptr = np.array([int(t) - 1 for t in f["csr_row_ptr"]], dtype=np.int64)
    col = np.array([int(t) - 1 for t in f["csr_col"]], dtype=np.int32)
    vals = np.array([float(t) for t in f["values"]])
    crac_ptr = np.array([int(t) - 1 for t in f["crac_row_ptr"]], dtype=np.int64)
    ca = f["col_align"]
    return f, row_ptr, col, vals, crac_ptr, ca


def test_fig1_csr_to_crac_exact():
    f, row_ptr, col, vals, crac_ptr_exp, ca_exp = _fig1_zero_based()
    n = row_ptr.shape[0] - 1
    crac_ptr, col_align = oracle.crac_from_csr(row_ptr, col, n_cols=n)
    assert crac_ptr.tolist() == crac_ptr_exp.tolist()
    # pairs: column is 1-based in the figure, value position 1-based
    exp = []
    for k in range(0, len(ca_exp), 2):
        c = ca_exp[k]
        exp.append(n if c == "-" else int(c) - 1)  # final pair's column: n_cols
        exp.append(int(ca_exp[k + 1]) - 1)
    assert col_align.tolist() == exp
    assert col_align.shape[0] == 2 * (7 + 1)


def test_fig1_lookups_all_36():
    f, row_ptr, col, vals, _, _ = _fig1_zero_based()
    n = row_ptr.shape[0] - 1
    crac_ptr, col_align = oracle.crac_from_csr(row_ptr, col, n_cols=n)
    dense = {}
    for i in range(n):
        for k in range(row_ptr[i], row_ptr[i + 1]):
            dense[(i, int(col[k]))] = k
    for i in range(n):
        for j in range(n):
            exp = dense.get((i, j), -1)
            assert oracle.csr_lookup(row_ptr, col, i, j) == exp
            assert oracle.crac_lookup(crac_ptr, col_align, i, j) == exp
    li, lj, lpos, lval = f["lookup"]
    pos = oracle.crac_lookup(crac_ptr, col_align, int(li) - 1, int(lj) - 1)
    assert pos == int(lpos) - 1
    assert vals[pos] == float(lval)


def test_fig1_matrix_through_crac_spmv_matches_dense():
    f, row_ptr, col, vals, _, _ = _fig1_zero_based()
    n = 6
    crac_ptr, col_align = oracle.crac_from_csr(row_ptr, col, n_cols=n)
    A = np.zeros((n, n))
    for i in range(n):
        for k in range(row_ptr[i], row_ptr[i + 1]):
            A[i, col[k]] = vals[k]
    x = np.arange(1, n + 1, dtype=np.float64)
    y_crac = oracle.spmv_crac(crac_ptr, col_align, vals, x)
    y_csr = oracle.spmv_csr(row_ptr, col, vals, x)
    assert np.array_equal(y_crac, y_csr)
    np.testing.assert_allclose(y_csr, A @ x, rtol=1e-14)


# ------------------------------------------------------- §2.1 compression ---

def test_compressed_dofs_example():
    g = golden.compressed_dofs()
    assert oracle.compress_dofs(np.array(g["plain"])).tolist() == g["compressed"]


def test_compressed_dofs_edge_cases():
    assert oracle.compress_dofs(np.array([7])).tolist() == [7, 1]
    assert oracle.compress_dofs(np.array([5, 4, 3])).tolist() == [5, 1, 4, 1, 3, 1]
    assert oracle.compress_dofs(np.arange(10, 40)).tolist() == [10, 30]
    assert oracle.compress_dofs(np.array([1, 2, 4, 5, 6, 0])).tolist() == [1, 2, 4, 3, 0, 1]


# ------------------------------------------------- brute force, tiny meshes ---

def _tiny_meshes():
    yield "quad_q1_3x3_d1", wl.quad_q1_grid(3, 1)
    yield "quad_q1_2x3_d2", (lambda c: c)(wl.quad_q1_grid(2, 2))
    yield "quad_q2_2x2_d1", wl.quad_qp_grid(2, 2, 1)
    yield "hex_q1_2_d3", wl.hex_q1_grid(2, 3)
    yield "tet_p2_1_d1_perm", wl.tet_p2_kuhn(1, d=1, seed=3)
    # irregular: element sizes equal, DOFs scattered, some DOFs unused (empty rows)
    rng = np.random.default_rng(11)
    D = np.stack([rng.choice(40, size=5, replace=False) for _ in range(9)]).astype(np.int32)
    yield "random_5dof_els_with_empty_rows", (D, 45)


def _brute_force(D, K, n_dofs, order=None):
    """Dense assembly by pure Python loops, Listing 2's loop nest verbatim."""
    n_e, n_loc = D.shape
    G = [[0.0] * n_dofs for _ in range(n_dofs)]
    touched = [[False] * n_dofs for _ in range(n_dofs)]
    for e in (range(n_e) if order is None else order):
        for r in range(n_loc):
            for c in range(n_loc):
                i, j = int(D[e, r]), int(D[e, c])
                G[i][j] = G[i][j] + float(K[e, r, c])
                touched[i][j] = True
    return G, touched


@pytest.mark.parametrize("name,mesh", list(_tiny_meshes()))
def test_brute_force_pattern_and_values(name, mesh):
    D, n_dofs = mesh
    n_e, n_loc = D.shape
    K = wl.random_matrices(n_e, n_loc, seed=5)  # unsymmetric: catches K^T
    G, touched = _brute_force(D, K, n_dofs)
    row_ptr, col_idx = oracle.csr_pattern(D, n_dofs)
    exp_ptr = [0]
    exp_col = []
    for i in range(n_dofs):
        cols = [j for j in range(n_dofs) if touched[i][j]]
        exp_col += cols
        exp_ptr.append(len(exp_col))
    assert row_ptr.tolist() == exp_ptr
    assert col_idx.tolist() == exp_col
    v = oracle.assemble_csr(D, K, row_ptr, col_idx)
    exp_v = [G[i][j] for i in range(n_dofs) for j in range(n_dofs) if touched[i][j]]
    assert v.tolist() == exp_v  # bit-exact: same (e, r, c) order, same adds
    # CRAC route gives the identical array
    crac_ptr, col_align = oracle.crac_from_csr(row_ptr, col_idx, n_dofs)
    v2 = oracle.assemble_crac(D, K, crac_ptr, col_align, col_idx.shape[0])
    assert np.array_equal(v, v2)


def test_brute_force_permuted_element_order():
    D, n_dofs = wl.hex_q1_grid(2, 1)
    K = wl.random_matrices(D.shape[0], D.shape[1], seed=9)
    order = np.random.default_rng(4).permutation(D.shape[0])
    G, touched = _brute_force(D, K, n_dofs, order=order)
    row_ptr, col_idx = oracle.csr_pattern(D, n_dofs)
    v = oracle.assemble_csr(D, K, row_ptr, col_idx, order=order)
    exp_v = [G[i][j] for i in range(n_dofs) for j in range(n_dofs) if touched[i][j]]
    assert v.tolist() == exp_v


def test_accumulate_onto_existing_values():
    D, n_dofs = wl.quad_q1_grid(3, 1)
    K = wl.random_matrices(D.shape[0], 4, seed=1)
    row_ptr, col_idx = oracle.csr_pattern(D, n_dofs)
    v1 = oracle.assemble_csr(D, K, row_ptr, col_idx)
    v2 = oracle.assemble_csr(D, K, row_ptr, col_idx, values=v1)
    G, touched = _brute_force(np.concatenate([D, D]), np.concatenate([K, K]), n_dofs)
    exp = [G[i][j] for i in range(n_dofs) for j in range(n_dofs) if touched[i][j]]
    assert v2.tolist() == exp


# ---------------------------------------------------------- closed forms ---

@pytest.mark.parametrize("m", [1, 2, 5, 16])
@pytest.mark.parametrize("d", [1, 2, 3])
def test_nnz_quad_q1_closed_form(m, d):
    D, n_dofs = wl.quad_q1_grid(m, d)
    row_ptr, _ = oracle.csr_pattern(D, n_dofs)
    assert row_ptr[-1] == d * d * (3 * m + 1) ** 2


@pytest.mark.parametrize("n", [3, 4, 6])
@pytest.mark.parametrize("d", [1, 3])
def test_nnz_and_nca_hex_q1_closed_form(n, d):
    D, n_dofs = wl.hex_q1_grid(n, d)
    row_ptr, col_idx = oracle.csr_pattern(D, n_dofs)
    assert row_ptr[-1] == d * d * (3 * n + 1) ** 3
    _, col_align = oracle.crac_from_csr(row_ptr, col_idx, n_dofs)
    # natural numbering: one run per (y, z) neighbour pair, d DOFs merge;
    # for n >= 3 the x-run of one grid line never touches the next line's
    assert col_align.shape[0] == 2 * (d * (n + 1) * (3 * n + 1) ** 2 + 1)


@pytest.mark.parametrize("m,p", [(1, 2), (3, 2), (2, 3), (2, 5)])
def test_nnz_quad_qp_closed_form(m, p):
    D, n_dofs = wl.quad_qp_grid(m, p, 1)
    row_ptr, _ = oracle.csr_pattern(D, n_dofs)
    s = m * (p - 1) * (p + 1) + (m - 1) * (2 * p + 1) + 2 * (p + 1)
    assert row_ptr[-1] == s * s


def test_nnz_invariant_under_node_permutation():
    Dn, n_dofs = wl.tet_p2_kuhn(3, d=3, permute=False)
    Dp, _ = wl.tet_p2_kuhn(3, d=3, seed=7, permute=True)
    rn, cn = oracle.csr_pattern(Dn, n_dofs)
    rp, cp = oracle.csr_pattern(Dp, n_dofs)
    assert rn[-1] == rp[-1]
    assert np.array_equal(np.sort(np.diff(rn)), np.sort(np.diff(rp)))


# ------------------------------------------- values printed in the paper ---

_PAPER_ROWS = golden.structured_patterns()


def _mesh_for(row):
    if row["p"] == 1:
        return wl.quad_q1_grid(row["m"], row["d"])
    return wl.quad_qp_grid(row["m"], row["p"], row["d"])


_SMALL = [r for r in _PAPER_ROWS if r["nnz"] <= 6_000_000]
_LARGE = [r for r in _PAPER_ROWS if r["nnz"] > 6_000_000 and r["source"].startswith("nnz_table")]


@pytest.mark.parametrize("row", _SMALL, ids=lambda r: f"{r['source']}-m{r['m']}p{r['p']}d{r['d']}")
def test_paper_printed_nnz(row):
    D, n_dofs = _mesh_for(row)
    assert n_dofs == row["n_dofs"]
    row_ptr, _ = oracle.csr_pattern(D, n_dofs)
    assert row_ptr[-1] == row["nnz"]


@pytest.mark.slow
@pytest.mark.parametrize("row", _LARGE, ids=lambda r: f"{r['source']}-m{r['m']}p{r['p']}d{r['d']}")
def test_paper_printed_nnz_large(row):
    D, n_dofs = _mesh_for(row)
    assert n_dofs == row["n_dofs"]
    row_ptr, _ = oracle.csr_pattern(D, n_dofs)
    assert row_ptr[-1] == row["nnz"]


def _dscale(nca1, d):
    return 2 * (d * (nca1 // 2 - 1) + 1)


def test_paper_nca_obeys_d_scaling_reading():
    """The paper's own n_ca data fix two readings: one pair per maximal run
    plus ONE final pair, and a node's d DOFs forming runs that merge."""
    rows = {(r["source"], r["m"], r["p"], r["d"]): r for r in _PAPER_ROWS}
    n1 = rows[("dgamma", 192, 1, 1)]["n_ca"]
    for d in range(2, 9):
        assert rows[("dgamma", 192, 1, d)]["n_ca"] == _dscale(n1, d)
    un = golden.unstructured_nca()
    for d, ndofs, nnz, nca in un:
        assert nca == _dscale(un[0][3], d)
        assert nnz == d * d * un[0][2]
    for m in (6, 12, 24, 48, 96, 192):
        assert rows[("hgamma_d4", m, 1, 4)]["n_ca"] == _dscale(rows[("hgamma_d1", m, 1, 1)]["n_ca"], 4)


@pytest.mark.parametrize("mesh", ["quad", "qp", "tet"])
def test_oracle_nca_obeys_d_scaling(mesh):
    def build(d):
        if mesh == "quad":
            return wl.quad_q1_grid(5, d)
        if mesh == "qp":
            return wl.quad_qp_grid(3, 3, d)
        return wl.tet_p2_kuhn(2, d=d, seed=1)
    D1, n1 = build(1)
    r1, c1 = oracle.csr_pattern(D1, n1)
    _, ca1 = oracle.crac_from_csr(r1, c1, n1)
    for d in (2, 3, 4):
        Dd, nd = build(d)
        rd, cd = oracle.csr_pattern(Dd, nd)
        _, cad = oracle.crac_from_csr(rd, cd, nd)
        assert cad.shape[0] == _dscale(ca1.shape[0], d)
        assert rd[-1] == d * d * r1[-1]


# -------------------------------------------------- value invariants ---

def test_all_ones_gives_incidence_counts():
    """Paper's dummy element (all ones, §2.1): G_ij = #elements holding i and j."""
    D, n_dofs = wl.tet_p2_kuhn(2, d=1, seed=2)
    n_e, n_loc = D.shape
    row_ptr, col_idx, v = oracle.assemble(D, wl.ones_matrices(n_e, n_loc), n_dofs)
    sets = [set(map(int, D[e])) for e in range(n_e)]
    elems_of = [[] for _ in range(n_dofs)]
    for e, s in enumerate(sets):
        for i in s:
            elems_of[i].append(e)
    for i in range(n_dofs):
        for k in range(row_ptr[i], row_ptr[i + 1]):
            j = int(col_idx[k])
            assert v[k] == sum(1 for e in elems_of[i] if j in sets[e])


def test_laplace_q1_quad_closed_form_rows():
    """16 x 16 Q1 Laplace: interior rows 8/3 on the diagonal, -1/3 for the 8
    neighbours; every row sums to zero."""
    m = 16
    D, n_dofs = wl.quad_q1_grid(m, 1)
    K = wl.broadcast_matrices(wl.laplace_q1_quad(), D.shape[0])
    row_ptr, col_idx, v = oracle.assemble(D, K, n_dofs)
    assert row_ptr[-1] == 2401
    s = m + 1
    for j in range(1, m):
        for i in range(1, m):
            node = i + s * j
            a, b = row_ptr[node], row_ptr[node + 1]
            assert b - a == 9
            for k in range(a, b):
                exp = 8.0 / 3.0 if col_idx[k] == node else -1.0 / 3.0
                assert abs(v[k] - exp) <= 4e-16 * 8
    sums = np.add.reduceat(v, row_ptr[:-1])
    assert np.max(np.abs(sums)) <= 1e-14


def test_elasticity_translations_in_null_space_and_symmetry():
    n = 3
    D, n_dofs = wl.hex_q1_grid(n, 3)
    K = wl.broadcast_matrices(wl.elasticity_q1_hex(1.0 / n), D.shape[0], 1.0)
    row_ptr, col_idx, v = oracle.assemble(D, K, n_dofs)
    rows = np.repeat(np.arange(n_dofs), np.diff(row_ptr))
    for comp in range(3):
        t = np.zeros(n_dofs)
        t[comp::3] = 1.0
        y = np.zeros(n_dofs)
        np.add.at(y, rows, v * t[col_idx])
        assert np.max(np.abs(y)) <= 1e-13
    # bit symmetry: K is bit-symmetric and every slot is summed in the same element order
    lookup = {(int(rows[k]), int(col_idx[k])): v[k] for k in range(v.shape[0])}
    for (i, j), x in lookup.items():
        assert lookup[(j, i)] == x


def test_sum_of_values_equals_sum_of_entries():
    D, n_dofs = wl.tet_p2_kuhn(2, d=3, seed=5)
    n_e, n_loc = D.shape
    K = wl.random_spd_matrices(n_e, n_loc, seed=8)
    _, _, v = oracle.assemble(D, K, n_dofs)
    exact_v = math.fsum(v.tolist())
    exact_k = math.fsum(K.ravel().tolist())
    bound = K.size * 2.0 ** -53 * float(np.abs(K).sum())
    assert abs(exact_v - exact_k) <= bound


def test_crac_equals_csr_on_spd_p2_mesh():
    D, n_dofs = wl.tet_p2_kuhn(2, d=3, seed=12)
    K = wl.random_spd_matrices(D.shape[0], D.shape[1], seed=3)
    row_ptr, col_idx, v = oracle.assemble(D, K, n_dofs)
    crac_ptr, col_align = oracle.crac_from_csr(row_ptr, col_idx, n_dofs)
    v2 = oracle.assemble_crac(D, K, crac_ptr, col_align, col_idx.shape[0])
    assert np.array_equal(v, v2)


def test_lookup_round_trip_and_misses():
    D, n_dofs = wl.tet_p2_kuhn(2, d=2, seed=4)
    row_ptr, col_idx = oracle.csr_pattern(D, n_dofs)
    crac_ptr, col_align = oracle.crac_from_csr(row_ptr, col_idx, n_dofs)
    rng = np.random.default_rng(0)
    for i in rng.choice(n_dofs, 60, replace=False):
        present = set(col_idx[row_ptr[i]:row_ptr[i + 1]].tolist())
        for j in range(n_dofs):
            exp = oracle.csr_lookup(row_ptr, col_idx, i, j)
            assert (exp >= 0) == (j in present)
            if exp >= 0:
                assert col_idx[exp] == j
            assert oracle.crac_lookup(crac_ptr, col_align, i, j) == exp


def test_empty_rows_in_crac():
    D = np.array([[0, 1], [4, 5]], dtype=np.int32)  # DOFs 2, 3, 6 unused
    row_ptr, col_idx = oracle.csr_pattern(D, 7)
    assert row_ptr.tolist() == [0, 2, 4, 4, 4, 6, 8, 8]
    crac_ptr, col_align = oracle.crac_from_csr(row_ptr, col_idx, 7)
    assert crac_ptr.tolist() == [0, 2, 4, 4, 4, 6, 8, 8]
    assert col_align.tolist() == [0, 0, 0, 2, 4, 4, 4, 6, 7, 8]
    for i in (2, 3, 6):
        for j in range(7):
            assert oracle.crac_lookup(crac_ptr, col_align, i, j) == -1


def test_invalid_connectivity_rejected():
    with pytest.raises(oracle.OracleError, match="out of range"):
        oracle.csr_pattern(np.array([[0, 9]], dtype=np.int32), 5)
    with pytest.raises(oracle.OracleError, match="duplicate"):
        oracle.csr_pattern(np.array([[1, 2, 1]], dtype=np.int32), 5)
    with pytest.raises(oracle.OracleError, match="out of range"):
        oracle.csr_pattern(np.array([[-1, 2]], dtype=np.int32), 5)


# ----------------------------------------------------------- colouring ---

def test_greedy_colouring_structured_quads_four_equal_colours():
    """Structured quads: 4 colours of 25 % each (§4, colouring statistics)."""
    D, n_dofs = wl.quad_q1_grid(48, 1)
    k, colour = oracle.greedy_colouring(D, n_dofs)
    assert k == 4
    assert np.bincount(colour).tolist() == [D.shape[0] // 4] * 4


def test_greedy_colouring_is_proper_and_first_fit():
    D, n_dofs = wl.tet_p2_kuhn(2, d=1, seed=6)
    k, colour = oracle.greedy_colouring(D, n_dofs)
    sets = [set(map(int, row)) for row in D]
    for e in range(D.shape[0]):
        nb = {colour[f] for f in range(e) if sets[e] & sets[f]}
        assert colour[e] not in nb
        assert colour[e] == min(set(range(k + 1)) - nb)  # smallest free colour
        for f in range(D.shape[0]):
            if f != e and sets[e] & sets[f]:
                assert colour[f] != colour[e]


# -------------------------------------------------------------- SpMV ---

def test_spmv_matches_dense_product():
    D, n_dofs = wl.tet_p2_kuhn(2, d=2, seed=21)
    K = wl.random_matrices(D.shape[0], D.shape[1], seed=2)
    row_ptr, col_idx, v = oracle.assemble(D, K, n_dofs)
    A = np.zeros((n_dofs, n_dofs))
    rows = np.repeat(np.arange(n_dofs), np.diff(row_ptr))
    A[rows, col_idx] = v
    x = np.random.default_rng(1).standard_normal(n_dofs)
    y = oracle.spmv_csr(row_ptr, col_idx, v, x)
    np.testing.assert_allclose(y, A @ x, rtol=1e-12, atol=1e-12)
    crac_ptr, col_align = oracle.crac_from_csr(row_ptr, col_idx, n_dofs)
    assert np.array_equal(oracle.spmv_crac(crac_ptr, col_align, v, x), y)


# ---------------------------------------------------- element matrices ---

def test_laplace_q1_quad_matches_closed_form():
    exp = np.array([[4, -1, -2, -1], [-1, 4, -1, -2], [-2, -1, 4, -1], [-1, -2, -1, 4]]) / 6.0
    np.testing.assert_allclose(wl.laplace_q1_quad(), exp, atol=1e-15)


def test_elasticity_q1_hex_rigid_modes():
    h = 0.25
    K = wl.elasticity_q1_hex(h)
    X = np.array([[dx, dy, dz] for dz in (0, 1) for dy in (0, 1) for dx in (0, 1)], float) * h
    modes = []
    for c in range(3):
        t = np.zeros(24)
        t[c::3] = 1
        modes.append(t)
    for a, b in ((0, 1), (1, 2), (0, 2)):
        r = np.zeros(24)
        r[a::3] = -X[:, b]
        r[b::3] = X[:, a]
        modes.append(r)
    for mode in modes:
        assert np.max(np.abs(K @ mode)) <= 1e-14
    w = np.linalg.eigvalsh(K)
    assert np.sum(np.abs(w) < 1e-12) == 6 and w.min() > -1e-12
    np.testing.assert_allclose(wl.elasticity_q1_hex(2 * h), 2 * K, rtol=1e-13)


def test_laplace_q1_hex_row_sums():
    K = wl.laplace_q1_hex(0.5)
    assert np.max(np.abs(K.sum(axis=1))) <= 1e-15
    assert np.all(np.linalg.eigvalsh(K) > -1e-14)


def test_tet_p2_kuhn_counts():
    n = 3
    D, n_dofs = wl.tet_p2_kuhn(n, d=3, seed=0)
    assert D.shape == (6 * n ** 3, 30)
    assert n_dofs == 3 * (2 * n + 1) ** 3
    assert np.unique(D).shape[0] == n_dofs  # every half-lattice point is a P2 node
