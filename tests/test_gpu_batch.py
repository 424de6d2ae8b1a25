"""Batched assembly (one persistent launch over many meshes) against the
per-mesh path and the oracle: every schedule, both formats, both modes;
the autotuner; CUDA-graph replay with new element values."""

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


def _meshes():
    out = []
    for n in (3, 5, 8):
        out.append(wl.hex_q1_grid(n, 1) + (wl.laplace_q1_hex(1.0 / n),))
    for n in (2, 4, 6):
        out.append(wl.hex_q1_grid(n, 3) + (wl.elasticity_q1_hex(1.0 / n),))
    out.append(wl.tet_p2_kuhn(2, d=3, seed=3) + (None,))     # 30 x 30, runs vary per element
    out.append(wl.quad_qp_grid(3, 3, 1) + (None,))           # 16 x 16, no specialised kernel
    out.append(wl.quad_q1_grid(5, 1) + (wl.laplace_q1_quad(),))
    out.append(wl.quad_qp_grid(2, 8, 1) + (None,))           # rows over 256: 16-bit maps
    return out


@pytest.fixture(scope="module")
def batch(ctx):
    import torch
    from paper_2012_00585_gb300 import feasm
    rows = []
    for k, (D, n_dofs, Kr) in enumerate(_meshes()):
        if Kr is None:
            K = wl.random_matrices(D.shape[0], D.shape[1], seed=k)
        else:
            K = wl.scaled_matrices(Kr, D.shape[0], seed=k)
        pat = feasm.Pattern(ctx, torch.from_numpy(D).cuda(), n_dofs)
        rp, ci = oracle.csr_pattern(D, n_dofs)
        v_o = oracle.assemble_csr(D, K, rp, ci)
        tau = gu.row_tolerance(rp, v_o, gu.contribution_abs_row_sums(D, K, n_dofs))
        rows.append(dict(D=D, n_dofs=n_dofs, K=K, Kd=torch.from_numpy(K).cuda(), pat=pat, rp=rp, v_o=v_o, tau=tau,
                         v=torch.empty(pat.info["nnz"], dtype=torch.float64, device="cuda")))
    yield rows
    for r in rows:
        r["pat"].free()


def _items(rows):
    return [(r["pat"], r["Kd"], r["v"]) for r in rows]


def _check(rows, mode):
    from paper_2012_00585_gb300 import feasm
    for r in rows:
        got = r["v"].cpu().numpy()
        if mode == feasm.FE_DETERMINISTIC:
            assert np.array_equal(got.view(np.uint64), r["v_o"].view(np.uint64))
        else:
            gu.assert_within_row_tol(r["rp"], got, r["v_o"], r["tau"])


@pytest.mark.parametrize("fmt", [0, 1])
@pytest.mark.parametrize("sched", [(4, 1), (4, 16), (4, 64)])
def test_batch_deterministic_bit_exact(ctx, batch, fmt, sched):
    import torch
    from paper_2012_00585_gb300 import feasm
    for r in batch:
        r["v"].fill_(float("nan"))
    feasm.fe_assemble_batch(ctx, _items(batch), fmt, feasm.FE_DETERMINISTIC, 0, sched)
    torch.cuda.synchronize()
    _check(batch, feasm.FE_DETERMINISTIC)


@pytest.mark.parametrize("fmt", [0, 1])
@pytest.mark.parametrize("sched", [(1, 1), (1, 16), (2, 1), (2, 4), (3, 1), (3, 4), (5, 1), (5, 16), (5, 64)])
def test_batch_atomic_schedules(ctx, batch, fmt, sched):
    import torch
    from paper_2012_00585_gb300 import feasm
    for r in batch:
        r["v"].fill_(float("nan"))
    feasm.fe_assemble_batch(ctx, _items(batch), fmt, feasm.FE_ATOMIC, 0, sched)
    torch.cuda.synchronize()
    _check(batch, feasm.FE_ATOMIC)


def test_batch_accumulate_and_bad_schedule(ctx, batch):
    import torch
    from paper_2012_00585_gb300 import feasm
    feasm.fe_assemble_batch(ctx, _items(batch), 0, feasm.FE_DETERMINISTIC)
    feasm.fe_assemble_batch(ctx, _items(batch), 0, feasm.FE_DETERMINISTIC, accumulate=1)
    torch.cuda.synchronize()
    for r in batch:
        exp = oracle.assemble_csr(r["D"], r["K"], r["rp"], oracle.csr_pattern(r["D"], r["n_dofs"])[1], values=r["v_o"])
        assert np.array_equal(r["v"].cpu().numpy(), exp)
    with pytest.raises(feasm.FeError):
        feasm.fe_assemble_batch(ctx, _items(batch), 0, feasm.FE_DETERMINISTIC, 0, (1, 16))  # atomic-only kind
    with pytest.raises(feasm.FeError):
        feasm.fe_assemble_batch(ctx, _items(batch), 0, feasm.FE_ATOMIC, 0, (1, 0))  # tile 0


@pytest.mark.parametrize("mode", [0, 1])
def test_autotune_then_default_uses_it(ctx, batch, mode):
    import torch
    from paper_2012_00585_gb300 import feasm
    kind, tile, ms = feasm.fe_batch_autotune(ctx, _items(batch), 0, mode)
    assert ms > 0 and tile >= 1
    assert kind == feasm.FE_SCHED_WARP_PER_ROW if mode == 1 else kind in (1, 2, 3, 5)
    for r in batch:
        r["v"].fill_(float("nan"))
    feasm.fe_assemble_batch(ctx, _items(batch), 0, mode)
    torch.cuda.synchronize()
    _check(batch, mode)


@pytest.mark.parametrize("mode", [0, 1])
def test_graph_replay_with_new_values(ctx, batch, mode):
    import torch
    from paper_2012_00585_gb300 import feasm
    g = feasm.fe_batch_graph_create(ctx, _items(batch), 1, mode)
    try:
        for rep in range(2):
            # new element values in the same buffers, then replay
            for k, r in enumerate(batch):
                K2 = wl.random_matrices(r["D"].shape[0], r["D"].shape[1], seed=100 + 10 * rep + k)
                r["Kd"].copy_(torch.from_numpy(K2))
                r["K2"] = K2
                r["v"].fill_(float("nan"))
            feasm.fe_batch_graph_launch(g)
            torch.cuda.synchronize()
            for r in batch:
                rp, ci = oracle.csr_pattern(r["D"], r["n_dofs"])
                exp = oracle.assemble_csr(r["D"], r["K2"], rp, ci)
                got = r["v"].cpu().numpy()
                if mode == 1:
                    assert np.array_equal(got, exp)
                else:
                    tau = gu.row_tolerance(rp, exp, gu.contribution_abs_row_sums(r["D"], r["K2"], r["n_dofs"]))
                    gu.assert_within_row_tol(rp, got, exp, tau)
    finally:
        feasm.fe_batch_graph_destroy(g)
        for r in batch:  # restore the module's K for other tests
            r["Kd"].copy_(torch.from_numpy(r["K"]))


@pytest.mark.parametrize("fmt", [0, 1])
def test_batch_staged_schedule_with_unaligned_matrices(ctx, batch, fmt):
    """A K buffer that is only 8-byte aligned cannot be moved by bulk copies:
    that item takes the warp-per-element path inside the same launch, and the
    result is unchanged."""
    import torch
    from paper_2012_00585_gb300 import feasm
    items = _items(batch)
    r = batch[4]  # hex 4^3, d = 3 (24 x 24)
    buf = torch.empty(r["Kd"].numel() + 1, dtype=torch.float64, device="cuda")
    k_odd = buf[1:].view(r["Kd"].shape)
    k_odd.copy_(r["Kd"])
    assert k_odd.data_ptr() % 16 == 8
    items[4] = (r["pat"], k_odd, r["v"])
    feasm.fe_assemble_batch(ctx, items, fmt, feasm.FE_ATOMIC, 0, (feasm.FE_SCHED_WARP_PER_ELEMENT_TMA, 8))
    _check(batch, feasm.FE_ATOMIC)
    assert feasm.fe_device_status(ctx) == 0


@pytest.mark.slow
@pytest.mark.parametrize("mode", [0, 1])
def test_batch_full_size_sampled(ctx, mode):
    """The batched workload at full size in the bench's launch configuration
    (256 hex meshes, n ~ logU[8, 48], half Q1 Laplace and half Q1 elasticity,
    autotuned schedule, one CUDA-graph launch): sampled meshes -- the two
    largest and the two smallest of each kind -- against the oracle."""
    import torch
    from paper_2012_00585_gb300 import feasm
    sizes = wl.batched_mesh_sizes(256, seed=0)
    rows = []
    for k, (n, d) in enumerate(sizes):
        D, n_dofs = wl.hex_q1_grid(n, d)
        Kr = wl.laplace_q1_hex(1.0 / n) if d == 1 else wl.elasticity_q1_hex(1.0 / n)
        Kd = wl.scaled_matrices(Kr, D.shape[0], seed=k, device="cuda")
        pat = feasm.Pattern(ctx, torch.from_numpy(D).cuda(), n_dofs)
        v = torch.empty(pat.info["nnz"], dtype=torch.float64, device="cuda")
        rows.append((k, n, d, D, n_dofs, Kd, pat, v))
    items = [(r[6], r[5], r[7]) for r in rows]
    feasm.fe_batch_autotune(ctx, items, feasm.FE_FORMAT_CSR, mode)
    g = feasm.fe_batch_graph_create(ctx, items, feasm.FE_FORMAT_CSR, mode)
    for _, _, _, _, _, _, _, v in rows:
        v.fill_(float("nan"))
    feasm.fe_batch_graph_launch(g)
    torch.cuda.synchronize()
    assert feasm.fe_device_status(ctx) == 0
    picks = []
    for d in (1, 3):
        kind = sorted((r for r in rows if r[2] == d), key=lambda r: r[1])
        picks += kind[:2] + kind[-2:]
    for k, n, d, D, n_dofs, Kd, pat, v in picks:
        K = Kd.cpu().numpy()
        rp, ci = oracle.csr_pattern(D, n_dofs)
        exp = oracle.assemble_csr(D, K, rp, ci)
        got = v.cpu().numpy()
        if mode == feasm.FE_DETERMINISTIC:
            assert np.array_equal(got.view(np.uint64), exp.view(np.uint64)), (k, n, d)
        else:
            gu.assert_within_row_tol(rp, got, exp, gu.row_tolerance(rp, exp, gu.contribution_abs_row_sums(D, K, n_dofs)))
    feasm.fe_batch_graph_destroy(g)
    for r in rows:
        r[6].free()


def test_tune_cache_file(tmp_path, monkeypatch):
    """With FEASM_TUNE_CACHE naming a file, the autotuner's result reaches a
    context created later (as in another process): the file holds one line
    per result keyed by GPU model, SM count and batch signature; a line edited
    by hand is what a new context then takes; without the variable nothing is
    known."""
    import torch
    from paper_2012_00585_gb300 import feasm
    path = tmp_path / "tune.txt"
    monkeypatch.setenv("FEASM_TUNE_CACHE", str(path))
    c1 = feasm.fe_create(0)
    pats, items = [], []
    try:
        for n, d in ((4, 3), (6, 1)):
            D, n_dofs = wl.hex_q1_grid(n, d)
            Kr = wl.laplace_q1_hex(1.0 / n) if d == 1 else wl.elasticity_q1_hex(1.0 / n)
            p = feasm.Pattern(c1, torch.from_numpy(D).cuda(), n_dofs)
            pats.append(p)
            items.append((p, torch.from_numpy(wl.scaled_matrices(Kr, D.shape[0], seed=n)).cuda(),
                          torch.empty(p.info["nnz"], dtype=torch.float64, device="cuda")))
        assert feasm.fe_batch_tuned(c1, items, 0, feasm.FE_ATOMIC) is None
        kind, tile, _ = feasm.fe_batch_autotune(c1, items, 0, feasm.FE_ATOMIC)
        assert feasm.fe_batch_tuned(c1, items, 0, feasm.FE_ATOMIC) == (kind, tile)
        lines = path.read_text().splitlines()
        assert len(lines) == 1 and lines[0].split()[-2:] == [str(kind), str(tile)]
        c2 = feasm.fe_create(0)
        assert feasm.fe_batch_tuned(c2, items, 0, feasm.FE_ATOMIC) == (kind, tile)
        assert feasm.fe_batch_tuned(c2, items, 0, feasm.FE_DETERMINISTIC) is None
        feasm.fe_destroy(c2)
        f = lines[0].split()
        path.write_text(" ".join(f[:-2] + [str(feasm.FE_SCHED_WARP_PER_ELEMENT), "3"]) + "\n")
        c3 = feasm.fe_create(0)
        assert feasm.fe_batch_tuned(c3, items, 0, feasm.FE_ATOMIC) == (feasm.FE_SCHED_WARP_PER_ELEMENT, 3)
        feasm.fe_destroy(c3)
        monkeypatch.delenv("FEASM_TUNE_CACHE")
        c4 = feasm.fe_create(0)
        assert feasm.fe_batch_tuned(c4, items, 0, feasm.FE_ATOMIC) is None
        feasm.fe_destroy(c4)
    finally:
        for p in pats:
            p.free()
        feasm.fe_destroy(c1)


@pytest.mark.parametrize("mode", [0, 1])
def test_per_item_timestamps(ctx, batch, mode):
    """With a times array per item, one batched launch (and its graph replay)
    records when each item's first tile started and its last tile finished:
    every item gets both, start <= finish, all within the launch, and the
    results are unchanged."""
    import torch
    from paper_2012_00585_gb300 import feasm
    times = torch.zeros((len(batch), 2), dtype=torch.int64, device="cuda")
    items = [(r["pat"], r["Kd"], r["v"], times[k]) for k, r in enumerate(batch)]
    for launch in ("direct", "graph"):
        times.zero_()
        for r in batch:
            r["v"].fill_(float("nan"))
        if launch == "direct":
            feasm.fe_assemble_batch(ctx, items, 0, mode)
        else:
            g = feasm.fe_batch_graph_create(ctx, items, 0, mode)
            feasm.fe_batch_graph_launch(g)
        torch.cuda.synchronize()
        t = times.cpu().numpy()
        assert np.all(t[:, 0] > 0) and np.all(t[:, 1] >= t[:, 0])
        assert t[:, 1].max() - t[:, 0].min() < 10 * 10 ** 9  # one launch, well under 10 s
        _check(batch, mode)
        if launch == "graph":
            feasm.fe_batch_graph_destroy(g)
