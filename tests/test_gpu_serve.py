"""Serving loop: results served alone and in a mix equal the oracle's
assembly of the same element values (bit for bit in deterministic mode,
within the row tolerance in atomic mode), at small sizes and in a trace of
the served workload's real sizes (meshes of the batched size distribution
and a 128^3 elasticity request); admission, cancellation, deadlines and bad
input fail cleanly while the server keeps serving; the element-value
generator matches its published definition."""

import numpy as np
import pytest

import oracle
import workloads as wl
from tests import gpu_util as gu

pytestmark = pytest.mark.gpu

M64 = (1 << 64) - 1


def splitmix64(x):
    """Steele, Lea & Flood's SplitMix64 step with Vigna's 64-bit finaliser."""
    x = (x + 0x9E3779B97F4A7C15) & M64
    x = ((x ^ (x >> 30)) * 0xBF58476D1CE4E5B9) & M64
    x = ((x ^ (x >> 27)) * 0x94D049BB133111EB) & M64
    return x ^ (x >> 31)


def alphas(seed, n_e):
    return np.array([0.5 + (splitmix64((seed + e) & M64) >> 44) / 2.0 ** 20 for e in range(n_e)])


@pytest.fixture(scope="module")
def ctx():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2012_00585_gb300 import feasm
    c = feasm.fe_create(0)
    yield c
    feasm.fe_destroy(c)


def test_generator_matches_definition(ctx):
    import torch
    from paper_2012_00585_gb300 import feasm
    Kr = wl.elasticity_q1_hex(0.25)
    Krd = torch.from_numpy(Kr).cuda()
    n_e = 37
    out = torch.empty((n_e, 24, 24), dtype=torch.float64, device="cuda")
    seed = 0xDEADBEEF12345678
    feasm.fe_generate_scaled(ctx, Krd, 24, n_e, seed, out)
    torch.cuda.synchronize()
    exp = alphas(seed, n_e)[:, None, None] * Kr[None]
    assert np.array_equal(out.cpu().numpy(), exp)


def _mesh_set():
    out = []
    for k, (n, d) in enumerate([(4, 1), (6, 3), (3, 3), (7, 1), (5, 3)]):
        D, n_dofs = wl.hex_q1_grid(n, d)
        Kr = wl.laplace_q1_hex(1.0 / n) if d == 1 else wl.elasticity_q1_hex(1.0 / n)
        out.append((1000 + k, D, n_dofs, Kr))
    return out


def _oracle_values(D, n_dofs, Kr, seed):
    """The oracle's assembly of K_e = alpha_e * K_ref (alpha_e from the
    generator's published definition, computed here on the host)."""
    K = alphas(seed, D.shape[0])[:, None, None] * Kr[None]
    rp, ci = oracle.csr_pattern(D, n_dofs)
    return rp, ci, oracle.assemble_csr(D, K, rp, ci), K


def _pattern_of(fe, res, n_dofs):
    import torch
    rp = fe.device_view(res["row_ptr"], n_dofs + 1, torch.int64).cpu().numpy()
    ci = fe.device_view(res["col_idx"], res["nnz"], torch.int32).cpu().numpy()
    return rp, ci


def _values_of(fe, res):
    import torch
    return fe.device_view(res["values"], res["nnz"], torch.float64).cpu().numpy()


@pytest.mark.parametrize("mode", [0, 1])
def test_same_result_alone_and_in_the_mix(ctx, mode):
    import torch
    from paper_2012_00585_gb300 import feasm as fe
    sv = fe.fe_server_start(ctx, n_streams=3, max_batch=8, hbm_budget_bytes=2 << 30)
    try:
        meshes = _mesh_set()
        dev = {key: (torch.from_numpy(D).cuda(), torch.from_numpy(Kr).cuda(), n_dofs, D, Kr)
               for key, D, n_dofs, Kr in meshes}
        # alone: one request, waited for
        key0 = meshes[1][0]
        Dd, Krd, n_dofs, D, Kr = dev[key0]
        r = fe.make_request(key0, Dd, n_dofs, k_ref=Krd, seed=77, fmt=1, mode=mode)
        (t,) = fe.fe_batch_submit(sv, [r])
        res = fe.fe_wait(sv, t, 60)
        assert res["state"] == fe.FE_STATE_DONE and res["cold"] == 1
        alone = _values_of(fe, res)
        fe.fe_release(sv, t)
        # in the mix: 40 requests over 5 meshes, the same one among them
        reqs, meta = [], []
        for k in range(40):
            key, D, n_dofs, Kr = meshes[k % len(meshes)]
            seed = 77 if key == key0 and k == 21 else 1000 + k
            Dd, Krd, _, _, _ = dev[key]
            reqs.append(fe.make_request(key, Dd, n_dofs, k_ref=Krd, seed=seed, fmt=1, mode=mode))
            meta.append((key, seed))
        tickets = fe.fe_batch_submit(sv, reqs)
        for t, (key, seed) in zip(tickets, meta):
            res = fe.fe_wait(sv, t, 60)
            assert res["state"] == fe.FE_STATE_DONE, res
            got = _values_of(fe, res)
            _, Krd, n_dofs, D, Kr = dev[key]
            rp, ci, v_o, K = _oracle_values(D, n_dofs, Kr, seed)
            rp_g, ci_g = _pattern_of(fe, res, n_dofs)
            assert np.array_equal(rp_g, rp) and np.array_equal(ci_g, ci)
            if mode == fe.FE_DETERMINISTIC:
                assert np.array_equal(got.view(np.uint64), v_o.view(np.uint64))  # Listing 2's order, bit for bit
                if key == key0 and seed == 77:
                    assert np.array_equal(got, alone)  # alone == in the mix, bit for bit
            else:
                tau = gu.row_tolerance(rp, v_o, gu.contribution_abs_row_sums(D, K, n_dofs))
                gu.assert_within_row_tol(rp, got, v_o, tau)
                if key == key0 and seed == 77:
                    gu.assert_within_row_tol(rp, got, alone, 2 * tau)
            fe.fe_release(sv, t)
        st = fe.fe_server_stats_get(sv)
        assert st["completed"] == 41 and st["patterns_built"] == 5  # warm requests skip the symbolic phase
        assert st["launches"] < 41  # requests shared launches
    finally:
        fe.fe_server_stop(sv)


def test_admission_cancel_and_bad_input(ctx):
    import torch
    from paper_2012_00585_gb300 import feasm as fe
    D, n_dofs = wl.hex_q1_grid(6, 3)
    Dd = torch.from_numpy(D).cuda()
    Krd = torch.from_numpy(wl.elasticity_q1_hex(1 / 6)).cuda()
    # a budget too small for this request: it fails with an admission error
    sv = fe.fe_server_start(ctx, 1, 4, hbm_budget_bytes=1 << 20)
    try:
        (t,) = fe.fe_batch_submit(sv, [fe.make_request(1, Dd, n_dofs, k_ref=Krd, seed=1)])
        res = fe.fe_wait(sv, t, 30)
        assert res["state"] == fe.FE_STATE_FAILED and res["status"] == fe.FE_ERR_ADMISSION
        fe.fe_release(sv, t)
    finally:
        fe.fe_server_stop(sv)
    # strict FIFO (one request at a time): later ones stay pending; cancel one
    sv = fe.fe_server_start(ctx, 1, 1, hbm_budget_bytes=40 << 20)
    try:
        reqs = [fe.make_request(2, Dd, n_dofs, k_ref=Krd, seed=s) for s in range(6)]
        tickets = fe.fe_batch_submit(sv, reqs)
        cancelled = None
        for t in reversed(tickets):
            try:
                fe.fe_cancel(sv, t)
                cancelled = t
                break
            except fe.FeError:
                continue
        assert cancelled is not None
        for t in tickets:
            res = fe.fe_wait(sv, t, 60)
            if t == cancelled:
                assert res["state"] == fe.FE_STATE_CANCELLED and res["status"] == fe.FE_ERR_CANCELLED
            else:
                assert res["state"] == fe.FE_STATE_DONE
            fe.fe_release(sv, t)
        # bad connectivity: that request fails, the next one is served
        bad = Dd.clone()
        bad[3, 2] = n_dofs + 5
        t_bad, t_ok = fe.fe_batch_submit(sv, [fe.make_request(3, bad, n_dofs, k_ref=Krd, seed=9),
                                              fe.make_request(2, Dd, n_dofs, k_ref=Krd, seed=10)])
        r_bad = fe.fe_wait(sv, t_bad, 60)
        r_ok = fe.fe_wait(sv, t_ok, 60)
        assert r_bad["state"] == fe.FE_STATE_FAILED and r_bad["status"] == fe.FE_ERR_DOF_RANGE
        assert r_ok["state"] == fe.FE_STATE_DONE
        fe.fe_release(sv, t_bad)
        fe.fe_release(sv, t_ok)
    finally:
        fe.fe_server_stop(sv)


def _alphas_at(seed, els):
    return np.array([0.5 + (splitmix64((seed + int(e)) & M64) >> 44) / 2.0 ** 20 for e in els])


def _check_served_rows(fe, res, D, n_dofs, Kr, seed, rows, mode):
    """Rows `rows` of a served result against the oracle run on the sub-mesh
    of the elements touching them, in ascending element order (which leaves
    those rows' sums and their order unchanged)."""
    import torch
    els = np.nonzero(np.isin(D, rows).any(axis=1))[0]
    Dsub = np.ascontiguousarray(D[els])
    Ksub = _alphas_at(seed, els)[:, None, None] * Kr[None]
    rp_o, ci_o = oracle.csr_pattern(Dsub, n_dofs)
    v_o = oracle.assemble_csr(Dsub, Ksub, rp_o, ci_o)
    rp = fe.device_view(res["row_ptr"], n_dofs + 1, torch.int64)
    ci = fe.device_view(res["col_idx"], res["nnz"], torch.int32)
    v = fe.device_view(res["values"], res["nnz"], torch.float64)
    rp_h = rp.cpu().numpy()
    assert rp_h[-1] == res["nnz"] and np.all(np.diff(rp_h) >= 0)
    for i in rows:
        a, b = int(rp_h[i]), int(rp_h[i + 1])
        ao, bo = int(rp_o[i]), int(rp_o[i + 1])
        assert np.array_equal(ci[a:b].cpu().numpy(), ci_o[ao:bo])
        got, exp = v[a:b].cpu().numpy(), v_o[ao:bo]
        if mode == FE_DET:
            assert np.array_equal(got.view(np.uint64), exp.view(np.uint64)), i
        else:
            assert np.all(np.abs(got - exp) <= 1e-12 * np.abs(exp).sum()), i


FE_DET = 1


@pytest.mark.slow
@pytest.mark.parametrize("mode", [0, 1])
def test_served_real_sizes_alone_and_in_the_mix(ctx, mode):
    """A trace at the served workload's real sizes: 24 hex meshes from the
    batched size distribution (n ~ logU[8, 48], half Q1 Laplace, half Q1
    elasticity) and a 128^3 Q1 elasticity request (6,440,067 DOFs, 1.21e9
    entries, K generated on the device after admission: 9.7 GB).  The large
    request is served alone (cold: its pattern is built), then again with the
    same seed inside the mix (warm: numeric only).  Deterministic mode: the two
    results are equal bit for bit, and sampled rows of every result equal the
    oracle's; atomic mode: within the row tolerance.  Meshes up to n = 20 are
    checked whole, larger ones on sampled rows."""
    import torch
    from paper_2012_00585_gb300 import feasm as fe
    rng = np.random.default_rng(5)
    D_big, n_big = wl.hex_q1_grid(128, 3)
    Kr_big = wl.elasticity_q1_hex(1.0 / 128)
    big = (torch.from_numpy(D_big).cuda(), torch.from_numpy(Kr_big).cuda())
    rows_big = np.unique(np.concatenate([rng.choice(n_big, 40, replace=False), [0, n_big - 1]]))
    small = []
    for k, (n, d) in enumerate(wl.batched_mesh_sizes(24, seed=3)):
        D, n_dofs = wl.hex_q1_grid(n, d)
        Kr = wl.laplace_q1_hex(1.0 / n) if d == 1 else wl.elasticity_q1_hex(1.0 / n)
        small.append((100 + k, D, n_dofs, Kr, torch.from_numpy(D).cuda(), torch.from_numpy(Kr).cuda()))
    sv = fe.fe_server_start(ctx, n_streams=4, max_batch=8, hbm_budget_bytes=0)
    try:
        (t_alone,) = fe.fe_batch_submit(sv, [fe.make_request(7, big[0], n_big, k_ref=big[1], seed=4242, mode=mode)])
        r_alone = fe.fe_wait(sv, t_alone, 300)
        assert r_alone["state"] == fe.FE_STATE_DONE and r_alone["cold"] == 1, r_alone
        reqs = [fe.make_request(key, Dd, n_dofs, k_ref=Krd, seed=900 + key, mode=mode)
                for key, _, n_dofs, _, Dd, Krd in small]
        reqs.insert(len(reqs) // 2, fe.make_request(7, big[0], n_big, k_ref=big[1], seed=4242, mode=mode))
        tickets = fe.fe_batch_submit(sv, reqs)
        results = [fe.fe_wait(sv, t, 300) for t in tickets]
        assert all(r["state"] == fe.FE_STATE_DONE for r in results), [r["status"] for r in results]
        r_mix = results[len(reqs) // 2]
        assert r_mix["cold"] == 0  # the cached pattern was reused
        v_alone = fe.device_view(r_alone["values"], r_alone["nnz"], torch.float64)
        v_mix = fe.device_view(r_mix["values"], r_mix["nnz"], torch.float64)
        if mode == FE_DET:
            assert torch.equal(v_alone.view(torch.int64), v_mix.view(torch.int64))
        else:
            assert float((v_alone - v_mix).abs().max()) <= 2e-12 * float(v_alone.abs().max()) * 81
        for r in (r_alone, r_mix):
            _check_served_rows(fe, r, D_big, n_big, Kr_big, 4242, rows_big, mode)
        del v_alone, v_mix
        small_results = results[:len(reqs) // 2] + results[len(reqs) // 2 + 1:]
        for (key, D, n_dofs, Kr, _, _), r in zip(small, small_results):
            n = round(D.shape[0] ** (1 / 3))
            if n <= 20:
                rp, ci, v_o, K = _oracle_values(D, n_dofs, Kr, 900 + key)
                rp_g, ci_g = _pattern_of(fe, r, n_dofs)
                assert np.array_equal(rp_g, rp) and np.array_equal(ci_g, ci)
                got = _values_of(fe, r)
                if mode == FE_DET:
                    assert np.array_equal(got.view(np.uint64), v_o.view(np.uint64))
                else:
                    tau = gu.row_tolerance(rp, v_o, gu.contribution_abs_row_sums(D, K, n_dofs))
                    gu.assert_within_row_tol(rp, got, v_o, tau)
            else:
                rows = np.unique(np.concatenate([rng.choice(n_dofs, 12, replace=False), [0, n_dofs - 1]]))
                _check_served_rows(fe, r, D, n_dofs, Kr, 900 + key, rows, mode)
        for t in [t_alone] + tickets:
            fe.fe_release(sv, t)
        st = fe.fe_server_stats_get(sv)
        assert st["patterns_built"] == 25 and st["completed"] == 26
        assert fe.fe_device_status(ctx) == 0
    finally:
        fe.fe_server_stop(sv)
        torch.cuda.empty_cache()


def test_deadline_watchdog(ctx):
    """A request that cannot be launched before its deadline (it queues
    behind others on a strict-FIFO server) fails with FE_ERR_TIMEOUT and
    gives its memory back; requests with no deadline or a generous one
    complete exactly, and the server keeps serving."""
    import torch
    from paper_2012_00585_gb300 import feasm as fe
    D, n_dofs = wl.hex_q1_grid(8, 3)
    Kr = wl.elasticity_q1_hex(1 / 8)
    Dd, Krd = torch.from_numpy(D).cuda(), torch.from_numpy(Kr).cuda()
    sv = fe.fe_server_start(ctx, 1, 1, hbm_budget_bytes=1 << 30)
    try:
        deadlines = [0.0, 0.0, 0.0, 1e-6, 0.0, 60.0]
        reqs = [fe.make_request(5, Dd, n_dofs, k_ref=Krd, seed=10 + k, deadline_s=dl)
                for k, dl in enumerate(deadlines)]
        tickets = fe.fe_batch_submit(sv, reqs)
        for k, t in enumerate(tickets):
            res = fe.fe_wait(sv, t, 60)
            if deadlines[k] == 1e-6:
                assert res["state"] == fe.FE_STATE_FAILED and res["status"] == fe.FE_ERR_TIMEOUT, res
            else:
                assert res["state"] == fe.FE_STATE_DONE, res
                rp, ci, v_o, _ = _oracle_values(D, n_dofs, Kr, 10 + k)
                assert np.array_equal(_values_of(fe, res).view(np.uint64), v_o.view(np.uint64))
            fe.fe_release(sv, t)
        st = fe.fe_server_stats_get(sv)
        assert st["expired"] == 1 and st["completed"] == 5
    finally:
        fe.fe_server_stop(sv)
    with pytest.raises(fe.FeError):
        sv2 = fe.fe_server_start(ctx, 1, 1, hbm_budget_bytes=1 << 30)
        try:
            fe.fe_batch_submit(sv2, [fe.make_request(5, Dd, n_dofs, k_ref=Krd, seed=1, deadline_s=-1.0)])
        finally:
            fe.fe_server_stop(sv2)


def test_timeline_and_one_off_eviction(ctx):
    """The device timeline lists every launched group and build with
    non-negative durations; a budget that holds only a few patterns evicts
    one-off meshes before a mesh that is reassembled repeatedly (which is then
    never rebuilt)."""
    import torch
    from paper_2012_00585_gb300 import feasm as fe
    D, n_dofs = wl.hex_q1_grid(10, 3)
    Kr = wl.elasticity_q1_hex(1 / 10)
    Dd, Krd = torch.from_numpy(D).cuda(), torch.from_numpy(Kr).cuda()
    probe = fe.Pattern(ctx, Dd, n_dofs)
    pat_bytes, nnz = probe.info["device_bytes"], probe.info["nnz"]
    probe.free()
    n_e, n_loc = D.shape
    # the server's admission charge for a request on an uncached mesh: its K,
    # an upper bound of its values (nnz <= entries) and of its pattern
    cold_need = 2 * n_e * n_loc * n_loc * 8 + n_e * n_loc * n_loc * 6 + n_dofs * 64 + (1 << 20)
    # room for the cold request plus about four cached patterns
    sv = fe.fe_server_start(ctx, 2, 4, hbm_budget_bytes=cold_need + 4 * pat_bytes + nnz * 8)
    try:
        hot = 1
        order = [hot, hot]
        for r in range(3):
            order += [1000 + 10 * r + k for k in range(6)] + [hot]
        for k, key in enumerate(order):
            (t,) = fe.fe_batch_submit(sv, [fe.make_request(key, Dd, n_dofs, k_ref=Krd, seed=k)])
            res = fe.fe_wait(sv, t, 60)
            assert res["state"] == fe.FE_STATE_DONE, res
            fe.fe_release(sv, t)
        st = fe.fe_server_stats_get(sv)
        # more one-off meshes than the budget holds: they are evicted, the hot one never
        assert st["evictions"] >= 10 and st["rebuilds"] == 0
        assert st["patterns_built"] == 19  # the hot mesh once, each one-off mesh once
        spans = fe.fe_server_timeline(sv)
        launches = [s for s in spans if s[2] >= 0]
        builds = [s for s in spans if s[2] == -1]
        assert len(launches) == st["launches"] == len(order) and len(builds) == 19
        assert all(0 <= a <= b for a, b, _, _ in spans)
    finally:
        fe.fe_server_stop(sv)


def test_small_request_passes_a_waiting_large_one(ctx):
    """Admission keeps arrival order, except that a small request may pass a
    large one waiting for memory.  Request A holds its memory on the GPU (its
    assembly waits for an event recorded after a bounded sleep kernel on
    another stream); B, as large and on a new mesh, cannot fit beside A and
    waits; S, tiny, arrives after B and completes while B is still waiting.
    Then A, B and S are all exact."""
    import torch
    from paper_2012_00585_gb300 import feasm as fe
    D, n_dofs = wl.hex_q1_grid(20, 3)
    Kr = wl.elasticity_q1_hex(1 / 20)
    Dd, Krd = torch.from_numpy(D).cuda(), torch.from_numpy(Kr).cuda()
    Ds, ns = wl.hex_q1_grid(3, 1)
    Krs = wl.laplace_q1_hex(1 / 3)
    Dsd, Krsd = torch.from_numpy(Ds).cuda(), torch.from_numpy(Krs).cuda()
    n_e, n_loc = D.shape
    # the server's charge for a request on a new mesh: K, values bound, pattern bound
    need = 2 * n_e * n_loc * n_loc * 8 + n_e * n_loc * n_loc * 6 + n_dofs * 64 + (1 << 20)
    sv = fe.fe_server_start(ctx, 4, 8, hbm_budget_bytes=int(1.3 * need))
    try:
        side = torch.cuda.Stream()
        ev = torch.cuda.Event()
        with torch.cuda.stream(side):
            for _ in range(3):  # about 2.2 s at GB300 clocks (3 x 1.5e9 cycles): S is done long before
                torch.cuda._sleep(int(1.5e9))
            ev.record(side)
        (ta,) = fe.fe_batch_submit(sv, [fe.make_request(1, Dd, n_dofs, k_ref=Krd, seed=1, ready_event=ev)])
        (tb,) = fe.fe_batch_submit(sv, [fe.make_request(2, Dd, n_dofs, k_ref=Krd, seed=2)])
        (ts,) = fe.fe_batch_submit(sv, [fe.make_request(3, Dsd, ns, k_ref=Krsd, seed=3)])
        rs = fe.fe_wait(sv, ts, 30)
        rb = fe.fe_poll(sv, tb)
        assert rs["state"] == fe.FE_STATE_DONE
        assert rb["state"] == fe.FE_STATE_PENDING  # still waiting for A's memory
        for t, (DD, nd, KR, seed) in ((ta, (D, n_dofs, Kr, 1)), (tb, (D, n_dofs, Kr, 2)), (ts, (Ds, ns, Krs, 3))):
            r = fe.fe_wait(sv, t, 60)
            assert r["state"] == fe.FE_STATE_DONE, r
            _, _, v_o, _ = _oracle_values(DD, nd, KR, seed)
            assert np.array_equal(_values_of(fe, r).view(np.uint64), v_o.view(np.uint64))
            fe.fe_release(sv, t)
        st = fe.fe_server_stats_get(sv)
        assert st["admission_waits"] >= 1 and st["peak_bytes_in_use"] <= st["budget_bytes"]
    finally:
        fe.fe_server_stop(sv)
