"""Serving loop: results served alone and in a mix equal the standalone
assembly of the same element values; admission, cancellation and bad input
fail cleanly while the server keeps serving; the element-value generator
matches its published definition."""

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


def _expected(ctx, fe, D, n_dofs, Kr, seed, mode, fmt):
    """Standalone: generate the same K, assemble with the single-mesh path."""
    import torch
    Dd = torch.from_numpy(D).cuda()
    Krd = torch.from_numpy(Kr).cuda()
    n_e, n_loc = D.shape
    K = torch.empty((n_e, n_loc, n_loc), dtype=torch.float64, device="cuda")
    fe.fe_generate_scaled(ctx, Krd, n_loc, n_e, seed, K)
    p = fe.Pattern(ctx, Dd, n_dofs)
    v = torch.empty(p.info["nnz"], dtype=torch.float64, device="cuda")
    (fe.fe_assemble_csr if fmt == 0 else fe.fe_assemble_crac)(ctx, p.handle, K, v, mode, 0)
    torch.cuda.synchronize()
    out = v.cpu().numpy(), K.cpu().numpy()
    p.free()
    return out


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
            exp, K = _expected(ctx, fe, D, n_dofs, Kr, seed, mode, 1)
            if mode == fe.FE_DETERMINISTIC:
                assert np.array_equal(got, exp)
                if key == key0 and seed == 77:
                    assert np.array_equal(got, alone)  # alone == in the mix, bit for bit
            else:
                rp, ci = oracle.csr_pattern(D, n_dofs)
                v_o = oracle.assemble_csr(D, K, rp, ci)
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
