"""Greedy element colouring on the GPU and colour-ordered assembly (the
colouring method of Listing 6), against the oracle: the colouring must equal
the sequential first-fit colouring element by element, and the assembled
values must equal the oracle's sequential assembly run in colour order."""

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
    rng = np.random.default_rng(3)
    scattered = np.stack([rng.choice(300, size=6, replace=False) for _ in range(200)]).astype(np.int32)
    return [
        ("quad48", *wl.quad_q1_grid(48, 1)),
        ("hex6_d3", *wl.hex_q1_grid(6, 3)),
        ("tet3_d3", *wl.tet_p2_kuhn(3, d=3, seed=4)),
        ("qp3", *wl.quad_qp_grid(4, 3, 2)),
        ("scattered", scattered, 300),
    ]


@pytest.mark.parametrize("name,D,n_dofs", _meshes(), ids=[m[0] for m in _meshes()])
def test_colouring_equals_sequential_first_fit(ctx, name, D, n_dofs):
    import torch
    from paper_2012_00585_gb300 import feasm
    g = gu.GpuAssembly(ctx, D, n_dofs)
    nc = feasm.fe_pattern_colour(ctx, g.pattern.handle)
    n2, cptr = feasm.fe_pattern_colours(g.pattern.handle)
    got = feasm.device_view(cptr, D.shape[0], torch.int32).cpu().numpy()
    k_o, exp = oracle.greedy_colouring(D, n_dofs)
    assert nc == n2 == k_o
    assert np.array_equal(got, exp)
    if name == "quad48":
        assert nc == 4 and np.bincount(got).tolist() == [D.shape[0] // 4] * 4  # 4 colours of 25 %
    g.free()


@pytest.mark.parametrize("fmt", ["csr", "crac"])
def test_coloured_assembly_is_the_colour_ordered_sum(ctx, fmt):
    from paper_2012_00585_gb300 import feasm
    for name, D, n_dofs in _meshes():
        K = wl.random_matrices(D.shape[0], D.shape[1], seed=len(name))
        g = gu.GpuAssembly(ctx, D, n_dofs)
        feasm.fe_pattern_colour(ctx, g.pattern.handle)
        _, colour = oracle.greedy_colouring(D, n_dofs)
        order = np.lexsort((np.arange(D.shape[0]), colour))  # by colour, then element
        rp, ci = oracle.csr_pattern(D, n_dofs)
        exp = oracle.assemble_csr(D, K, rp, ci, order=order)
        got = g.assemble(K, fmt, feasm.FE_COLOURED).cpu().numpy()
        assert np.array_equal(got.view(np.uint64), exp.view(np.uint64)), name
        again = g.assemble(K, fmt, feasm.FE_COLOURED).cpu().numpy()
        assert np.array_equal(again, got)
        g.free()


def test_coloured_mode_needs_a_colouring(ctx):
    from paper_2012_00585_gb300 import feasm
    D, n_dofs = wl.quad_q1_grid(4, 1)
    g = gu.GpuAssembly(ctx, D, n_dofs)
    with pytest.raises(feasm.FeError) as ei:
        g.assemble(np.ones((16, 4, 4)), "csr", feasm.FE_COLOURED)
    assert ei.value.code == feasm.FE_ERR_NOT_BUILT
    g.free()
