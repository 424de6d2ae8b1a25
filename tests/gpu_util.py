"""Helpers shared by the GPU tests: run the CUDA path through the C ABI and
compare it with the oracle."""

import numpy as np

import oracle

TOL_REL = 1e-12  # atomic mode: |G_gpu - G_oracle| <= 1e-12 * sum_j |G_oracle(i, j)| per row


def row_tolerance(row_ptr, values, K_abs_row_sums=None):
    """tau_i = 1e-12 * sum_j |G_ij| (oracle values); rows whose sum is zero
    fall back to 1e-12 * (sum of |contributions| into the row)."""
    absv = np.abs(values)
    nrow = row_ptr.shape[0] - 1
    s = np.zeros(nrow)
    nz = np.diff(row_ptr) > 0
    s[nz] = np.add.reduceat(absv, row_ptr[:-1][nz])
    tau = TOL_REL * s
    if K_abs_row_sums is not None:
        tau = np.where(tau > 0, tau, TOL_REL * K_abs_row_sums)
    return tau


def contribution_abs_row_sums(D, K, n_dofs):
    """sum over (e, r, c) with D_e(r) = i of |K_e(r, c)|, per row i."""
    out = np.zeros(n_dofs)
    np.add.at(out, D.ravel(), np.abs(K).sum(axis=2).ravel())
    return out


def assert_within_row_tol(row_ptr, got, exp, tau):
    diff = np.abs(got - exp)
    rows = np.repeat(np.arange(row_ptr.shape[0] - 1), np.diff(row_ptr))
    bad = diff > tau[rows]
    assert not bad.any(), (f"{int(bad.sum())} entries outside 1e-12*rowsum; worst rel "
                           f"{float(np.max(diff / np.maximum(tau[rows], 1e-300)) * 1e-12):.3e}")


class GpuAssembly:
    """Pattern + assemblies of one mesh through the C ABI (torch for memory)."""

    def __init__(self, ctx, D, n_dofs, flags=None, device="cuda"):
        import torch
        from paper_2012_00585_gb300 import feasm
        self.fe = feasm
        self.ctx = ctx
        self.D = np.ascontiguousarray(D, dtype=np.int32)
        self.n_dofs = n_dofs
        self.Dd = torch.from_numpy(self.D).to(device)
        self.pattern = feasm.Pattern(ctx, self.Dd, n_dofs, feasm.FE_PATTERN_ALL if flags is None else flags)
        torch.cuda.synchronize()

    def csr_host(self):
        rp, ci = self.pattern.csr()
        return rp.cpu().numpy(), ci.cpu().numpy()

    def crac_host(self):
        rp, ca = self.pattern.crac()
        return rp.cpu().numpy(), ca.cpu().numpy()

    def assemble(self, K, fmt="csr", mode=0, accumulate=0, values=None):
        import torch
        Kd = K if isinstance(K, torch.Tensor) else torch.from_numpy(np.ascontiguousarray(K)).to("cuda")
        nnz = self.pattern.info["nnz"]
        if values is None:
            v = torch.full((nnz,), float("nan"), dtype=torch.float64, device="cuda")
        else:
            v = values if isinstance(values, torch.Tensor) else torch.from_numpy(values).to("cuda")
        f = self.fe.fe_assemble_csr if fmt == "csr" else self.fe.fe_assemble_crac
        f(self.ctx, self.pattern.handle, Kd, v, mode, accumulate)
        torch.cuda.synchronize()
        return v

    def free(self):
        self.pattern.free()


def oracle_reference(D, K, n_dofs):
    row_ptr, col_idx = oracle.csr_pattern(D, n_dofs)
    vals = oracle.assemble_csr(D, K, row_ptr, col_idx)
    return row_ptr, col_idx, vals
