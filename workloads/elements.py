"""Dense element matrices K (float64, row-major per element).

The paper uses a dummy element, a matrix of ones (§2.1), because it times the
assembly alone.  The workloads here also use physical element matrices so
that the assembled matrix has checkable structure (zero row sums, rigid body
modes), and random SPD matrices so that no two entries are alike.  Reference
matrices are computed on the host by Gauss quadrature; per-element copies
can be materialised on the host (numpy) or on a CUDA device (torch), the
latter only as memory plumbing.
"""

import numpy as np

_GAUSS2 = np.array([-1.0, 1.0]) / np.sqrt(3.0)


def laplace_q1_quad() -> np.ndarray:
    """4x4 stiffness of -Laplace on a square bilinear element (scale free in 2-D).

    Local nodes counter-clockwise (0,0), (1,0), (1,1), (0,1); 2x2 Gauss
    quadrature, which is exact for this integrand on an affine square.
    """
    xi_a = np.array([-1.0, 1.0, 1.0, -1.0])
    eta_a = np.array([-1.0, -1.0, 1.0, 1.0])
    K = np.zeros((4, 4))
    for xi in _GAUSS2:
        for eta in _GAUSS2:
            # reference square [-1,1]^2 mapped to a side-h square: the h factors cancel in 2-D
            dN = np.stack([0.25 * xi_a * (1 + eta * eta_a), 0.25 * eta_a * (1 + xi * xi_a)], axis=1)
            K += dN @ dN.T  # |J| * J^-T J^-1 = 1 for the map with J = h/2 I in 2-D
    return K


def _hex_grad(xi, eta, zeta):
    """Reference gradients [8, 3] of the trilinear shape functions, x-fastest order."""
    s = np.array([[-1.0, -1.0, -1.0], [1.0, -1.0, -1.0], [-1.0, 1.0, -1.0], [1.0, 1.0, -1.0],
                  [-1.0, -1.0, 1.0], [1.0, -1.0, 1.0], [-1.0, 1.0, 1.0], [1.0, 1.0, 1.0]])
    fx = 1 + xi * s[:, 0]
    fy = 1 + eta * s[:, 1]
    fz = 1 + zeta * s[:, 2]
    return 0.125 * np.stack([s[:, 0] * fy * fz, s[:, 1] * fx * fz, s[:, 2] * fx * fy], axis=1)


def laplace_q1_hex(h: float = 1.0) -> np.ndarray:
    """8x8 stiffness of -Laplace on a cube of side h (2x2x2 Gauss); scales as h."""
    K = np.zeros((8, 8))
    for xi in _GAUSS2:
        for eta in _GAUSS2:
            for zeta in _GAUSS2:
                g = _hex_grad(xi, eta, zeta) * (2.0 / h)
                K += (g @ g.T) * (h / 2.0) ** 3
    return K


def elasticity_q1_hex(h: float = 1.0, E: float = 1.0, nu: float = 0.3) -> np.ndarray:
    """24x24 isotropic linear-elastic stiffness of a cube of side h (2x2x2 Gauss).

    Local DOF ``3*node + comp`` with nodes in x-fastest order.  Voigt strains
    (xx, yy, zz, yz, xz, xy) with engineering shears.  Scales as h.
    """
    lam = E * nu / ((1 + nu) * (1 - 2 * nu))
    mu = E / (2 * (1 + nu))
    D = np.zeros((6, 6))
    D[:3, :3] = lam
    D[np.arange(3), np.arange(3)] += 2 * mu
    D[np.arange(3, 6), np.arange(3, 6)] = mu
    K = np.zeros((24, 24))
    for xi in _GAUSS2:
        for eta in _GAUSS2:
            for zeta in _GAUSS2:
                g = _hex_grad(xi, eta, zeta) * (2.0 / h)
                B = np.zeros((6, 24))
                for a in range(8):
                    gx, gy, gz = g[a]
                    c = 3 * a
                    B[0, c + 0] = gx
                    B[1, c + 1] = gy
                    B[2, c + 2] = gz
                    B[3, c + 1] = gz
                    B[3, c + 2] = gy
                    B[4, c + 0] = gz
                    B[4, c + 2] = gx
                    B[5, c + 0] = gy
                    B[5, c + 1] = gx
                K += (B.T @ D @ B) * (h / 2.0) ** 3
    return 0.5 * (K + K.T)


def ones_matrices(n_e: int, n_loc: int) -> np.ndarray:
    """The paper's dummy element: every entry 1.0 (§2.1)."""
    return np.ones((n_e, n_loc, n_loc), dtype=np.float64)


def broadcast_matrices(K_ref: np.ndarray, n_e: int, scale: float = 1.0, device=None):
    """n_e materialised copies of ``scale * K_ref``.

    With ``device`` set (a torch device string) the copies are made on that
    device with torch; otherwise a numpy array is returned.
    """
    K1 = np.ascontiguousarray(K_ref * scale, dtype=np.float64)
    if device is None:
        return np.broadcast_to(K1, (n_e,) + K1.shape).copy()
    import torch
    t = torch.from_numpy(K1).to(device)
    return t.unsqueeze(0).expand(n_e, *K1.shape).contiguous()


def random_matrices(n_e: int, n_loc: int, seed: int = 0) -> np.ndarray:
    """Unsymmetric N(0,1) element matrices (host); catches transposed operands."""
    rng = np.random.default_rng(seed)
    return rng.standard_normal((n_e, n_loc, n_loc))


def random_spd_matrices(n_e: int, n_loc: int, seed: int = 0, device=None, chunk: int = 1 << 16):
    """Random SPD element matrices ``K = G G^T + n_loc*I`` with G ~ N(0,1).

    The product is symmetrised as ``(M + M^T)/2`` so that K is bit-symmetric.
    Host (numpy) by default; with ``device`` the matrices are drawn on that
    torch device from a seeded torch generator, in chunks of ``chunk``
    elements (the host and device draws are different samples of the same
    distribution).
    """
    if device is None:
        rng = np.random.default_rng(seed)
        out = np.empty((n_e, n_loc, n_loc), dtype=np.float64)
        eye = np.eye(n_loc) * float(n_loc)
        for s in range(0, n_e, chunk):
            t = min(chunk, n_e - s)
            G = rng.standard_normal((t, n_loc, n_loc))
            M = G @ G.transpose(0, 2, 1)
            out[s:s + t] = 0.5 * (M + M.transpose(0, 2, 1)) + eye
        return out
    import torch
    gen = torch.Generator(device=device)
    gen.manual_seed(seed)
    out = torch.empty((n_e, n_loc, n_loc), dtype=torch.float64, device=device)
    eye = torch.eye(n_loc, dtype=torch.float64, device=device) * float(n_loc)
    for s in range(0, n_e, chunk):
        t = min(chunk, n_e - s)
        G = torch.randn((t, n_loc, n_loc), generator=gen, dtype=torch.float64, device=device)
        M = torch.bmm(G, G.transpose(1, 2))
        out[s:s + t] = 0.5 * (M + M.transpose(1, 2)) + eye
    return out


def scaled_matrices(K_ref: np.ndarray, n_e: int, seed: int = 0, device=None):
    """``K_e = alpha_e * K_ref`` with alpha_e = 0.5 + u_e, u_e dyadic uniform in [0,1).

    u_e has 20 random bits, so alpha_e is exact and the product is one IEEE
    multiply per entry: symmetry and zero row sums of K_ref carry over.
    """
    if device is None:
        rng = np.random.default_rng(seed)
        u = rng.integers(0, 1 << 20, size=n_e).astype(np.float64) / float(1 << 20)
        alpha = 0.5 + u
        return alpha[:, None, None] * np.asarray(K_ref, dtype=np.float64)[None]
    import torch
    gen = torch.Generator(device=device)
    gen.manual_seed(seed)
    u = torch.randint(0, 1 << 20, (n_e,), generator=gen, device=device).to(torch.float64) / float(1 << 20)
    alpha = 0.5 + u
    Kr = torch.as_tensor(np.asarray(K_ref, dtype=np.float64), device=device)
    return alpha[:, None, None] * Kr[None]
