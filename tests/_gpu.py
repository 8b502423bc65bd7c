"""Helpers for the GPU parity tests (compare the CUDA path with the oracle)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")


def need_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1110_0836_gb300 as phb
    phb.build()
    return phb


def sets_of(off, idx):
    off = off.cpu().numpy()
    idx = idx.cpu().numpy()
    return [idx[off[i]:off[i + 1]] for i in range(len(off) - 1)]


def kind_err(a, o, floor_frac=0.0):
    """Per field: max |a - o| / max |o| over particles and components (absolute when o == 0).
    a, o: [8][ncomp][n] or [8][n].  With floor_frac > 0 every field's scale is
    at least floor_frac times the largest field scale: a field whose exact
    value vanishes (its oracle value is cancellation noise) is then measured
    against the dominant field instead of against that noise."""
    a = np.asarray(a)
    o = np.asarray(o)
    if a.ndim == 2:
        a, o = a[:, None, :], o[:, None, :]
    num = np.abs(a - o).max(axis=(1, 2))
    den = np.abs(o).max(axis=(1, 2))
    if floor_frac > 0:
        den = np.maximum(den, floor_frac * den.max())
    return np.where(den > 0, num / np.where(den > 0, den, 1.0), num)


RHS_FLOOR = 1e-2  # field-scale floor used for time-derivative comparisons


def rhs_term_scales(U, grad, hess, gamma, zeta=None, eta=None):
    """Per field, the largest magnitude over particles of the terms combined in
    that field's equation (the scale against which rounding errors of the
    right-hand side are measured; a field whose terms cancel keeps the terms'
    scale).  U [8][n], grad [8][3][n], hess [8][6][n] (oracle values)."""
    n = U.shape[1]
    z = np.zeros(n) if zeta is None else np.abs(zeta)
    e = np.zeros(n) if eta is None else np.abs(eta)
    rho, sig, B = np.abs(U[0]), np.abs(U[7]), np.abs(U[4:7])
    gV = np.abs(grad[1:4])            # [a][b][n] = |dV_a/dx_b|
    gB = np.abs(grad[4:7])
    divabs = gV[0, 0] + gV[1, 1] + gV[2, 2]
    hV = np.abs(hess[1:4]).sum(axis=1).max(axis=0)
    hB = np.abs(hess[4:7]).sum(axis=1).max(axis=0)
    J = gB.sum(axis=(0, 1))
    Bmax = B.max(axis=0)
    sc = np.zeros(8)
    sc[0] = (rho * divabs).max()
    sc[1:4] = (((gamma - 1) * np.abs(grad[7]).max(axis=0) + J * Bmax) / rho + z * hV).max()
    for a in range(3):
        sc[4 + a] = ((B * gV[a]).sum(axis=0) + B[a] * divabs + e * hB).max()
    sc[7] = (gamma * sig * divabs + rho * z * divabs ** 2).max()
    return sc


def rhs_err(a, o, scales):
    """Per field: max_i |a - o| / (that field's term scale)."""
    num = np.abs(np.asarray(a) - np.asarray(o)).max(axis=-1)
    return num / np.where(scales > 0, scales, 1.0)


def sample(n, k, seed=0):
    rng = np.random.default_rng(seed)
    return np.sort(rng.choice(n, min(n, k), replace=False)).astype(np.int64)
