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


def sample(n, k, seed=0):
    rng = np.random.default_rng(seed)
    return np.sort(rng.choice(n, min(n, k), replace=False)).astype(np.int64)
