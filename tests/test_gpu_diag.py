"""GPU Kelvin-Helmholtz mode-amplitude diagnostic (Sec. 3.4) against the
oracle's plain FP64 sums, on the paper's seeded mode and on the 8M shear
layer."""
import numpy as np
import pytest

import oracle
import workloads
from _gpu import need_gpu, torch

pytestmark = pytest.mark.gpu


def _kh_lattice(nx=64, ny=256, amp=0.01):
    """The paper's set-up in a 1 x 4 slab: Vy = amp sin(4 pi x) exp(-4 pi |y~ - 1|)."""
    x = (np.arange(nx) + 0.5) / nx
    y = (np.arange(ny) + 0.5) * 4.0 / ny
    X, Y = np.meshgrid(x, y, indexing="ij")
    pos = np.stack([X.ravel(), Y.ravel(), np.full(X.size, 0.01)])
    yt = np.where(pos[1] < 2, pos[1], 4 - pos[1])
    U = np.zeros((8, pos.shape[1]))
    U[0] = 1.0
    U[2] = amp * np.sin(4 * np.pi * pos[0]) * np.exp(-4 * np.pi * np.abs(yt - 1.0))
    U[7] = 2.5 / (5.0 / 3.0 - 1.0)
    return pos, U


def test_seeded_mode_amplitude():
    phb = need_gpu()
    pos, U = _kh_lattice()
    plan = phb.Plan([0, 0, 0], [1.0, 4.0, 1.0], [1, 1, 0], pos.shape[1], 1 / 64, 1 / 64)
    out = phb.kh_mode_amplitude(plan, torch.tensor(pos, device="cuda"), torch.tensor(U, device="cuda"))
    out = out.cpu().numpy()
    M, (s, c, d) = oracle.kh_mode_amplitude(pos, U)
    assert abs(out[3] - 0.01) <= 1e-13
    assert np.allclose(out[:3], [s, c, d], rtol=1e-12, atol=1e-16)
    assert abs(out[3] - M) <= 1e-13 * M


def test_shear_layer_full_size_and_repeatable():
    """The 8,000,000-particle shear layer (layers at y = 0.25 and 0.75 of the
    unit box, a random Vy seed): sums and M equal the oracle's within FP64
    summation-order rounding, and two calls agree bit for bit."""
    phb = need_gpu()
    w = workloads.config("C5")
    plan = phb.Plan.for_workload(w)
    pos, lam, U = phb.tensors_of(w)
    k = 2 * np.pi * 4
    a = phb.kh_mode_amplitude(plan, pos, U, k=k, y0=0.25, ly=1.0)
    b = phb.kh_mode_amplitude(plan, pos, U, k=k, y0=0.25, ly=1.0)
    assert torch.equal(a, b)
    M, (s, c, d) = oracle.kh_mode_amplitude(w.pos, w.U, k=k, y0=0.25, ly=1.0)
    got = a.cpu().numpy()
    scale = np.abs(w.U[2]).sum()
    assert abs(got[0] - s) <= 1e-12 * scale and abs(got[1] - c) <= 1e-12 * scale
    assert abs(got[2] - d) <= 1e-12 * d
    assert abs(got[3] - M) <= 1e-9 * max(M, 1e-12)
    del plan
    torch.cuda.empty_cache()


def test_invalid_arguments():
    phb = need_gpu()
    pos, U = _kh_lattice(8, 16)
    plan = phb.Plan([0, 0, 0], [1.0, 4.0, 1.0], [1, 1, 0], pos.shape[1], 1 / 8, 1 / 8)
    with pytest.raises(phb.PhbError):
        phb.kh_mode_amplitude(plan, torch.tensor(pos, device="cuda"), torch.tensor(U, device="cuda"),
                              k=-1.0)
