"""Oracle: the Kelvin-Helmholtz mode-amplitude diagnostic (Sec. 3.4), pinned
by closed forms on lattices that sample whole periods of the mode."""
import numpy as np

import oracle


def _lattice(nx=32, ny=128, lx=1.0, ly=4.0):
    x = (np.arange(nx) + 0.5) * lx / nx
    y = (np.arange(ny) + 0.5) * ly / ny
    X, Y = np.meshgrid(x, y, indexing="ij")
    pos = np.stack([X.ravel(), Y.ravel(), np.zeros(X.size)])
    return pos


def _vy_mode(pos, amp, k=4 * np.pi, phase=0.0, y0=1.0, ly=4.0, decay=None):
    y = pos[1]
    yt = np.where(y < ly / 2, y, ly - y)
    dk = k if decay is None else decay
    U = np.zeros((8, pos.shape[1]))
    U[2] = amp * np.sin(k * pos[0] + phase) * np.exp(-dk * np.abs(yt - y0))
    return U


def test_seeded_mode_gives_its_amplitude():
    """Vy = A sin(4 pi x) exp(-4 pi |y - 1|) (and the mirror form above y = 2),
    the paper's initial perturbation: s_i = A sin^2 d_i, so sum s / sum d = A/2
    on x points spread evenly over whole periods, and M = A."""
    pos = _lattice()
    for amp in (1e-2, 0.3):
        M, (s, c, d) = oracle.kh_mode_amplitude(pos, _vy_mode(pos, amp))
        assert abs(M - amp) <= 1e-13 * amp
        assert abs(c) <= 1e-13 * abs(s)


def test_phase_and_scale():
    """A phase shift of the mode moves weight between the sine and cosine sums
    without changing M; M is linear in the amplitude."""
    pos = _lattice()
    for ph in (0.3, 1.2, np.pi / 2, 2.5):
        M, (s, c, d) = oracle.kh_mode_amplitude(pos, _vy_mode(pos, 0.02, phase=ph))
        assert abs(M - 0.02) <= 1e-13
        assert abs(s / d - 0.01 * np.cos(ph)) <= 1e-14 and abs(c / d - 0.01 * np.sin(ph)) <= 1e-14


def test_other_wavenumbers_are_not_seen():
    """Modes of other whole wavenumbers (2 pi, 8 pi) are orthogonal to sin and
    cos(4 pi x) on the even x points: M = 0 up to rounding."""
    pos = _lattice()
    for k in (2 * np.pi, 8 * np.pi):
        M, _ = oracle.kh_mode_amplitude(pos, _vy_mode(pos, 0.05, k=k, decay=4 * np.pi))
        assert M < 1e-15


def test_layer_weighting_and_mirror():
    """Only the y profile's overlap with exp(-4 pi |y~ - 1|) matters: a mode
    with a flat profile in y gives sum s / sum d = (A/2) sum e / sum e^2, the
    closed form of the lattice sums; the mirror image above y = 2 counts the
    same as the lower layer."""
    pos = _lattice()
    U = np.zeros((8, pos.shape[1]))
    U[2] = 0.04 * np.sin(4 * np.pi * pos[0])
    M, (s, c, d) = oracle.kh_mode_amplitude(pos, U)
    y = pos[1]
    yt = np.where(y < 2, y, 4 - y)
    e = np.exp(-4 * np.pi * np.abs(yt - 1.0))
    assert abs(M - 2 * 0.02 * e.sum() / (e * e).sum()) <= 1e-13 * M
    lower = pos[1] < 2
    M1, _ = oracle.kh_mode_amplitude(pos[:, lower], U[:, lower])
    M2, _ = oracle.kh_mode_amplitude(pos[:, ~lower], U[:, ~lower])
    assert abs(M1 - M2) <= 1e-13 * M1 and abs(M - M1) <= 1e-13 * M1
