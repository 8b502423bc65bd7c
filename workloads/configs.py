"""Seeded synthetic particle sets shaped like the test problems of Phurbas Paper II.

The paper's own initial conditions (relaxed glass distributions, Athena
reference states) are not available as data, so these generators stand in for
them: jittered lattices or density-sampled random placements, with the field
profiles of the paper's tests (linear waves, App. A; shock-tube states,
Table 1; Kelvin-Helmholtz shear layer, Sec. 3.4).

This module holds input recipes only.  It contains none of the arithmetic of
the MLS fit or of the MHD right-hand side.

Layout: ``pos`` is float64 ``[3][n]``, ``lam`` float64 ``[n]``, ``U`` float64
``[8][n]`` with the field order (rho, Vx, Vy, Vz, Bx, By, Bz, sigma), where
sigma is the internal energy density, P = (gamma - 1) sigma.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

from . import rng

FIELDS = ("rho", "Vx", "Vy", "Vz", "Bx", "By", "Bz", "sigma")

# stream ids: one per purpose so that sub-draws never overlap
_S_JITTER, _S_MODE_K, _S_MODE_A, _S_MODE_PHI, _S_X, _S_Y, _S_Z, _S_PERT, _S_WEIGHTS = range(1, 10)


@dataclass
class Workload:
    name: str
    box_lo: np.ndarray          # [3]
    box_len: np.ndarray         # [3]
    periodic: np.ndarray        # [3] int32
    pos: np.ndarray             # [3][n] float64
    lam: np.ndarray             # [n] float64
    U: np.ndarray               # [8][n] float64
    gamma: float
    meta: dict = field(default_factory=dict)

    @property
    def n(self) -> int:
        return int(self.lam.shape[0])


def _box(lo, ln, per):
    return (np.asarray(lo, np.float64), np.asarray(ln, np.float64), np.asarray(per, np.int32))


def lattice_positions(n_side: int, seed: int, jitter: float = 0.1, box_len: float = 1.0,
                      stream: int = _S_JITTER) -> tuple[np.ndarray, float]:
    """Cubic lattice of n_side**3 points at (idx + 0.5) h with uniform jitter of
    +-jitter*h per axis, x-major particle order.  Returns (pos[3][n], h)."""
    h = box_len / n_side
    idx = np.arange(n_side, dtype=np.float64)
    gx, gy, gz = np.meshgrid(idx, idx, idx, indexing="ij")
    n = n_side ** 3
    base = np.stack([gx.ravel(), gy.ravel(), gz.ravel()])
    jit = rng.uniform(seed, stream, 3 * n, -jitter * h, jitter * h).reshape(3, n)
    pos = (base + 0.5) * h + jit
    return np.ascontiguousarray(pos), h


def background(n: int, rho0=1.0, V0=(0.0, 0.0, 0.0), B0=(1.0, np.sqrt(2.0), 0.5), P0=1.0,
               gamma=5.0 / 3.0) -> np.ndarray:
    U = np.empty((8, n), np.float64)
    U[0] = rho0
    U[1:4] = np.asarray(V0, np.float64)[:, None]
    U[4:7] = np.asarray(B0, np.float64)[:, None]
    U[7] = P0 / (gamma - 1.0)
    return U


def linear_mhd_modes(kvec, B0, rho0, P0, gamma):
    """Eigen-decomposition of the undamped linear MHD momentum operator of
    App. A: omega^2 V = (k.vA)^2 V + [(vs^2+vA^2) k - (k.vA) vA](k.V) - (k.vA)(vA.V) k.
    Returns (omega^2 ascending, unit eigenvectors as columns)."""
    k = np.asarray(kvec, np.float64)
    vA = np.asarray(B0, np.float64) / np.sqrt(rho0)
    vs2 = gamma * P0 / rho0
    kvA = k @ vA
    K = kvA ** 2 * np.eye(3) + np.outer((vs2 + vA @ vA) * k - kvA * vA, k) - kvA * np.outer(k, vA)
    w2, vec = np.linalg.eig(K)
    order = np.argsort(w2.real)
    w2 = w2.real[order]
    vec = vec.real[:, order]
    vec /= np.linalg.norm(vec, axis=0)
    return w2, vec


def linear_wave(n_side: int = 16, seed: int = rng.DEFAULT_SEED, amplitude: float = 1e-6,
                mode: str = "fast", B0=(1.0, np.sqrt(2.0), 0.5), rho0=1.0, P0=1.0,
                gamma=5.0 / 3.0, kx: int = 1, jitter: float = 0.1) -> Workload:
    """Jittered lattice in the periodic unit box with a linear MHD eigenmode
    along x (App. A):  V = A Vhat sin(k x),  rho = rho0 (k Vhat_x / omega) A sin,
    P = gamma P0 (k Vhat_x / omega) A sin,  B = [(k Vhat_x) B0 - (k B0_x) Vhat] / omega A sin.
    The time derivative of this state is -omega times the same amplitudes with
    cos(k x) in place of sin(k x)."""
    pos, h = lattice_positions(n_side, seed, jitter)
    n = pos.shape[1]
    k = 2.0 * np.pi * kx
    w2, vec = linear_mhd_modes((k, 0.0, 0.0), B0, rho0, P0, gamma)
    pick = {"slow": 0, "alfven": 1, "fast": 2}[mode]
    if mode != "fast":
        # identify the Alfven branch as the one with omega^2 = (k.vA)^2
        kvA2 = (k * B0[0]) ** 2 / rho0
        ia = int(np.argmin(np.abs(w2 - kvA2)))
        rest = [i for i in range(3) if i != ia]
        pick = ia if mode == "alfven" else rest[0]
    omega = float(np.sqrt(w2[pick]))
    vhat = vec[:, pick].copy()
    if vhat[np.argmax(np.abs(vhat))] < 0:
        vhat = -vhat
    s = amplitude * np.sin(k * pos[0])
    kv = k * vhat[0]
    U = background(n, rho0=rho0, B0=B0, P0=P0, gamma=gamma)
    U[0] += rho0 * kv / omega * s
    U[1:4] += vhat[:, None] * s
    U[4:7] += ((kv * np.asarray(B0)[:, None] - k * B0[0] * vhat[:, None]) / omega) * s
    U[7] += gamma * P0 * kv / omega * s / (gamma - 1.0)
    lo, ln, per = _box((0, 0, 0), (1, 1, 1), (1, 1, 1))
    lam = np.full(n, h)
    meta = dict(omega=omega, vhat=vhat, k=k, amplitude=amplitude, B0=np.asarray(B0), rho0=rho0,
                P0=P0, mode=mode, h=h, seed=seed)
    return Workload(f"linear_wave_{mode}_{n_side}^3", lo, ln, per, pos, lam, U, gamma, meta)


def random_modes(n_side: int = 64, seed: int = rng.DEFAULT_SEED, nmodes: int = 8,
                 amp: float = 1e-2, kmax: int = 4, jitter: float = 0.1,
                 gamma=5.0 / 3.0) -> Workload:
    """Jittered lattice, constant lambda = h, fields = C1 background plus
    sum_m a_m sin(2 pi k_m.x + phi_m), k_m in {-kmax..kmax}^3 minus 0, one
    amplitude a_m ~ U(-amp, amp) per field, phi_m ~ U(0, 2 pi)."""
    pos, h = lattice_positions(n_side, seed, jitter)
    n = pos.shape[1]
    side = 2 * kmax + 1
    choices = side ** 3 - 1
    pick = rng.integers(seed, _S_MODE_K, nmodes, choices)
    pick = pick + (pick >= choices // 2)           # skip the zero vector (centre of the cube)
    kv = np.stack([pick // (side * side), (pick // side) % side, pick % side], axis=1) - kmax
    a = rng.uniform(seed, _S_MODE_A, nmodes * 8, -amp, amp).reshape(nmodes, 8)
    phi = rng.uniform(seed, _S_MODE_PHI, nmodes, 0.0, 2.0 * np.pi)
    U = background(n, gamma=gamma)
    for m in range(nmodes):
        s = np.sin(2.0 * np.pi * (kv[m] @ pos) + phi[m])
        U += a[m][:, None] * s[None, :]
    lo, ln, per = _box((0, 0, 0), (1, 1, 1), (1, 1, 1))
    lam = np.full(n, h)
    meta = dict(k=kv, a=a, phi=phi, h=h, seed=seed)
    return Workload(f"random_modes_{n_side}^3", lo, ln, per, pos, lam, U, gamma, meta)


def _inverse_cdf(grid: np.ndarray, dens: np.ndarray, u: np.ndarray) -> np.ndarray:
    cdf = np.concatenate([[0.0], np.cumsum(0.5 * (dens[1:] + dens[:-1]) * np.diff(grid))])
    cdf /= cdf[-1]
    return np.interp(u, cdf, grid)


def shock_tube(n: int = 1 << 20, seed: int = rng.DEFAULT_SEED, gamma: float = 2.0) -> Workload:
    """Magnetised shock-tube profile in a periodic 8x1x1 box (Brio-Wu-like states of
    Table 1 with B_x = 0.75), two mirrored tanh interfaces at x = 2 and x = 6 of
    width 2 lambda_L, lambda = lambda_L rho^(-1/3), particles drawn with number
    density 1/lambda^3 (x by inverse CDF, y and z uniform)."""
    lamL = (4.5 / n) ** (1.0 / 3.0)
    w = 2.0 * lamL
    rhoL, rhoR, PL, PR, ByL, ByR = 1.0, 0.125, 1.0, 0.1, 1.0, -1.0

    def sfun(x):
        return 0.5 * (np.tanh((x - 2.0) / w) - np.tanh((x - 6.0) / w))

    grid = np.linspace(0.0, 8.0, (1 << 20) + 1)
    dens = rhoL + (rhoR - rhoL) * sfun(grid)
    x = _inverse_cdf(grid, dens, rng.uniform(seed, _S_X, n))
    y = rng.uniform(seed, _S_Y, n)
    z = rng.uniform(seed, _S_Z, n)
    pos = np.ascontiguousarray(np.stack([x, y, z]))
    s = sfun(x)
    rho = rhoL + (rhoR - rhoL) * s
    P = PL + (PR - PL) * s
    U = np.zeros((8, n), np.float64)
    U[0] = rho
    U[4] = 0.75
    U[5] = ByL + (ByR - ByL) * s
    U[7] = P / (gamma - 1.0)
    lam = lamL * rho ** (-1.0 / 3.0)
    lo, ln, per = _box((0, 0, 0), (8, 1, 1), (1, 1, 1))
    meta = dict(lambda_L=lamL, width=w, seed=seed)
    return Workload(f"shock_tube_{n}", lo, ln, per, pos, lam, U, gamma, meta)


def shear_layer(n: int = 8_000_000, seed: int = rng.DEFAULT_SEED, gamma: float = 5.0 / 3.0) -> Workload:
    """Kelvin-Helmholtz-like double shear layer in the periodic unit box
    (Sec. 3.4 shapes): Vx = +-0.5 across tanh layers of width 0.05 at y = 0.25
    and 0.75, rho 1 outside and 2 between the layers, P = 2.5, B = (0.1, 0, 0),
    Vy = 1e-2 U(-1,1) exp(-(dy/0.05)^2), lambda = lambda0/2 within 0.1 of a
    layer and lambda0 elsewhere, placement with number density 1/lambda^3."""
    lam0 = ((0.4 * 8.0 + 0.6) / n) ** (1.0 / 3.0)
    w = 0.05
    # piecewise-constant number density in y: exact inverse CDF on the breakpoints
    yb = np.array([0.0, 0.15, 0.35, 0.65, 0.85, 1.0])
    db = np.array([1.0, 8.0, 1.0, 8.0, 1.0])
    cum = np.concatenate([[0.0], np.cumsum(db * np.diff(yb))])
    cum /= cum[-1]
    y = np.interp(rng.uniform(seed, _S_Y, n), cum, yb)
    x = rng.uniform(seed, _S_X, n)
    z = rng.uniform(seed, _S_Z, n)
    pos = np.ascontiguousarray(np.stack([x, y, z]))
    band = 0.5 * (np.tanh((y - 0.25) / w) - np.tanh((y - 0.75) / w))
    dy = np.minimum(np.abs(y - 0.25), np.abs(y - 0.75))
    U = np.zeros((8, n), np.float64)
    U[0] = 1.0 + band
    U[1] = -0.5 + band
    U[2] = 1e-2 * rng.uniform(seed, _S_PERT, n, -1.0, 1.0) * np.exp(-(dy / w) ** 2)
    U[4] = 0.1
    U[7] = 2.5 / (gamma - 1.0)
    lam = np.where(dy < 0.1, 0.5 * lam0, lam0)
    lo, ln, per = _box((0, 0, 0), (1, 1, 1), (1, 1, 1))
    meta = dict(lambda0=lam0, seed=seed)
    return Workload(f"shear_layer_{n}", lo, ln, per, pos, lam, U, gamma, meta)


def loss_weights(n: int, seed: int = rng.DEFAULT_SEED) -> np.ndarray:
    """r in U(-1, 1)^[8][n] for the scalar functional L = sum_i sum_k r_ik (dU_k/dt)_i."""
    return rng.uniform(seed, _S_WEIGHTS, 8 * n, -1.0, 1.0).reshape(8, n)


CONFIGS = {
    "C1": ("linear fast wave, 16^3 jittered lattice", lambda seed: linear_wave(16, seed)),
    "C2": ("random Fourier modes, 64^3 jittered lattice", lambda seed: random_modes(64, seed)),
    "C3": ("shock tube, 1,048,576 density-sampled particles, 8x1x1", lambda seed: shock_tube(1 << 20, seed)),
    "C4": ("adjoint workload, 64^3 jittered lattice with random modes", lambda seed: random_modes(64, seed)),
    "C5": ("double shear layer, 8,000,000 density-sampled particles", lambda seed: shear_layer(8_000_000, seed)),
}


def config(name: str, seed: int = rng.DEFAULT_SEED) -> Workload:
    return CONFIGS[name][1](seed)
