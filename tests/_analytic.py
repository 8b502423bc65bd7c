"""Closed-form expectations used by the tests (test-only helpers).

Nothing here evaluates the MLS fit: these are exact solutions of the model
equations (Paper II, App. A; the circularly polarised Alfven wave of Sec. 3.2)
and exact derivatives of polynomial fields.
"""
from __future__ import annotations

import numpy as np


def linear_wave_dudt(w) -> np.ndarray:
    """Time derivative at t = 0 of the linear eigenmode built by
    workloads.linear_wave: every perturbation a sin(kx) has d/dt = -omega a cos(kx)
    (App. A: rho = rho0 k.V/omega, P = gamma P0 k.V/omega,
    B = [(k.V) B0 - (k.B0) V] / omega)."""
    m = w.meta
    k, A, om, vh, B0 = m["k"], m["amplitude"], m["omega"], m["vhat"], m["B0"]
    c = A * np.cos(k * w.pos[0])
    kv = k * vh[0]
    out = np.zeros((8, w.n))
    out[0] = -m["rho0"] * kv * c
    out[1:4] = -om * vh[:, None] * c
    out[4:7] = -(kv * B0[:, None] - k * B0[0] * vh[:, None]) * c
    out[7] = -w.gamma * m["P0"] * kv / (w.gamma - 1.0) * c
    return out


def circular_alfven_state(pos, gamma=5.0 / 3.0):
    """Sec. 3.2: rho = 1, Vx = 0, Bx = 1, Vy = By = 0.1 sin 2 pi x,
    Vz = Bz = 0.1 cos 2 pi x, P = 0.1.  An exact travelling solution U(x + t)."""
    x = pos[0]
    n = x.shape[0]
    U = np.zeros((8, n))
    U[0] = 1.0
    U[4] = 1.0
    U[2] = U[5] = 0.1 * np.sin(2 * np.pi * x)
    U[3] = U[6] = 0.1 * np.cos(2 * np.pi * x)
    U[7] = 0.1 / (gamma - 1.0)
    return U


def circular_alfven_dudt(pos):
    x = pos[0]
    out = np.zeros((8, x.shape[0]))
    out[2] = out[5] = 0.2 * np.pi * np.cos(2 * np.pi * x)
    out[3] = out[6] = -0.2 * np.pi * np.sin(2 * np.pi * x)
    return out


def damped_sound_wave(pos, zeta, A=1e-6, rho0=1.0, P0=1.0, gamma=5.0 / 3.0, kx=1):
    """Sound wave along x with bulk viscosity zeta (App. A, B = 0).  With the
    dependence exp(i(kx - omega t)) the dispersion relation is
    omega^2 + i zeta k^2 omega - c_s^2 k^2 = 0, i.e.
    omega = sqrt(c_s^2 k^2 - zeta^2 k^4 / 4) - i zeta k^2 / 2  (|Re omega|/k and
    |Im omega| = k^2 zeta / 2 as printed in App. A).  Returns (U, dU/dt) of the
    real part of the eigenmode with V-hat = A."""
    k = 2 * np.pi * kx
    cs2 = gamma * P0 / rho0
    om = np.sqrt(cs2 * k * k - zeta * zeta * k ** 4 / 4) - 0.5j * zeta * k * k
    e = np.exp(1j * k * pos[0])
    Vh = A
    rh = rho0 * k * Vh / om
    Ph = gamma * P0 * k * Vh / om
    n = pos.shape[1]
    U = np.zeros((8, n))
    d = np.zeros((8, n))
    U[0] = rho0 + (rh * e).real
    U[1] = (Vh * e).real
    U[7] = (P0 + (Ph * e).real) / (gamma - 1.0)
    d[0] = (-1j * om * rh * e).real
    d[1] = (-1j * om * Vh * e).real
    d[7] = (-1j * om * Ph * e).real / (gamma - 1.0)
    return U, d


def poly3(coef, x):
    """Full cubic sum_{|a|<=3} coef[a] x^a at points x [3][n]; coef: dict a->c.
    Returns (value, grad [3][n], hess [6][n] in xx,xy,xz,yy,yz,zz order)."""
    n = x.shape[1]
    val = np.zeros(n)
    grad = np.zeros((3, n))
    hess = np.zeros((6, n))
    pairs = [(0, 0), (0, 1), (0, 2), (1, 1), (1, 2), (2, 2)]
    for a, c in coef.items():
        a = np.asarray(a)
        val += c * np.prod(x ** a[:, None], axis=0)
        for ax in range(3):
            if a[ax] > 0:
                b = a.copy(); b[ax] -= 1
                grad[ax] += c * a[ax] * np.prod(x ** b[:, None], axis=0)
        for h, (p, q) in enumerate(pairs):
            b = a.copy()
            f = b[p]; b[p] -= 1
            if f <= 0:
                continue
            g = b[q]; b[q] -= 1
            if g <= 0:
                continue
            hess[h] += c * f * g * np.prod(x ** b[:, None], axis=0)
    return val, grad, hess


def cubic_exponents():
    return [(i, j, k) for i in range(4) for j in range(4) for k in range(4) if i + j + k <= 3]


def rel_err(a, o):
    """max_i |a - o| / max_i |o| over the last axis (absolute when o == 0)."""
    a = np.asarray(a)
    o = np.asarray(o)
    num = np.abs(a - o).max(axis=-1)
    den = np.abs(o).max(axis=-1)
    return np.where(den > 0, num / np.where(den > 0, den, 1.0), num)
