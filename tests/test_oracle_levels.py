"""Pins of the oracle's individual time-step levels (Paper II Sec. 2, Sec. 2.1).

The rule has a hand-derived golden case and is checked against what the text
fixes: steps rounded down to powers of two, independence of the bulk
velocity, the limiter's guarantee towards neighbours (and nothing more), and
exact scalings of the Courant step with lambda, rho and the signal speed."""
import json
import os

import numpy as np
import pytest

import oracle
import workloads

HERE = os.path.dirname(os.path.abspath(__file__))


def _state_line(g):
    n = len(g["pos_x"])
    pos = np.zeros((3, n))
    pos[0] = g["pos_x"]
    pos[1:] = 0.5
    lam = np.full(n, g["lambda"])
    U = np.zeros((8, n))
    U[0] = 1.0
    gam = g["gamma"]
    U[7] = np.asarray(g["sound_speed"]) ** 2 / (gam * (gam - 1.0))
    return pos, lam, U


def test_golden_line():
    g = json.load(open(os.path.join(HERE, "golden", "timestep_levels_line.json")))
    pos, lam, U = _state_line(g)
    box = oracle.make_box((0, 0, 0), (8, 1, 1), (0, 0, 0))
    nb = oracle.neighbors(box, pos, lam)
    kw = dict(gamma=g["gamma"], cfl=g["cfl"], dt_max=g["dt_max"], max_level=g["max_level"])
    none = (np.zeros(len(lam) + 1, np.int64), np.zeros(0, np.int64))
    assert oracle.timestep_levels(lam, U, none, **kw).tolist() == g["unlimited_levels"]
    assert oracle.timestep_levels(lam, U, nb, **kw).tolist() == g["levels"]


def _random_case(seed=3, n=4000):
    w = workloads.shock_tube(n, seed=seed)
    rng = np.random.default_rng(seed)
    w.U[7] *= rng.uniform(0.5, 40.0, w.n)      # spread of sound speeds
    w.U[4:7] *= rng.uniform(0.2, 3.0, w.n)     # and of Alfven speeds
    nb = oracle.neighbors(oracle.box_of(w), w.pos, w.lam)
    return w, nb


def _fast_speed(w):
    """Textbook upper bound of the fast magnetosonic speed, c_s^2 + v_A^2."""
    rho = w.U[0]
    cs2 = w.gamma * (w.gamma - 1.0) * w.U[7] / rho
    va2 = (w.U[4] ** 2 + w.U[5] ** 2 + w.U[6] ** 2) / rho
    return np.sqrt(cs2 + va2)


def test_power_of_two_rounding_against_the_courant_step():
    w, _ = _random_case()
    none = (np.zeros(w.n + 1, np.int64), np.zeros(0, np.int64))
    cfl, dt_max = 0.3, 0.05
    L = oracle.timestep_levels(w.lam, w.U, none, gamma=w.gamma, cfl=cfl, dt_max=dt_max)
    dt = cfl * w.lam / _fast_speed(w)
    lo = dt_max / 2.0 ** L
    assert (lo <= dt * (1 + 1e-12)).all()                          # rounded down
    assert ((L == 0) | (2 * lo > dt * (1 - 1e-12))).all()          # to the nearest power
    assert L.max() > L.min() + 2


def test_bulk_velocity_does_not_change_levels():
    w, nb = _random_case()
    kw = dict(gamma=w.gamma, cfl=0.2, dt_max=0.05)
    L = oracle.timestep_levels(w.lam, w.U, nb, **kw)
    U2 = w.U.copy()
    U2[1:4] += np.array([[3.0], [-1.5], [0.25]])
    assert np.array_equal(oracle.timestep_levels(w.lam, U2, nb, **kw), L)


def test_limiter_guarantee_and_minimality():
    w, nb = _random_case()
    kw = dict(gamma=w.gamma, cfl=0.2, dt_max=0.05)
    off, idx = nb
    none = (np.zeros(w.n + 1, np.int64), np.zeros(0, np.int64))
    L0 = oracle.timestep_levels(w.lam, w.U, none, **kw)
    L = oracle.timestep_levels(w.lam, w.U, nb, **kw)
    src = np.repeat(np.arange(w.n), np.diff(off))
    assert (L[idx] >= L0[src] - 1).all()                 # every neighbour within one level
    assert (L >= L0).all()
    lifted = np.full(w.n, -1)
    np.maximum.at(lifted, idx, L0[src] - 1)
    assert np.array_equal(L, np.maximum(L0, lifted))     # raised no further than needed
    assert (L > L0).any()


@pytest.mark.parametrize("change", ["dt_max", "lambda", "rho", "speed"])
def test_exact_scalings_shift_levels_by_one(change):
    w, _ = _random_case(n=1500)
    none = (np.zeros(w.n + 1, np.int64), np.zeros(0, np.int64))
    kw = dict(gamma=w.gamma, cfl=0.2, dt_max=0.05, max_level=40)
    L = oracle.timestep_levels(w.lam, w.U, none, **kw)
    lam, U = w.lam.copy(), w.U.copy()
    if change == "dt_max":
        kw["dt_max"] *= 2.0
    elif change == "lambda":
        lam *= 0.5
    elif change == "rho":
        U[0] *= 0.25           # c = sqrt((gamma P + B^2) / rho) doubles
    else:
        U[7] *= 4.0            # P x 4 and |B|^2 x 4: c doubles
        U[4:7] *= 2.0
    assert np.array_equal(oracle.timestep_levels(lam, U, none, **kw), L + 1)


def test_cap_and_invalid_arguments():
    w, nb = _random_case(n=500)
    L = oracle.timestep_levels(w.lam, w.U, nb, gamma=w.gamma, cfl=0.01, dt_max=10.0, max_level=3)
    assert L.max() == 3
    with pytest.raises(ValueError):
        oracle.timestep_levels(w.lam, w.U, nb, gamma=w.gamma, cfl=0.1, dt_max=0.0)
