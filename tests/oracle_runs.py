"""Oracle trajectories used as expected values by the GPU parity tests (test helper)."""
import numpy as np

import synth
from oracle import spai as SP
from oracle.fem import FEM
from oracle.gym import GYM, DipoleSource
from oracle.mesh import KuhnMesh

_cache = {}


def oracle_model(n, k, eps_seed=None, eps_range=(1.0, 4.0), pattern=None):
    key = (n, k, eps_seed, eps_range, pattern)
    if key not in _cache:
        eps = None if eps_seed is None else synth.tet_eps(eps_seed, n, *eps_range)
        f = FEM(KuhnMesh(n, k), eps=eps)
        M1 = f.M1()
        Q, info = SP.gym_q1(f, M1, pattern_kind=pattern)
        g = GYM(f.C(), f.M2(), Q, M1)
        _cache[key] = (f, g, eps, info)
    return _cache[key]


def te110(x):
    x = np.atleast_2d(x)
    return np.stack([0 * x[:, 0], 0 * x[:, 0], np.sin(np.pi * x[:, 0]) * np.sin(np.pi * x[:, 1])], axis=1)


def run_oracle(f, g, e0, b0, tau, nsteps, sources=(), energy_every=0):
    """(e_n, b_{n-1/2}, b_n synced, W history) after nsteps from a synchronised (e0, b0)."""
    J = DipoleSource(f, list(sources), tau) if sources else None
    b = g.half_init(e0, b0, tau)
    e, b, W = g.run(e0.copy(), b, tau, nsteps, source=J, energy_every=energy_every)
    return e, b, g.sync(e, b, tau), np.array(W)


def rel_l2(a, b):
    return float(np.linalg.norm(np.asarray(a, float) - np.asarray(b, float)) / max(np.linalg.norm(b), 1e-300))


def golden(name):
    """Rows of a golden fixture under tests/golden/ (whitespace-separated, '#' comments)."""
    import os
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", name)
    rows = []
    with open(path) as f:
        for line in f:
            line = line.split("#", 1)[0].strip()
            if line:
                rows.append(line.split())
    return rows


def fraction(text):
    """'4/9' -> 0.444..., '1' -> 1.0, '+0.145' -> 0.145."""
    if "/" in text:
        a, b = text.split("/")
        return float(a) / float(b)
    return float(text)
