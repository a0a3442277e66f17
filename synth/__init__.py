"""Seeded synthetic inputs shared by the oracle and the CUDA path.

This module holds random-number generation and workload recipes only; it
contains none of the method's arithmetic (no mesh, basis, mass matrix, SPAI
or time stepping).  Every draw comes from the counter form of splitmix64:
output i of the stream with seed s is mix(s + (i + 1) * 0x9E3779B97F4A7C15),
where mix is the published splitmix64 finaliser (Steele, Lea, Flood 2014).
Seeds follow the rule  seed = 1000 * config_index + purpose  with purposes
0 = per-tet permittivity, 1 = source positions, 2 = source orientations,
3 = mesh size / order draws, 4 = finite-difference tets, 5 = probe region.
"""
import numpy as np

_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(seed: int, n: int, start: int = 0) -> np.ndarray:
    """Outputs start .. start+n-1 of the splitmix64 stream for `seed` (uint64)."""
    with np.errstate(over="ignore"):
        i = np.arange(start + 1, start + n + 1, dtype=np.uint64)
        z = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + i * _GAMMA
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return z


def uniform(seed: int, n: int, lo: float = 0.0, hi: float = 1.0, start: int = 0) -> np.ndarray:
    """n doubles uniform in [lo, hi): the top 53 bits of each output times 2^-53."""
    u = (splitmix64(seed, n, start) >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)
    return lo + (hi - lo) * u


def normal(seed: int, n: int) -> np.ndarray:
    """n standard normal doubles by Box-Muller on consecutive uniform pairs."""
    u = uniform(seed, 2 * n)
    u1 = 1.0 - u[0::2]            # (0, 1]
    u2 = u[1::2]
    return np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * np.pi * u2)


def tet_eps(seed: int, n_cubes: int, lo: float, hi: float) -> np.ndarray:
    """Per-tet permittivity, i.i.d. uniform in [lo, hi), length 6 n^3 (tet order of the mesh)."""
    return uniform(seed, 6 * n_cubes ** 3, lo, hi)


def source_positions(seed: int, count: int, lo: float = 0.2, hi: float = 0.8, side: float = 1.0) -> np.ndarray:
    """count points uniform in [lo, hi)^3 * side, shape (count, 3)."""
    return (uniform(seed, 3 * count, lo, hi) * side).reshape(count, 3)


def unit_vectors(seed: int, count: int) -> np.ndarray:
    """count unit vectors (normalised Gaussian triples), shape (count, 3)."""
    g = normal(seed, 3 * count).reshape(count, 3)
    return g / np.linalg.norm(g, axis=1, keepdims=True)


# ---- workload recipes (sizes and seeds of the benchmark cavities) ----------

def cavity_config(index: int) -> dict:
    """The synthetic PEC-cube cavity workloads.

    1: N=4, k=1, eps=mu=1, analytic (1,1,0) mode E = z sin(pi x) sin(pi y), 1000 steps, FP64.
    2: N=32, k=2, eps_T ~ U[1,4) (seed 2000), mu=1, one z-dipole pulse at a point
       ~ U[0.2,0.8)^3 (seed 2001), centre frequency pi*sqrt(5), width 20 steps, 2000 steps.
    3: N=48, k=3, eps_T ~ U[1,4) (seed 3000), 64 dipoles (positions seed 3001,
       orientations seed 3002), 1000 steps.
    """
    if index == 1:
        return dict(n=4, order=1, eps=None, mu=None, steps=1000, n_rhs=1,
                    mode="te110", sources=[])
    if index == 2:
        n = 32
        x0 = source_positions(2001, 1)[0]
        return dict(n=n, order=2, eps=tet_eps(2000, n, 1.0, 4.0), mu=None, steps=2000, n_rhs=1,
                    mode="zero", sources=[dict(x=x0, d=np.array([0.0, 0.0, 1.0]), amp=1.0,
                                               omega=np.pi * np.sqrt(5.0), width_steps=20.0, rhs=0)])
    if index == 3:
        n = 48
        xs = source_positions(3001, 64)
        ds = unit_vectors(3002, 64)
        return dict(n=n, order=3, eps=tet_eps(3000, n, 1.0, 4.0), mu=None, steps=1000, n_rhs=64,
                    mode="zero", sources=[dict(x=xs[r], d=ds[r], amp=1.0, omega=np.pi * np.sqrt(5.0),
                                               width_steps=20.0, rhs=r) for r in range(64)])
    raise ValueError(index)
