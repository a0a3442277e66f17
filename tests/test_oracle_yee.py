"""Sec. 4 pin: the oracle's GYM leapfrog with cubical Whitney forms and lumped masses
(Q1 = Delta_V^-1 I, M2 = Delta_V I) equals a textbook Yee FDTD loop to machine precision."""
import numpy as np
import scipy.sparse as sp

from oracle.gym import GYM
from oracle.yee3d import PeriodicCubes, yee_textbook
from oracle_runs import fraction, golden


def test_gym_with_lumped_cubical_whitney_is_yee():
    g = PeriodicCubes()
    nx, ny, nz = g.n
    rng = np.random.default_rng(0)
    E = [rng.standard_normal((nx, ny, nz), ) for _ in range(3)]
    C = g.C()
    gym = GYM(C, sp.identity(g.N2) * g.dV, sp.identity(g.N1) / g.dV)
    # field coefficients of the average-normalised basis are the Yee values; e = M1^Y E = dV E
    a_E = np.concatenate([E[a].transpose(2, 1, 0).ravel() for a in range(3)])
    e0 = g.dV * a_E
    b0 = np.zeros(g.N2)
    tau = 0.4 * gym.tau_cfl()
    for nsteps in (1, 25):
        e, b, _ = gym.run(e0.copy(), gym.half_init(e0, b0, tau), tau, nsteps)
        # textbook Yee from E^0, B^0 = 0 with the same initial half step B^{-1/2} = B^0 + tau/2 curl E^0
        hx, hy, hz = g.h
        d = lambda a, ax: np.roll(a, -1, axis=ax) - a
        Bh = [(tau / 2) * (d(E[2], 1) / hy - d(E[1], 2) / hz), (tau / 2) * (d(E[0], 2) / hz - d(E[2], 0) / hx),
              (tau / 2) * (d(E[1], 0) / hx - d(E[0], 1) / hy)]
        Ey_, By_ = yee_textbook(E, Bh, tau, g.h, nsteps)
        e_yee = np.concatenate([Ey_[a].transpose(2, 1, 0).ravel() for a in range(3)])
        b_yee = np.concatenate([By_[a].transpose(2, 1, 0).ravel() for a in range(3)])
        assert np.linalg.norm(e / g.dV - e_yee) / np.linalg.norm(e_yee) < 1e-14
        assert np.linalg.norm(b - b_yee) / np.linalg.norm(b_yee) < 1e-14


def test_cubical_complex_identities():
    g = PeriodicCubes()
    C = g.C()
    # grad: vertex -> edges (a_e = phi(head) - phi(tail)) / h : curl grad = 0
    nx, ny, nz = g.n
    r, c, v = [], [], []
    for k in range(nz):
        for j in range(ny):
            for i in range(nx):
                for a, (di, dj, dk) in enumerate(((1, 0, 0), (0, 1, 0), (0, 0, 1))):
                    e = g.edge(a, i, j, k)
                    r += [e, e]
                    c += [g.cell(i + di, j + dj, k + dk), g.cell(i, j, k)]
                    v += [1.0 / g.h[a], -1.0 / g.h[a]]
    G = sp.csr_matrix((v, (r, c)), shape=(g.N1, g.nc))
    assert abs(C @ G).max() < 1e-12


def test_whitney_cube_masses_match_printed_values():
    """The oracle's consistent cubical Whitney masses, assembled by quadrature, reproduce the
    entries printed in Sec. 4 (Eq. whitMassMatrices) and the unit row sums that motivate the
    lumped Yee masses (tests/golden/whitney_cube_masses.txt)."""
    ref = {(r[0], r[1]): fraction(r[2]) for r in golden("whitney_cube_masses.txt")}
    g = PeriodicCubes()
    nx, ny, nz = g.n
    M1, M2 = g.M1().tocsr(), g.M2().tocsr()

    def decode(idx):
        a, cell = divmod(idx, g.nc)
        return a, (cell % nx, (cell // nx) % ny, cell // (nx * ny))

    def wrap(d, n):
        d = d % n
        return d - n if d > n // 2 else d

    seen1, seen2 = set(), set()
    for M, seen, kind in ((M1, seen1, "M1"), (M2, seen2, "M2")):
        for i in range(M.shape[0]):
            ai, pi = decode(i)
            row = M.getrow(i)
            assert abs(row.sum() / g.dV - ref[("rowsum", "every_row_of_M1_and_M2")]) < 1e-13
            for j, v in zip(row.indices, row.data):
                aj, pj = decode(j)
                assert ai == aj                       # perpendicular functions are L2-orthogonal
                d = [wrap(pj[t] - pi[t], g.n[t]) for t in range(3)]
                perp = [abs(d[t]) for t in range(3) if t != ai]
                if kind == "M1":
                    assert d[ai] == 0
                    rel = {0: "same_edge", 1: "parallel_edges_sharing_a_face",
                           2: "parallel_edges_sharing_only_a_cell"}[sum(perp)]
                    assert max(perp) <= 1
                else:
                    assert perp == [0, 0] and abs(d[ai]) <= 1
                    rel = "same_face" if d[ai] == 0 else "parallel_faces_of_one_cell"
                assert abs(v / g.dV - ref[(kind, rel)]) < 1e-13, (kind, rel, v / g.dV)
                seen.add(rel)
    assert len(seen1) == 3 and len(seen2) == 2
