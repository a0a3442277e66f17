"""Pins of the oracle's SPAI (Sec. 5, Eq. NormalEqSolve) against brute force, closed forms and
the frequencies printed in Table dispersionTable."""
import numpy as np

from oracle_runs import fraction, golden
import pytest
import scipy.sparse as sp

import synth
from oracle import spai as SP
from oracle.cubical2d import Torus2D, zero_crossing_frequency
from oracle.fem import FEM
from oracle.gym import GYM
from oracle.mesh import KuhnMesh


def test_diagonal_spai_closed_form():
    f = FEM(KuhnMesh(3, 2), eps=synth.tet_eps(11, 3, 1, 4))
    M = f.M1()
    Q = SP.spai_columns(M, SP.pattern("diag", M)).diagonal()
    Md = M.toarray()
    assert np.allclose(Q, np.diag(Md) / np.sum(Md ** 2, axis=0), rtol=1e-13)


@pytest.mark.parametrize("n,k,kind", [(3, 1, "sm1"), (2, 2, "sm1"), (2, 2, "sm1sq")])
def test_columns_solve_the_least_squares_problem(n, k, kind):
    """Each column minimises ||M q - 1_l|| over its pattern: compare with dense lstsq on all rows."""
    f = FEM(KuhnMesh(n, k), eps=synth.tet_eps(12, n, 1, 4))
    M = f.M1()
    S = SP.pattern(kind, M, f.dof1)
    Q = SP.spai_columns(M, S).toarray()
    Md = M.toarray()
    Sc = S.tocsc()
    rng = np.random.default_rng(0)
    for l in rng.choice(M.shape[0], size=6, replace=False):
        I = Sc.indices[Sc.indptr[l]:Sc.indptr[l + 1]]
        rhs = np.zeros(M.shape[0])
        rhs[l] = 1.0
        q, *_ = np.linalg.lstsq(Md[:, I], rhs, rcond=None)
        assert np.allclose(Q[I, l], q, rtol=1e-8, atol=1e-10 * abs(q).max())
        assert np.count_nonzero(Q[:, l]) <= len(I)


def test_structural_pattern_is_tet_sharing():
    f = FEM(KuhnMesh(2, 1))
    S = SP.pattern("sm1", f.M1(), f.dof1).toarray() > 0
    ref = np.zeros_like(S)
    for d in f.dof1:
        d = d[d >= 0]
        ref[np.ix_(d, d)] = True
    assert np.array_equal(S, ref)


@pytest.mark.parametrize("n,k", [(4, 1), (3, 2), (2, 3)])
def test_default_policy_gives_spd_without_shift(n, k):
    f = FEM(KuhnMesh(n, k), eps=synth.tet_eps(13, n, 1, 4))
    Q, info = SP.gym_q1(f)
    assert info["shift"] == 0.0 and info["lmin"] > 0
    assert abs(Q - Q.T).max() < 1e-12 * abs(Q).max()
    # the pattern of Q1 stays inside the requested structural pattern
    S = SP.pattern(info["pattern"], f.M1(), f.dof1)
    assert ((abs(Q) > 0).astype(int) - (S > 0).astype(int)).max() <= 0


def test_ortho_basis_keeps_the_dynamics_and_pattern():
    """Q1 = T^T Q' T: the GYM of basis Lambda' in integer-C variables; T is invertible, block
    diagonal over entities, and orthonormalises each entity's DoFs in the M1 inner product."""
    f = FEM(KuhnMesh(2, 2), eps=synth.tet_eps(14, 2, 1, 4))
    M1 = f.M1()
    T = SP.ortho_basis_transform(f, M1).toarray()
    Mp = T @ M1.toarray() @ T.T
    # T is block diagonal over the entities: it never couples DoFs of different entities
    Sm = SP.pattern("sm1", M1, f.dof1).toarray() > 0
    assert np.all((np.abs(T) > 0) <= Sm)
    gid = np.zeros(f.mesh.N1, int)
    for i, g in enumerate(sum(SP.entity_groups(f), [])):
        gid[list(g)] = i
    rr, cc = np.nonzero(np.abs(T) > 0)
    assert np.all(gid[rr] == gid[cc])
    # exact inverse is basis independent: T^T (T M T^T)^-1 T = M^-1
    assert np.allclose(T.T @ np.linalg.inv(Mp) @ T, np.linalg.inv(M1.toarray()), rtol=1e-8, atol=1e-10)
    # the primed mass matrix is normalised inside each entity
    for g in sum(SP.entity_groups(f), []):
        g = list(g)
        assert np.allclose(Mp[np.ix_(g, g)], np.eye(len(g)), atol=1e-10)


# ---------------------------------------------------------------- Table dispersionTable
def _dispersion(kind):
    t = Torus2D(20, 20)
    M1, C, M2 = t.M1(), t.C(), t.M2()
    if kind == "exact":
        Q = sp.csr_matrix(np.linalg.inv(M1.toarray()))
    else:
        Q, _ = SP.spai(M1, kind)
    g = GYM(C, M2, Q)
    a = t.mode_sin_y()
    omega_space = np.sqrt((a @ (Q @ (g.P2 @ a))) / (a @ a))
    # time domain: the lowest exact eigenmode v of M1^-1 P2 (here e = M1 a), CFL factor 0.3,
    # 200 periods, zero crossings of <e(t), e(0)>
    v = M1 @ a
    v /= np.linalg.norm(v)
    tau = 0.3 * g.tau_cfl()
    n = int(200 * 2 * np.pi / omega_space / tau)
    e, b = v.copy(), g.half_init(v, np.zeros(t.N2), tau)
    proj = [v @ v]
    for _ in range(n):
        e, b, _, _ = g.step(e, b, tau)
        proj.append(e @ v)
    return omega_space, zero_crossing_frequency(np.array(proj), tau), t.hx


# printed values of Table dispersionTable (tests/golden/dispersion_table.txt)
_TABLE = {r[0]: (fraction(r[1]), fraction(r[2])) for r in golden("dispersion_table.txt")}


def test_dispersion_exact_feec():
    w, wt, h = _dispersion("exact")
    assert np.isclose(w, np.sqrt(6 / h ** 2 * (1 - np.cos(h)) / (2 + np.cos(h))), rtol=1e-12)
    w0 = _TABLE["exact_feec"][0]
    assert abs(w / w0 - 1) < 1e-4 and abs(wt / w0 - 1) < 3e-4


def test_dispersion_diagonal_spai_matches_yee_row():
    w, wt, h = _dispersion("diag")
    assert np.isclose(w, np.sqrt(4.0 / 3.0) * 2 / h * np.sin(h / 2), rtol=1e-12)
    w0 = _TABLE["exact_feec"][0]
    wp, dev = _TABLE["diagonal_yee"]
    assert abs(w / wp - 1) < 1e-4 and abs(wt / wp - 1) < 3e-4
    assert abs((w - w0) / w0 - dev) < 5e-4
    # Sec. 7.6: after 200 periods the Yee-like run is ~29 periods ahead of the exact mode
    assert round(200 * (wt - w0) / w0) == 29


def test_dispersion_spai_sm1_matches_printed_value():
    w, wt, h = _dispersion("sm1")
    w0 = _TABLE["exact_feec"][0]
    wp, dev = _TABLE["spai_sm1"]
    assert abs(wt / wp - 1) < 3e-4 and abs(w / wp - 1) < 3e-4
    assert abs((wt - w0) / w0 - dev) < 5e-4
    # Sec. 7.6: and the SPAI run ~8 periods behind
    assert round(200 * (wt - w0) / w0) == -8


# ---------------------------------------------------------------- Table SPAIOPeigTable, SPAI rows
def test_spai_eigen_residual_table_rows():
    """Sec. 7.2: residual eigenvalue errors of the column SPAI on the 20 x 80 torus, per pattern,
    against the printed table (tests/golden/spai_eig_table.txt); eigenvectors of the exact
    generalised problem P2 v = lam M1 v with unit 2-norm."""
    import scipy.linalg as sl
    t = Torus2D(20, 80, Lx=5.0, Ly=20.0)
    M1, C, M2 = t.M1(), t.C(), t.M2()
    P2 = (C.T @ M2 @ C).tocsr()
    w, V = sl.eigh(P2.toarray(), M1.toarray())
    nz = np.where(w > 1e-8 * w[-1])[0]
    assert len(nz) == 1599 and t.N1 - len(nz) == 1601
    V = V[:, nz] / np.linalg.norm(V[:, nz], axis=0)
    lam = w[nz]
    for row in golden("spai_eig_table.txt"):
        Q, _ = SP.spai(M1, row[0])
        eps = np.linalg.norm(Q @ (P2 @ V) - V * lam, axis=0) / np.abs(lam)
        got = (eps.mean(), eps[:100].mean(), eps[100:].mean())
        for g, printed in zip(got, map(fraction, row[1:])):
            assert abs(g - printed) <= 5e-5, (row[0], got)


def test_spai_consistency_error_does_not_refine_away():
    """Sec. 7.1: the sparse approximation Q1 ~ M1^-1 adds a consistency error independent of h
    (first Strang lemma) that wider stencils reduce.  Lowest cavity eigenvalue of the unit PEC cube
    (2 pi^2), k = 1: exact FEEC converges at ~h^2; S(1) and S(M1) SPAI errors plateau, S(M1)'s well
    below S(1)'s."""
    import scipy.linalg as sl
    w0 = 2 * np.pi ** 2
    err = {}
    for n in (3, 6):
        f = FEM(KuhnMesh(n, 1))
        M1 = f.M1()
        P2 = (f.C().T @ f.M2() @ f.C()).tocsr().toarray()
        we = sl.eigh(P2, M1.toarray(), eigvals_only=True)
        err[n, "exact"] = (we[we > 1e-8 * we[-1]][0] - w0) / w0
        for kind in ("diag", "sm1"):
            Q, _ = SP.spai(M1, kind)
            wq = np.sort(np.linalg.eigvals(Q.toarray() @ P2).real)
            err[n, kind] = (wq[wq > 1e-8 * wq[-1]][0] - w0) / w0
    assert 3.0 < err[3, "exact"] / err[6, "exact"] < 5.0                 # ~ (6/3)^2
    for kind in ("diag", "sm1"):
        assert abs(err[6, kind]) > 0.9 * abs(err[3, kind])                # no convergence
    assert abs(err[6, "sm1"]) < 0.5 * abs(err[6, "diag"])                  # the wider stencil helps


@pytest.mark.parametrize("n,k,tol", [(3, 2, 0.015), (4, 2, 0.015), (2, 3, 0.05), (3, 3, 0.10)])
def test_default_policy_keeps_the_lowest_cavity_modes(n, k, tol):
    """Reading R2 (k >= 2: S(M1^2) SPAI in the entity-orthonormal basis): Q1 P2 keeps the three
    lowest non-kernel eigenvalues of the unit PEC cube within ~1 % (k = 2) and ~8 % (k = 3) of the
    exact FEEC values M1^-1 P2."""
    import scipy.linalg as sl
    f = FEM(KuhnMesh(n, k))
    M1 = f.M1()
    P2 = (f.C().T @ f.M2() @ f.C()).tocsr().toarray()
    we = sl.eigh(P2, M1.toarray(), eigvals_only=True)
    we = we[we > 1e-8 * we[-1]][:3]
    Q, info = SP.gym_q1(f, M1)
    assert info["shift"] == 0.0 and info["lmin"] > 0
    wq = np.sort(np.linalg.eigvals(Q.toarray() @ P2).real)
    wq = wq[wq > 1e-8 * wq[-1]][:3]
    assert np.all(np.abs(wq - we) / we < tol)


@pytest.mark.parametrize("k", [2, 3])
def test_primed_basis_assembled_tet_by_tet_gives_the_same_q1(k):
    """Reading R2, pinned from a second route: the primed mass matrix assembled tet by tet from the
    transformed local blocks (T restricted to each tet's DoFs: every entity lies in the tet)
    equals T M1 T^T, is the identity inside every entity, and its column SPAI mapped back as
    T^T Q' T is, entry by entry, the Q1 of gym_q1."""
    f = FEM(KuhnMesh(2, k), eps=synth.tet_eps(15 + k, 2, 1, 4))
    M1 = f.M1()
    T = SP.ortho_basis_transform(f, M1).toarray()
    N1 = f.mesh.N1
    Mp = np.zeros((N1, N1))
    for t in range(f.mesh.n_tets):
        d = f.dof1[t]
        ok = np.nonzero(d >= 0)[0]
        g = d[ok]
        blk = f.eps[t] * f.local(f.mesh.tet_shape[t])["M1"][np.ix_(ok, ok)]
        Tt = T[np.ix_(g, g)]
        Mp[np.ix_(g, g)] += Tt @ blk @ Tt.T
    assert np.allclose(Mp, T @ M1.toarray() @ T.T, rtol=0, atol=1e-12 * np.abs(Mp).max())
    for grp in sum(SP.entity_groups(f), []):
        grp = list(grp)
        assert np.allclose(Mp[np.ix_(grp, grp)], np.eye(len(grp)), atol=1e-10)
    S = SP.pattern("sm1sq", M1, f.dof1)
    Qp = SP.symmetrize(SP.spai_columns(sp.csr_matrix(Mp), S)).toarray()
    Q_route2 = T.T @ Qp @ T
    Q_route2 = 0.5 * (Q_route2 + Q_route2.T)
    Q, _ = SP.gym_q1(f, M1)
    assert np.abs(Q_route2 - Q.toarray()).max() <= 1e-9 * np.abs(Q.toarray()).max()
