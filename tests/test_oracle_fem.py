"""Pins of the oracle's bases and mass matrices: finite differences, closed forms,
polynomial reproduction, the L2 re-derivation of C, and the cavity spectrum."""
import numpy as np
import pytest
import scipy.linalg as sl
import scipy.sparse.linalg as spl

from oracle import basis as B
from oracle.mesh import KuhnMesh, LOCAL_EDGES
from oracle.fem import FEM


def _random_tet(rng):
    X = rng.normal(size=(4, 3))
    return X if np.linalg.det(X[1:] - X[0]) > 0.3 else _random_tet(rng)


@pytest.mark.parametrize("k", [1, 2, 3])
def test_curls_match_finite_differences(k):
    rng = np.random.default_rng(k)
    X = _random_tet(rng)
    g = B.bary_gradients(X)
    A = np.vstack([np.ones(4), X.T])
    pts = rng.dirichlet(np.ones(4), size=5) @ X
    h = 1e-6
    for f in B.one_forms(k):
        def val(x):
            L = np.linalg.solve(A, np.concatenate([[1.0], x]))[None, :]
            return B.eval1(f, L, g)[0][0]
        for x in pts:
            J = np.stack([(val(x + h * e) - val(x - h * e)) / (2 * h) for e in np.eye(3)], axis=1)
            fd = np.array([J[2, 1] - J[1, 2], J[0, 2] - J[2, 0], J[1, 0] - J[0, 1]])
            L = np.linalg.solve(A, np.concatenate([[1.0], x]))[None, :]
            assert np.allclose(B.eval1(f, L, g)[1][0], fd, atol=1e-6)


def test_quadrature_exact_for_barycentric_monomials():
    """int_T l^a = |T| a! 3! / (|a| + 3)!  (a textbook identity), up to degree 7."""
    from math import factorial
    rng = np.random.default_rng(0)
    X = _random_tet(rng)
    L, W = B.tet_quadrature(X, 6)
    vol = B.tet_volume(X)
    for a in [(0, 0, 0, 0), (2, 1, 0, 0), (1, 1, 1, 1), (3, 0, 2, 1), (0, 4, 0, 3), (6, 0, 0, 1)]:
        exact = vol * np.prod([factorial(x) for x in a]) * 6 / factorial(sum(a) + 3)
        assert np.isclose(np.sum(W * np.prod(L ** np.array(a), axis=1)), exact, rtol=1e-12)


def test_whitney_mass_closed_form():
    """k = 1: (M1)_{ab,cd} = int (l_a g_b - l_b g_a).(l_c g_d - l_d g_c) with int l_i l_j = |T|(1+d_ij)/20."""
    f = FEM(KuhnMesh(1, 1))
    for s in range(6):
        loc = f.local(s)
        g, vol = loc["g"], loc["vol"]
        mij = lambda i, j: vol * (1 + (i == j)) / 20.0
        M = np.zeros((6, 6))
        for p, (a, b) in enumerate(LOCAL_EDGES):
            for q, (c, d) in enumerate(LOCAL_EDGES):
                M[p, q] = (mij(a, c) * g[b] @ g[d] - mij(a, d) * g[b] @ g[c]
                           - mij(b, c) * g[a] @ g[d] + mij(b, d) * g[a] @ g[c])
        assert np.allclose(loc["M1"], M, rtol=1e-13, atol=1e-15)


@pytest.mark.parametrize("k", [1, 2, 3])
def test_local_blocks_identical_for_all_kuhn_shapes(k):
    """The six Kuhn tets are congruent (axis permutations); in local order their blocks coincide."""
    f = FEM(KuhnMesh(1, k))
    for key in ("M1", "M2"):
        ref = f.local(0)[key]
        for s in range(1, 6):
            assert np.allclose(f.local(s)[key], ref, rtol=1e-12, atol=1e-14 * abs(ref).max())


@pytest.mark.parametrize("n,k", [(2, 1), (3, 1), (2, 2), (2, 3)])
def test_curl_rederived_by_l2_projection(n, k):
    """M2 C_num = B with B_ij = int curl(Lambda1_j) . Lambda2_i must give the integer C."""
    f = FEM(KuhnMesh(n, k))
    solve = lambda M, Bm: np.asarray(sl.solve(M.toarray(), Bm.toarray(), assume_a="pos"))
    Cn = solve(f.M2(), f.B_curl())
    C = f.C().toarray()
    assert np.array_equal(np.round(Cn), C)
    assert abs(Cn - C).max() < 1e-9
    Gn = solve(f.M1(), f.B_grad())
    assert abs(Gn - f.G().toarray()).max() < 1e-9
    Dn = solve(f.M3(), f.B_div())
    assert abs(Dn - f.D().toarray()).max() < 1e-9


def test_constant_field_interpolant_reproduces_load_vector():
    """Whitney forms reproduce constant fields: (M1 Pi^1 E)_i = int E . Lambda1_i, checked on the
    DoFs whose every tet keeps all its DoFs (PEC removes the boundary ones)."""
    f = FEM(KuhnMesh(4, 1))
    E = np.array([0.3, -1.2, 0.7])
    field = lambda x: np.broadcast_to(E, x.shape) * 1.0
    c = f.edge_interpolant(field)
    F = f.load_vector(field)
    full = np.all(f.dof1 >= 0, axis=1)
    deep = np.ones(f.mesh.N1, bool)
    for t in np.where(~full)[0]:
        deep[f.dof1[t][f.dof1[t] >= 0]] = False
    assert deep.sum() > 20
    assert np.allclose((f.M1() @ c)[deep], F[deep], rtol=1e-12, atol=1e-15)


@pytest.mark.parametrize("k", [2, 3])
def test_linear_field_reproduced_by_l2_projection(k):
    f = FEM(KuhnMesh(2, k))
    A = np.array([[0.2, -1.0, 0.5], [1.1, 0.3, -0.4], [0.0, 0.7, 0.9]])
    b = np.array([0.1, 0.2, -0.3])
    # PEC removes boundary DoFs, so test on a field with zero tangential trace: use the full
    # local reproduction on one tet instead (local space contains P1 fields)
    X = f.mesh.tet_vx[17]
    g = B.bary_gradients(X)
    L, W = B.tet_quadrature(X, 6)
    x = L @ X
    vals = np.stack([B.eval1(fn, L, g)[0] for fn in f.F1])
    Mloc = np.einsum("ipx,jpx,p->ij", vals, vals, W)
    Fv = np.einsum("ipx,px,p->i", vals, x @ A.T + b, W)
    c = np.linalg.solve(Mloc, Fv)
    rng = np.random.default_rng(1)
    Lp = rng.dirichlet(np.ones(4), size=7)
    approx = np.einsum("i,ipx->px", c, np.stack([B.eval1(fn, Lp, g)[0] for fn in f.F1]))
    assert np.allclose(approx, (Lp @ X) @ A.T + b, atol=1e-10)


def _cavity(n, k):
    f = FEM(KuhnMesh(n, k))
    C = f.C()
    P2 = (C.T @ f.M2() @ C).toarray()
    w = sl.eigh(P2, f.M1().toarray(), eigvals_only=True)
    tol = 1e-8 * w.max()
    return f.mesh, np.sum(np.abs(w) < tol), np.sort(w[w > tol])


@pytest.mark.parametrize("k,ns,min_order", [(1, (2, 4), 1.6), (2, (3, 4), 3.3), (3, (2, 3), 5.0)])
def test_cavity_spectrum_converges_to_analytic_modes(k, ns, min_order):
    """Exact FEEC (dense generalized eigenproblem P2 v = w^2 M1 v) on the PEC unit cube:
    kernel multiplicity N0 and the lowest eigenvalues -> pi^2 (m^2 + n^2 + l^2) = 2pi^2 (x3), 3pi^2 (x2)."""
    exact = np.pi ** 2 * np.array([2, 2, 2, 3, 3])
    errs = []
    for n in ns:
        mesh, nzero, w = _cavity(n, k)
        assert nzero == mesh.N0
        errs.append(np.abs(w[:5] - exact) / exact)
    order = np.log(errs[0].max() / errs[1].max()) / np.log(ns[1] / ns[0])
    assert order > min_order
    assert errs[1].max() < [0.15, 0.01, 1e-3][k - 1]
