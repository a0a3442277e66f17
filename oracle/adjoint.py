"""Discrete adjoint of the GYM leapfrog: gradient of a probe-region field energy with respect to
the per-tet permittivity (order 1, column SPAI on S(M1)).

Oracle (test infrastructure; see oracle/__init__.py).  Plain, dense, for tiny meshes.

Loss (a reading: the paper defines no loss; this is the probe-region energy of the adjoint row)
    L(eps) = tau sum_{n=0}^{N-1} [ 1/2 x_n^T M1^R x_n + 1/2 b_{n+1/2}^T M2^R b_{n+1/2} ],
    x_n = Q1 e_n, with M1^R, M2^R the mass matrices assembled over the tets of a region R only.
The forward map is the leapfrog of Eq. YeeLeapfrog in the GYM form of Eq. preYeeFEECEqns, from
e_0 = b_0 = 0 and driven by a dipole current (the current term of Eq. allEOM); tau is held fixed.
eps enters through M1(eps) = sum_T eps_T M1^T (Sec. 2), hence through M1^R and through
Q1 = (P + P^T) / 2, P the column SPAI of Eq. NormalEqSolve on the structural pattern S(M1).

Reverse sweep (transposes of the three shear-map operations, newest step first):
    bbar   += tau M2 C ebar + tau M2^R b_{n+1/2}        (b_{n+1/2} feeds e_{n+1} and the loss)
    xbar    = -tau C^T bbar + tau M1^R x_n              (x_n feeds b_{n+1/2} and the loss)
    ebar   += Q1 xbar ;  Q1bar += xbar e_n^T             (x_n = Q1 e_n)
SPAI derivative (per column l, A = M1(:, I_l), q = (A^T A)^-1 A^T 1_l, r = 1_l - A q):
    dq = (A^T A)^-1 (dA^T r - A^T dA q),  so  g^T dq = (dA z)^T r - (A z)^T (dA q),  z = (A^T A)^-1 g,
with g = Pbar(I_l, l), Pbar = (Q1bar + Q1bar^T) / 2 and dA = M1^T(:, I_l) for d eps_T.
Pinned by tests/test_oracle_adjoint.py against central finite differences of the whole pipeline.
"""
import numpy as np
import scipy.sparse as sp

from . import spai as SP


def element_M1(fem, t):
    """Unweighted element matrix of tet t as a dense N1 x N1 array (dM1 / d eps_t)."""
    N1 = fem.mesh.N1
    D = np.zeros((N1, N1))
    blk = fem.local(fem.mesh.tet_shape[t])["M1"]
    dofs = fem.dof1[t]
    for a, i in enumerate(dofs):
        if i < 0:
            continue
        for b, j in enumerate(dofs):
            if j >= 0:
                D[i, j] += blk[a, b]
    return D


def region_mass(fem, region):
    """(M1^R, M2^R): mass matrices over the tets in `region` only (boolean per tet)."""
    w1 = np.where(region, fem.eps, 0.0)
    w2 = np.where(region, 1.0 / fem.mu, 0.0)
    N1, N2 = fem.mesh.N1, fem.mesh.N2
    return (fem._sparse("M1", fem.dof1, fem.dof1, w1, (N1, N1)).toarray(),
            fem._sparse("M2", fem.dof2, fem.dof2, w2, (N2, N2)).toarray())


def q1_of(fem, S):
    """Q1 = (P + P^T) / 2 with P the column SPAI of M1(eps) on the fixed pattern S."""
    return SP.symmetrize(SP.spai_columns(fem.M1(), S)).toarray()


def forward(C, M2, Q, MR1, MR2, J, tau, nsteps):
    """Leapfrog from e = b = 0 with currents J[n] at t_{n+1/2}; returns (L, e_n list, x_n list, b_{n+1/2} list)."""
    N1, N2 = Q.shape[0], C.shape[0]
    e, b = np.zeros(N1), np.zeros(N2)
    es, xs, bs = [], [], []
    L = 0.0
    for n in range(nsteps):
        x = Q @ e
        b = b - tau * (C @ x)
        es.append(e)
        xs.append(x)
        bs.append(b)
        L += tau * (0.5 * x @ (MR1 @ x) + 0.5 * b @ (MR2 @ b))
        e = e + tau * (C.T @ (M2 @ b)) - tau * J[n]
    return L, es, xs, bs


def reverse(C, M2, Q, MR1, MR2, tau, es, xs, bs):
    """Reverse sweep; returns (Q1bar, M1Rbar) = (dL/dQ1, dL/dM1^R) as dense arrays."""
    N1, N2 = Q.shape[0], C.shape[0]
    ebar, bbar = np.zeros(N1), np.zeros(N2)
    Qbar = np.zeros((N1, N1))
    MRbar = np.zeros((N1, N1))
    for n in range(len(es) - 1, -1, -1):
        bbar = bbar + tau * (M2 @ (C @ ebar)) + tau * (MR2 @ bs[n])
        xbar = -tau * (C.T @ bbar) + tau * (MR1 @ xs[n])
        ebar = ebar + Q @ xbar
        Qbar += np.outer(xbar, es[n])
        MRbar += 0.5 * tau * np.outer(xs[n], xs[n])
    return Qbar, MRbar


def spai_vjp(fem, S, Pbar):
    """sum_l g_l^T dq_l / d eps_t for every tet t (the column SPAI of Eq. NormalEqSolve)."""
    M = fem.M1().toarray()
    S = sp.csc_matrix(S)
    T = fem.mesh.n_tets
    dM = [element_M1(fem, t) for t in range(T)]
    grad = np.zeros(T)
    N = M.shape[0]
    for l in range(N):
        I = S.indices[S.indptr[l]:S.indptr[l + 1]]
        A = M[:, I]
        AtA = A.T @ A
        one = np.zeros(N)
        one[l] = 1.0
        q = np.linalg.solve(AtA, A.T @ one)
        r = one - A @ q
        z = np.linalg.solve(AtA, Pbar[I, l])
        Az = A @ z
        for t in range(T):
            dA = dM[t][:, I]
            grad[t] += (dA @ z) @ r - Az @ (dA @ q)
    return grad


def loss_and_gradient(make_fem, eps, region, source, tau, nsteps):
    """L and dL/d eps (per tet) for the recipe above.  make_fem(eps) builds the FEM object;
    source(fem) returns the list of per-step currents J[n]."""
    fem = make_fem(eps)
    S = SP.pattern("sm1", fem.M1(), fem.dof1)
    Q = q1_of(fem, S)
    C, M2 = fem.C().toarray(), fem.M2().toarray()
    MR1, MR2 = region_mass(fem, region)
    J = source(fem)
    L, es, xs, bs = forward(C, M2, Q, MR1, MR2, J, tau, nsteps)
    Qbar, MRbar = reverse(C, M2, Q, MR1, MR2, tau, es, xs, bs)
    Sd = S.toarray() != 0
    Pbar = 0.5 * (Qbar + Qbar.T) * Sd
    grad = spai_vjp(fem, S, Pbar)
    for t in np.nonzero(region)[0]:
        grad[t] += np.sum(MRbar * element_M1(fem, t))
    return L, grad
