"""Discrete adjoint of the GYM leapfrog: gradient of a probe-region field energy with respect to
the per-tet permittivity, through the Q1 policy of each order (order 1: column SPAI on S(M1);
orders >= 2: the entity-orthonormal S(M1^2) SPAI of reading R2, see the second block below).

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


# ----------------------------------------------------------------------------
# Orders >= 2: Q1 = T Q' T in the entity-orthonormal basis (reading R2 of the column SPAI)
#   T = blockdiag_g (M1[g, g])^(-1/2),  M' = T M1 T,  Q' = (P' + P'^T) / 2,  P' = SPAI(M') on S.
# Reverse mode, T and Q' symmetric:
#   Q'bar = T Q1bar T,                      Tbar  = Q1bar T Q' + Q' T Q1bar
#   P'bar = (Q'bar + Q'bar^T) / 2 on S,     M'bar = sum_l [r z^T - (A z) q^T] in the columns I_l
#   M1bar = T M'bar T,                      Tbar += M'bar T M1 + M1 T M'bar
#   M1bar[g, g] += V (Gamma o (V^T Tbar[g, g] V)) V^T  (derivative of A^(-1/2), A = M1[g, g] = V w V^T,
#                  Gamma_ij = (w_i^-1/2 - w_j^-1/2) / (w_i - w_j), or -w_i^-3/2 / 2 when w_i = w_j)
#   dL/d eps_T = sum_ij M1bar_ij (M1^T)_ij
# ----------------------------------------------------------------------------
def _groups(fem):
    e, f, c = SP.entity_groups(fem)
    return [list(g) for g in e + f + c]


def q1_ortho_of(fem, S):
    """Q1 of the k >= 2 policy, dense (the same steps as oracle.spai.gym_q1 with the ortho basis)."""
    M1 = fem.M1()
    T = SP.ortho_basis_transform(fem, M1)
    Mp = (T @ M1 @ T.T).tocsr()
    return SP.symmetrize((T.T @ SP.symmetrize(SP.spai_columns(Mp, S)) @ T).tocsr()).toarray()


def spai_vjp_matrix(M, S, Pbar):
    """dL/dM (dense, all entries) of the column SPAI P = SPAI(M) for a given Pbar on S."""
    S = sp.csc_matrix(S)
    N = M.shape[0]
    Mbar = np.zeros((N, N))
    for l in range(N):
        I = S.indices[S.indptr[l]:S.indptr[l + 1]]
        A = M[:, I]
        AtA = A.T @ A
        one = np.zeros(N)
        one[l] = 1.0
        q = np.linalg.solve(AtA, A.T @ one)
        r = one - A @ q
        z = np.linalg.solve(AtA, Pbar[I, l])
        Mbar[:, I] += np.outer(r, z) - np.outer(A @ z, q)
    return Mbar


def q1_ortho_vjp(fem, S, Q1bar):
    """dL/d eps per tet through the k >= 2 Q1 (see the block comment above)."""
    M1 = fem.M1().toarray()
    N = M1.shape[0]
    groups = _groups(fem)
    T = np.zeros((N, N))
    eig = []
    for g in groups:
        w, V = np.linalg.eigh(M1[np.ix_(g, g)])
        T[np.ix_(g, g)] = (V / np.sqrt(w)) @ V.T
        eig.append((w, V))
    Mp = T @ M1 @ T
    Pp = SP.spai_columns(sp.csr_matrix(Mp), S).toarray()
    Qp = 0.5 * (Pp + Pp.T)
    Sd = sp.csr_matrix(S).toarray() != 0
    Qpbar = T @ Q1bar @ T
    Tbar = Q1bar @ T @ Qp + Qp @ T @ Q1bar
    Ppbar = 0.5 * (Qpbar + Qpbar.T) * Sd
    Mpbar = spai_vjp_matrix(Mp, S, Ppbar)
    M1bar = T @ Mpbar @ T
    Tbar += Mpbar @ T @ M1 + M1 @ T @ Mpbar
    for g, (w, V) in zip(groups, eig):
        f = w ** -0.5
        dw = w[:, None] - w[None, :]
        same = np.abs(dw) <= 1e-12 * np.abs(w).max()
        Gam = np.where(same, -0.5 * w[:, None] ** -1.5, (f[:, None] - f[None, :]) / np.where(same, 1.0, dw))
        M1bar[np.ix_(g, g)] += V @ (Gam * (V.T @ Tbar[np.ix_(g, g)] @ V)) @ V.T
    return np.array([np.sum(M1bar * element_M1(fem, t)) for t in range(fem.mesh.n_tets)])


def loss_and_gradient_policy(make_fem, eps, region, source, tau, nsteps):
    """loss_and_gradient under the Q1 policy of the order: the column SPAI on S(M1) at k = 1, the
    entity-orthonormal S(M1^2) SPAI at k >= 2."""
    fem = make_fem(eps)
    if fem.mesh.k == 1:
        return loss_and_gradient(make_fem, eps, region, source, tau, nsteps)
    S = SP.pattern("sm1sq", fem.M1(), fem.dof1)
    Q = q1_ortho_of(fem, S)
    C, M2 = fem.C().toarray(), fem.M2().toarray()
    MR1, MR2 = region_mass(fem, region)
    J = source(fem)
    L, es, xs, bs = forward(C, M2, Q, MR1, MR2, J, tau, nsteps)
    Qbar, MRbar = reverse(C, M2, Q, MR1, MR2, tau, es, xs, bs)
    Qbar = Qbar * (S.toarray() != 0)              # T Q' T vanishes off S for every eps (S is entity-closed)
    grad = q1_ortho_vjp(fem, S, Qbar)
    for t in np.nonzero(region)[0]:
        grad[t] += np.sum(MRbar * element_M1(fem, t))
    return L, grad
