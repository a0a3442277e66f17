"""Operator-probed SPAI (SPAI-OP, Sec. 5.1), FP64, dense and plain.

Oracle (test infrastructure; see oracle/__init__.py).  Follows the paper's steps in its notation:

  objective      O(Q1) = ||M1 Q1 - 1||_F^2 + lam sum_k ||(M1 Q1 - 1) P2 v_k||^2   (Eq. SPAIOPobjective)
  definitions    U = M1^2,  W = P2 V,  T^ = 1 + lam W W^T,  R^ = M1 T^ + T^ M1      (Eq. ThatDefinition)
  stationarity   (U Q1 T^ + T^ Q1 U)_ij = R^_ij  for every (i, j) in S               (Eq. SPAIOPSylvester)
  vector form    A q = r with A_jk = U_{ir(j) ir(k)} T^_{ic(k) ic(j)}
                                    + T^_{ir(j) ir(k)} U_{ic(k) ic(j)}               (Eq. SPAIOPcoefficient)
  solver         PCG with the diagonal preconditioner of Eq. diagonalPreconditioner,
                 A q evaluated matrix-free (assemble Q1 on S, form U Q1 T^ + T^ Q1 U,
                 read it on S), warm start from the symmetrised column-wise SPAI.

Matrices are dense here (the meshes the oracle runs are small): every product is the one the
paper writes, with no reordering.  `sylvester_matrix` builds A entry by entry from Eq.
SPAIOPcoefficient, so tiny cases can be solved directly as an independent check of the PCG.

Readings (the paper leaves them open):
  - the Tikhonov term eps of A + eps 1 defaults to 0: A is already positive definite when M1 is
    (it is a principal submatrix of the Kronecker sum of two SPD matrices);
  - the PCG stops when ||r_k|| <= tol ||r_0|| with the residual of A q = r;
  - probe vectors are used as given; the pins use eigenvectors normalised in the M1 inner
    product (v^T M1 v = 1), the normalisation that reproduces the printed SPAI-OP numbers.

Parity is pinned in tests/test_oracle_spai_op.py: the lam = 0 solution equals the column-wise
SPAI on the periodic grid (Sec. 7.2), PCG at lam = 0 converges in two iterations (Sec. 5.1), the
solution is symmetric, PCG agrees with the dense solve of the explicit A, and the single-mode
probe of Sec. 7.6 (lam = 5e5) reproduces the SPAI-OP row of Table dispersionTable, and probing the
100 lowest modes at the lambda* of Table kneeTable reproduces the SPAI-OP rows of Table
SPAIOPeigTable.  `spai_op_sparse` evaluates the same products on the pattern only (for the 3200-DoF
torus of Sec. 7.2); it is pinned to the dense form on a small torus.
"""
import numpy as np
import scipy.sparse as sp


def pattern_pairs(S):
    """(i_r(k), i_c(k)) of a sparse pattern S, row-major order."""
    S = sp.csr_matrix(S)
    S.sort_indices()
    rows = np.repeat(np.arange(S.shape[0]), np.diff(S.indptr))
    return rows, S.indices.copy()


def t_hat(n, W=None, lam=0.0):
    """T^ = 1 + lam W W^T (Eq. ThatDefinition), dense."""
    T = np.eye(n)
    if W is not None and lam != 0.0:
        W = np.asarray(W, dtype=float).reshape(n, -1)
        T = T + lam * (W @ W.T)
    return T


def sylvester_apply(q, ir, ic, U, T, n):
    """(A q)_j = (U Q1 T^ + T^ Q1 U)_{ir(j), ic(j)} with Q1 assembled from q on S."""
    Q = np.zeros((n, n))
    Q[ir, ic] = q
    Smat = U @ Q @ T + T @ Q @ U
    return Smat[ir, ic]


def sylvester_matrix(ir, ic, U, T):
    """Explicit A of Eq. SPAIOPcoefficient (tiny cases only)."""
    return U[np.ix_(ir, ir)] * T[np.ix_(ic, ic)].T + T[np.ix_(ir, ir)] * U[np.ix_(ic, ic)].T


def spai_op(M1, S, P2=None, V=None, lam=0.0, q0=None, tol=1e-13, maxiter=5000, eps=0.0):
    """Symmetric Q1 on pattern S minimising Eq. SPAIOPobjective.

    M1: SPD mass matrix (n x n); S: symmetric sparsity pattern; P2: C^T M2 C; V: probe modes
    (n x n_probe); q0: warm start (a matrix on S, e.g. the symmetrised column SPAI).
    Returns (Q1 as CSR, dict(iters, residual history))."""
    M = np.asarray(sp.csr_matrix(M1).toarray())
    n = M.shape[0]
    ir, ic = pattern_pairs(S)
    U = M @ M
    W = None
    if V is not None and lam != 0.0:
        W = np.asarray(sp.csr_matrix(P2) @ np.asarray(V, dtype=float).reshape(n, -1))
    T = t_hat(n, W, lam)
    R = M @ T + T @ M
    r = R[ir, ic]
    prec = U[ir, ir] * T[ic, ic] + T[ir, ir] * U[ic, ic] + eps

    def A(x):
        return sylvester_apply(x, ir, ic, U, T, n) + eps * x

    if q0 is None:
        q = np.zeros(len(ir))
    else:
        q = np.asarray(sp.csr_matrix(q0)[ir, ic]).ravel()
    res = r - A(q)
    z = res / prec
    p = z.copy()
    rz = res @ z
    r0 = np.linalg.norm(r)
    hist = [np.linalg.norm(res)]
    it = 0
    while it < maxiter and hist[-1] > tol * r0:
        Ap = A(p)
        alpha = rz / (p @ Ap)
        q = q + alpha * p
        res = res - alpha * Ap
        hist.append(np.linalg.norm(res))
        it += 1
        z = res / prec
        rz_new = res @ z
        p = z + (rz_new / rz) * p
        rz = rz_new
    Q = sp.csr_matrix((q, (ir, ic)), shape=(n, n))
    return Q, dict(iters=it, history=np.array(hist), rel_residual=hist[-1] / r0)


def frobenius_error(M1, Q1):
    """||M1 Q1 - 1||_F (Eq. FrobeniusDecomp)."""
    D = np.asarray(sp.csr_matrix(M1) @ sp.csr_matrix(Q1).toarray()) - np.eye(M1.shape[0])
    return float(np.linalg.norm(D))


def eig_residual(Q1, P2, v, lam_k):
    """epsilon_k = ||Q1 P2 v - lam_k v|| / |lam_k| (Eq. eigError)."""
    return float(np.linalg.norm(Q1 @ (P2 @ v) - lam_k * v) / abs(lam_k))


def spai_op_q1(fem, M1, P2, V, lam, tol=1e-13, maxiter=20000):
    """SPAI-OP Q1 under the pattern and basis policy of oracle.spai.gym_q1.

    Order 1: Eq. SPAIOPSylvester on M1 with the S(M1) pattern, warm start the symmetrised column
    SPAI.  Orders >= 2 (reading R2 of the column SPAI): the same system in the entity-orthonormal
    basis, M' = T M1 T^T on S(M1^2), probes W' = T P2 V (the probe term (M1 Q1 - 1) P2 v equals
    T^-1 (M' Q' - 1) T P2 v), warm start the column SPAI of M', and Q1 = T^T Q' T."""
    from oracle import spai as SP
    pattern_kind, _ = SP.default_policy(fem.mesh.k)
    basis = SP.basis_for(fem.mesh.k, pattern_kind)
    S = SP.pattern(pattern_kind, M1, fem.dof1)
    if basis == "plain":
        Q0 = SP.symmetrize(SP.spai_columns(M1, S))
        return spai_op(M1, S, P2=P2, V=V, lam=lam, q0=Q0, tol=tol, maxiter=maxiter)
    T = SP.ortho_basis_transform(fem, M1)
    Mp = (T @ M1 @ T.T).tocsr()
    Q0 = SP.symmetrize(SP.spai_columns(Mp, S))
    Qp, info = spai_op(Mp, S, P2=(T @ P2).tocsr(), V=V, lam=lam, q0=Q0, tol=tol, maxiter=maxiter)
    return SP.symmetrize((T.T @ Qp @ T).tocsr()), info


def spai_op_sparse(M1, S, P2=None, V=None, lam=0.0, q0=None, tol=1e-13, maxiter=5000):
    """The same PCG as spai_op for meshes where dense n x n products are too slow.

    The products are the ones of Eq. SPAIOPSylvester, evaluated only on the pattern: with Q1 and
    U = M1^2 symmetric and T^ = 1 + lam W W^T,
        (U Q1 T^)_ij = (U Q1)_ij + lam ((U Q1 W) W^T)_ij,   (T^ Q1 U)_ij = (U Q1)_ji + lam (W (U Q1 W)^T)_ij,
        R^_ij = 2 (M1)_ij + lam ((M1 W) W^T + W (M1 W)^T)_ij."""
    M = sp.csr_matrix(M1)
    n = M.shape[0]
    ir, ic = pattern_pairs(S)
    U = (M @ M).tocsr()
    if V is not None and lam != 0.0:
        W = np.asarray(sp.csr_matrix(P2) @ np.asarray(V, dtype=float).reshape(n, -1))
    else:
        W = np.zeros((n, 0))
    Z = M @ W
    Ud = U.diagonal()
    Td = 1.0 + lam * np.sum(W * W, axis=1)
    r = 2.0 * np.asarray(M[ir, ic]).ravel() + lam * (np.sum(Z[ir] * W[ic], axis=1) + np.sum(W[ir] * Z[ic], axis=1))
    prec = Ud[ir] * Td[ic] + Td[ir] * Ud[ic]

    def A(x):
        Q = sp.csr_matrix((x, (ir, ic)), shape=(n, n))
        G = (U @ Q).tocsr()
        Y = U @ (Q @ W)
        out = np.asarray(G[ir, ic]).ravel() + np.asarray(G[ic, ir]).ravel()
        return out + lam * (np.sum(Y[ir] * W[ic], axis=1) + np.sum(W[ir] * Y[ic], axis=1))

    q = np.zeros(len(ir)) if q0 is None else np.asarray(sp.csr_matrix(q0)[ir, ic]).ravel()
    res = r - A(q)
    z = res / prec
    p = z.copy()
    rz = res @ z
    r0 = np.linalg.norm(r)
    hist = [np.linalg.norm(res)]
    it = 0
    while it < maxiter and hist[-1] > tol * r0:
        Ap = A(p)
        alpha = rz / (p @ Ap)
        q = q + alpha * p
        res = res - alpha * Ap
        hist.append(np.linalg.norm(res))
        it += 1
        z = res / prec
        rz_new = res @ z
        p = z + (rz_new / rz) * p
        rz = rz_new
    return sp.csr_matrix((q, (ir, ic)), shape=(n, n)), dict(iters=it, history=np.array(hist), rel_residual=hist[-1] / r0)
