"""Sparse approximate inverse Q ~ M^-1 on a prescribed sparsity pattern (Sec. 5, SPAI paragraph).

Oracle (test infrastructure).  Column by column (Eq. FrobeniusDecomp), the
entries allowed in column l, I_l, solve the small normal-equation system of
Eq. NormalEqSolve,
    q_l(I_l) = [M(:, I_l)^T M(:, I_l)]^-1 M(:, I_l)^T 1_l ,
then Q <- (Q + Q^T)/2 (symmetrisation, same paragraph), then an SPD check and,
if needed, a diagonal shift (Sec. 5.1, practical considerations).
Reading for the shift size (the paper leaves it open): Q += (|lmin| + 1e-12 lmax) I.

Patterns (Sec. 5.1: S(M^k)):
  'diag'  S(1): q_l = M_ll / sum_k M_kl^2
  'sm1'   S(M1): DoF pairs that share a tetrahedron (the structural pattern of M1)
  'sm1sq' S(M1^2): pairs joined by a path of two such steps
Pins: tests/test_oracle_spai.py (brute-force least squares on the full matrix,
the S(1) closed form, the printed SPAI dispersion numbers of Table dispersionTable).
"""
import numpy as np
import scipy.sparse as sp


def structural_pattern(dof_map, n):
    """Boolean CSR of DoF pairs (i, j) that appear together in some row of dof_map (per-tet DoFs)."""
    T, m = dof_map.shape
    R = np.repeat(dof_map[:, :, None], m, axis=2)
    C = np.repeat(dof_map[:, None, :], m, axis=1)
    ok = (R >= 0) & (C >= 0)
    S = sp.csr_matrix((np.ones(ok.sum()), (R[ok], C[ok])), shape=(n, n))
    S.data[:] = 1.0
    return S


def pattern(kind, M, dof_map=None):
    n = M.shape[0]
    if kind == "diag":
        return sp.identity(n, format="csr")
    if kind == "sm1":
        return structural_pattern(dof_map, n) if dof_map is not None else (abs(M) > 0).astype(float).tocsr()
    if kind == "sm1sq":
        S = pattern("sm1", M, dof_map)
        S2 = (S @ S).tocsr()
        S2.data[:] = 1.0
        return S2
    raise ValueError(kind)


def spai_columns(M, S):
    """Unsymmetrised column-wise SPAI of Eq. NormalEqSolve on pattern S (both sparse, n x n)."""
    M = sp.csc_matrix(M)
    S = sp.csc_matrix(S)
    n = M.shape[0]
    rows, cols, vals = [], [], []
    for l in range(n):
        I = S.indices[S.indptr[l]:S.indptr[l + 1]]
        A = M[:, I]                                   # n x |I|, sparse
        J = np.unique(A.indices)
        Ad = A[J, :].toarray()                        # the nonzero rows
        rhs = np.zeros(len(J))
        pos = np.searchsorted(J, l)
        if pos < len(J) and J[pos] == l:
            rhs[pos] = 1.0
        q = np.linalg.solve(Ad.T @ Ad, Ad.T @ rhs)
        rows.append(I)
        cols.append(np.full(len(I), l))
        vals.append(q)
    return sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))), shape=(n, n))


def symmetrize(Q):
    return ((Q + Q.T) * 0.5).tocsr()


def spd_shift(Q, dense_limit=4000):
    """Smallest / largest eigenvalue of symmetric Q, and Q shifted to SPD if needed."""
    n = Q.shape[0]
    if n <= dense_limit:
        w = np.linalg.eigvalsh(Q.toarray())
        lmin, lmax = w[0], w[-1]
    else:
        import scipy.sparse.linalg as spl
        lmax = spl.eigsh(Q, k=1, which="LA", return_eigenvectors=False)[0]
        lmin = spl.eigsh(Q, k=1, which="SA", return_eigenvectors=False)[0]
    shift = 0.0
    if lmin <= 0:
        shift = abs(lmin) + 1e-12 * lmax
        Q = (Q + shift * sp.identity(n)).tocsr()
    return Q, lmin, lmax, shift


def spai(M, kind="sm1", dof_map=None):
    """Symmetric SPD SPAI Q1 ~ M^-1 (Sec. 5): columns, symmetrise, SPD check."""
    S = pattern(kind, M, dof_map)
    Q = symmetrize(spai_columns(M, S))
    Q, lmin, lmax, shift = spd_shift(Q)
    return Q, dict(lmin=lmin, lmax=lmax, shift=shift, nnz=Q.nnz)


# ----------------------------------------------------------------------------
# SPAI in an entity-orthonormalised basis (reading for orders k >= 2)
#
# SPAI is not invariant under a change of basis (Sec. 5: the column problems
# depend on the basis through M).  For k >= 2 the integer-curl hierarchical
# basis gives an ill-conditioned M1 and an indefinite symmetrised SPAI.  The
# SPAI is then computed in the basis Lambda' = T Lambda, T block diagonal over
# the mesh entities: the DoFs of one edge (or face, or cell) are replaced by
# their symmetric (Lowdin) orthonormalisation in the M1(eps) inner product,
#     Lambda'_g = (M1[g,g])^(-1/2) Lambda_g ,
# and the result is mapped back as Q1 = T^T Q' T.  Every DoF of an entity lives
# on the same tets, so T keeps the sparsity of M1, Q1 keeps the pattern of Q'
# (S(M1) or S(M1^2)), and Q1 is SPD exactly when Q' is.  The GYM with (Q1,
# integer C) is the GYM of the basis Lambda' with (Q', C T^T): the same b and E.
# ----------------------------------------------------------------------------

def entity_groups(fem):
    """Lists of global 1-form DoFs per entity: edges, faces, cells (each a tuple)."""
    k = fem.mesh.k
    per_f = k * (k - 1)
    d1 = fem.dof1
    edges, faces, cells = {}, {}, {}
    for t in range(d1.shape[0]):
        d = d1[t]
        for le in range(6):
            g = tuple(int(x) for x in d[le * k:(le + 1) * k] if x >= 0)
            if g:
                edges[g[0]] = g
        for lf in range(4):
            g = tuple(int(x) for x in d[6 * k + lf * per_f:6 * k + (lf + 1) * per_f] if x >= 0)
            if g:
                faces[g[0]] = g
        if k >= 3:
            g = tuple(int(x) for x in d[6 * k + 4 * per_f:])
            cells[g[0]] = g
    return list(edges.values()), list(faces.values()), list(cells.values())


def ortho_basis_transform(fem, M1):
    """Block-diagonal T: per entity group g, T[g, g] = (M1[g, g])^(-1/2) (sparse, N1 x N1)."""
    M = sp.csr_matrix(M1)
    N1 = fem.mesh.N1
    edges, faces, cells = entity_groups(fem)
    r, c, v = [], [], []
    for g in edges + faces + cells:
        g = list(g)
        w, V = np.linalg.eigh(M[g][:, g].toarray())
        Lg = (V / np.sqrt(w)) @ V.T
        for ii, x in enumerate(g):
            for jj, y in enumerate(g):
                r.append(x)
                c.append(y)
                v.append(Lg[ii, jj])
    return sp.csr_matrix((v, (r, c)), shape=(N1, N1))


def default_policy(order):
    """(pattern, basis) used for each order: k = 1 S(M1) in the Whitney basis; k >= 2 S(M1^2), orthogonalised."""
    return ("sm1", "plain") if order == 1 else ("sm1sq", "ortho")


def basis_for(order, pattern_kind):
    """The orthogonalised basis is used exactly for S(M1^2) at orders k >= 2; otherwise the plain basis."""
    return "ortho" if (order >= 2 and pattern_kind == "sm1sq") else "plain"


def gym_q1(fem, M1=None, pattern_kind=None, basis_kind=None):
    """Q1 for the GYM of this mesh: SPAI (Eq. NormalEqSolve), symmetrised, SPD-checked."""
    M1 = fem.M1() if M1 is None else M1
    dp, _ = default_policy(fem.mesh.k)
    pattern_kind = pattern_kind or dp
    basis_kind = basis_kind or basis_for(fem.mesh.k, pattern_kind)
    S = pattern(pattern_kind, M1, fem.dof1)
    if basis_kind == "plain":
        Q = symmetrize(spai_columns(M1, S))
    elif basis_kind == "ortho":
        T = ortho_basis_transform(fem, M1)
        Mp = (T @ M1 @ T.T).tocsr()
        Q = (T.T @ symmetrize(spai_columns(Mp, S)) @ T).tocsr()
        Q = symmetrize(Q)
    else:
        raise ValueError(basis_kind)
    Q, lmin, lmax, shift = spd_shift(Q)
    return Q, dict(lmin=lmin, lmax=lmax, shift=shift, nnz=Q.nnz, pattern=pattern_kind, basis=basis_kind)


# ----------------------------------------------------------------------------
# Sampled rows of Q1 on large meshes (the same definitions, evaluated locally)
# ----------------------------------------------------------------------------

class LocalQ1:
    """Rows of the default-policy Q1 computed one by one from their neighbourhood, for meshes
    where the whole SPAI is too slow in Python.  Same steps as gym_q1: structural pattern,
    entity Lowdin basis (k >= 2 with S(M1^2)), column SPAI (Eq. NormalEqSolve), symmetrisation."""

    def __init__(self, fem, M1, pattern_kind=None):
        self.fem = fem
        self.M1 = sp.csr_matrix(M1)
        k = fem.mesh.k
        self.kind = pattern_kind or default_policy(k)[0]
        self.ortho = basis_for(k, self.kind) == "ortho"
        # entity group of every DoF (tuple of the entity's DoFs)
        self.group = {}
        for g in sum(entity_groups(fem), []):
            for i in g:
                self.group[i] = g
        self._T = {}
        self._col = {}
        self._mp = {}

    def s1(self, i):
        M = self.M1
        return M.indices[M.indptr[i]:M.indptr[i + 1]]

    def pattern_row(self, i):
        if self.kind == "diag":
            return np.array([i])
        if self.kind == "sm1":
            return np.sort(self.s1(i))
        return np.unique(np.concatenate([self.s1(m) for m in self.s1(i)]))

    def T_block(self, g):
        if g not in self._T:
            if self.ortho:
                w, V = np.linalg.eigh(self.M1[list(g)][:, list(g)].toarray())
                self._T[g] = (V / np.sqrt(w)) @ V.T
            else:
                self._T[g] = np.eye(len(g))
        return self._T[g]

    def Mp_col(self, c):
        """Column c of M' = T M1 T^T as a dict {row: value} (cached)."""
        if c in self._mp:
            return self._mp[c]
        gc = self.group[c]
        Tc = self.T_block(gc)
        jc = gc.index(c)
        # M1 T^T column c: sum_b M1[:, b] T[c, b] over b in the group of c
        col = {}
        for bb, b in enumerate(gc):
            t = Tc[jc, bb]
            if t == 0.0:
                continue
            M = self.M1
            for p in range(M.indptr[b], M.indptr[b + 1]):
                col[M.indices[p]] = col.get(M.indices[p], 0.0) + M.data[p] * t
        out = {}
        for r0, v in col.items():
            g = self.group[r0]
            Tg = self.T_block(g)
            j0 = g.index(r0)
            for aa, a in enumerate(g):
                out[a] = out.get(a, 0.0) + Tg[aa, j0] * v
        self._mp[c] = out
        return out

    def column(self, l):
        """q'_l on its pattern (dict row -> value), Eq. NormalEqSolve in the primed basis."""
        if l not in self._col:
            I = self.pattern_row(l)
            cols = [self.Mp_col(int(i)) for i in I]
            rows = sorted(set().union(*[c.keys() for c in cols]))
            ridx = {r: n for n, r in enumerate(rows)}
            A = np.zeros((len(rows), len(I)))
            for p, c in enumerate(cols):
                for r, v in c.items():
                    A[ridx[r], p] = v
            rhs = np.zeros(len(rows))
            if l in ridx:
                rhs[ridx[l]] = 1.0
            q = np.linalg.solve(A.T @ A, A.T @ rhs)
            self._col[l] = dict(zip((int(i) for i in I), q))
        return self._col[l]

    def qp(self, a, b):
        """Symmetrised primed entry Q'(a, b) = (q'_b[a] + q'_a[b]) / 2."""
        return 0.5 * (self.column(b).get(a, 0.0) + self.column(a).get(b, 0.0))

    def row(self, i):
        """Row i of Q1 = T^T Q' T as a dict {column: value}."""
        gi = self.group[i]
        Ti = self.T_block(gi)
        ji = gi.index(i)
        out = {}
        for aa, a in enumerate(gi):
            ta = Ti[aa, ji]
            for b in self.pattern_row(a):
                b = int(b)
                gb = self.group[b]
                Tb = self.T_block(gb)
                v = ta * self.qp(a, b)
                if v == 0.0:
                    continue
                jb = gb.index(b)
                for cc, c in enumerate(gb):
                    out[c] = out.get(c, 0.0) + v * Tb[jb, cc]
        return out
