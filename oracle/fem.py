"""Assembly of the mass matrices and the integer matrices of the discrete de Rham complex.

Oracle (test infrastructure).  Follows Sec. 2:
  (M_p)_ij = int (Lambda^p_i, Lambda^p_j) dx                                      (mass matrices)
  G^T Lambda^1 = d Lambda^0,  C^T Lambda^2 = d Lambda^1,  D^T Lambda^3 = d Lambda^2 (Eq. discreteDeRham)
with M1 weighted by the per-tet permittivity and M2 by the inverse per-tet
permeability (units eps0 = mu0 = c = 1, Sec. 7).  Local matrices are computed
with tetrahedron quadrature on the actual tet coordinates of every Kuhn shape;
the integer matrices are written from incidence (Whitney part) and from the
definition of the higher-order 2-forms as curls of 1-forms.
Pins: tests/test_oracle_fem.py and tests/test_oracle_topology.py.
"""
import numpy as np
import scipy.sparse as sp
from . import basis as B
from .mesh import KuhnMesh, LOCAL_EDGES, LOCAL_FACES


class FEM:
    def __init__(self, mesh: KuhnMesh, eps=None, mu=None, quad_pts=6):
        self.mesh = mesh
        k = mesh.k
        T = mesh.n_tets
        self.eps = np.ones(T) if eps is None else np.asarray(eps, float)
        self.mu = np.ones(T) if mu is None else np.asarray(mu, float)
        assert self.eps.shape == (T,) and self.mu.shape == (T,)
        self.F1, self.F2 = B.one_forms(k), B.two_forms(k)
        self.F0, self.F3 = B.zero_forms(k), B.three_forms(k)
        self.n1, self.n2, self.n0, self.n3 = len(self.F1), len(self.F2), len(self.F0), len(self.F3)
        self.quad_pts = quad_pts
        self.dof0, self.dof1, self.dof2, self.dof3 = mesh.dof_maps()
        assert self.dof1.shape[1] == self.n1 and self.dof2.shape[1] == self.n2
        assert self.dof0.shape[1] == self.n0 and self.dof3.shape[1] == self.n3
        self._local = [self._local_matrices(s) for s in range(6)]

    # ------------------------------------------------------------ local blocks
    def shape_vertices(self, s):
        """Coordinates of the Kuhn tet of shape s in the first cube."""
        return self.mesh.tet_vx[s]

    def _local_matrices(self, s):
        X = self.shape_vertices(s)
        g = B.bary_gradients(X)
        L, W = B.tet_quadrature(X, self.quad_pts)
        v1 = [B.eval1(f, L, g) for f in self.F1]
        v2 = [B.eval2(f, L, g) for f in self.F2]
        val1 = np.stack([v[0] for v in v1])          # (n1, P, 3)
        cur1 = np.stack([v[1] for v in v1])
        val2 = np.stack([v[0] for v in v2])
        div2 = np.stack([v[1] for v in v2])          # (n2, P)
        val0 = np.stack([B.eval0(f, L, g)[0] for f in self.F0])
        grd0 = np.stack([B.eval0(f, L, g)[1] for f in self.F0])
        vol = B.tet_volume(X)
        val3 = np.stack([B.eval3(f, L, g, vol) for f in self.F3])
        M1 = np.einsum("ipx,jpx,p->ij", val1, val1, W)
        M2 = np.einsum("ipx,jpx,p->ij", val2, val2, W)
        M0 = np.einsum("ip,jp,p->ij", val0, val0, W)
        M3 = np.einsum("ip,jp,p->ij", val3, val3, W)
        Bc = np.einsum("ipx,jpx,p->ij", val2, cur1, W)    # int Lambda2_i . curl Lambda1_j
        Bg = np.einsum("ipx,jpx,p->ij", val1, grd0, W)    # int Lambda1_i . grad Lambda0_j
        Bd = np.einsum("ip,jp,p->ij", val3, div2, W)      # int Lambda3_i div Lambda2_j
        return dict(M1=M1, M2=M2, M0=M0, M3=M3, Bc=Bc, Bg=Bg, Bd=Bd, g=g, vol=vol)

    def local(self, s):
        return self._local[s]

    # ------------------------------------------------------------ assembly helpers
    def _assemble(self, rows_map, cols_map, blocks, weight):
        T = self.mesh.n_tets
        nr, nc = rows_map.shape[1], cols_map.shape[1]
        R = np.repeat(rows_map[:, :, None], nc, axis=2)
        Cc = np.repeat(cols_map[:, None, :], nr, axis=1)
        V = blocks[self.mesh.tet_shape] * weight[:, None, None]
        m = (R >= 0) & (Cc >= 0)
        return R[m], Cc[m], V[m]

    def _sparse(self, key, rows_map, cols_map, weight, shape):
        blocks = np.stack([self._local[s][key] for s in range(6)])
        r, c, v = self._assemble(rows_map, cols_map, blocks, weight)
        return sp.csr_matrix((v, (r, c)), shape=shape)

    def M1(self):
        N1 = self.mesh.N1
        return self._sparse("M1", self.dof1, self.dof1, self.eps, (N1, N1))

    def M2(self):
        N2 = self.mesh.N2
        return self._sparse("M2", self.dof2, self.dof2, 1.0 / self.mu, (N2, N2))

    def M0(self):
        N0 = self.mesh.N0
        return self._sparse("M0", self.dof0, self.dof0, np.ones(self.mesh.n_tets), (N0, N0))

    def M3(self):
        N3 = self.mesh.N3
        return self._sparse("M3", self.dof3, self.dof3, np.ones(self.mesh.n_tets), (N3, N3))

    def B_curl(self):
        """B_ij = int Lambda2_i . curl Lambda1_j  (so that M2 C = B)."""
        return self._sparse("Bc", self.dof2, self.dof1, np.ones(self.mesh.n_tets), (self.mesh.N2, self.mesh.N1))

    def B_grad(self):
        return self._sparse("Bg", self.dof1, self.dof0, np.ones(self.mesh.n_tets), (self.mesh.N1, self.mesh.N0))

    def B_div(self):
        return self._sparse("Bd", self.dof3, self.dof2, np.ones(self.mesh.n_tets), (self.mesh.N3, self.mesh.N2))

    # ------------------------------------------------------------ integer complex
    def local_C(self):
        """Local curl block (n2, n1): d Lambda1_j = sum_i C_ij Lambda2_i on one tet."""
        k = self.mesh.k
        C = np.zeros((self.n2, self.n1), dtype=np.int64)
        le_index = {e: i for i, e in enumerate(LOCAL_EDGES)}
        per_f1 = k * (k - 1)
        row = 0
        for lf, (a, b, c) in enumerate(LOCAL_FACES):
            # Stokes on the face: flux of curl w_e = circulation of w_e around the boundary
            C[row, le_index[(b, c)] * k] = 1
            C[row, le_index[(a, c)] * k] = -1
            C[row, le_index[(a, b)] * k] = 1
            row += 1
            for j in range(per_f1):
                col = 6 * k + lf * per_f1 + j
                if self.F1[col][0] != "grad":
                    C[row, col] = 1
                    row += 1
        if k >= 3:
            for j in range(3):
                C[row, 6 * k + 4 * per_f1 + j] = 1
                row += 1
        return C

    def local_G(self):
        k = self.mesh.k
        G = np.zeros((self.n1, self.n0), dtype=np.int64)
        for le, (a, b) in enumerate(LOCAL_EDGES):
            G[le * k, a] = -1      # grad l_v = sum over edges of +-w_e (head +, tail -)
            G[le * k, b] = 1
            for j in range(k - 1):
                G[le * k + 1 + j, 4 + le * (k - 1) + j] = 1
        if k >= 3:
            per_f1 = k * (k - 1)
            for lf in range(4):
                G[6 * k + lf * per_f1 + 5, 4 + 6 * (k - 1) + lf] = 1
        return G

    def local_D(self, s):
        """Local divergence block (n3, n2) of Kuhn shape s."""
        k = self.mesh.k
        loc = self._local[s]
        g, vol = loc["g"], loc["vol"]
        D = np.zeros((self.n3, self.n2), dtype=np.int64)
        per_f2 = k * (k + 1) // 2
        for lf, (a, b, c) in enumerate(LOCAL_FACES):
            flux = 6.0 * vol * np.dot(g[a], np.cross(g[b], g[c]))   # int_T div W_abc
            D[0, lf * per_f2] = int(round(flux))
        j3 = 1
        for j, f in enumerate(self.F2):
            if f[0] == "pW" and f[1] is not B.ONE:
                D[j3, j] = 1
                j3 += 1
        return D

    def _int_assemble(self, rows_map, cols_map, locs, shape):
        T = self.mesh.n_tets
        blocks = np.stack(locs)[self.mesh.tet_shape] if isinstance(locs, list) else np.broadcast_to(locs, (T,) + locs.shape)
        nr, nc = rows_map.shape[1], cols_map.shape[1]
        R = np.repeat(rows_map[:, :, None], nc, axis=2)
        Cc = np.repeat(cols_map[:, None, :], nr, axis=1)
        m = (R >= 0) & (Cc >= 0) & (blocks != 0)
        r, c, v = R[m], Cc[m], blocks[m]
        # every tet that contains both DoFs must agree on the entry: set, not add
        key = r.astype(np.int64) * shape[1] + c
        order = np.argsort(key, kind="stable")
        key, v = key[order], v[order]
        uniq, first = np.unique(key, return_index=True)
        vals = v[first]
        # consistency check
        counts = np.diff(np.append(first, len(key)))
        assert np.all(np.repeat(vals, counts) == v), "inconsistent integer entries"
        return sp.csr_matrix((vals.astype(np.float64), (uniq // shape[1], uniq % shape[1])), shape=shape)

    def C(self):
        return self._int_assemble(self.dof2, self.dof1, self.local_C(), (self.mesh.N2, self.mesh.N1))

    def G(self):
        return self._int_assemble(self.dof1, self.dof0, self.local_G(), (self.mesh.N1, self.mesh.N0))

    def D(self):
        return self._int_assemble(self.dof3, self.dof2, [self.local_D(s) for s in range(6)],
                                  (self.mesh.N3, self.mesh.N2))

    # ------------------------------------------------------------ projections
    def load_vector(self, E0):
        """F_i = int E0 . Lambda1_i dx (quadrature).  E0 maps (P, 3) points to (P, 3)."""
        mesh = self.mesh
        F = np.zeros(mesh.N1)
        for t in range(mesh.n_tets):
            X = mesh.tet_vx[t]
            g = B.bary_gradients(X)
            L, W = B.tet_quadrature(X, self.quad_pts)
            x = L @ X
            Ev = E0(x)
            for i, f in enumerate(self.F1):
                gi = self.dof1[t, i]
                if gi >= 0:
                    F[gi] += np.sum(np.einsum("px,px->p", B.eval1(f, L, g)[0], Ev) * W)
        return F

    def edge_interpolant(self, E0, npts=10):
        """Canonical Whitney interpolant (k = 1): c_e = int_e E0 . t ds (Eq. WhitneyFormDefn, integral form)."""
        assert self.mesh.k == 1
        mesh = self.mesh
        s, w = np.polynomial.legendre.leggauss(npts)
        s = 0.5 * (s + 1.0)
        w = 0.5 * w
        c = np.zeros(mesh.N1)
        done = np.zeros(mesh.N1, bool)
        for t in range(mesh.n_tets):
            X = mesh.tet_vx[t]
            for le, (a, b) in enumerate(LOCAL_EDGES):
                gi = self.dof1[t, le]
                if gi < 0 or done[gi]:
                    continue
                pts = X[a][None, :] + s[:, None] * (X[b] - X[a])[None, :]
                c[gi] = np.sum(w * (E0(pts) @ (X[b] - X[a])))
                done[gi] = True
        return c

    def point_values(self, t, x):
        """Values of the 1-form basis functions of tet t at point x: (n1, 3)."""
        X = self.mesh.tet_vx[t]
        g = B.bary_gradients(X)
        L = B.bary_of(X, np.asarray(x, float))[None, :]
        return np.stack([B.eval1(f, L, g)[0][0] for f in self.F1])
