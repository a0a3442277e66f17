"""Local order-k bases of the discrete de Rham complex on one tetrahedron, and quadrature.

Oracle (test infrastructure).  Pinned by tests/test_oracle_fem.py: curls against
finite differences, reproduction of polynomial fields, exactness d(d(.)) = 0,
the L2-projection re-derivation of the integer curl, and convergence of the
cavity spectrum to pi^2 (m^2 + n^2 + l^2).

The paper requires de Rham-conforming elements (Def. GYM (i), Eq. eqnCommute)
and names Whitney forms and Nedelec elements on simplices (Sec. 2) but gives
no 3-D higher-order basis.  Reading taken here (fixed for the project): the
trimmed spaces P_k^- Lambda^p, k = 1, 2, 3, in a hierarchical exact-sequence
basis, written with barycentric coordinates l_i, their gradients g_i,
  w_ab  = l_a g_b - l_b g_a                       (Whitney 1-form)
  W_abc = 2 (l_a g_b x g_c + l_b g_c x g_a + l_c g_a x g_b)   (Whitney 2-form)
and vertices a < b < c < d of the tet (local order = global order):

1-forms, per edge (a,b):  w_ab ; grad(l_a l_b) ; grad(l_a l_b (l_b - l_a))
         per face (a,b,c): k=2: l_c w_ab, l_b w_ac
                           k=3: l_c w_ab, l_b w_ac, l_a l_c w_ab, l_b l_c w_ab,
                                l_a l_b w_ac, grad(l_a l_b l_c)
         cell (k=3):       l_c l_d w_ab, l_b l_d w_ac, l_b l_c w_ad
2-forms, per face: W_abc, then curl of every non-gradient face 1-form above
         cell: curl of the cell 1-forms (k=3), then the divergence part
               k=2: l_d W_abc, l_c W_abd, l_b W_acd
               k=3: for (S, m) in ((abc, d), (abd, c), (acd, b)):
                    l_m^2 W_S, l_m l_S0 W_S, l_m l_S1 W_S
0-forms: l_v ; l_a l_b ; l_a l_b (l_b - l_a) ; l_a l_b l_c
3-forms: 1/|T| and the divergences of the divergence-part 2-forms.
With this basis the matrices G, C, D of the complex have entries in {0, +-1}.
"""
import numpy as np
from .mesh import LOCAL_EDGES, LOCAL_FACES


# ------------------------------------------------------------------ polynomials
def mono(*idx):
    """Monomial prod_i l_{idx_i} as {exponent tuple: coefficient}."""
    a = [0, 0, 0, 0]
    for i in idx:
        a[i] += 1
    return {tuple(a): 1.0}


def padd(p, q, s=1.0):
    r = dict(p)
    for k, v in q.items():
        r[k] = r.get(k, 0.0) + s * v
    return r


def peval(p, L):
    out = np.zeros(L.shape[0])
    for a, c in p.items():
        out += c * np.prod(L ** np.array(a), axis=1)
    return out


def pgrad(p, L, g):
    """Cartesian gradient sum_m dP/dl_m g_m at barycentric points L (P, 4)."""
    out = np.zeros((L.shape[0], 3))
    for a, c in p.items():
        for m in range(4):
            if a[m] == 0:
                continue
            b = list(a)
            b[m] -= 1
            out += (c * a[m] * np.prod(L ** np.array(b), axis=1))[:, None] * g[m]
    return out


ONE = {(0, 0, 0, 0): 1.0}


# ------------------------------------------------------------------ function lists
def one_forms(k):
    """Local 1-form basis: list of ('pw', P, a, b) or ('grad', P)."""
    F = []
    for a, b in LOCAL_EDGES:
        F.append(("pw", ONE, a, b))
        if k >= 2:
            F.append(("grad", mono(a, b)))
        if k >= 3:
            F.append(("grad", padd(mono(a, b, b), mono(a, a, b), -1.0)))
    for a, b, c in LOCAL_FACES:
        if k >= 2:
            F.append(("pw", mono(c), a, b))
            F.append(("pw", mono(b), a, c))
        if k >= 3:
            F.append(("pw", mono(a, c), a, b))
            F.append(("pw", mono(b, c), a, b))
            F.append(("pw", mono(a, b), a, c))
            F.append(("grad", mono(a, b, c)))
    if k >= 3:
        F.append(("pw", mono(2, 3), 0, 1))
        F.append(("pw", mono(1, 3), 0, 2))
        F.append(("pw", mono(1, 2), 0, 3))
    return F


def two_forms(k):
    """Local 2-form basis: ('pW', P, a, b, c) or ('curl', one_form)."""
    F1 = one_forms(k)
    per_e = k
    per_f = k * (k - 1)
    F = []
    for lf, (a, b, c) in enumerate(LOCAL_FACES):
        F.append(("pW", ONE, a, b, c))
        for j in range(per_f):
            f = F1[6 * per_e + lf * per_f + j]
            if f[0] != "grad":
                F.append(("curl", f))
    if k >= 3:
        for j in range(3):
            F.append(("curl", F1[6 * per_e + 4 * per_f + j]))
    if k == 2:
        F += [("pW", mono(3), 0, 1, 2), ("pW", mono(2), 0, 1, 3), ("pW", mono(1), 0, 2, 3)]
    if k == 3:
        for (s0, s1, s2), m in (((0, 1, 2), 3), ((0, 1, 3), 2), ((0, 2, 3), 1)):
            for extra in (m, s0, s1):
                F.append(("pW", mono(m, extra), s0, s1, s2))
    return F


def zero_forms(k):
    F = [("p", mono(v)) for v in range(4)]
    for a, b in LOCAL_EDGES:
        if k >= 2:
            F.append(("p", mono(a, b)))
        if k >= 3:
            F.append(("p", padd(mono(a, b, b), mono(a, a, b), -1.0)))
    if k >= 3:
        for a, b, c in LOCAL_FACES:
            F.append(("p", mono(a, b, c)))
    # local order must match the mesh's 0-form map: vertices, edges (k-1 each), faces
    return F


def three_forms(k):
    """('vol',) then ('div', two_form) for the divergence-part 2-forms."""
    F2 = two_forms(k)
    return [("vol",)] + [("div", f) for f in F2 if f[0] == "pW" and f[1] is not ONE]


# ------------------------------------------------------------------ evaluation
def _w(L, g, a, b):
    return L[:, a:a + 1] * g[b] - L[:, b:b + 1] * g[a]


def _W(L, g, a, b, c):
    return 2.0 * (L[:, a:a + 1] * np.cross(g[b], g[c]) + L[:, b:b + 1] * np.cross(g[c], g[a])
                  + L[:, c:c + 1] * np.cross(g[a], g[b]))


def eval1(f, L, g):
    """(value, curl) of a 1-form basis function, each (P, 3)."""
    if f[0] == "grad":
        return pgrad(f[1], L, g), np.zeros((L.shape[0], 3))
    _, p, a, b = f
    w = _w(L, g, a, b)
    P = peval(p, L)[:, None]
    curl = np.cross(pgrad(p, L, g), w) + P * (2.0 * np.cross(g[a], g[b]))
    return P * w, curl


def eval2(f, L, g):
    """(value, divergence) of a 2-form basis function."""
    if f[0] == "curl":
        return eval1(f[1], L, g)[1], np.zeros(L.shape[0])
    _, p, a, b, c = f
    W = _W(L, g, a, b, c)
    P = peval(p, L)
    divW = 6.0 * np.dot(g[a], np.cross(g[b], g[c]))
    div = np.einsum("pi,pi->p", pgrad(p, L, g), W) + P * divW
    return P[:, None] * W, div


def eval0(f, L, g):
    return peval(f[1], L), pgrad(f[1], L, g)


def eval3(f, L, g, vol):
    if f[0] == "vol":
        return np.full(L.shape[0], 1.0 / vol)
    return eval2(f[1], L, g)[1]


# ------------------------------------------------------------------ geometry, quadrature
def bary_gradients(X):
    """Gradients g_i of the barycentric coordinates of the tet with vertices X (4, 3)."""
    A = np.vstack([np.ones(4), X.T])
    return np.linalg.inv(A)[:, 1:]


def tet_volume(X):
    return abs(np.linalg.det(X[1:] - X[0])) / 6.0


def tet_quadrature(X, npts=6):
    """Collapsed (Duffy) Gauss-Legendre rule on tet X: barycentric points (P, 4), weights (P,).

    With npts nodes per direction it integrates polynomials of degree 2*npts - 3 exactly.
    """
    t, w = np.polynomial.legendre.leggauss(npts)
    t = 0.5 * (t + 1.0)
    w = 0.5 * w
    x1, x2, x3 = np.meshgrid(t, t, t, indexing="ij")
    w1, w2, w3 = np.meshgrid(w, w, w, indexing="ij")
    l1 = x1
    l2 = (1 - x1) * x2
    l3 = (1 - x1) * (1 - x2) * x3
    l0 = 1 - l1 - l2 - l3
    L = np.stack([l0, l1, l2, l3], axis=-1).reshape(-1, 4)
    W = (w1 * w2 * w3 * (1 - x1) ** 2 * (1 - x2)).reshape(-1) * 6.0 * tet_volume(X)
    return L, W


def bary_of(X, x):
    """Barycentric coordinates of point x in tet X."""
    A = np.vstack([np.ones(4), X.T])
    return np.linalg.solve(A, np.concatenate([[1.0], x]))
