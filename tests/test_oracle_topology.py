"""Pins of the oracle's mesh, numbering and integer de Rham complex (Sec. 2, Eq. discreteDeRham)."""
import numpy as np
import pytest

from oracle.mesh import KuhnMesh
from oracle.fem import FEM


def euler_counts(n):
    """Entity counts of the Kuhn cube from the Euler characteristic (chi = 1 solid, chi = 2 sphere)."""
    V = (n + 1) ** 3
    E = 3 * n * (n + 1) ** 2 + 3 * n * n * (n + 1) + n ** 3
    T = 6 * n ** 3
    F = 1 - V + E + T
    Vb = (n + 1) ** 3 - (n - 1) ** 3
    Fb = 12 * n * n
    Eb = Vb + Fb - 2
    return V - Vb, E - Eb, F - Fb, T


@pytest.mark.parametrize("n", [1, 2, 3, 4, 7])
@pytest.mark.parametrize("k", [1, 2, 3])
def test_dof_counts_match_closed_form(n, k):
    m = KuhnMesh(n, k)
    Vi, Ei, Fi, T = euler_counts(n)
    assert m.N1 == k * Ei + k * (k - 1) * Fi + k * (k - 1) * (k - 2) // 2 * T
    assert m.N2 == k * (k + 1) // 2 * Fi + (k - 1) * k * (k + 1) // 2 * T
    assert m.N0 == Vi + (k - 1) * Ei + (k - 1) * (k - 2) // 2 * Fi
    assert m.N3 == T * k * (k + 1) * (k + 2) // 6


def test_config1_sizes():
    m = KuhnMesh(4, 1)
    assert (m.n_tets, m.N1, m.N2) == (384, 316, 672)


def test_every_interior_dof_is_used():
    for n, k in [(3, 1), (3, 2), (2, 3)]:
        m = KuhnMesh(n, k)
        d0, d1, d2, d3 = m.dof_maps()
        for d, N in ((d0, m.N0), (d1, m.N1), (d2, m.N2)):
            used = np.unique(d[d >= 0])
            assert len(used) == N and used[0] == 0 and used[-1] == N - 1


@pytest.mark.parametrize("n,k", [(1, 1), (2, 1), (4, 1), (2, 2), (3, 2), (2, 3), (3, 3)])
def test_complex_identities_exact_in_integers(n, k):
    f = FEM(KuhnMesh(n, k))
    C, G, D = f.C(), f.G(), f.D()
    for A in (C, G, D):
        assert set(np.unique(A.data)).issubset({-1.0, 1.0})
    assert abs(C @ G).max() == 0 if (C @ G).nnz else True
    assert abs(D @ C).max() == 0 if (D @ C).nnz else True


@pytest.mark.parametrize("n,k", [(2, 1), (4, 1), (2, 2), (3, 2), (2, 3)])
def test_exactness_rank_of_curl(n, k):
    """The cube with PEC is contractible: no harmonic fields, so ker C = im G (rank C = N1 - N0)."""
    f = FEM(KuhnMesh(n, k))
    C, G = f.C().toarray(), f.G().toarray()
    assert np.linalg.matrix_rank(G) == f.mesh.N0
    assert np.linalg.matrix_rank(C) == f.mesh.N1 - f.mesh.N0
    # and D is onto the 3-forms minus the constants? With PEC (no boundary flux) the total
    # divergence integrates to zero, so rank D = N3 - 1.
    assert np.linalg.matrix_rank(f.D().toarray()) == f.mesh.N3 - 1


def test_n4_k1_kernel_dimension():
    f = FEM(KuhnMesh(4, 1))
    C = f.C().toarray()
    assert C.shape[1] - np.linalg.matrix_rank(C) == 27


def test_locate_returns_containing_tet():
    m = KuhnMesh(3, 1)
    rng = np.random.default_rng(3)
    from oracle.basis import bary_of
    for x in rng.uniform(0, 1, size=(50, 3)):
        t = m.locate(x)
        lam = bary_of(m.tet_vx[t], x)
        assert lam.min() > -1e-12
