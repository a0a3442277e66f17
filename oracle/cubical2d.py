"""2-D periodic cubical Whitney GYM (Q1^- Lambda^p on squares), used only to pin the oracle.

Oracle (test infrastructure).  Reproduces the setting of Sec. 7.5 / 7.6: a
20 x 20 periodic cubical mesh, first-order cubical Whitney forms, Q1 from the
column-wise SPAI of Eq. NormalEqSolve on S(1) (the "Diagonal (Yee)" row of
Table dispersionTable) or S(M1), or the exact inverse, Strang splitting at CFL
safety factor 0.3, the lowest non-kernel eigenmode of M1^-1 P2 as initial e,
b = 0, and the numerical frequency from zero crossings of <e(t), e(0)>.

Readings (the paper does not state them): the torus is [0, 2 pi]^2 (so the
fundamental mode sin(y) dx has continuum frequency 1 and the exact-FEEC value is
1.0041); DoFs use the average normalisation of Eq. WhitneyFormDefn, so the
1-form mass matrix has 2/3 (diagonal) and 1/6 (parallel edges of a common
cell) times the cell area (Eq. whitMassMatrices in 2-D), M2 = area * I and C
is the difference of Eq. dIsFiniteDiff with coefficients +-1/h.
"""
import numpy as np
import scipy.sparse as sp


class Torus2D:
    def __init__(self, nx=20, ny=20, Lx=2 * np.pi, Ly=2 * np.pi):
        self.nx, self.ny = nx, ny
        self.hx, self.hy = Lx / nx, Ly / ny
        self.area = self.hx * self.hy
        # DoFs: x-edges ex(i, j) from (i, j) to (i+1, j): index i + nx j
        #       y-edges ey(i, j) from (i, j) to (i, j+1): nx ny + i + nx j
        #       cells  c(i, j) = [i, i+1] x [j, j+1]:     i + nx j
        self.N1 = 2 * nx * ny
        self.N2 = nx * ny

    def ex(self, i, j):
        return (i % self.nx) + self.nx * (j % self.ny)

    def ey(self, i, j):
        return self.nx * self.ny + (i % self.nx) + self.nx * (j % self.ny)

    def cell(self, i, j):
        return (i % self.nx) + self.nx * (j % self.ny)

    def M1(self):
        """Per cell: 1/3 area on the diagonal, 1/6 area between the two parallel edges (Sec. 7.2)."""
        r, c, v = [], [], []
        for j in range(self.ny):
            for i in range(self.nx):
                for a, b in ((self.ex(i, j), self.ex(i, j + 1)), (self.ey(i, j), self.ey(i + 1, j))):
                    r += [a, b, a, b]
                    c += [a, b, b, a]
                    v += [self.area / 3, self.area / 3, self.area / 6, self.area / 6]
        return sp.csr_matrix((v, (r, c)), shape=(self.N1, self.N1))

    def M2(self):
        return sp.identity(self.N2, format="csr") * self.area

    def C(self):
        """(C a)_cell = (a_right - a_left)/hx - (a_top - a_bottom)/hy  (Eq. dIsFiniteDiff)."""
        r, c, v = [], [], []
        for j in range(self.ny):
            for i in range(self.nx):
                k = self.cell(i, j)
                r += [k, k, k, k]
                c += [self.ey(i + 1, j), self.ey(i, j), self.ex(i, j + 1), self.ex(i, j)]
                v += [1 / self.hx, -1 / self.hx, -1 / self.hy, 1 / self.hy]
        return sp.csr_matrix((v, (r, c)), shape=(self.N2, self.N1))

    def mode_sin_y(self):
        """Coefficients of the field sin(y) dx: x-edge values sin(y_j), y-edges 0."""
        a = np.zeros(self.N1)
        for j in range(self.ny):
            for i in range(self.nx):
                a[self.ex(i, j)] = np.sin(j * self.hy)
        return a


def zero_crossing_frequency(signal, tau):
    """omega from the mean spacing of sign changes (linear interpolation between samples)."""
    s = np.asarray(signal)
    idx = np.where(np.sign(s[:-1]) * np.sign(s[1:]) < 0)[0]
    tz = (idx + s[idx] / (s[idx] - s[idx + 1])) * tau
    if len(tz) < 3:
        return np.nan
    half_period = (tz[-1] - tz[0]) / (len(tz) - 1)
    return np.pi / half_period
