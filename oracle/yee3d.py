"""3-D periodic cubical Whitney complex (Q1^- Lambda^p on cubes), used only to pin the oracle's
leapfrog against a textbook Yee FDTD loop (Sec. 4: Yee's method is the GYM with cubical Whitney
forms, lumped masses and Strang splitting; the paper reports agreement to < 1e-15).

Oracle (test infrastructure).  DoFs use the average normalisation of Eq. WhitneyFormDefn, so
the curl is the finite difference of Eq. dIsFiniteDiff with coefficients +-1/Delta, the lumped
masses are M1^Y = M2^Y = Delta_V I (Eq. YeeMassMatrices), and the GYM shear maps become
Eq. shearMapsBE with Q1 = Delta_V^-1 I.
"""
import numpy as np
import scipy.sparse as sp


class PeriodicCubes:
    def __init__(self, n=(6, 5, 4), h=(0.3, 0.25, 0.2)):
        self.n = tuple(n)
        self.h = tuple(h)
        self.dV = h[0] * h[1] * h[2]
        self.nc = n[0] * n[1] * n[2]
        self.N1 = 3 * self.nc         # edges: x, y, z edges anchored at every vertex
        self.N2 = 3 * self.nc         # faces: normals x, y, z anchored at every vertex

    def cell(self, i, j, k):
        nx, ny, nz = self.n
        return (i % nx) + nx * ((j % ny) + ny * (k % nz))

    def edge(self, a, i, j, k):       # edge along axis a starting at vertex (i, j, k)
        return a * self.nc + self.cell(i, j, k)

    def face(self, a, i, j, k):       # face with normal a, lower corner at vertex (i, j, k)
        return a * self.nc + self.cell(i, j, k)

    def C(self):
        """b_face = sum over the face's boundary of +-(1/Delta) a_edge (Eq. dIsFiniteDiff)."""
        hx, hy, hz = self.h
        r, c, v = [], [], []
        nx, ny, nz = self.n
        for k in range(nz):
            for j in range(ny):
                for i in range(nx):
                    # normal z (face in the xy plane): (1/hx)(a_y(i+1) - a_y(i)) - (1/hy)(a_x(j+1) - a_x(j))
                    f = self.face(2, i, j, k)
                    r += [f] * 4
                    c += [self.edge(1, i + 1, j, k), self.edge(1, i, j, k), self.edge(0, i, j + 1, k), self.edge(0, i, j, k)]
                    v += [1 / hx, -1 / hx, -1 / hy, 1 / hy]
                    # normal x (yz plane): (1/hy)(a_z(j+1) - a_z(j)) - (1/hz)(a_y(k+1) - a_y(k))
                    f = self.face(0, i, j, k)
                    r += [f] * 4
                    c += [self.edge(2, i, j + 1, k), self.edge(2, i, j, k), self.edge(1, i, j, k + 1), self.edge(1, i, j, k)]
                    v += [1 / hy, -1 / hy, -1 / hz, 1 / hz]
                    # normal y (zx plane): (1/hz)(a_x(k+1) - a_x(k)) - (1/hx)(a_z(i+1) - a_z(i))
                    f = self.face(1, i, j, k)
                    r += [f] * 4
                    c += [self.edge(0, i, j, k + 1), self.edge(0, i, j, k), self.edge(2, i + 1, j, k), self.edge(2, i, j, k)]
                    v += [1 / hz, -1 / hz, -1 / hx, 1 / hx]
        return sp.csr_matrix((v, (r, c)), shape=(self.N2, self.N1))

    # ---- consistent (unlumped) masses of the cubical Whitney forms, by quadrature ----------
    # In a cell with local coordinates (s, t, u) in [0,1]^3, the x-edge function of the local
    # edge at (t, u) = (bt, bu) is hat_bt(t) hat_bu(u) e_x (hat_0 = 1 - s, hat_1 = s), and the
    # face with normal x at s = bs is hat_bs(s) e_x: the average-normalised Whitney forms
    # (Eq. WhitneyFormDefn).  Their L2 products, summed over cells, give M1 and M2.
    def _mass(self, kind):
        nx, ny, nz = self.n
        g, w = np.polynomial.legendre.leggauss(3)
        g, w = 0.5 * (g + 1.0), 0.5 * w                 # Gauss-Legendre on [0, 1], exact to degree 5
        hat = lambda b, x: x if b else 1.0 - x
        N = self.N1 if kind == 1 else self.N2
        r, c, v = [], [], []
        for k in range(nz):
            for j in range(ny):
                for i in range(nx):
                    loc = []                            # (global index, axis, function of (x, y, z))
                    for a in range(3):
                        o1, o2 = (a + 1) % 3, (a + 2) % 3
                        if kind == 1:
                            for b1 in (0, 1):
                                for b2 in (0, 1):
                                    off = [0, 0, 0]
                                    off[o1], off[o2] = b1, b2
                                    loc.append((self.edge(a, i + off[0], j + off[1], k + off[2]), a,
                                                (lambda p, b1=b1, b2=b2, o1=o1, o2=o2: hat(b1, p[o1]) * hat(b2, p[o2]))))
                        else:
                            for b0 in (0, 1):
                                off = [0, 0, 0]
                                off[a] = b0
                                loc.append((self.face(a, i + off[0], j + off[1], k + off[2]), a,
                                            (lambda p, b0=b0, a=a: hat(b0, p[a]))))
                    for (gi, ai, fi) in loc:
                        for (gj, aj, fj) in loc:
                            if ai != aj:
                                continue                # orthogonal directions
                            val = 0.0
                            for x, wx in zip(g, w):
                                for y, wy in zip(g, w):
                                    for z, wz in zip(g, w):
                                        val += wx * wy * wz * fi((x, y, z)) * fj((x, y, z))
                            r.append(gi)
                            c.append(gj)
                            v.append(val * self.dV)
        return sp.csr_matrix((v, (r, c)), shape=(N, N))

    def M1(self):
        return self._mass(1)

    def M2(self):
        return self._mass(2)


def yee_textbook(E, B, tau, h, nsteps):
    """Standard Yee update on a periodic grid (c = 1): B^{n+1/2} = B^{n-1/2} - tau curl E^n,
    E^{n+1} = E^n + tau curl^T B^{n+1/2}; arrays indexed [axis][i, j, k] on staggered positions.
    B is given at half step -1/2 (the caller applies the initial half step)."""
    Ex, Ey, Ez = [a.copy() for a in E]
    Bx, By, Bz = [a.copy() for a in B]
    hx, hy, hz = h
    d = lambda a, ax, s: (np.roll(a, -1, axis=ax) - a) if s > 0 else (a - np.roll(a, 1, axis=ax))
    for _ in range(nsteps):
        Bz = Bz - tau * (d(Ey, 0, 1) / hx - d(Ex, 1, 1) / hy)
        Bx = Bx - tau * (d(Ez, 1, 1) / hy - d(Ey, 2, 1) / hz)
        By = By - tau * (d(Ex, 2, 1) / hz - d(Ez, 0, 1) / hx)
        Ex = Ex + tau * (d(Bz, 1, -1) / hy - d(By, 2, -1) / hz)
        Ey = Ey + tau * (d(Bx, 2, -1) / hz - d(Bz, 0, -1) / hx)
        Ez = Ez + tau * (d(By, 0, -1) / hx - d(Bx, 1, -1) / hy)
    return (Ex, Ey, Ez), (Bx, By, Bz)
