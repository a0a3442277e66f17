"""Structured PEC cube [0, side]^3 cut into n^3 cubes, each split into 6 Kuhn tetrahedra.

Oracle (test infrastructure).  Pinned by tests/test_oracle_topology.py:
entity counts against the Euler characteristic, N1/N2 against the closed-form
DoF counts, exactness (rank C = N1 - N0) and C.G = 0, D.C = 0 in integers.

The paper works on a simplicial complex T_h (Sec. 2) and names Whitney /
Nedelec elements on simplicial meshes; the cube and its Kuhn split are the
synthetic workload.  Every Kuhn simplex has its vertices on a monotone lattice
path, so the vertex order along the path equals the order of the lexicographic
vertex numbering i + (n+1)(j + (n+1)k): local orientation is global orientation.

Lattice offsets are 3-bit masks (bit 0 = x, bit 1 = y, bit 2 = z).  An entity is
anchored at its smallest vertex v and described by the chain of offsets of its
other vertices:
  edge  (v, v+d)                       d  in 1..7                  7 shapes
  face  (v, v+d1, v+d2), d1 subset d2   (d1, d2) in FACE_SHAPES     12 shapes
  tet   (v, v+d1, v+d2, v+7)            (d1, d2) in TET_SHAPES      6 shapes
A tet is numbered  6 * (cx + n*(cy + n*cz)) + shape.

DoF numbering (shared layout with the C-ABI, stated there too): DoFs come in
classes = (entity shape, index of the DoF inside the entity).  Class c owns the
anchors v whose entity is interior (PEC removes entities lying in the boundary):
along axis a, v_a runs over [0, n-1] if the entity extends along a, else over
[1, n-1].  Global index = offset[c] + ((vz-lo)*ny + (vy-lo))*nx + (vx-lo), the
classes in order edges, faces, tets (shape-major, then DoF inside the entity).
"""
import numpy as np

EDGE_SHAPES = [1, 2, 3, 4, 5, 6, 7]
FACE_SHAPES = [(1, 3), (2, 3), (1, 5), (4, 5), (2, 6), (4, 6),
               (1, 7), (2, 7), (3, 7), (4, 7), (5, 7), (6, 7)]
TET_SHAPES = [(1, 3), (1, 5), (2, 3), (2, 6), (4, 5), (4, 6)]
LOCAL_EDGES = [(0, 1), (0, 2), (0, 3), (1, 2), (1, 3), (2, 3)]
LOCAL_FACES = [(0, 1, 2), (0, 1, 3), (0, 2, 3), (1, 2, 3)]

_FACE_INDEX = {fs: i for i, fs in enumerate(FACE_SHAPES)}


def bits(mask):
    """Offset vector (x, y, z) of a 3-bit mask; works elementwise on arrays."""
    mask = np.asarray(mask)
    return np.stack([(mask >> 0) & 1, (mask >> 1) & 1, (mask >> 2) & 1], axis=-1)


def dofs_per_entity(order):
    """(edge, face, cell) 1-form DoFs and (face, cell) 2-form DoFs of P_k^- on a tet."""
    k = order
    return dict(e1=k, f1=k * (k - 1), c1=k * (k - 1) * (k - 2) // 2,
                f2=k * (k + 1) // 2, c2=(k - 1) * k * (k + 1) // 2,
                v0=1, e0=k - 1, f0=(k - 1) * (k - 2) // 2,
                t3=k * (k + 1) * (k + 2) // 6)


class KuhnMesh:
    def __init__(self, n, order=1, side=1.0):
        assert n >= 1 and order in (1, 2, 3)
        self.n, self.k, self.side = n, order, float(side)
        self.h = self.side / n
        self.cnt = dofs_per_entity(order)
        T = 6 * n ** 3
        self.n_tets = T
        t = np.arange(T)
        cube = t // 6
        self.tet_shape = t % 6
        self.tet_cube = np.stack([cube % n, (cube // n) % n, cube // (n * n)], axis=1)
        off = np.array([[0, d1, d2, 7] for d1, d2 in TET_SHAPES])          # (6, 4)
        self.tet_off = off[self.tet_shape]                                   # (T, 4) masks
        self.tet_vlat = self.tet_cube[:, None, :] + bits(self.tet_off)      # (T, 4, 3) lattice coords
        self.tet_vx = self.tet_vlat * self.h                                 # coordinates
        self._build_classes()

    # ---------------------------------------------------------------- numbering
    def _box(self, extent):
        n = self.n
        e = bits(extent)
        lo = np.where(e == 1, 0, 1)
        num = np.where(e == 1, n, n - 1)
        return lo, num

    def _make_classes(self, spec):
        """spec: list of (kind, shape_index, extent_mask, j).  Returns offsets and boxes."""
        offs, boxes, total = [], [], 0
        for kind, s, ext, j in spec:
            lo, num = self._box(ext)
            offs.append(total)
            boxes.append((lo, num))
            total += int(np.prod(num))
        return offs, boxes, total

    def _build_classes(self):
        c = self.cnt
        s1 = []
        for s, d in enumerate(EDGE_SHAPES):
            for j in range(c["e1"]):
                s1.append(("e", s, d, j))
        for s, (d1, d2) in enumerate(FACE_SHAPES):
            for j in range(c["f1"]):
                s1.append(("f", s, d2, j))
        for s in range(6):
            for j in range(c["c1"]):
                s1.append(("t", s, 7, j))
        s2 = []
        for s, (d1, d2) in enumerate(FACE_SHAPES):
            for j in range(c["f2"]):
                s2.append(("f", s, d2, j))
        for s in range(6):
            for j in range(c["c2"]):
                s2.append(("t", s, 7, j))
        s0 = [("v", 0, 0, 0)]
        for s, d in enumerate(EDGE_SHAPES):
            for j in range(c["e0"]):
                s0.append(("e", s, d, j))
        for s, (d1, d2) in enumerate(FACE_SHAPES):
            for j in range(c["f0"]):
                s0.append(("f", s, d2, j))
        self.classes1, self.classes2, self.classes0 = s1, s2, s0
        self.off1, self.box1, self.N1 = self._make_classes(s1)
        self.off2, self.box2, self.N2 = self._make_classes(s2)
        self.off0, self.box0, self.N0 = self._make_classes(s0)
        self.cid1 = {(kd, s, j): i for i, (kd, s, _, j) in enumerate(s1)}
        self.cid2 = {(kd, s, j): i for i, (kd, s, _, j) in enumerate(s2)}
        self.cid0 = {(kd, s, j): i for i, (kd, s, _, j) in enumerate(s0)}
        self.N3 = self.n_tets * self.cnt["t3"]

    def _index(self, offs, boxes, cls, anchor):
        """Global index of DoFs of class `cls` (array) at lattice anchors (array, 3) or -1."""
        cls = np.asarray(cls)
        lo = np.array([boxes[c][0] for c in cls.ravel()]).reshape(cls.shape + (3,))
        num = np.array([boxes[c][1] for c in cls.ravel()]).reshape(cls.shape + (3,))
        o = np.array([offs[c] for c in cls.ravel()]).reshape(cls.shape)
        r = anchor - lo
        inside = np.all((r >= 0) & (r < num), axis=-1)
        idx = o + (r[..., 2] * num[..., 1] + r[..., 1]) * num[..., 0] + r[..., 0]
        return np.where(inside, idx, -1)

    def _local_entities(self):
        """Per tet: (shape index, anchor) of its 6 edges, 4 faces, and itself."""
        T = self.n_tets
        off = self.tet_off
        e_shape = np.zeros((T, 6), int)
        e_anchor = np.zeros((T, 6, 3), int)
        for le, (i, j) in enumerate(LOCAL_EDGES):
            d = off[:, j] ^ off[:, i]
            e_shape[:, le] = d - 1
            e_anchor[:, le] = self.tet_vlat[:, i]
        f_shape = np.zeros((T, 4), int)
        f_anchor = np.zeros((T, 4, 3), int)
        for lf, (i, j, l) in enumerate(LOCAL_FACES):
            d1 = off[:, j] ^ off[:, i]
            d2 = off[:, l] ^ off[:, i]
            f_shape[:, lf] = [_FACE_INDEX[(a, b)] for a, b in zip(d1, d2)]
            f_anchor[:, lf] = self.tet_vlat[:, i]
        return e_shape, e_anchor, f_shape, f_anchor

    def dof_maps(self):
        """(dof0, dof1, dof2, dof3): per-tet arrays of global DoF indices, -1 where removed.

        Local order: 1-forms edges (LOCAL_EDGES, k each), faces (LOCAL_FACES, k(k-1)
        each), cell; 2-forms faces (k(k+1)/2 each), cell; 0-forms vertices, edges,
        faces; 3-forms the tet's own k(k+1)(k+2)/6 DoFs.
        """
        if hasattr(self, "_maps"):
            return self._maps
        c = self.cnt
        es, ea, fs, fa = self._local_entities()
        T = self.n_tets
        cols1, cols2, cols0 = [], [], []
        for le in range(6):
            for j in range(c["e1"]):
                cols1.append(self._index(self.off1, self.box1, es[:, le] * c["e1"] + j, ea[:, le]))
        base_f1 = 7 * c["e1"]
        for lf in range(4):
            for j in range(c["f1"]):
                cols1.append(self._index(self.off1, self.box1, base_f1 + fs[:, lf] * c["f1"] + j, fa[:, lf]))
        base_c1 = base_f1 + 12 * c["f1"]
        for j in range(c["c1"]):
            cols1.append(self._index(self.off1, self.box1, base_c1 + self.tet_shape * c["c1"] + j, self.tet_cube))
        for lf in range(4):
            for j in range(c["f2"]):
                cols2.append(self._index(self.off2, self.box2, fs[:, lf] * c["f2"] + j, fa[:, lf]))
        base_c2 = 12 * c["f2"]
        for j in range(c["c2"]):
            cols2.append(self._index(self.off2, self.box2, base_c2 + self.tet_shape * c["c2"] + j, self.tet_cube))
        for lv in range(4):
            cols0.append(self._index(self.off0, self.box0, np.zeros(T, int), self.tet_vlat[:, lv]))
        for le in range(6):
            for j in range(c["e0"]):
                cols0.append(self._index(self.off0, self.box0, 1 + es[:, le] * c["e0"] + j, ea[:, le]))
        base_f0 = 1 + 7 * c["e0"]
        for lf in range(4):
            for j in range(c["f0"]):
                cols0.append(self._index(self.off0, self.box0, base_f0 + fs[:, lf] * c["f0"] + j, fa[:, lf]))
        dof1 = np.stack(cols1, axis=1)
        dof2 = np.stack(cols2, axis=1)
        dof0 = np.stack(cols0, axis=1)
        dof3 = np.arange(T)[:, None] * c["t3"] + np.arange(c["t3"])[None, :]
        self._maps = (dof0, dof1, dof2, dof3)
        return self._maps

    def locate(self, x):
        """Index of the tet containing point x (lowest index if x lies on shared faces)."""
        x = np.asarray(x, float) / self.h
        cube = np.clip(np.floor(x).astype(int), 0, self.n - 1)
        r = x - cube
        best = None
        for s, (d1, d2) in enumerate(TET_SHAPES):
            # Kuhn tet of permutation (a1, a2, a3): 1 >= r[a1] >= r[a2] >= r[a3] >= 0
            a1 = int(np.log2(d1))
            a2 = int(np.log2(d2 ^ d1))
            a3 = int(np.log2(7 ^ d2))
            if r[a1] >= r[a2] - 1e-14 and r[a2] >= r[a3] - 1e-14:
                t = 6 * (cube[0] + self.n * (cube[1] + self.n * cube[2])) + s
                best = t if best is None else min(best, t)
        return best
