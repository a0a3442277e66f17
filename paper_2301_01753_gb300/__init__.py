"""Python binding of libygm (the GB300 generalized Yee method leapfrog library).

Argument marshalling only: every step of the time integration runs in the library's CUDA
kernels, and the FP64 operator set-up runs in its C++ host code.  Names follow the C ABI
in include/ygm.h.  The library is built in-tree (paper_2301_01753_gb300/libygm.so); if it
is missing, importing this module raises -- there is no fallback path.
"""
import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libygm.so")

YGM_OK, YGM_EINVAL, YGM_ECFL, YGM_ENOTSPD, YGM_ENOMEM, YGM_ECUDA, YGM_ETIMEOUT, YGM_ENODEV = 0, -1, -2, -3, -4, -5, -6, -7
YGM_FP64, YGM_FP32, YGM_FP32_TC_TF32, YGM_FP32_TC_3XTF32 = 0, 1, 2, 3
YGM_Q1_DEFAULT, YGM_Q1_DIAG, YGM_Q1_SM1, YGM_Q1_SM1SQ = 0, 1, 2, 3

EXPORTED = ["ygm_create", "ygm_create_like", "ygm_sizes", "ygm_set_state", "ygm_get_state", "ygm_project_E", "ygm_step", "ygm_step_noalloc",
            "ygm_energy", "ygm_energy_history", "ygm_time", "ygm_export_q1", "ygm_set_q1", "ygm_spai_op", "ygm_cavity_modes", "ygm_q1_vjp", "ygm_q1_info",
            "ygm_local_blocks", "ygm_kernel_timing", "ygm_kernel_times", "ygm_set_qapply", "ygm_set_launch", "ygm_launch_count", "ygm_adjoint", "ygm_set_splitting",
            "ygm_yee_create", "ygm_yee_sizes", "ygm_yee_set_state", "ygm_yee_step", "ygm_yee_get_state",
            "ygm_yee_last_error", "ygm_yee_destroy",
            "ygm_batch_create", "ygm_batch_step", "ygm_batch_status", "ygm_batch_status_clear", "ygm_batch_wait_limit",
            "ygm_batch_tune", "ygm_batch_last_error",
            "ygm_batch_destroy",
            "ygm_qapply_counts", "ygm_last_error", "ygm_destroy"]
KERNEL_KINDS = ["k_qapply", "k_curl_b", "k_curlT_e", "k_source", "k_energy"]


class YgmError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"ygm error {code}: {msg}")
        self.code = code


class ygm_mesh(C.Structure):
    _fields_ = [("n", C.c_int32), ("side", C.c_double)]


class ygm_opts(C.Structure):
    _fields_ = [("precision", C.c_int32), ("q1_pattern", C.c_int32), ("n_rhs", C.c_int32),
                ("energy_every", C.c_int32), ("threads", C.c_int32), ("device", C.c_int32),
                ("stream", C.c_void_p)]


class ygm_source(C.Structure):
    _fields_ = [("x", C.c_double * 3), ("d", C.c_double * 3), ("amp", C.c_double), ("omega", C.c_double),
                ("t0", C.c_double), ("sigma", C.c_double), ("rhs", C.c_int32)]


E0_CB = C.CFUNCTYPE(None, C.POINTER(C.c_double), C.POINTER(C.c_double), C.c_void_p)


def load_library(path=LIB_PATH):
    if not os.path.exists(path):
        raise ImportError(f"{path} is missing: build it with __graft_entry__.build() "
                          "(python -m paper_2301_01753_gb300._build)")
    lib = C.CDLL(path)
    P, I64, D = C.c_void_p, C.c_int64, C.c_double
    pI64, pD, pI32 = C.POINTER(C.c_int64), C.POINTER(C.c_double), C.POINTER(C.c_int32)
    sig = {
        "ygm_create": (C.c_int, [C.POINTER(ygm_mesh), C.c_int, pD, pD, C.POINTER(ygm_opts), C.POINTER(P)]),
        "ygm_create_like": (C.c_int, [P, C.POINTER(ygm_opts), C.POINTER(P)]),
        "ygm_sizes": (C.c_int, [P, pI64, pI64, pI64, pD]),
        "ygm_set_state": (C.c_int, [P, P, P, C.c_int]),
        "ygm_get_state": (C.c_int, [P, P, P, C.c_int, C.c_int]),
        "ygm_project_E": (C.c_int, [P, E0_CB, P, C.c_int32]),
        "ygm_step": (C.c_int, [P, I64, D, C.POINTER(ygm_source), C.c_int32]),
        "ygm_step_noalloc": (C.c_int, [P, P, P, P, D]),
        "ygm_energy": (C.c_int, [P, pD, pD]),
        "ygm_energy_history": (C.c_int, [P, pD, I64, pI64]),
        "ygm_time": (C.c_int, [P, pI64, pD]),
        "ygm_export_q1": (C.c_int, [P, pI64, pI64, pD]),
        "ygm_set_q1": (C.c_int, [P, pI64, pI64, pD]),
        "ygm_spai_op": (C.c_int, [P, pD, C.c_int32, D, C.c_int32, D, pI32, pD]),
        "ygm_cavity_modes": (C.c_int, [P, C.c_int32, pD, pD, C.c_int32, D, pI32]),
        "ygm_q1_vjp": (C.c_int, [P, pD, pD]),
        "ygm_set_splitting": (C.c_int, [P, C.c_int32]),
        "ygm_adjoint": (C.c_int, [P, I64, D, C.POINTER(ygm_source), C.c_int32, C.POINTER(C.c_uint8), C.c_int32, pD, pD]),
        "ygm_q1_info": (C.c_int, [P, pD, pD, pD, pD, pI32, pI32]),
        "ygm_local_blocks": (C.c_int, [P, pI32, pI32, pD, pD]),
        "ygm_kernel_timing": (C.c_int, [P, C.c_int]),
        "ygm_set_qapply": (C.c_int, [P, C.c_int32, C.c_int32, C.POINTER(C.c_int32)]),
        "ygm_set_launch": (C.c_int, [P, C.c_int32]),
        "ygm_kernel_times": (C.c_int, [P, pD, pI64]),
        "ygm_launch_count": (C.c_int, [P, pI64]),
        "ygm_qapply_counts": (C.c_int, [P, C.c_int, pI64, pI64, pI64]),
        "ygm_batch_create": (C.c_int, [C.POINTER(P), C.c_int32, C.POINTER(P)]),
        "ygm_batch_step": (C.c_int, [P, I64, pD, C.POINTER(ygm_source), C.c_int32]),
        "ygm_batch_status": (C.c_int, [P]),
        "ygm_batch_status_clear": (C.c_int, [P]),
        "ygm_batch_wait_limit": (C.c_int, [P, I64]),
        "ygm_batch_tune": (C.c_int, [P, C.c_int32, pD, C.POINTER(ygm_source), pI32, pI32, pD]),
        "ygm_batch_last_error": (C.c_char_p, [P]),
        "ygm_batch_destroy": (None, [P]),
        "ygm_yee_create": (C.c_int, [C.POINTER(C.c_int32), pD, pD, pD, C.c_int32, C.c_int32, P, C.POINTER(P)]),
        "ygm_yee_sizes": (C.c_int, [P, pI64, pI64, pD]),
        "ygm_yee_set_state": (C.c_int, [P, P, P, C.c_int]),
        "ygm_yee_step": (C.c_int, [P, I64, D]),
        "ygm_yee_get_state": (C.c_int, [P, P, P, C.c_int, C.c_int]),
        "ygm_yee_last_error": (C.c_char_p, [P]),
        "ygm_yee_destroy": (None, [P]),
        "ygm_last_error": (C.c_char_p, [P]),
        "ygm_destroy": (None, [P]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    return lib


_lib = load_library()


def _ptr(a):
    """Raw pointer of a numpy array or a torch tensor (contiguous), and whether it is on a device."""
    if hasattr(a, "data_ptr"):
        assert a.is_contiguous()
        return C.c_void_p(a.data_ptr()), 1 if a.is_cuda else 0
    assert isinstance(a, np.ndarray) and a.flags.c_contiguous
    return a.ctypes.data_as(C.c_void_p), 0


def _stream_arg(stream):
    """cudaStream_t for the opts: None lets the context create its own non-blocking stream; 0 is
    the legacy default stream (the handle torch reports for its default stream), passed as
    cudaStreamLegacy so that work and events on torch's default stream are ordered with it."""
    if stream is None:
        return None
    return C.c_void_p(1 if int(stream) == 0 else int(stream))


class Context:
    """One GYM cavity: operators on the device plus the state (e, b)."""

    def __init__(self, n, order, eps=None, mu=None, side=1.0, precision=YGM_FP64, q1_pattern=YGM_Q1_DEFAULT,
                 n_rhs=1, energy_every=0, threads=0, device=0, stream=None):
        self._h = C.c_void_p()
        mesh = ygm_mesh(int(n), float(side))
        opts = ygm_opts(precision, q1_pattern, n_rhs, energy_every, threads, device,
                        _stream_arg(stream))
        T = 6 * n ** 3
        self._eps = None if eps is None else np.ascontiguousarray(eps, np.float64)
        self._mu = None if mu is None else np.ascontiguousarray(mu, np.float64)
        for a in (self._eps, self._mu):
            if a is not None and a.shape != (T,):
                raise ValueError(f"per-tet arrays must have length 6 n^3 = {T}")
        pe = self._eps.ctypes.data_as(C.POINTER(C.c_double)) if self._eps is not None else None
        pm = self._mu.ctypes.data_as(C.POINTER(C.c_double)) if self._mu is not None else None
        rc = _lib.ygm_create(C.byref(mesh), int(order), pe, pm, C.byref(opts), C.byref(self._h))
        if rc:
            raise YgmError(rc, _lib.ygm_last_error(None).decode())
        self.n, self.order, self.precision, self.n_rhs, self.device = n, order, precision, n_rhs, device
        self.dtype = np.float64 if precision == YGM_FP64 else np.float32
        self.N1, self.N2, self.q1_nnz, self.tau_cfl = self.sizes()

    def like(self, precision=None, n_rhs=1, energy_every=0, device=None, stream=None):
        """A second context of the same problem (ygm_create_like): same mesh, materials and
        operators, its own precision / columns / device; no operator set-up is recomputed."""
        new = Context.__new__(Context)
        new._h = C.c_void_p()
        precision = self.precision if precision is None else precision
        dev = self.device if device is None else device
        opts = ygm_opts(precision, 0, n_rhs, energy_every, 0, dev, _stream_arg(stream))
        rc = _lib.ygm_create_like(self._h, C.byref(opts), C.byref(new._h))
        if rc:
            raise YgmError(rc, _lib.ygm_last_error(None).decode())
        new._eps, new._mu = self._eps, self._mu
        new.n, new.order, new.precision, new.n_rhs, new.device = self.n, self.order, precision, n_rhs, dev
        new.dtype = np.float64 if precision == YGM_FP64 else np.float32
        new.N1, new.N2, new.q1_nnz, new.tau_cfl = new.sizes()
        return new

    # ---------------------------------------------------------------- helpers
    def _check(self, rc):
        if rc:
            raise YgmError(rc, _lib.ygm_last_error(self._h).decode())

    def close(self):
        if self._h:
            _lib.ygm_destroy(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    # ---------------------------------------------------------------- ABI calls
    def sizes(self):
        n1, n2, nnz, dt = C.c_int64(), C.c_int64(), C.c_int64(), C.c_double()
        self._check(_lib.ygm_sizes(self._h, C.byref(n1), C.byref(n2), C.byref(nnz), C.byref(dt)))
        return n1.value, n2.value, nnz.value, dt.value

    def set_state(self, e, b):
        pe, de = _ptr(e)
        pb, db = _ptr(b)
        assert de == db
        self._check(_lib.ygm_set_state(self._h, pe, pb, de))

    def get_state(self, synced=True, out_e=None, out_b=None):
        R = self.n_rhs
        e = out_e if out_e is not None else np.empty(self.N1 * R, self.dtype)
        b = out_b if out_b is not None else np.empty(self.N2 * R, self.dtype)
        pe, de = _ptr(e)
        pb, db = _ptr(b)
        self._check(_lib.ygm_get_state(self._h, pe, pb, de, 1 if synced else 0))
        return e, b

    def project_E(self, E0, rhs=0):
        """E0(x: ndarray(3)) -> ndarray(3), evaluated on host points by the library."""
        def cb(xp, outp, user):
            v = E0(np.array([xp[0], xp[1], xp[2]]))
            outp[0], outp[1], outp[2] = float(v[0]), float(v[1]), float(v[2])
        self._cb = E0_CB(cb)
        self._check(_lib.ygm_project_E(self._h, self._cb, None, rhs))

    def set_splitting(self, order):
        """2: Strang leapfrog (default); 4: fourth-order symmetric composition (ygm_set_splitting)."""
        self._check(_lib.ygm_set_splitting(self._h, int(order)))

    def step(self, n, dt, sources=()):
        self._check(_lib.ygm_step(self._h, int(n), float(dt), _source_array(sources), len(sources)))

    def adjoint(self, nsteps, dt, sources, region, checkpoint_every=100, gradient=True):
        """(L, dL/d eps) of the probe-region energy of ygm_adjoint: the leapfrog from rest under
        `sources` for `nsteps` steps of `dt`, region = boolean per tet.  gradient=False returns
        (L, None) without the reverse sweep's host SPAI derivative.  Leaves the state at rest."""
        T = 6 * self.n ** 3
        reg = np.ascontiguousarray(np.asarray(region).astype(np.uint8))
        if reg.shape != (T,):
            raise ValueError(f"region must have 6 n^3 = {T} entries")
        L = C.c_double()
        g = np.zeros(T) if gradient else None
        self._check(_lib.ygm_adjoint(self._h, int(nsteps), float(dt), _source_array(sources), len(sources),
                                     reg.ctypes.data_as(C.POINTER(C.c_uint8)), int(checkpoint_every), C.byref(L),
                                     g.ctypes.data_as(C.POINTER(C.c_double)) if gradient else None))
        return L.value, g

    def step_noalloc(self, e, b_in, b_out, dt):
        """One leapfrog step on caller-owned device tensors, no device allocation (ygm_step_noalloc)."""
        pe, de = _ptr(e)
        pbi, dbi = _ptr(b_in)
        pbo, dbo = _ptr(b_out)
        assert de == dbi == dbo == 1, "ygm_step_noalloc works on device buffers"
        self._check(_lib.ygm_step_noalloc(self._h, pe, pbi, pbo, float(dt)))

    def energy(self):
        W = (C.c_double * self.n_rhs)()
        H = (C.c_double * self.n_rhs)()
        self._check(_lib.ygm_energy(self._h, W, H))
        return np.array(W[:]), np.array(H[:])

    def energy_history(self, max_count=1 << 16):
        out = np.empty(max_count * self.n_rhs)
        cnt = C.c_int64()
        self._check(_lib.ygm_energy_history(self._h, out.ctypes.data_as(C.POINTER(C.c_double)), max_count,
                                            C.byref(cnt)))
        return out[:cnt.value * self.n_rhs].copy()

    def time(self):
        s, t = C.c_int64(), C.c_double()
        self._check(_lib.ygm_time(self._h, C.byref(s), C.byref(t)))
        return s.value, t.value

    def export_q1(self):
        """(rowptr, colind, val) of the symmetric FP64 Q1 over the global numbering."""
        rp = np.empty(self.N1 + 1, np.int64)
        ci = np.empty(self.q1_nnz, np.int64)
        va = np.empty(self.q1_nnz, np.float64)
        self._check(_lib.ygm_export_q1(self._h, rp.ctypes.data_as(C.POINTER(C.c_int64)),
                                       ci.ctypes.data_as(C.POINTER(C.c_int64)),
                                       va.ctypes.data_as(C.POINTER(C.c_double))))
        return rp, ci, va

    def set_q1(self, Q):
        """Install a symmetric scipy.sparse Q1 (global numbering) in place of the SPAI."""
        import scipy.sparse as sp
        Q = sp.csr_matrix(Q)
        Q.sort_indices()
        rp = np.ascontiguousarray(Q.indptr, np.int64)
        ci = np.ascontiguousarray(Q.indices, np.int64)
        va = np.ascontiguousarray(Q.data, np.float64)
        self._check(_lib.ygm_set_q1(self._h, rp.ctypes.data_as(C.POINTER(C.c_int64)),
                                    ci.ctypes.data_as(C.POINTER(C.c_int64)),
                                    va.ctypes.data_as(C.POINTER(C.c_double))))
        self.N1, self.N2, self.q1_nnz, self.tau_cfl = self.sizes()

    def spai_op(self, V=None, lam=0.0, max_iter=5000, tol=1e-12):
        """Operator-probed SPAI (ygm_spai_op): V is N1 x n_probe (probe modes as columns).
        Returns (PCG iterations, final relative residual)."""
        if V is None:
            Vc, npb = None, 0
        else:
            V = np.asarray(V, dtype=np.float64).reshape(self.N1, -1)
            npb = V.shape[1]
            Vc = np.ascontiguousarray(V.T)             # column-major: mode k contiguous
        it, rr = C.c_int32(), C.c_double()
        self._check(_lib.ygm_spai_op(self._h, None if Vc is None else Vc.ctypes.data_as(C.POINTER(C.c_double)),
                                     npb, float(lam), int(max_iter), float(tol), C.byref(it), C.byref(rr)))
        self.N1, self.N2, self.q1_nnz, self.tau_cfl = self.sizes()
        return it.value, rr.value

    def cavity_modes(self, count, max_iter=500, tol=1e-10):
        """Lowest non-kernel eigenpairs of P2 v = omega^2 M1 v (ygm_cavity_modes):
        returns (omega_sq[count], V[N1, count]) with v^T M1 v = 1."""
        V = np.empty((count, self.N1), dtype=np.float64)          # row k = mode k (column-major N1 x count)
        w = np.empty(count, dtype=np.float64)
        it = C.c_int32()
        self._check(_lib.ygm_cavity_modes(self._h, int(count), V.ctypes.data_as(C.POINTER(C.c_double)),
                                          w.ctypes.data_as(C.POINTER(C.c_double)), int(max_iter), float(tol),
                                          C.byref(it)))
        return w, V.T.copy()

    def q1_vjp(self, q1bar):
        """dL/d eps per tet through Q1, given dL/dQ1 on the ygm_export_q1 pattern (ygm_q1_vjp)."""
        qb = np.ascontiguousarray(q1bar, dtype=np.float64)
        if qb.shape != (self.q1_nnz,):
            raise ValueError(f"q1bar must hold the {self.q1_nnz} stored entries of Q1")
        g = np.empty(6 * self.n ** 3, dtype=np.float64)
        self._check(_lib.ygm_q1_vjp(self._h, qb.ctypes.data_as(C.POINTER(C.c_double)),
                                    g.ctypes.data_as(C.POINTER(C.c_double))))
        return g

    def q1_info(self):
        lmin, lmax, sh, w2 = C.c_double(), C.c_double(), C.c_double(), C.c_double()
        pat, orth = C.c_int32(), C.c_int32()
        self._check(_lib.ygm_q1_info(self._h, C.byref(lmin), C.byref(lmax), C.byref(sh), C.byref(w2),
                                     C.byref(pat), C.byref(orth)))
        return dict(lmin=lmin.value, lmax=lmax.value, shift=sh.value, omega_max_sq=w2.value,
                    pattern=pat.value, ortho=orth.value)

    def local_blocks(self):
        n1, n2a = C.c_int32(), C.c_int32()
        self._check(_lib.ygm_local_blocks(self._h, C.byref(n1), C.byref(n2a), None, None))
        M1 = np.empty(n1.value ** 2)
        M2 = np.empty(n2a.value ** 2)
        self._check(_lib.ygm_local_blocks(self._h, C.byref(n1), C.byref(n2a),
                                          M1.ctypes.data_as(C.POINTER(C.c_double)),
                                          M2.ctypes.data_as(C.POINTER(C.c_double))))
        return M1.reshape(n1.value, -1), M2.reshape(n2a.value, -1)

    def set_qapply(self, kernel=0, stages=0):
        """Select the Q1 apply kernel (0 automatic, 1 per-thread loads, 2 bulk copies into shared-
        memory stages; stages 0 = as many as fit) and return its resident blocks per SM."""
        bps = C.c_int32(0)
        self._check(_lib.ygm_set_qapply(self._h, int(kernel), int(stages), C.byref(bps)))
        return bps.value

    def set_launch(self, pdl=True):
        """Programmatic dependent launch between the one-column step's kernels (on by default)."""
        self._check(_lib.ygm_set_launch(self._h, 1 if pdl else 0))

    def kernel_timing(self, enable=True):
        self._check(_lib.ygm_kernel_timing(self._h, 1 if enable else 0))

    def kernel_times(self):
        """{kernel: (total ms, launches)} since the last call (requires kernel_timing(True))."""
        ms = (C.c_double * 5)()
        cnt = (C.c_int64 * 5)()
        self._check(_lib.ygm_kernel_times(self._h, ms, cnt))
        return {k: (ms[i], cnt[i]) for i, k in enumerate(KERNEL_KINDS)}

    def launch_count(self):
        c = C.c_int64()
        self._check(_lib.ygm_launch_count(self._h, C.byref(c)))
        return c.value

    def qapply_counts(self, all_rows):
        """(rows, unique Q1 values, streamed Q1 entries) of one Q1 apply launch (roofline accounting)."""
        r, u, st = C.c_int64(), C.c_int64(), C.c_int64()
        self._check(_lib.ygm_qapply_counts(self._h, 1 if all_rows else 0, C.byref(r), C.byref(u), C.byref(st)))
        return r.value, u.value, st.value


class Yee:
    """Cubical Whitney GYM (Yee) on a periodic box (ygm_yee_*): n = (n0, n1, n2) cubes, h = edge
    lengths, optional diagonal q1 / m2 (3 n0 n1 n2 values each)."""

    def __init__(self, n, h, q1=None, m2=None, precision=YGM_FP64, device=0, stream=None):
        nn = (C.c_int32 * 3)(*[int(v) for v in n])
        hh = (C.c_double * 3)(*[float(v) for v in h])
        self._q = None if q1 is None else np.ascontiguousarray(q1, np.float64)
        self._m = None if m2 is None else np.ascontiguousarray(m2, np.float64)
        pq = self._q.ctypes.data_as(C.POINTER(C.c_double)) if self._q is not None else None
        pm = self._m.ctypes.data_as(C.POINTER(C.c_double)) if self._m is not None else None
        self._h = C.c_void_p()
        rc = _lib.ygm_yee_create(nn, hh, pq, pm, precision, device, _stream_arg(stream),
                                 C.byref(self._h))
        if rc:
            raise YgmError(rc, _lib.ygm_yee_last_error(None).decode())
        self.dtype = np.float64 if precision == YGM_FP64 else np.float32
        n1, n2, dt = C.c_int64(), C.c_int64(), C.c_double()
        self._check(_lib.ygm_yee_sizes(self._h, C.byref(n1), C.byref(n2), C.byref(dt)))
        self.N1, self.N2, self.tau_cfl = n1.value, n2.value, dt.value

    def _check(self, rc):
        if rc:
            raise YgmError(rc, _lib.ygm_yee_last_error(self._h).decode())

    def set_state(self, e, b):
        pe, de = _ptr(e)
        pb, db = _ptr(b)
        self._check(_lib.ygm_yee_set_state(self._h, pe, pb, de))

    def step(self, n, dt):
        self._check(_lib.ygm_yee_step(self._h, int(n), float(dt)))

    def get_state(self, synced=True):
        e = np.empty(self.N1, self.dtype)
        b = np.empty(self.N2, self.dtype)
        self._check(_lib.ygm_yee_get_state(self._h, _ptr(e)[0], _ptr(b)[0], 0, 1 if synced else 0))
        return e, b

    def close(self):
        if self._h:
            _lib.ygm_yee_destroy(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Batch:
    """Independent one-column contexts (any n, order) stepped together by one persistent launch
    (ygm_batch_*).  The contexts stay usable for set_state / get_state / energy and must outlive
    the batch."""

    def __init__(self, contexts):
        self._ctx = list(contexts)
        hs = (C.c_void_p * len(self._ctx))(*[c._h.value for c in self._ctx])
        self._h = C.c_void_p()
        rc = _lib.ygm_batch_create(hs, len(self._ctx), C.byref(self._h))
        if rc:
            raise YgmError(rc, _lib.ygm_last_error(None).decode())

    def _check(self, rc):
        if rc:
            raise YgmError(rc, _lib.ygm_batch_last_error(self._h).decode())

    def _args(self, dts, sources):
        d = np.ascontiguousarray(dts, np.float64)
        assert d.shape == (len(self._ctx),)
        src = _source_array(sources) if sources is not None else None
        return d, src

    def step(self, nsteps, dts, sources=None, use_graph=False):
        d, src = self._args(dts, sources)
        self._check(_lib.ygm_batch_step(self._h, int(nsteps), d.ctypes.data_as(C.POINTER(C.c_double)), src,
                                        1 if use_graph else 0))

    def status(self):
        self._check(_lib.ygm_batch_status(self._h))

    def status_clear(self):
        self._check(_lib.ygm_batch_status_clear(self._h))

    def wait_limit(self, polls):
        self._check(_lib.ygm_batch_wait_limit(self._h, int(polls)))

    def tune(self, trial_steps, dts, sources=None):
        """Autotune the launch shape; returns (CTAs per SM, work order, ms per step)."""
        d, src = self._args(dts, sources)
        c, o, ms = C.c_int32(), C.c_int32(), C.c_double()
        self._check(_lib.ygm_batch_tune(self._h, int(trial_steps), d.ctypes.data_as(C.POINTER(C.c_double)), src,
                                        C.byref(c), C.byref(o), C.byref(ms)))
        return c.value, o.value, ms.value

    def close(self):
        if self._h:
            _lib.ygm_batch_destroy(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _source_array(sources):
    arr = (ygm_source * max(1, len(sources)))()
    for i, s in enumerate(sources):
        arr[i].x[:] = list(map(float, s["x"]))
        arr[i].d[:] = list(map(float, s["d"]))
        arr[i].amp = float(s.get("amp", 1.0))
        arr[i].omega = float(s["omega"])
        arr[i].t0 = float(s["t0"])
        arr[i].sigma = float(s["sigma"])
        arr[i].rhs = int(s.get("rhs", 0))
    return arr


def probe_energy(eps, n, order, nsteps, dt, sources, region, checkpoint_every=100, precision=YGM_FP64, device=0):
    """The probe-region energy of ygm_adjoint as a differentiable function of the per-tet
    permittivity (a torch tensor of 6 n^3 entries): forward builds the operators for eps and runs
    the leapfrog, backward returns dL/d eps from the device adjoint.  dt is held fixed."""
    import torch

    class _ProbeEnergy(torch.autograd.Function):
        @staticmethod
        def forward(fctx, e):
            eh = e.detach().to("cpu", torch.float64).numpy()
            with Context(n, order, eps=eh, precision=precision, device=device) as c:
                L, g = c.adjoint(nsteps, dt, sources, region, checkpoint_every=checkpoint_every, gradient=True)
            fctx.save_for_backward(torch.as_tensor(g, dtype=e.dtype, device=e.device))
            return torch.tensor(L, dtype=e.dtype, device=e.device)

        @staticmethod
        def backward(fctx, gout):
            (g,) = fctx.saved_tensors
            return gout * g

    return _ProbeEnergy.apply(eps)


def pulse_source(x, d, omega, dt, width_steps=20.0, amp=1.0, t0_sigmas=4.0, rhs=0):
    """Dipole with s(t) = amp exp(-((t - t0)/sigma)^2) sin(omega (t - t0)), sigma = width * dt, t0 = 4 sigma."""
    sigma = width_steps * dt
    return dict(x=x, d=d, amp=amp, omega=omega, t0=t0_sigmas * sigma, sigma=sigma, rhs=rhs)
