"""CPU tests of the product's host logic: the C-ABI library loads and exports every declared
symbol, and the FP64 host builder (host-only contexts, no GPU) matches the oracle."""
import os
import re

import numpy as np
import pytest
import scipy.sparse as sp

import synth
from oracle_runs import oracle_model

Y = pytest.importorskip("paper_2301_01753_gb300")
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_every_declared_symbol_is_exported():
    hdr = open(os.path.join(ROOT, "include", "ygm.h")).read()
    declared = set(re.findall(r"\b(ygm_[A-Za-z0-9_]+)\s*\(", hdr))
    assert declared == set(Y.EXPORTED)
    for name in declared:
        assert hasattr(Y._lib, name), name


@pytest.mark.parametrize("n,k,pattern,tol", [(4, 1, None, 1e-13), (3, 2, None, 1e-12), (2, 3, None, 1e-11),
                                             (3, 2, "diag", 1e-13), (4, 1, "sm1sq", 1e-13), (3, 2, "sm1", 1e-12)])
def test_host_builder_matches_oracle(n, k, pattern, tol):
    code = {None: Y.YGM_Q1_DEFAULT, "diag": Y.YGM_Q1_DIAG, "sm1": Y.YGM_Q1_SM1, "sm1sq": Y.YGM_Q1_SM1SQ}[pattern]
    f, g, eps, info = oracle_model(n, k, eps_seed=5, pattern=pattern)
    c = Y.Context(n, k, eps=eps, device=-1, q1_pattern=code)
    assert (c.N1, c.N2) == (f.mesh.N1, f.mesh.N2)
    rp, ci, va = c.export_q1()
    Qb = sp.csr_matrix((va, ci, rp), shape=(c.N1, c.N1))
    assert Qb.nnz == g.Q1.nnz
    assert abs(Qb - g.Q1).max() <= tol * abs(g.Q1).max()
    if info["shift"] == 0.0:
        assert abs(c.tau_cfl / g.tau_cfl() - 1) < 1e-9
    M1l, M2l = c.local_blocks()
    assert np.allclose(M1l, f.local(0)["M1"], rtol=1e-12, atol=1e-16)


def test_host_only_context_refuses_stepping():
    c = Y.Context(2, 1, device=-1)
    with pytest.raises(Y.YgmError) as ei:
        c.step(1, 0.01)
    assert ei.value.code == Y.YGM_ENODEV


def test_invalid_arguments_are_rejected():
    with pytest.raises(Y.YgmError) as ei:
        Y.Context(0, 1, device=-1)
    assert ei.value.code == Y.YGM_EINVAL
    with pytest.raises(Y.YgmError):
        Y.Context(2, 4, device=-1)
    with pytest.raises(Y.YgmError):
        Y.Context(2, 1, eps=-np.ones(48), device=-1)
    with pytest.raises(Y.YgmError):
        Y.Context(2, 1, eps=np.full(48, np.nan), device=-1)


def test_set_q1_checks_pattern_symmetry_and_definiteness():
    f, g, eps, _ = oracle_model(2, 2, eps_seed=6)
    c = Y.Context(2, 2, eps=eps, device=-1)
    c.set_q1(g.Q1)
    assert abs(c.tau_cfl / g.tau_cfl() - 1) < 1e-9
    Q = g.Q1.tolil()
    i, j = 0, g.Q1.indices[g.Q1.indptr[0] + 1]
    Q[i, j] += 1.0                                     # breaks symmetry
    with pytest.raises(Y.YgmError):
        c.set_q1(Q.tocsr())
    rp0, ci0, va0 = c.export_q1()
    tau0 = c.tau_cfl
    with pytest.raises(Y.YgmError) as ei:
        c.set_q1(-g.Q1)                                # negative definite
    assert ei.value.code == Y.YGM_ENOTSPD
    rp1, ci1, va1 = c.export_q1()                      # the previous Q1 is kept
    assert np.array_equal(rp0, rp1) and np.array_equal(ci0, ci1) and np.array_equal(va0, va1)
    assert c.sizes()[3] == tau0 and c.q1_info()["lmin"] > 0


def _probe_modes(f, M1, count):
    """The lowest non-kernel eigenmodes of M1^-1 P2 (dense generalised eigensolver, test side),
    normalised to v^T M1 v = 1."""
    import scipy.linalg as sl
    P2 = (f.C().T @ f.M2() @ f.C()).tocsr()
    w, V = sl.eigh(P2.toarray(), M1.toarray())
    nz = np.where(w > 1e-8 * w[-1])[0][:count]
    return P2, w[nz], V[:, nz]


@pytest.mark.parametrize("lam", [0.0, 1e3])
def test_host_spai_op_matches_oracle(lam):
    """ygm_spai_op (Sec. 5.1) against the oracle's Sylvester PCG, same pattern, probes, warm start."""
    from oracle import spai as SP
    from oracle import spai_op as OP
    f, g, eps, _ = oracle_model(3, 1, eps_seed=5)
    M1 = f.M1()
    P2, w, V = _probe_modes(f, M1, 3)
    c = Y.Context(3, 1, eps=eps, device=-1)
    it, rr = c.spai_op(V, lam, tol=1e-13)
    assert rr <= 1e-13 and it > 0
    rp, ci, va = c.export_q1()
    Qb = sp.csr_matrix((va, ci, rp), shape=(c.N1, c.N1))
    Qo, _ = OP.spai_op(M1, SP.pattern("sm1", M1, f.dof1), P2=P2, V=V, lam=lam, q0=g.Q1, tol=1e-13)
    assert Qb.nnz == Qo.nnz
    assert abs(Qb - Qo).max() <= 1e-9 * abs(Qo).max()
    assert abs(Qb - Qb.T).max() == 0.0
    if lam > 0:    # the probed modes' residuals fall well below the column SPAI's
        for j in range(V.shape[1]):
            assert OP.eig_residual(Qb, P2, V[:, j], w[j]) < 0.05 * OP.eig_residual(g.Q1, P2, V[:, j], w[j])
    info = c.q1_info()
    assert info["lmin"] > 0 and abs(c.tau_cfl - 2 / np.sqrt(info["omega_max_sq"])) < 1e-12 * c.tau_cfl


def test_host_spai_op_rejects_bad_input():
    c = Y.Context(2, 1, device=-1)
    with pytest.raises(Y.YgmError) as ei:
        c.spai_op(np.full((c.N1, 1), np.nan), 1.0)
    assert ei.value.code == Y.YGM_EINVAL
    with pytest.raises(Y.YgmError) as ei:
        c.spai_op(np.ones((c.N1, 1)), -1.0)
    assert ei.value.code == Y.YGM_EINVAL
    with pytest.raises(Y.YgmError) as ei:
        c.spai_op(np.ones((c.N1, 1)), 1e3, max_iter=1, tol=1e-15)
    assert ei.value.code == Y.YGM_ETIMEOUT


def test_create_like_copies_the_operators_without_recomputing():
    f, g, eps, _ = oracle_model(3, 1, eps_seed=5)
    c = Y.Context(3, 1, eps=eps, device=-1)
    it, _ = c.spai_op(np.ones((c.N1, 1)) / np.sqrt(c.N1), 10.0, tol=1e-12)
    d = c.like(precision=Y.YGM_FP32, n_rhs=4, device=-1)
    assert (d.N1, d.N2, d.q1_nnz) == (c.N1, c.N2, c.q1_nnz) and d.tau_cfl == c.tau_cfl
    for a, b in zip(c.export_q1(), d.export_q1()):
        assert np.array_equal(a, b)
    assert d.q1_info() == c.q1_info()
    c.close()
    assert d.export_q1()[0].shape == (d.N1 + 1,)      # independent of the source's lifetime
    with pytest.raises(Y.YgmError) as ei:
        d.like(n_rhs=3, device=-1)
    assert ei.value.code == Y.YGM_EINVAL


def test_host_spai_op_orthogonal_basis_matches_oracle():
    """Order 2: SPAI-OP in the entity-orthonormal basis (builder against oracle).  The Sylvester
    system is ill-conditioned there once lam > 0 (Sec. 5.1: the rank-n_probe term degrades it), so
    both solve to 1e-11 and agree to the matching level."""
    from oracle import spai_op as OP
    f, g, eps, _ = oracle_model(2, 2, eps_seed=7)
    M1 = f.M1()
    P2, w, V = _probe_modes(f, M1, 2)
    c = Y.Context(2, 2, eps=eps, device=-1)
    assert c.q1_info()["ortho"] == 1
    it, rr = c.spai_op(V, 1.0, tol=1e-11, max_iter=50000)
    assert rr <= 1e-11
    rp, ci, va = c.export_q1()
    Qb = sp.csr_matrix((va, ci, rp), shape=(c.N1, c.N1))
    Qo, info = OP.spai_op_q1(f, M1, P2, V, 1.0, tol=1e-11)
    assert abs(Qb - Qo).max() <= 1e-8 * abs(Qo).max()
    for j in range(V.shape[1]):
        assert OP.eig_residual(Qb, P2, V[:, j], w[j]) < 0.6 * OP.eig_residual(g.Q1, P2, V[:, j], w[j])


@pytest.mark.parametrize("n,k,seed", [(3, 1, 5), (4, 1, None), (2, 2, 7)])
def test_cavity_modes_match_dense_eigenpairs(n, k, seed):
    """ygm_cavity_modes against a dense generalised eigensolver on the oracle's P2 and M1: the
    lowest non-kernel eigenvalues (degenerate ones included, N=4 unit cube), M1-orthonormal
    eigenvectors, and the same eigenspaces."""
    import scipy.linalg as sl
    f, g, eps, _ = oracle_model(n, k, eps_seed=seed)
    M1 = f.M1()
    P2 = (f.C().T @ f.M2() @ f.C()).tocsr()
    w, V = sl.eigh(P2.toarray(), M1.toarray())
    nz = np.where(w > 1e-8 * w[-1])[0][:5]
    c = Y.Context(n, k, eps=eps, device=-1)
    wb, Vb = c.cavity_modes(5, tol=1e-10)
    assert np.allclose(wb, w[nz], rtol=1e-10)
    Md = M1.toarray()
    assert np.allclose(Vb.T @ Md @ Vb, np.eye(5), atol=1e-9)
    assert np.linalg.norm(P2 @ Vb - (Md @ Vb) * wb) <= 1e-8 * wb.max() * np.linalg.norm(Md @ Vb)
    # eigenspaces: every dense eigenvector of the (closed) cluster lies in the returned span
    full = [i for i in range(len(w)) if w[i] > 1e-8 * w[-1] and w[i] <= wb[-1] * (1 + 1e-9)]
    if len(full) == 5:
        Pv = Vb @ (Vb.T @ Md)                          # M1-orthogonal projector onto span(Vb)
        assert np.linalg.norm(Pv @ V[:, full] - V[:, full]) < 1e-7 * np.linalg.norm(V[:, full])


def test_cavity_modes_as_spai_op_probes():
    """The workflow of Sec. 5.1 through the C ABI only: compute probe modes, probe them with
    SPAI-OP, and the probed residual eigenvalue errors fall well below the column SPAI's."""
    from oracle import spai_op as OP
    f, g, eps, _ = oracle_model(3, 1, eps_seed=5)
    P2 = (f.C().T @ f.M2() @ f.C()).tocsr()
    c = Y.Context(3, 1, eps=eps, device=-1)
    w, V = c.cavity_modes(3)
    c.spai_op(V, 1e3, tol=1e-12)
    rp, ci, va = c.export_q1()
    Q = sp.csr_matrix((va, ci, rp), shape=(c.N1, c.N1))
    for j in range(3):
        assert OP.eig_residual(Q, P2, V[:, j], w[j]) < 0.05 * OP.eig_residual(g.Q1, P2, V[:, j], w[j])


def test_cavity_modes_reject_bad_counts():
    c = Y.Context(2, 1, device=-1)
    for bad in (0, c.N1):
        with pytest.raises(Y.YgmError) as ei:
            c.cavity_modes(bad)
        assert ei.value.code == Y.YGM_EINVAL


def test_option_validation_before_any_set_up():
    """Bad options are refused by ygm_create before the operators are built (host-only)."""
    for kw in (dict(n_rhs=3), dict(n_rhs=512), dict(n_rhs=0), dict(precision=7), dict(q1_pattern=9),
               dict(energy_every=-1)):
        with pytest.raises(Y.YgmError) as ei:
            Y.Context(2, 1, device=-1, **kw)
        assert ei.value.code == Y.YGM_EINVAL, kw
    with pytest.raises(Y.YgmError) as ei:
        Y.Context(2, 1, side=0.0, device=-1)
    assert ei.value.code == Y.YGM_EINVAL
    with pytest.raises(ValueError):
        Y.Context(2, 1, eps=np.ones(47), device=-1)   # per-tet arrays must have 6 n^3 entries


@pytest.mark.parametrize("n", [2, 3])
def test_q1_vjp_matches_the_oracle_spai_derivative(n):
    """ygm_q1_vjp (the differentiated normal equations) against oracle.adjoint.spai_vjp, for a
    random dL/dQ1 on the pattern (order 1, random eps)."""
    from oracle import adjoint as AD
    from oracle import spai as SP
    from oracle.fem import FEM
    from oracle.mesh import KuhnMesh
    eps = synth.tet_eps(5002, n, 1.0, 4.0)
    f = FEM(KuhnMesh(n, 1), eps=eps)
    c = Y.Context(n, 1, eps=eps, device=-1)
    rp, ci, va = c.export_q1()
    rng = np.random.default_rng(n)
    qbar = rng.standard_normal(len(va))
    g = c.q1_vjp(qbar)
    Qbar = sp.csr_matrix((qbar, ci, rp), shape=(c.N1, c.N1)).toarray()
    S = SP.pattern("sm1", f.M1(), f.dof1)
    go = AD.spai_vjp(f, S, 0.5 * (Qbar + Qbar.T) * (S.toarray() != 0))
    assert np.allclose(g, go, rtol=1e-9, atol=1e-11 * np.abs(go).max())
    assert np.array_equal(g, c.q1_vjp(qbar))                  # reproducible


@pytest.mark.parametrize("n,k", [(2, 2), (3, 2)])
def test_q1_vjp_through_the_orthonormal_basis_matches_the_oracle(n, k):
    """Orders >= 2: ygm_q1_vjp through Q1 = T Q' T and T = blockdiag (M1[g,g])^(-1/2) (reading R2)
    against oracle.adjoint.q1_ortho_vjp, itself pinned to central differences."""
    from oracle import adjoint as AD
    from oracle import spai as SP
    from oracle.fem import FEM
    from oracle.mesh import KuhnMesh
    eps = synth.tet_eps(5004, n, 1.0, 4.0)
    f = FEM(KuhnMesh(n, k), eps=eps)
    c = Y.Context(n, k, eps=eps, device=-1)
    assert c.q1_info()["ortho"] == 1
    rp, ci, va = c.export_q1()
    qbar = np.random.default_rng(k).standard_normal(len(va))
    g = c.q1_vjp(qbar)
    Qbar = sp.csr_matrix((qbar, ci, rp), shape=(c.N1, c.N1)).toarray()
    go = AD.q1_ortho_vjp(f, SP.pattern("sm1sq", f.M1(), f.dof1), Qbar)
    assert np.abs(g - go).max() <= 1e-10 * np.abs(go).max()


def test_noalloc_step_argument_checks_without_a_device():
    """ygm_step_noalloc refuses NULL buffers and host-only contexts before any CUDA call."""
    import ctypes as C
    c = Y.Context(2, 1, device=-1)
    buf = np.zeros(max(c.N1, c.N2))
    p = buf.ctypes.data_as(C.c_void_p)
    assert Y._lib.ygm_step_noalloc(c._h, None, p, p, 0.01) == Y.YGM_EINVAL
    assert Y._lib.ygm_step_noalloc(c._h, p, p, p, 0.01) == Y.YGM_ENODEV
    assert b"host-only" in Y._lib.ygm_last_error(c._h)


def test_stream_handles_passed_to_the_opts():
    # None: the context makes its own stream; 0 (torch's default stream) is the legacy default
    # stream, so events recorded there order with the context's launches; others pass through
    import paper_2301_01753_gb300 as Y
    assert Y._stream_arg(None) is None
    assert Y._stream_arg(0).value == 1
    assert Y._stream_arg(0x5000).value == 0x5000


def test_q1_kernel_selection_needs_a_device():
    import paper_2301_01753_gb300 as Y
    c = Y.Context(3, 2, device=-1)
    with pytest.raises(Y.YgmError):
        c.set_qapply(2, 0)


def test_launch_mode_needs_a_device_and_checks_its_argument():
    import ctypes
    import paper_2301_01753_gb300 as Y
    c = Y.Context(3, 1, device=-1)
    with pytest.raises(Y.YgmError):
        c.set_launch(True)
    assert Y._lib.ygm_set_launch(c._h, 2) != 0
