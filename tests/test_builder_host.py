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
    with pytest.raises(Y.YgmError):
        c.set_q1(-g.Q1)                                # negative definite
