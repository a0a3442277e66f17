"""GPU cubical Whitney GYM (ygm_yee_*), the structured-grid kernel family of Sec. 4: the leapfrog with
the cubical curl and diagonal Q1, M2 against the oracle's GYM on the same periodic cubical complex
(oracle/yee3d.py, itself pinned to a textbook Yee loop and to the printed Whitney masses)."""
import numpy as np
import pytest
import scipy.sparse as sp

pytestmark = pytest.mark.gpu

from oracle.gym import GYM
from oracle.yee3d import PeriodicCubes
from oracle_runs import rel_l2

Y = pytest.importorskip("paper_2301_01753_gb300")

N, H = (6, 5, 4), (0.3, 0.25, 0.2)


def _oracle(q=None, m=None):
    g = PeriodicCubes(N, H)
    q = np.full(g.N1, 1.0 / g.dV) if q is None else q
    m = np.full(g.N2, g.dV) if m is None else m
    return g, GYM(g.C(), sp.diags(m), sp.diags(q))


@pytest.mark.parametrize("diag", [False, True])
def test_yee_follows_the_oracle_fp64(diag):
    rng = np.random.default_rng(1)
    g = PeriodicCubes(N, H)
    q = rng.uniform(0.5, 2.0, g.N1) / g.dV if diag else None
    m = rng.uniform(0.5, 2.0, g.N2) * g.dV if diag else None
    g, gym = _oracle(q, m)
    y = Y.Yee(N, H, q1=q, m2=m, precision=Y.YGM_FP64)
    assert y.N1 == g.N1 and y.N2 == g.N2
    e0 = rng.standard_normal(g.N1)
    b0 = g.C() @ rng.standard_normal(g.N1)
    tau = 0.4 * gym.tau_cfl()
    assert tau < y.tau_cfl
    y.set_state(e0, b0)
    y.step(10, tau)
    y.step(15, tau)
    e, b = y.get_state(synced=True)
    e_or, b_or, _ = gym.run(e0.copy(), gym.half_init(e0, b0, tau), tau, 25)
    assert rel_l2(e, e_or) < 1e-13
    assert rel_l2(b, gym.sync(e_or, b_or, tau)) < 1e-13
    _, bs = y.get_state(synced=False)                    # the read-out did not touch the state
    assert rel_l2(bs, b_or) < 1e-13
    y.close()


def test_yee_fp32_against_fp64():
    rng = np.random.default_rng(2)
    g, gym = _oracle()
    e0 = rng.standard_normal(g.N1)
    b0 = np.zeros(g.N2)
    out = []
    for p, dt in ((Y.YGM_FP64, np.float64), (Y.YGM_FP32, np.float32)):
        y = Y.Yee(N, H, precision=p)
        tau = 0.5 * y.tau_cfl
        y.set_state(e0.astype(dt), b0.astype(dt))
        y.step(200, tau)
        out.append(y.get_state(synced=True))
        y.close()
    assert rel_l2(out[1][0], out[0][0]) < 1e-5 and rel_l2(out[1][1], out[0][1]) < 1e-5


def test_yee_cfl_bound_is_safe_and_refused_beyond():
    y = Y.Yee(N, H)
    lam_exact = sum(4.0 / h ** 2 for h in H)              # lumped uniform grid: lambda_max(Q1 C^T M2 C)
    tau_exact = 2.0 / np.sqrt(lam_exact)
    assert 0.7 * tau_exact < y.tau_cfl <= tau_exact * (1 + 1e-12)
    y.set_state(np.ones(y.N1), np.zeros(y.N2))
    with pytest.raises(Y.YgmError) as ei:
        y.step(1, 1.01 * y.tau_cfl)
    assert ei.value.code == Y.YGM_ECFL
    y.close()
