"""GPU runs with the operator-probed Q1 of ygm_spai_op (Sec. 5.1).

The SPAI-OP set-up is host FP64 work; what the GPU path must show is that the refreshed device
operators step exactly the Q1 the set-up produced, and that probing improves the probed cavity
mode's time-domain frequency as Sec. 7.6 reports for the periodic grid."""
import numpy as np
import pytest
import scipy.linalg as sl
import scipy.sparse as sp

pytestmark = pytest.mark.gpu

from oracle.gym import GYM
from oracle.cubical2d import zero_crossing_frequency
from oracle_runs import oracle_model, rel_l2, run_oracle

Y = pytest.importorskip("paper_2301_01753_gb300")


def _modes(f, M1, count):
    P2 = (f.C().T @ f.M2() @ f.C()).tocsr()
    w, V = sl.eigh(P2.toarray(), M1.toarray())
    nz = np.where(w > 1e-8 * w[-1])[0][:count]
    return P2, w[nz], V[:, nz]


@pytest.mark.parametrize("precision,tol", [(0, 1e-12), (1, 5e-5)])
def test_spai_op_q1_steps_like_the_oracle(precision, tol):
    f, g, eps, _ = oracle_model(4, 1, eps_seed=31)
    M1 = f.M1()
    P2, w, V = _modes(f, M1, 3)
    c = Y.Context(4, 1, eps=eps, precision=precision)
    it, rr = c.spai_op(V, 1e3, tol=1e-12)
    assert rr <= 1e-12
    rp, ci, va = c.export_q1()
    Q = sp.csr_matrix((va, ci, rp), shape=(c.N1, c.N1))
    go = GYM(f.C(), f.M2(), Q, M1)
    assert abs(c.tau_cfl / go.tau_cfl() - 1) < 1e-9
    tau = 0.5 * c.tau_cfl
    e0 = M1 @ V[:, 0]
    b0 = np.zeros(f.mesh.N2)
    e_or, bst_or, bs_or, _ = run_oracle(f, go, e0, b0, tau, 400)
    dt = np.float64 if precision == 0 else np.float32
    c.set_state(e0.astype(dt), b0.astype(dt))
    c.step(400, tau)
    e, b = c.get_state(synced=True)
    assert rel_l2(e, e_or) < tol and rel_l2(b, bs_or) < tol


def test_probed_mode_frequency_on_the_gpu():
    """The lowest cavity mode propagated on the GPU (FP64, N=4, k=1): its zero-crossing frequency
    moves from the column SPAI's to within 1e-3 of the exact FEEC value once it is probed."""
    f, g, eps, _ = oracle_model(4, 1)
    M1 = f.M1()
    P2, w, V = _modes(f, M1, 1)
    omega = np.sqrt(w[0])
    v = V[:, 0]
    e0 = M1 @ v

    def freq(ctx):
        tau = 0.3 * ctx.tau_cfl
        periods = 40
        nsteps = int(periods * 2 * np.pi / omega / tau)
        ctx.set_state(e0, np.zeros(f.mesh.N2))
        proj = [e0 @ e0]
        chunk = 2
        for _ in range(nsteps // chunk):
            ctx.step(chunk, tau)
            e, _ = ctx.get_state(synced=False)
            proj.append(e @ e0)
        return zero_crossing_frequency(np.array(proj), chunk * tau)

    c = Y.Context(4, 1, precision=Y.YGM_FP64)
    w_spai = freq(c)
    c.spai_op(v.reshape(-1, 1), 5e5, tol=1e-12)
    w_op = freq(c)
    assert abs(w_op - omega) / omega < 1e-3
    assert abs(w_op - omega) < 0.1 * abs(w_spai - omega)
