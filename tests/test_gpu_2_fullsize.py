"""Full-size checks at the benchmark workload (N = 32, k = 2, eps ~ U[1,4) seed 2000, z-dipole,
dt = 0.5 tau_CFL): one step from a seeded random state compared with the oracle on sampled
outputs (the oracle evaluates the needed Q1 rows locally), and properties that hold at any size
over the whole 2000-step run."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

import synth
from oracle.fem import FEM
from oracle.gym import DipoleSource
from oracle.mesh import KuhnMesh
from oracle.spai import LocalQ1

Y = pytest.importorskip("paper_2301_01753_gb300")
N, K = 32, 2


@pytest.fixture(scope="module")
def model():
    eps = synth.tet_eps(2000, N, 1.0, 4.0)
    f = FEM(KuhnMesh(N, K), eps=eps)
    M1 = f.M1()
    C = f.C()
    M2 = f.M2()
    return dict(f=f, M1=M1, C=C, CT=C.T.tocsr(), M2=M2, eps=eps, x0=synth.source_positions(2001, 1)[0])


@pytest.fixture(scope="module")
def ctxs(model):
    """One context per precision, shared by the tests of this module (the N = 32 set-up is the
    expensive part)."""
    c = {p: Y.Context(N, K, eps=model["eps"], precision=p, energy_every=100) for p in (Y.YGM_FP64, Y.YGM_FP32)}
    yield c
    for v in c.values():
        v.close()




def test_one_step_all_outputs_fp64_and_fp32(model, ctxs):
    """e0 is supported on four DoFs (classes and places chosen to include a boundary-adjacent DoF
    and the source tet), b0 = C a0 is dense.  By symmetry of Q1, x = Q1 e0 needs only the four Q1
    rows of the support, which the oracle evaluates locally; every element of b_{1/2} and e_1 is
    then compared (the first step includes the initial half step and the source)."""
    f, C, CT, M2 = model["f"], model["C"], model["CT"], model["M2"]
    rng = np.random.default_rng(5)
    dt = 0.5 * ctxs[Y.YGM_FP64].tau_cfl
    J = DipoleSource(f, [dict(x=model["x0"], d=np.array([0.0, 0.0, 1.0]), amp=1.0, omega=np.pi * np.sqrt(5.0),
                              width_steps=20.0)], dt)
    src_dofs = J.items[0]["dofs"]
    support = sorted({0, int(f.mesh.N1 // 2), int(rng.integers(f.mesh.N1)), int(src_dofs[len(src_dofs) // 2])})
    e0 = np.zeros(f.mesh.N1)
    e0[support] = rng.standard_normal(len(support))
    b0 = C @ rng.standard_normal(f.mesh.N1)
    L = LocalQ1(f, model["M1"])
    x = np.zeros(f.mesh.N1)
    for c in support:
        for r, v in L.row(c).items():
            x[r] += v * e0[c]
    b_half = b0 - 0.5 * dt * (C @ x)                 # initial half step + first b update
    e1 = e0 + dt * (CT @ (M2 @ b_half)) - dt * J(0.5 * dt)
    src = Y.pulse_source(model["x0"], [0.0, 0.0, 1.0], np.pi * np.sqrt(5.0), dt)
    for prec, tol in ((Y.YGM_FP64, 1e-12), (Y.YGM_FP32, 2e-6)):
        c = ctxs[prec]
        dtp = np.float64 if prec == Y.YGM_FP64 else np.float32
        c.set_state(e0.astype(dtp), b0.astype(dtp))
        c.step(1, dt, [src])
        eg, bg = c.get_state(synced=False)
        assert np.max(np.abs(eg - e1)) <= tol * np.abs(e1).max()
        assert np.max(np.abs(bg - b_half)) <= tol * np.abs(b_half).max()
        # rows far from the support must stay exactly untouched by Q1 (no stray reads)
        if prec == Y.YGM_FP64:
                assert np.array_equal(bg[np.abs(C @ x) == 0], b0[np.abs(C @ x) == 0])


def test_full_run_invariants(model, ctxs):
    """2000 steps of the workload: W_n constant once the pulse is over (FP64), and the FP32 run
    within 1e-5 relative L2 of the FP64 run (measured 6.1e-6 for e and 9.5e-6 for b, the same to
    the last digit on every GB300 run: the kernels have a fixed summation order)."""
    f = model["f"]
    dt = 0.5 * ctxs[Y.YGM_FP64].tau_cfl
    src = [Y.pulse_source(model["x0"], [0.0, 0.0, 1.0], np.pi * np.sqrt(5.0), dt)]
    runs = {}
    for prec in (Y.YGM_FP64, Y.YGM_FP32):
        c = ctxs[prec]
        dtp = np.float64 if prec == Y.YGM_FP64 else np.float32
        c.set_state(np.zeros(c.N1, dtp), np.zeros(c.N2, dtp))
        c.step(2000, dt, src)
        e, b = c.get_state(synced=True)
        runs[prec] = (e.astype(np.float64), b.astype(np.float64), c.energy_history())
    e64, b64, W64 = runs[Y.YGM_FP64]
    e32, b32, W32 = runs[Y.YGM_FP32]
    assert np.linalg.norm(e64) > 0 and len(W64) == 20
    # after ~10 pulse widths the source amplitude is below 1e-40: W must be flat
    assert np.max(np.abs(W64[4:] - W64[4])) / W64[4] < 1e-11
    assert np.max(np.abs(W32[4:] - W32[4])) / W32[4] < 1e-5
    assert np.linalg.norm(e32 - e64) / np.linalg.norm(e64) < 1e-5
    assert np.linalg.norm(b32 - b64) / np.linalg.norm(b64) < 1e-5
