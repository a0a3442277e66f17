"""GPU adjoint of the leapfrog (ygm_adjoint): the eps-gradient of a probe-region field energy,
by the transposed shear maps of Eq. shearMaps run newest step first on the device with
checkpointed recomputation, chained through the host SPAI derivative.

Checked against the FP64 CPU adjoint (oracle/adjoint.py, itself pinned to central differences),
against central differences of the GPU loss on seeded tets of a larger mesh, for independence of
the checkpoint interval, and through torch.autograd."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

import synth
from oracle import adjoint as AD
from oracle import spai as SP
from oracle.fem import FEM
from oracle.gym import GYM, DipoleSource
from oracle.mesh import KuhnMesh

Y = pytest.importorskip("paper_2301_01753_gb300")

SRC = dict(x=np.array([0.41, 0.52, 0.47]), d=np.array([0.3, 0.2, 1.0]), amp=1.0, omega=np.pi * np.sqrt(5.0))


def _gpu_source(tau, width=5.0):
    sigma = width * tau
    return [dict(SRC, t0=4 * sigma, sigma=sigma)]


def _oracle_problem(n, k, seed, steps):
    eps0 = synth.tet_eps(seed, n, 1.0, 4.0)
    make = lambda eps: FEM(KuhnMesh(n, k), eps=eps)
    f0 = make(eps0)
    region = np.all(f0.mesh.tet_vx.mean(axis=1) < 0.5, axis=1)
    M1 = f0.M1()
    Q, _ = SP.gym_q1(f0, M1)
    tau = 0.5 * GYM(f0.C(), f0.M2(), Q, M1).tau_cfl()
    src = [dict(SRC, width_steps=5.0)]

    def source(fem):
        J = DipoleSource(fem, src, tau)
        return [J((m + 0.5) * tau) for m in range(steps)]
    return make, eps0, region, source, tau


@pytest.mark.parametrize("k,steps", [(1, 40), (2, 30)])
def test_adjoint_matches_the_fp64_oracle(k, steps):
    make, eps0, region, source, tau = _oracle_problem(2, k, 5001 + 2 * (k - 1), steps)
    L_or, g_or = AD.loss_and_gradient_policy(make, eps0, region, source, tau, steps)
    c = Y.Context(2, k, eps=eps0, precision=Y.YGM_FP64)
    L, g = c.adjoint(steps, tau, _gpu_source(tau), region, checkpoint_every=7)
    assert abs(L - L_or) <= 1e-12 * abs(L_or)
    assert np.max(np.abs(g - g_or)) <= 1e-10 * np.max(np.abs(g_or))
    # the context is left at rest and steps normally afterwards
    e, b = c.get_state(synced=False)
    assert not np.any(e) and not np.any(b)
    c.close()


def test_checkpoint_interval_does_not_change_the_result():
    n, k, steps = 3, 2, 50
    eps = synth.tet_eps(5006, n, 1.0, 4.0)
    c = Y.Context(n, k, eps=eps, precision=Y.YGM_FP64)
    tau = 0.5 * c.tau_cfl
    region = np.zeros(6 * n ** 3, bool)
    region[:40] = True
    ref = c.adjoint(steps, tau, _gpu_source(tau), region, checkpoint_every=steps)
    for K in (1, 7, 16):
        L, g = c.adjoint(steps, tau, _gpu_source(tau), region, checkpoint_every=K)
        assert L == ref[0] and np.array_equal(g, ref[1]), K
    c.close()


def _subcube_region(n, seed, side=0.4):
    """Tets whose centroid lies in a side x side x side cube at a seeded corner of the unit cube."""
    m = KuhnMesh(n, 1)
    corner = synth.uniform(seed, 3) < 0.5
    lo = np.where(corner, 0.0, 1.0 - side)
    cen = m.tet_vx.mean(axis=1)
    return np.all((cen >= lo) & (cen < lo + side), axis=1)


def test_gradient_matches_central_differences_on_seeded_tets():
    """The differentiation workload at reduced size: N = 4, k = 2, eps ~ U[1,4), one dipole, 200
    steps, region a 0.4-side subcube at a seeded corner; central differences of the GPU loss
    (each a fresh operator set-up) on 20 seeded tets.  h = 1e-4 eps_t relative (reading: smaller
    steps drown in the rounding of the recomputed SPAI, larger ones in truncation)."""
    n, k, steps = 4, 2, 200
    eps0 = synth.tet_eps(5000, n, 1.0, 4.0)
    region = _subcube_region(n, 5001)
    assert region.any()
    c = Y.Context(n, k, eps=eps0, precision=Y.YGM_FP64)
    tau = 0.5 * c.tau_cfl
    L, g = c.adjoint(steps, tau, _gpu_source(tau, 20.0), region, checkpoint_every=50)
    c.close()
    tets = np.unique((synth.uniform(5004, 20) * len(eps0)).astype(int))
    for t in tets:
        h = 1e-4 * eps0[t]
        vals = []
        for sgn in (1.0, -1.0):
            e = eps0.copy()
            e[t] += sgn * h
            with Y.Context(n, k, eps=e, precision=Y.YGM_FP64) as cc:
                vals.append(cc.adjoint(steps, tau, _gpu_source(tau, 20.0), region, gradient=False)[0])
        fd = (vals[0] - vals[1]) / (2 * h)
        assert abs(g[t] - fd) <= 1e-6 * np.max(np.abs(g)), (t, g[t], fd)


def test_fp32_adjoint_against_fp64():
    n, k, steps = 4, 2, 200
    eps0 = synth.tet_eps(5000, n, 1.0, 4.0)
    region = _subcube_region(n, 5001)
    out = {}
    for p in (Y.YGM_FP64, Y.YGM_FP32):
        with Y.Context(n, k, eps=eps0, precision=p) as c:
            tau = 0.5 * c.tau_cfl
            out[p] = c.adjoint(steps, tau, _gpu_source(tau, 20.0), region, checkpoint_every=50)
    L64, g64 = out[Y.YGM_FP64]
    L32, g32 = out[Y.YGM_FP32]
    assert abs(L32 - L64) <= 1e-5 * abs(L64)
    assert np.linalg.norm(g32 - g64) <= 1e-4 * np.linalg.norm(g64)


def test_probe_energy_through_torch_autograd():
    torch = pytest.importorskip("torch")
    n, k, steps = 3, 1, 60
    eps0 = synth.tet_eps(5007, n, 1.0, 4.0)
    region = _subcube_region(n, 5001, side=0.5)
    with Y.Context(n, k, eps=eps0, precision=Y.YGM_FP64) as c:
        tau = 0.5 * c.tau_cfl
        L, g = c.adjoint(steps, tau, _gpu_source(tau), region)
    eps = torch.tensor(eps0, dtype=torch.float64, requires_grad=True)
    loss = Y.probe_energy(eps, n, k, steps, tau, _gpu_source(tau), region)
    (3.0 * loss).backward()
    assert abs(loss.item() - L) <= 1e-14 * abs(L)
    assert np.allclose(eps.grad.numpy(), 3.0 * g, rtol=0, atol=1e-14 * np.abs(g).max())
