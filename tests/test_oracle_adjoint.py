"""Pins of the adjoint oracle (oracle/adjoint.py): the eps-gradient of a probe-region field energy
through the leapfrog, M1^R and the column SPAI, against central finite differences of the whole
pipeline; the reverse sweep alone against a directional derivative in Q1."""
import numpy as np
import pytest

import synth
from oracle import adjoint as AD
from oracle import spai as SP
from oracle.fem import FEM
from oracle.gym import GYM, DipoleSource
from oracle.mesh import KuhnMesh

N, K, STEPS = 2, 1, 40


def _problem():
    eps0 = synth.tet_eps(5001, N, 1.0, 4.0)
    make = lambda eps: FEM(KuhnMesh(N, K), eps=eps)
    f0 = make(eps0)
    region = np.all(f0.mesh.tet_vx.mean(axis=1) < 0.5, axis=1)        # tets of the corner cube
    M1 = f0.M1()
    Q, _ = SP.gym_q1(f0, M1)
    tau = 0.5 * GYM(f0.C(), f0.M2(), Q, M1).tau_cfl()                  # fixed, not a function of eps
    src = [dict(x=np.array([0.41, 0.52, 0.47]), d=np.array([0.3, 0.2, 1.0]), amp=1.0,
                omega=np.pi * np.sqrt(5.0), width_steps=5.0)]

    def source(fem):
        J = DipoleSource(fem, src, tau)
        return [J((m + 0.5) * tau) for m in range(STEPS)]
    return make, eps0, region, source, tau


def test_gradient_matches_central_differences_on_every_tet():
    make, eps0, region, source, tau = _problem()
    L, grad = AD.loss_and_gradient(make, eps0, region, source, tau, STEPS)
    assert L > 0 and region.any() and (~region).any()
    for t in range(len(eps0)):
        h = 1e-5 * eps0[t]
        ep, em = eps0.copy(), eps0.copy()
        ep[t] += h
        em[t] -= h
        fd = (AD.loss_and_gradient(make, ep, region, source, tau, STEPS)[0]
              - AD.loss_and_gradient(make, em, region, source, tau, STEPS)[0]) / (2 * h)
        assert abs(grad[t] - fd) <= 1e-7 * np.max(np.abs(grad)), (t, grad[t], fd)


def test_reverse_sweep_is_the_transpose_of_the_step():
    """<dL/dQ1, dQ> equals the directional derivative of L along a symmetric dQ on the pattern,
    with eps (hence M1^R and everything else) held fixed."""
    make, eps0, region, source, tau = _problem()
    fem = make(eps0)
    S = SP.pattern("sm1", fem.M1(), fem.dof1)
    Q = AD.q1_of(fem, S)
    C, M2 = fem.C().toarray(), fem.M2().toarray()
    MR1, MR2 = AD.region_mass(fem, region)
    J = source(fem)
    L, es, xs, bs = AD.forward(C, M2, Q, MR1, MR2, J, tau, STEPS)
    Qbar, _ = AD.reverse(C, M2, Q, MR1, MR2, tau, es, xs, bs)
    rng = np.random.default_rng(7)
    D = rng.standard_normal(Q.shape) * (S.toarray() != 0)
    D = 0.5 * (D + D.T)
    h = 1e-6 * np.abs(Q).max()
    Lp = AD.forward(C, M2, Q + h * D, MR1, MR2, J, tau, STEPS)[0]
    Lm = AD.forward(C, M2, Q - h * D, MR1, MR2, J, tau, STEPS)[0]
    assert abs(np.sum(Qbar * D) - (Lp - Lm) / (2 * h)) <= 1e-7 * abs(np.sum(Qbar * D))


def test_spai_term_is_needed_outside_the_region():
    """Outside R, eps acts only through Q1: the SPAI derivative carries the whole gradient there
    (a gradient built from M1^R alone would be zero on those tets)."""
    make, eps0, region, source, tau = _problem()
    _, grad = AD.loss_and_gradient(make, eps0, region, source, tau, STEPS)
    assert np.max(np.abs(grad[~region])) > 1e-2 * np.max(np.abs(grad))


def test_order2_gradient_through_the_orthonormal_basis():
    """k = 2: Q1 = T Q' T with T = blockdiag (M1[g,g])^(-1/2) depending on eps as well (reading R2);
    the chained gradient against central differences (h = 1e-4 relative: smaller steps drown in the
    rounding of the recomputed SPAI, larger ones in truncation)."""
    n, k, steps = 2, 2, 30
    eps0 = synth.tet_eps(5003, n, 1.0, 4.0)
    make = lambda eps: FEM(KuhnMesh(n, k), eps=eps)
    f0 = make(eps0)
    region = np.all(f0.mesh.tet_vx.mean(axis=1) < 0.5, axis=1)
    M1 = f0.M1()
    Q, _ = SP.gym_q1(f0, M1)
    tau = 0.5 * GYM(f0.C(), f0.M2(), Q, M1).tau_cfl()
    src = [dict(x=np.array([0.41, 0.52, 0.47]), d=np.array([0.3, 0.2, 1.0]), amp=1.0,
                omega=np.pi * np.sqrt(5.0), width_steps=5.0)]

    def source(fem):
        J = DipoleSource(fem, src, tau)
        return [J((m + 0.5) * tau) for m in range(steps)]
    L, grad = AD.loss_and_gradient_policy(make, eps0, region, source, tau, steps)
    assert np.allclose(AD.q1_ortho_of(f0, SP.pattern("sm1sq", M1, f0.dof1)), Q.toarray(), rtol=0, atol=1e-12 * abs(Q).max())
    for t in (0, 3, 7, 20, 40, 47):
        h = 1e-4 * eps0[t]
        ep, em = eps0.copy(), eps0.copy()
        ep[t] += h
        em[t] -= h
        fd = (AD.loss_and_gradient_policy(make, ep, region, source, tau, steps)[0]
              - AD.loss_and_gradient_policy(make, em, region, source, tau, steps)[0]) / (2 * h)
        assert abs(grad[t] - fd) <= 1e-6 * np.max(np.abs(grad)), (t, grad[t], fd)
