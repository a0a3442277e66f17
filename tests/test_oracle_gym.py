"""Pins of the oracle's time stepping: Theorem symplecticity, Eq. eigenvaluePairs, Prop. stability,
the exactly conserved discrete energy, the tau^2 scaling of the modified Hamiltonian's
oscillation (Sec. 7.5), Gauss' law, the (a, e) / (b, e) equivalence and the source work identity."""
import numpy as np
import pytest
import scipy.sparse as sp

import synth
from oracle import spai as SP
from oracle.fem import FEM
from oracle import gym as G
from oracle.gym import GYM, DipoleSource
from oracle.mesh import KuhnMesh


def _setup(n, k, seed=21, eps_range=(1, 4)):
    f = FEM(KuhnMesh(n, k), eps=synth.tet_eps(seed, n, *eps_range))
    M1 = f.M1()
    Q, _ = SP.gym_q1(f, M1)
    return f, GYM(f.C(), f.M2(), Q, M1)


@pytest.mark.parametrize("n,k", [(2, 1), (2, 2)])
def test_strang_map_is_symplectic(n, k):
    f, g = _setup(n, k)
    tau = 0.5 * g.tau_cfl()
    J = g.strang_jacobian(tau)
    N = f.mesh.N1
    Om = np.block([[np.zeros((N, N)), np.eye(N)], [-np.eye(N), np.zeros((N, N))]])
    assert abs(J.T @ Om @ J - Om).max() < 1e-12 * max(1.0, abs(J).max() ** 2)


def test_symplectic_even_for_indefinite_symmetric_q1():
    f, g = _setup(2, 1)
    Q = g.Q1.toarray()
    Q = Q - 1.5 * np.linalg.eigvalsh(Q)[-1] * np.eye(Q.shape[0]) * 0.5
    g2 = GYM(f.C(), f.M2(), sp.csr_matrix(Q))
    J = g2.strang_jacobian(0.01)
    N = f.mesh.N1
    Om = np.block([[np.zeros((N, N)), np.eye(N)], [-np.eye(N), np.zeros((N, N))]])
    assert abs(J.T @ Om @ J - Om).max() < 1e-11 * abs(J).max() ** 2


def test_eigenvalues_of_one_step_map_follow_the_2x2_blocks():
    """eig(J) = 1 - z/2 +- sqrt(z(z-4))/2 with z = tau^2 w^2, w^2 in eig(Q1 P2)."""
    f, g = _setup(2, 1)
    tau = 0.7 * g.tau_cfl()
    lam = np.linalg.eigvals(g.strang_jacobian(tau))
    w2 = np.linalg.eigvals(g.Q1.toarray() @ g.P2.toarray()).real
    z = tau ** 2 * np.clip(w2, 0, None)
    pred = np.concatenate([1 - z / 2 + 0.5 * np.sqrt(z * (z - 4) + 0j), 1 - z / 2 - 0.5 * np.sqrt(z * (z - 4) + 0j)])
    key = lambda x: (np.round(x.real, 8), np.round(abs(x.imag), 8))
    assert np.allclose(sorted(lam, key=key), sorted(pred, key=key), atol=1e-8)


@pytest.mark.parametrize("k", [1, 2])
def test_cfl_bound_separates_stable_and_unstable(k):
    f, g = _setup(2, k)
    tc = g.tau_cfl()
    lam_s = np.linalg.eigvals(g.strang_jacobian(0.9 * tc))
    # gradient fields (omega = 0) form Jordan blocks at lambda = 1 whose computed eigenvalues
    # carry sqrt(machine epsilon) noise; every other eigenvalue sits on the unit circle
    osc = np.abs(lam_s - 1) > 1e-6
    assert abs(np.abs(lam_s[osc]) - 1).max() < 1e-10
    assert abs(np.abs(lam_s) - 1).max() < 1e-7
    lam_u = np.linalg.eigvals(g.strang_jacobian(1.1 * tc))
    big = lam_u[np.abs(lam_u) > 1 + 1e-6]
    assert len(big) > 0 and np.all(abs(big.imag) < 1e-8)          # leave along the real axis
    for x in big:                                                   # reciprocal partners
        assert np.min(np.abs(lam_u - 1 / x)) < 1e-6


def test_time_domain_growth_beyond_cfl_and_for_indefinite_q1():
    f, g = _setup(2, 1)
    tc = g.tau_cfl()
    rng = np.random.default_rng(0)
    e0 = rng.standard_normal(f.mesh.N1)
    e, b, _ = g.run(e0, g.half_init(e0, np.zeros(f.mesh.N2), 1.1 * tc), 1.1 * tc, 400)
    assert np.linalg.norm(e) > 1e3 * np.linalg.norm(e0)
    e, b, _ = g.run(e0, g.half_init(e0, np.zeros(f.mesh.N2), 0.9 * tc), 0.9 * tc, 400)
    assert np.linalg.norm(e) < 1e2 * np.linalg.norm(e0)
    Q = g.Q1.toarray()
    wp, Vp = np.linalg.eigh(g.P2.toarray())
    u = Vp[:, -1]                                                   # a curl-carrying direction
    Q_ind = Q - 2.0 * (u @ Q @ u) * np.outer(u, u)                 # u^T Q_ind u < 0
    g2 = GYM(f.C(), f.M2(), sp.csr_matrix(Q_ind))
    w2 = np.linalg.eigvals(Q_ind @ g.P2.toarray()).real
    assert w2.min() < 0
    tau = 0.05 * tc
    e, b, _ = g2.run(e0, g2.half_init(e0, np.zeros(f.mesh.N2), tau), tau, 4000)
    assert np.linalg.norm(e) > 1e3 * np.linalg.norm(e0)


def test_discrete_energy_conserved_config1_like():
    """N=4, k=1, TE(1,1,0) mode E = z sin(pi x) sin(pi y), dt = 0.5 tau_CFL, 1000 steps."""
    f = FEM(KuhnMesh(4, 1))
    M1 = f.M1()
    Q, _ = SP.gym_q1(f, M1)
    g = GYM(f.C(), f.M2(), Q, M1)
    E0 = lambda x: np.stack([0 * x[:, 0], 0 * x[:, 0], np.sin(np.pi * x[:, 0]) * np.sin(np.pi * x[:, 1])], axis=1)
    e0 = M1 @ f.edge_interpolant(E0)
    tau = 0.5 * g.tau_cfl()
    b = g.half_init(e0, np.zeros(f.mesh.N2), tau)
    W0 = g.W(e0, b, tau)
    e, b, W = g.run(e0, b, tau, 1000, energy_every=1)
    drift = np.max(np.abs(np.array(W) - W0)) / W0
    assert drift < 1e-13
    # the paper's H~ oscillates boundedly (Sec. 7.5)
    H = [g.H_tilde(e0, np.zeros(f.mesh.N2))]
    e2, b2 = e0.copy(), g.half_init(e0, np.zeros(f.mesh.N2), tau)
    for n in range(200):
        e2, b2, _, _ = g.step(e2, b2, tau)
        H.append(g.H_tilde(e2, g.sync(e2, b2, tau)))
    H = np.array(H)
    assert np.max(np.abs(H - H[0])) / H[0] < 0.05


@pytest.mark.parametrize("n,k", [(3, 1), (2, 2)])
def test_gauss_law_and_divergence_free_b(n, k):
    f, g = _setup(n, k)
    G, D = f.G(), f.D()
    rng = np.random.default_rng(5)
    e0 = rng.standard_normal(f.mesh.N1)
    tau = 0.5 * g.tau_cfl()
    b = g.half_init(e0, np.zeros(f.mesh.N2), tau)
    e, b, _ = g.run(e0, b, tau, 300)
    assert abs(G.T @ e - G.T @ e0).max() < 1e-11 * abs(e0).max()
    assert abs(D @ b).max() < 1e-11 * abs(b).max()


def test_leapfrog_equals_strang_in_a_e_variables():
    """(b, e) leapfrog with half steps equals Phi_tau (Eq. strangSplit) on (a, e) with b = C a."""
    f, g = _setup(2, 2)
    rng = np.random.default_rng(8)
    a0 = rng.standard_normal(f.mesh.N1)
    e0 = rng.standard_normal(f.mesh.N1)
    tau = 0.4 * g.tau_cfl()
    a, e = a0.copy(), e0.copy()
    for _ in range(25):
        a, e = g.strang(a, e, tau)
    b = g.half_init(e0, g.C @ a0, tau)
    e2, b2, _ = g.run(e0.copy(), b, tau, 25)
    assert np.allclose(e2, e, rtol=1e-12, atol=1e-12 * abs(e).max())
    assert np.allclose(g.sync(e2, b2, tau), g.C @ a, rtol=1e-11, atol=1e-11 * abs(g.C @ a).max())


def test_source_work_identity_and_linearity():
    """W_{n+1} - W_n = -tau (e_n + e_{n+1})^T Q1 j_{n+1/2} / 2, and the response is linear in s."""
    f, g = _setup(3, 2, seed=31)
    tau = 0.5 * g.tau_cfl()
    src = [dict(x=np.array([0.41, 0.52, 0.47]), d=np.array([0.0, 0.0, 1.0]), amp=1.0,
                omega=np.pi * np.sqrt(5.0), width_steps=5.0)]
    J = DipoleSource(f, src, tau)
    e = np.zeros(f.mesh.N1)
    b = np.zeros(f.mesh.N2)
    res = []
    for n in range(60):
        j = J((n + 0.5) * tau)
        W0 = g.W(e, b, tau)
        e1, b1, _, _ = g.step(e, b, tau, j)
        W1 = g.W(e1, b1, tau)
        work = -tau * 0.5 * (e + e1) @ (g.Q1 @ j)
        res.append(abs(W1 - W0 - work) / max(abs(W1), 1e-300))
        e, b = e1, b1
    assert np.linalg.norm(e) > 0 and max(res) < 1e-10
    J2 = DipoleSource(f, [dict(src[0], amp=2.0)], tau)
    e2, b2, _ = g.run(np.zeros(f.mesh.N1), np.zeros(f.mesh.N2), tau, 60, source=J2)
    assert np.allclose(e2, 2 * e, rtol=1e-12, atol=1e-14)


def test_modified_hamiltonian_oscillation_scales_with_dt_squared():
    """Sec. 7.5: H~ = e^T Q1 e / 2 + b^T M2 b / 2 oscillates without secular drift, with an amplitude
    of order tau^2 omega_max^2.  Halving tau must divide the amplitude by ~4, and the deviation over
    the second half of the run must not exceed the first half's."""
    f = FEM(KuhnMesh(4, 1))
    M1 = f.M1()
    Q, _ = SP.gym_q1(f, M1)
    g = GYM(f.C(), f.M2(), Q, M1)
    E0 = lambda x: np.stack([0 * x[:, 0], 0 * x[:, 0], np.sin(np.pi * x[:, 0]) * np.sin(np.pi * x[:, 1])], axis=1)
    e0 = M1 @ f.edge_interpolant(E0)
    T = 6 * 2 * np.pi / (np.pi * np.sqrt(2.0))          # six periods of the (1,1,0) mode

    def deviation(tau):
        n = int(round(T / tau))
        e, b = e0.copy(), g.half_init(e0, np.zeros(f.mesh.N2), tau)
        H0 = g.H_tilde(e0, np.zeros(f.mesh.N2))
        dev = []
        for _ in range(n):
            e, b, _, _ = g.step(e, b, tau)
            dev.append(abs(g.H_tilde(e, g.sync(e, b, tau)) - H0) / H0)
        dev = np.array(dev)
        return dev.max(), dev[: n // 2].max(), dev[n // 2:].max()

    tau = 0.2 * g.tau_cfl()
    a1, h1, h2 = deviation(tau)
    a2, _, _ = deviation(tau / 2)
    assert 3.4 < a1 / a2 < 4.6
    assert h2 <= 1.05 * h1


# ---------------------------------------------------------------- composed (higher-order) splittings
def _exact_semidiscrete(g, e0, b0, T):
    """(e, b)(T) of the semi-discrete system b' = -C Q1 e, e' = C^T M2 b (Eq. preYeeFEECEqns),
    exactly, by the matrix exponential (tiny meshes)."""
    import scipy.linalg as sla
    N1, N2 = g.Q1.shape[0], g.C.shape[0]
    A = np.zeros((N1 + N2, N1 + N2))
    A[N1:, :N1] = -(g.C @ g.Q1).toarray()
    A[:N1, N1:] = (g.CT @ g.M2).toarray()
    y = sla.expm(A * T) @ np.concatenate([e0, b0])
    return y[:N1], y[N1:]


def test_yoshida_weights_are_the_fourth_order_triple_jump():
    w = G.yoshida4()
    assert abs(sum(w) - 1) < 1e-15                      # consistency
    assert abs(sum(x ** 3 for x in w)) < 1e-14           # the third-order condition of a symmetric composition
    assert w[0] == w[2] and w[1] < 0


@pytest.mark.parametrize("weights,order", [((1.0,), 2), (None, 4)])
def test_composed_splitting_converges_at_its_order(weights, order):
    """Against the exact semi-discrete solution: halving tau divides the error by 2^order."""
    weights = weights or G.yoshida4()
    f = FEM(KuhnMesh(2, 1), eps=synth.tet_eps(61, 2, 1.0, 4.0))
    M1 = f.M1()
    Q, _ = SP.gym_q1(f, M1)
    g = G.GYM(f.C(), f.M2(), Q, M1)
    rng = np.random.default_rng(5)
    e0 = rng.standard_normal(f.mesh.N1)
    b0 = f.C() @ rng.standard_normal(f.mesh.N1)
    T = 0.6
    ee, be = _exact_semidiscrete(g, e0, b0, T)
    errs = []
    for m in (80, 160, 320):
        e, b = g.run_composed(e0.copy(), b0.copy(), T / m, m, weights)
        errs.append(np.linalg.norm(np.concatenate([e - ee, b - be])) / np.linalg.norm(np.concatenate([ee, be])))
    rates = [np.log2(errs[i] / errs[i + 1]) for i in range(2)]
    assert all(abs(r - order) < 0.15 for r in rates), (errs, rates)
    if order == 4:
        assert errs[-1] < 1e-7


def test_composed_step_is_symplectic_and_time_symmetric():
    f = FEM(KuhnMesh(2, 1))
    M1 = f.M1()
    Q, _ = SP.gym_q1(f, M1)
    g = G.GYM(f.C(), f.M2(), Q, M1)
    tau = 0.3 * g.tau_cfl()
    J = g.composed_jacobian(tau, G.yoshida4())
    n = Q.shape[0]
    Om = np.block([[np.zeros((n, n)), np.eye(n)], [-np.eye(n), np.zeros((n, n))]])
    assert np.abs(J.T @ Om @ J - Om).max() < 1e-10 * np.abs(J).max() ** 2
    Jb = g.composed_jacobian(-tau, G.yoshida4())
    assert np.abs(Jb @ J - np.eye(2 * n)).max() < 1e-10 * np.abs(J).max() ** 2


def _exact_driven(g, j, s, T):
    """(e, b)(T) of the driven semi-discrete system e' = C^T M2 b - s(t) j, b' = -C Q1 e from rest
    (Eq. preYeeFEECEqns with the current term of Eq. allEOM), by SciPy's DOP853 at tight tolerance."""
    from scipy.integrate import solve_ivp
    N1 = g.Q1.shape[0]
    CQ = (g.C @ g.Q1).toarray()
    CTM = (g.CT @ g.M2).toarray()

    def rhs(t, y):
        return np.concatenate([CTM @ y[N1:] - s(t) * j, -CQ @ y[:N1]])

    sol = solve_ivp(rhs, (0.0, T), np.zeros(N1 + g.C.shape[0]), method="DOP853", rtol=1e-12, atol=1e-14)
    return sol.y[:N1, -1], sol.y[N1:, -1]


def test_driven_leapfrog_converges_to_the_exact_driven_solution():
    """The dipole current enters the e update at the half step t_{n+1/2}: from rest, the leapfrog
    converges at order 2 to the exact driven solution.  Sampling the current at t_n instead (a
    half-step shift planted here in the oracle) drops the rate to 1, so the pin sees the time
    placement, the sign and the weight of the source term."""
    f = FEM(KuhnMesh(2, 1), eps=synth.tet_eps(62, 2, 1.0, 4.0))
    M1 = f.M1()
    Q, _ = SP.gym_q1(f, M1)
    g = G.GYM(f.C(), f.M2(), Q, M1)
    T = 1.0
    src = DipoleSource(f, [dict(x=np.array([0.37, 0.58, 0.44]), d=np.array([0.2, 0.1, 1.0]), omega=np.pi * np.sqrt(5.0),
                               width_steps=5.0)], T / 80)      # sigma = T / 16, t0 = T / 4: over by T
    j = src(0.3)
    a = src.items[0]
    s = lambda t: G.pulse(t, a["amp"], a["omega"], a["t0"], a["sigma"])
    assert np.allclose(src(0.3), s(0.3) * (j / s(0.3)))
    jw = j / s(0.3)
    ee, be = _exact_driven(g, jw, s, T)
    assert np.linalg.norm(ee) > 1e-3
    scale = np.linalg.norm(np.concatenate([ee, be]))

    def err(m, shift):
        tau = T / m
        z1, z2 = np.zeros(f.mesh.N1), np.zeros(f.C().shape[0])
        e, b, _ = g.run(z1, g.half_init(z1, z2, tau), tau, m, source=lambda t: src(t - shift * tau))
        b = g.sync(e, b, tau)
        return np.linalg.norm(np.concatenate([e - ee, b - be])) / scale

    errs = [err(m, 0.0) for m in (80, 160, 320)]
    rates = [np.log2(errs[i] / errs[i + 1]) for i in range(2)]
    assert all(abs(r - 2) < 0.15 for r in rates), (errs, rates)
    assert errs[-1] < 1e-3
    shifted = [err(m, 0.5) for m in (160, 320)]
    r_shift = np.log2(shifted[0] / shifted[1])
    assert abs(r_shift - 1) < 0.2 and shifted[1] > 10 * errs[-1], (shifted, r_shift)
