"""GPU (sm_103a) parity of the C-ABI leapfrog against the FP64 oracle.

Tolerances (relative L2 of e and b): FP64 1e-12 (same operators and operation order up to
summation order); FP32 1e-5 after the run (float state and Q1 with compensated Q1 sums and a hi/lo
step size: rounding errors of about 6e-8 per operation, accumulated over a few hundred
norm-preserving steps; measured 1.3e-6 / 2.2e-6 on the dipole case)."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

import synth
from oracle.gym import DipoleSource
from oracle_runs import oracle_model, run_oracle, rel_l2, te110

Y = pytest.importorskip("paper_2301_01753_gb300")

FP64_TOL = 1e-12
FP32_TOL = 1e-5


def _dipole(tau, x=(0.41, 0.52, 0.47), d=(0.0, 0.0, 1.0), width=20.0):
    sigma = width * tau
    return dict(x=np.array(x), d=np.array(d), amp=1.0, omega=np.pi * np.sqrt(5.0), width_steps=width,
                t0=4 * sigma, sigma=sigma)


def _gpu_run(n, k, eps, e0, b0, tau, nsteps, precision, sources=(), energy_every=0, pattern=0):
    c = Y.Context(n, k, eps=eps, precision=precision, energy_every=energy_every, q1_pattern=pattern)
    dt = np.float64 if precision == Y.YGM_FP64 else np.float32
    c.set_state(np.ascontiguousarray(e0, dt), np.ascontiguousarray(b0, dt))
    c.step(nsteps, tau, [dict(s) for s in sources])
    e, b = c.get_state(synced=True)
    _, bs = c.get_state(synced=False)
    W = c.energy_history() if energy_every else None
    return c, e, b, bs, W


def test_config1_te110_fp64_1000_steps():
    """N=4, k=1, eps=mu=1, TE(1,1,0) mode, dt = 0.5 tau_CFL, 1000 steps, FP64."""
    f, g, eps, _ = oracle_model(4, 1)
    tau = 0.5 * g.tau_cfl()
    e0 = f.M1() @ f.edge_interpolant(te110)
    b0 = np.zeros(f.mesh.N2)
    e_or, bst_or, bs_or, W_or = run_oracle(f, g, e0, b0, tau, 1000, energy_every=10)
    c = Y.Context(4, 1, precision=Y.YGM_FP64, energy_every=10)
    assert abs(c.tau_cfl / g.tau_cfl() - 1) < 1e-9
    c.project_E(lambda x: te110(x)[0])
    e_gpu0, _ = c.get_state()
    assert rel_l2(e_gpu0, e0) < 1e-13
    c.step(1000, tau)
    e, b = c.get_state(synced=True)
    assert rel_l2(e, e_or) < FP64_TOL
    assert rel_l2(b, bs_or) < FP64_TOL
    W = c.energy_history()
    assert len(W) == 100
    assert np.max(np.abs(W - W_or)) / W_or[0] < 1e-12
    assert np.max(np.abs(W - W[0])) / W[0] < 1e-12        # exact invariant up to round-off
    assert c.time()[0] == 1000


@pytest.mark.parametrize("precision,tol", [(0, FP64_TOL), (1, FP32_TOL)])
def test_k2_random_eps_dipole(precision, tol):
    n, k, steps = 4, 2, 300
    f, g, eps, _ = oracle_model(n, k, eps_seed=2000)
    tau = 0.5 * g.tau_cfl()
    src = [_dipole(tau)]
    z1, z2 = np.zeros(f.mesh.N1), np.zeros(f.mesh.N2)
    e_or, bst_or, bs_or, _ = run_oracle(f, g, z1, z2, tau, steps, sources=src)
    c, e, b, bs, _ = _gpu_run(n, k, eps, z1, z2, tau, steps, precision, sources=src)
    assert np.linalg.norm(e_or) > 0
    assert rel_l2(e, e_or) < tol
    assert rel_l2(b, bs_or) < tol
    assert rel_l2(bs, bst_or) < tol


# Full pipeline (host set-up + kernels).  The builder's FP64 SPAI agrees with the oracle's to
# ~1e-15 (k=1), ~1e-13 (k=2), ~2e-12 (k=3: the normal equations square the column problem's
# condition number); over 120 steps that perturbation grows by < 25x, hence 5e-11 at k=3.
PIPE_TOL = {1: FP64_TOL, 2: FP64_TOL, 3: 5e-11}


@pytest.mark.parametrize("n,k", [(2, 3), (3, 1), (3, 2)])
def test_random_state_fp64(n, k):
    f, g, eps, _ = oracle_model(n, k, eps_seed=77)
    tau = 0.45 * g.tau_cfl()
    rng = np.random.default_rng(n * 10 + k)
    e0 = rng.standard_normal(f.mesh.N1)
    b0 = f.C() @ rng.standard_normal(f.mesh.N1)          # b in the range of C (div-free)
    e_or, bst_or, bs_or, _ = run_oracle(f, g, e0, b0, tau, 120)
    _, e, b, bs, _ = _gpu_run(n, k, eps, e0, b0, tau, 120, Y.YGM_FP64)
    assert rel_l2(e, e_or) < PIPE_TOL[k]
    assert rel_l2(b, bs_or) < PIPE_TOL[k]


@pytest.mark.parametrize("n,k", [(2, 3), (3, 3), (3, 2), (4, 1)])
def test_kernels_with_oracle_q1_fp64(n, k):
    """Operator-identical parity: the GPU runs the oracle's own Q1 (ygm_set_q1), so only the
    summation order differs."""
    f, g, eps, _ = oracle_model(n, k, eps_seed=78)
    tau = 0.45 * g.tau_cfl()
    rng = np.random.default_rng(n * 7 + k)
    e0 = rng.standard_normal(f.mesh.N1)
    b0 = f.C() @ rng.standard_normal(f.mesh.N1)
    e_or, bst_or, bs_or, _ = run_oracle(f, g, e0, b0, tau, 150)
    c = Y.Context(n, k, eps=eps, precision=Y.YGM_FP64)
    c.set_q1(g.Q1)
    assert abs(c.tau_cfl / g.tau_cfl() - 1) < 1e-9
    c.set_state(e0, b0)
    c.step(150, tau)
    e, b = c.get_state(synced=True)
    _, bs = c.get_state(synced=False)
    assert rel_l2(e, e_or) < FP64_TOL and rel_l2(b, bs_or) < FP64_TOL and rel_l2(bs, bst_or) < FP64_TOL


def test_single_step_elementwise_fp64():
    """One step from a random staggered state: every element of e_1 and b_{1/2}."""
    f, g, eps, _ = oracle_model(3, 2, eps_seed=5)
    tau = 0.5 * g.tau_cfl()
    rng = np.random.default_rng(0)
    e0 = rng.standard_normal(f.mesh.N1)
    b0 = f.C() @ rng.standard_normal(f.mesh.N1)
    e_or, bst_or, bs_or, _ = run_oracle(f, g, e0, b0, tau, 1)
    _, e, b, bs, _ = _gpu_run(3, 2, eps, e0, b0, tau, 1, Y.YGM_FP64)
    scale_e, scale_b = np.abs(e_or).max(), np.abs(bst_or).max()
    assert np.all(np.abs(e - e_or) <= 1e-13 * scale_e)
    assert np.all(np.abs(bs - bst_or) <= 1e-13 * scale_b)


def test_ragged_rows_longer_than_a_warp():
    """n = 34: class rows of 33/34 entries take two 32-lane passes per warp."""
    n, k = 34, 1
    c = Y.Context(n, k, precision=Y.YGM_FP64)
    f, g, eps, _ = oracle_model(6, 1)     # only for the property checks below
    rng = np.random.default_rng(1)
    e0 = rng.standard_normal(c.N1)
    b0 = np.zeros(c.N2)
    c.set_state(e0, b0)
    tau = 0.5 * c.tau_cfl
    c.step(1, tau)
    W0, _ = c.energy()
    c.step(200, tau)
    W1, _ = c.energy()
    assert abs(W1[0] - W0[0]) / W0[0] < 1e-12           # conserved at any size


def test_tiny_mesh_n1_and_empty_classes():
    c = Y.Context(1, 1, precision=Y.YGM_FP64)
    assert (c.N1, c.N2) == (1, 6)
    c.set_state(np.ones(1), np.zeros(6))
    c.step(10, 0.5 * c.tau_cfl)
    e, b = c.get_state()
    assert np.all(np.isfinite(e)) and np.all(np.isfinite(b))


def test_cfl_refused_and_nothing_run():
    c = Y.Context(2, 1, precision=Y.YGM_FP64)
    c.set_state(np.ones(c.N1), np.zeros(c.N2))
    n0 = c.launch_count()
    with pytest.raises(Y.YgmError) as ei:
        c.step(5, c.tau_cfl * 1.01)
    assert ei.value.code == Y.YGM_ECFL
    assert c.launch_count() == n0
    c.step(3, c.tau_cfl)                                  # exactly at the bound is allowed


def test_dt_change_is_an_exact_strang_restaggering():
    f, g, eps, _ = oracle_model(3, 1, eps_seed=9)
    t1, t2 = 0.4 * g.tau_cfl(), 0.3 * g.tau_cfl()
    rng = np.random.default_rng(4)
    e0 = rng.standard_normal(f.mesh.N1)
    b0 = np.zeros(f.mesh.N2)
    e, bst, bs, _ = run_oracle(f, g, e0, b0, t1, 40)
    e, bst, bs, _ = run_oracle(f, g, e, bs, t2, 25)        # restart from the synchronised state
    c = Y.Context(3, 1, eps=eps, precision=Y.YGM_FP64)
    c.set_state(e0, b0)
    c.step(40, t1)
    c.step(25, t2)
    eg, bg = c.get_state(synced=True)
    assert rel_l2(eg, e) < FP64_TOL and rel_l2(bg, bs) < FP64_TOL
    assert abs(c.time()[1] - (40 * t1 + 25 * t2)) < 1e-12


def test_energy_api_matches_oracle():
    f, g, eps, _ = oracle_model(3, 2, eps_seed=12)
    tau = 0.5 * g.tau_cfl()
    rng = np.random.default_rng(2)
    e0 = rng.standard_normal(f.mesh.N1)
    b0 = np.zeros(f.mesh.N2)
    e, bst, bs, _ = run_oracle(f, g, e0, b0, tau, 50)
    c = Y.Context(3, 2, eps=eps, precision=Y.YGM_FP64)
    c.set_state(e0, b0)
    c.step(50, tau)
    W, H = c.energy()
    assert abs(W[0] - g.W(e, bst, tau)) / abs(W[0]) < 1e-12
    assert abs(H[0] - g.H_tilde(e, bs)) / abs(H[0]) < 1e-12


def test_device_pointer_state_roundtrip():
    torch = pytest.importorskip("torch")
    c = Y.Context(3, 1, precision=Y.YGM_FP32)
    e = torch.randn(c.N1, device="cuda", dtype=torch.float32)
    b = torch.zeros(c.N2, device="cuda", dtype=torch.float32)
    c.set_state(e, b)
    torch.cuda.synchronize()
    e2 = torch.empty_like(e)
    b2 = torch.empty_like(b)
    c.get_state(synced=False, out_e=e2, out_b=b2)
    torch.cuda.synchronize()
    assert torch.equal(e, e2) and torch.equal(b, b2)


def test_nonuniform_mu_uses_per_tet_path():
    import scipy.sparse as sp
    from oracle import spai as SP
    from oracle.fem import FEM
    from oracle.gym import GYM
    from oracle.mesh import KuhnMesh
    n, k = 3, 2
    eps = synth.tet_eps(41, n, 1.0, 4.0)
    mu = synth.tet_eps(42, n, 1.0, 2.0)
    f = FEM(KuhnMesh(n, k), eps=eps, mu=mu)
    M1 = f.M1()
    Q, _ = SP.gym_q1(f, M1)
    g = GYM(f.C(), f.M2(), Q, M1)
    tau = 0.5 * g.tau_cfl()
    rng = np.random.default_rng(3)
    e0 = rng.standard_normal(f.mesh.N1)
    b0 = np.zeros(f.mesh.N2)
    e_or, bst_or, bs_or, _ = run_oracle(f, g, e0, b0, tau, 80)
    c = Y.Context(n, k, eps=eps, mu=mu, precision=Y.YGM_FP64)
    assert abs(c.tau_cfl / g.tau_cfl() - 1) < 1e-9
    c.set_state(e0, b0)
    c.step(80, tau)
    e, b = c.get_state(synced=True)
    assert rel_l2(e, e_or) < FP64_TOL and rel_l2(b, bs_or) < FP64_TOL


def test_energy_history_keeps_every_record():
    """More W_n records than the initial history capacity (65,536): the history grows inside
    ygm_step, every record is kept, and W_n stays conserved over the whole run."""
    c = Y.Context(2, 1, precision=Y.YGM_FP64, energy_every=1)
    rng = np.random.default_rng(21)
    c.set_state(rng.standard_normal(c.N1), np.zeros(c.N2))
    tau = 0.5 * c.tau_cfl
    c.step(40000, tau)
    c.step(30000, tau)
    W = c.energy_history(max_count=1 << 20)
    assert len(W) == 70000
    assert np.max(np.abs(W - W[0])) / W[0] < 1e-11
    c.close()


@pytest.mark.parametrize("precision,tol", [(0, 1e-12), (1, 1e-5)])
def test_fourth_order_splitting_follows_the_oracle(precision, tol):
    """ygm_set_splitting(4): each step the symmetric composition of Strang steps w1, w0, w1 (with a
    negative middle weight) against the oracle's composed_step, sources at sub-step midpoints."""
    from oracle.gym import yoshida4
    n, k, steps = 3, 2, 60
    f, g, eps, _ = oracle_model(n, k, eps_seed=2000)
    w = yoshida4()
    tau = 0.5 * g.tau_cfl() / abs(w[1])
    src = [_dipole(tau, width=5.0)]
    J = DipoleSource(f, [dict(s) for s in src], tau)
    rng = np.random.default_rng(8)
    e0 = rng.standard_normal(f.mesh.N1)
    b0 = f.C() @ rng.standard_normal(f.mesh.N1)
    e_or, b_or = g.run_composed(e0.copy(), b0.copy(), tau, steps, w, source=J)
    c = Y.Context(n, k, eps=eps, precision=precision)
    c.set_splitting(4)
    dtp = np.float64 if precision == 0 else np.float32
    c.set_state(e0.astype(dtp), b0.astype(dtp))
    c.step(25, tau, [dict(s) for s in src])
    c.step(35, tau, [dict(s) for s in src])
    e, b = c.get_state(synced=True)
    assert rel_l2(e, e_or) < tol and rel_l2(b, b_or) < tol
    assert c.time()[0] == steps and abs(c.time()[1] - steps * tau) < 1e-12
    with pytest.raises(Y.YgmError) as ei:
        c.set_splitting(2)                                 # only before the first step
    assert ei.value.code == Y.YGM_EINVAL
    with pytest.raises(Y.YgmError) as ei:
        c.step(1, 1.01 * c.tau_cfl / abs(w[1]))           # CFL on the largest sub-step
    assert ei.value.code == Y.YGM_ECFL


# n = 17 and 12: planes of 24 x 17 and 16 x 12 lattice points, so a (class, plane) spans two
# blocks of 256 with a ragged second one; the small cases also follow the oracle
@pytest.mark.parametrize("n,k,precision,oracle", [(2, 2, 1, True), (5, 1, 1, True), (4, 2, 0, True), (3, 3, 0, True),
                                                  (17, 2, 1, False), (12, 3, 1, False), (17, 1, 0, False)])
def test_q1_kernels_agree_bit_for_bit(n, k, precision, oracle):
    """The bulk-copy Q1 apply (shared-memory stages) and the per-thread-load one add the same terms
    in the same order: the states and energies after a run with energy read-outs are identical,
    for every stage count."""
    if oracle:
        f, g, eps, _ = oracle_model(n, k, eps_seed=90 + n)
    else:
        eps = synth.tet_eps(90 + n, n, 1.0, 4.0)
    c0 = Y.Context(n, k, eps=eps, precision=precision, energy_every=7)
    tau = 0.45 * c0.tau_cfl
    rng = np.random.default_rng(n * 13 + k)
    e0 = rng.standard_normal(c0.N1)
    b0 = np.zeros(c0.N2)
    dt = np.float64 if precision == Y.YGM_FP64 else np.float32
    runs = []
    for kernel, stages in [(1, 0), (2, 0), (2, 2), (2, 5)]:
        c = c0.like(energy_every=7)           # same operators, fresh state, clock and energy record
        assert c.set_qapply(kernel, stages) >= 1
        c.set_state(np.ascontiguousarray(e0, dt), np.ascontiguousarray(b0, dt))
        c.step(40, tau)
        e, b = c.get_state(synced=True)
        runs.append((e, b, c.energy_history()))
    assert np.linalg.norm(runs[0][1]) > 0
    for e, b, W in runs[1:]:
        assert np.array_equal(e, runs[0][0]) and np.array_equal(b, runs[0][1]) and np.array_equal(W, runs[0][2])
    if oracle:
        e_or, _, bs_or, _ = run_oracle(f, g, e0, b0, tau, 40)
        tol = FP32_TOL if precision == Y.YGM_FP32 else PIPE_TOL[k]
        assert rel_l2(runs[0][0], e_or) < tol and rel_l2(runs[0][1], bs_or) < tol


def test_q1_kernel_selection_rejects_bad_arguments():
    c = Y.Context(4, 2, precision=Y.YGM_FP32)
    for kernel, stages in [(3, 0), (-1, 0), (2, 1), (2, 9), (0, 99)]:
        with pytest.raises(Y.YgmError):
            c.set_qapply(kernel, stages)
    assert c.set_qapply(0, 0) >= 1
    r = Y.Context(4, 2, precision=Y.YGM_FP32, n_rhs=4)
    with pytest.raises(Y.YgmError):
        r.set_qapply(1, 0)


def test_programmatic_dependent_launch_changes_nothing():
    """The step's kernels launched with programmatic stream serialization (the default) and as
    ordinary stream-ordered launches give identical states, energies and source response."""
    n, k = 17, 2
    c0 = Y.Context(n, k, eps=synth.tet_eps(117, n, 1.0, 4.0), precision=Y.YGM_FP32, energy_every=9)
    tau = 0.5 * c0.tau_cfl
    src = [_dipole(tau, x=(0.43, 0.51, 0.48))]
    out = []
    for pdl in (True, False):
        c = c0.like(energy_every=9)
        c.set_launch(pdl)
        c.set_state(np.zeros(c.N1, np.float32), np.zeros(c.N2, np.float32))
        c.step(120, tau, [dict(s) for s in src])
        e, b = c.get_state(synced=True)
        out.append((e, b, c.energy_history()))
    assert np.linalg.norm(out[0][0]) > 0
    for a, b in zip(out[0], out[1]):
        assert np.array_equal(a, b)
