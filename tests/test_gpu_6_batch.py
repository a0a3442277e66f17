"""GPU uneven batch (ygm_batch_*): independent cavities of different size n and order k stepped by
one persistent launch.  Each member must follow the FP64 oracle run of its own cavity (the
leapfrog of Eq. YeeLeapfrog in the form of Eq. preYeeFEECEqns, its own dt and dipole), and must
give exactly what ygm_step gives for the same context."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

import synth
from oracle_runs import oracle_model, run_oracle, rel_l2

Y = pytest.importorskip("paper_2301_01753_gb300")

# (n, k, eps seed): mixed sizes and orders, small enough for the oracle
MEMBERS = [(3, 1, 4001), (2, 3, 4002), (4, 2, 4003), (5, 1, 4004), (3, 2, 4005)]


def _src(i, tau):
    x = synth.source_positions(4100 + i, 1)[0]
    d = synth.unit_vectors(4200 + i, 1)[0]
    sigma = 5.0 * tau
    return dict(x=x, d=d, amp=1.0, omega=np.pi * np.sqrt(5.0), t0=4 * sigma, sigma=sigma)


def _members(precision):
    out = []
    for i, (n, k, seed) in enumerate(MEMBERS):
        f, g, eps, _ = oracle_model(n, k, eps_seed=seed, eps_range=(1.0, 9.0))
        c = Y.Context(n, k, eps=eps, precision=precision)
        out.append((f, g, c))
    return out


# FP64: the single-column pipeline tolerances (host SPAI of the builder against the oracle's: ~1e-13
# at k <= 2, ~2e-12 at k = 3, carried by the run); FP32: the single-column FP32 bound
PIPE_TOL = {1: 1e-12, 2: 1e-12, 3: 5e-11}


@pytest.mark.parametrize("precision", [0, 1])
def test_batch_members_follow_the_oracle(precision):
    mem = _members(precision)
    dts = np.array([0.5 * c.tau_cfl for _, _, c in mem])
    srcs = [_src(i, dts[i]) for i in range(len(mem))]
    dtp = np.float64 if precision == 0 else np.float32
    for _, _, c in mem:
        c.set_state(np.zeros(c.N1, dtp), np.zeros(c.N2, dtp))
    B = Y.Batch([c for _, _, c in mem])
    B.step(40, dts, srcs)
    B.step(35, dts, srcs, use_graph=True)          # a second call continues the staggered run
    B.status()
    for i, (f, g, c) in enumerate(mem):
        s = dict(srcs[i], width_steps=5.0)
        z1, z2 = np.zeros(f.mesh.N1), np.zeros(f.mesh.N2)
        e_or, _, bs_or, _ = run_oracle(f, g, z1, z2, dts[i], 75, sources=[s])
        e, b = c.get_state(synced=True)
        tol = PIPE_TOL[MEMBERS[i][1]] if precision == 0 else 1e-5
        assert np.linalg.norm(e_or) > 0
        assert rel_l2(e, e_or) < tol, i
        assert rel_l2(b, bs_or) < tol, i
        assert c.time()[0] == 75
    B.close()


def test_batch_equals_ygm_step_exactly():
    """The batch runs the same item bodies as the one-column kernels: bitwise equal FP32 states."""
    mem_b = _members(Y.YGM_FP32)
    mem_s = _members(Y.YGM_FP32)
    dts = np.array([0.5 * c.tau_cfl for _, _, c in mem_b])
    srcs = [_src(i, dts[i]) for i in range(len(mem_b))]
    rng = np.random.default_rng(3)
    for (_, _, cb), (_, _, cs) in zip(mem_b, mem_s):
        e0 = rng.standard_normal(cb.N1).astype(np.float32)
        cb.set_state(e0, np.zeros(cb.N2, np.float32))
        cs.set_state(e0, np.zeros(cs.N2, np.float32))
    B = Y.Batch([c for _, _, c in mem_b])
    B.step(50, dts, srcs, use_graph=True)
    B.status()
    for i, ((_, _, cb), (_, _, cs)) in enumerate(zip(mem_b, mem_s)):
        cs.step(50, dts[i], [srcs[i]])
        eb, bb = cb.get_state(synced=False)
        es, bs = cs.get_state(synced=False)
        assert np.array_equal(eb, es) and np.array_equal(bb, bs), i
    B.close()


def test_tuner_restores_the_states_and_picks_a_shape():
    mem = _members(Y.YGM_FP64)
    dts = np.array([0.5 * c.tau_cfl for _, _, c in mem])
    rng = np.random.default_rng(4)
    states = []
    for _, _, c in mem:
        e0 = rng.standard_normal(c.N1)
        c.set_state(e0, np.zeros(c.N2))
        states.append(c.get_state(synced=False))
    B = Y.Batch([c for _, _, c in mem])
    cps, order, ms = B.tune(5, dts)
    assert 1 <= cps <= 4 and order in (0, 1) and ms > 0
    for (e0, b0), (_, _, c) in zip(states, mem):
        e, b = c.get_state(synced=False)
        assert np.array_equal(e, e0) and np.array_equal(b, b0)
        assert c.time()[0] == 0
    B.step(10, dts)
    B.status()
    B.close()


def test_batch_rejects_mismatched_members():
    a = Y.Context(2, 1, precision=Y.YGM_FP32)
    b = Y.Context(2, 1, precision=Y.YGM_FP64)
    with pytest.raises(Y.YgmError) as ei:
        Y.Batch([a, b])
    assert ei.value.code == Y.YGM_EINVAL
    c = Y.Context(2, 1, precision=Y.YGM_FP32)
    B = Y.Batch([a, c])
    with pytest.raises(Y.YgmError) as ei:
        B.step(3, [a.tau_cfl * 1.5, c.tau_cfl * 0.5])
    assert ei.value.code == Y.YGM_ECFL
    B.close()


def test_barrier_timeout_is_reported_and_the_batch_recovers():
    """A wait limit of zero polls makes every grid-barrier wait that does not find the barrier
    complete give up at once: the launch ends early with the error flag set (no hang), the host
    reads YGM_ETIMEOUT, and after clearing the flag and restoring the limit the batch steps
    correctly again from a fresh state."""
    mem = _members(Y.YGM_FP64)
    dts = np.array([0.5 * c.tau_cfl for _, _, c in mem])
    for _, _, c in mem:
        c.set_state(np.ones(c.N1), np.zeros(c.N2))
    B = Y.Batch([c for _, _, c in mem])
    B.wait_limit(0)
    B.step(20, dts)
    with pytest.raises(Y.YgmError) as ei:
        B.status()
    assert ei.value.code == Y.YGM_ETIMEOUT
    B.status_clear()
    B.wait_limit(1 << 24)
    srcs = [_src(i, dts[i]) for i in range(len(mem))]
    for _, _, c in mem:
        c.set_state(np.zeros(c.N1), np.zeros(c.N2))
    B.step(30, dts, srcs)
    B.status()
    for i, (f, g, c) in enumerate(mem):
        e_or, _, bs_or, _ = run_oracle(f, g, np.zeros(f.mesh.N1), np.zeros(f.mesh.N2), dts[i], 30,
                                       sources=[dict(srcs[i], width_steps=5.0)])
        e, b = c.get_state(synced=True)
        assert rel_l2(e, e_or) < PIPE_TOL[MEMBERS[i][1]], i
    B.close()
