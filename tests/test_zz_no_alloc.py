"""GPU test of ygm_step_noalloc: the leapfrog step for callers that cannot allocate device memory
(device memory reserved up front by another allocator, latency budgets that rule out
cudaMalloc).  It must give what the
regular entry point gives, on two calls in a row, and reject contexts beyond its fixed scratch.
This file is collected last on purpose."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

import synth

Y = pytest.importorskip("paper_2301_01753_gb300")
torch = pytest.importorskip("torch")


@pytest.mark.parametrize("precision,tol", [(0, 1e-12), (1, 1e-6)])
def test_noalloc_step_matches_ygm_step_twice(precision, tol):
    n, k = 4, 2
    eps = synth.tet_eps(91, n, 1.0, 4.0)
    c = Y.Context(n, k, eps=eps, precision=precision)
    dt = 0.5 * c.tau_cfl
    rng = np.random.default_rng(9)
    dtp = np.float64 if precision == Y.YGM_FP64 else np.float32
    tdt = torch.float64 if precision == Y.YGM_FP64 else torch.float32
    c.set_state(rng.standard_normal(c.N1).astype(dtp), np.zeros(c.N2, dtp))
    c.step(1, dt)                                       # staggered state (e_1, b_{1/2})
    e1, bh = c.get_state(synced=False)
    e_t = torch.tensor(e1, dtype=tdt, device="cuda")
    b_t = torch.tensor(bh, dtype=tdt, device="cuda")
    for _ in range(2):
        c.step(1, dt)                                   # regular entry point
        e_ref, b_ref = c.get_state(synced=False)
        c.step_noalloc(e_t, b_t, b_t, dt)               # no-allocation entry point, in place
        torch.cuda.synchronize()
        e_na, b_na = e_t.cpu().numpy(), b_t.cpu().numpy()
        assert np.max(np.abs(e_na - e_ref)) <= tol * np.abs(e_ref).max()
        assert np.max(np.abs(b_na - b_ref)) <= tol * np.abs(b_ref).max()


def test_noalloc_rejects_contexts_beyond_the_scratch():
    # k = 1, n = 68: N1 = 2,160,416 > 2,097,152 FP64 values of scratch
    c = Y.Context(68, 1, precision=Y.YGM_FP64, device=-1)
    assert c.N1 * 8 > 16 * 2 ** 20
    e = torch.zeros(8, dtype=torch.float64, device="cuda")
    with pytest.raises(Y.YgmError) as ei:
        c.step_noalloc(e, e, e, 1e-3)
    assert ei.value.code == Y.YGM_EINVAL and "16 MiB" in str(ei.value)
