"""Generalized Yee method: shear maps, Strang / leapfrog stepping, energies, CFL bound, sources.

Oracle (test infrastructure), FP64, plain sparse matrix-vector products.

Paper passages followed:
  Eq. discEOM          a' = -Q1 e,  e' = c^2 C^T M2 C a
  Eq. preYeeFEECEqns   b' = -C Q1 e, e' = c^2 C^T M2 b          (b = C a)
  Eq. shearMaps        Phi^e_tau (a, e) = (a - tau Q1 e, e);  Phi^a_tau (a, e) = (a, e + tau P2 a)
  Eq. strangSplit      Phi_tau = Phi^e_{tau/2} o Phi^a_tau o Phi^e_{tau/2}; higher-order
                       splittings as symmetric compositions of Strang maps (composed_step)
  Eq. YeeLeapfrog      initial half step of Phi^e, then alternate full steps
  Prop. stability      tau <= 2 / omega_max, omega_max^2 = lambda_max(Q1 P2)
  Eq. allEOM (3rd)     e' = -sum q xdot . Lambda1(x_s): template of the dipole current term
Readings (the paper is silent): state (e_n, b_{n-1/2}); one step is
  x = Q1 e_n;  b_{n+1/2} = b_{n-1/2} - tau C x;  e_{n+1} = e_n + tau (C^T M2 b_{n+1/2} - j_{n+1/2})
with j_i(t) = s(t) d . Lambda1_i(x0) for a point dipole d delta(x - x0) s(t),
s(t) = amp exp(-((t - t0)/sigma)^2) sin(omega0 (t - t0)), sigma = width * tau, t0 = 4 sigma.
The exactly conserved discrete energy (derived by telescoping, not stated in the
paper) is W_n = 1/2 e_n^T Q1 e_n + 1/2 b_{n+1/2}^T M2 b_{n-1/2}; the paper's
recorded energy is H~ = 1/2 e^T Q1 e + 1/2 b^T M2 b at synchronised times.
Pins: tests/test_oracle_gym.py (symplecticity, eigenvalue pairs, CFL, energy,
Gauss law, Yee equivalence, source work identity).
"""
import numpy as np
import scipy.sparse as sp
import scipy.linalg as sl


class GYM:
    def __init__(self, C, M2, Q1, M1=None):
        self.C = sp.csr_matrix(C)
        self.CT = self.C.T.tocsr()
        self.M2 = sp.csr_matrix(M2)
        self.Q1 = sp.csr_matrix(Q1)
        self.M1 = M1
        self.P2 = (self.CT @ self.M2 @ self.C).tocsr()

    # -------------------------------------------------------------- CFL
    def omega_max_sq(self, dense_limit=3000, iters=300, seed=0):
        """lambda_max(Q1 P2) (Prop. stability)."""
        n = self.Q1.shape[0]
        if n <= dense_limit:
            Q = self.Q1.toarray()
            w, V = np.linalg.eigh(Q)
            Qh = (V * np.sqrt(w)) @ V.T                # Q1^(1/2), Q1 SPD
            return float(np.linalg.eigvalsh(Qh @ self.P2.toarray() @ Qh)[-1])
        # Lanczos on P2 Q1, self-adjoint in the Q1 inner product <x, y> = x^T Q1 y
        rng = np.random.default_rng(seed)
        v = rng.standard_normal(n)
        v /= np.sqrt(v @ (self.Q1 @ v))
        v_prev = np.zeros(n)
        beta = 0.0
        al, be = [], []
        for _ in range(iters):
            w = self.P2 @ (self.Q1 @ v) - beta * v_prev
            a = w @ (self.Q1 @ v)
            w = w - a * v
            beta = np.sqrt(max(w @ (self.Q1 @ w), 0.0))
            al.append(a)
            be.append(beta)
            if beta == 0:
                break
            v_prev, v = v, w / beta
        Tm = np.diag(al) + np.diag(be[:-1], 1) + np.diag(be[:-1], -1)
        return float(np.linalg.eigvalsh(Tm)[-1])

    def tau_cfl(self, **kw):
        return 2.0 / np.sqrt(self.omega_max_sq(**kw))

    # -------------------------------------------------------------- (a, e) form
    def phi_e(self, a, e, tau):
        return a - tau * (self.Q1 @ e), e

    def phi_a(self, a, e, tau):
        return a, e + tau * (self.P2 @ a)

    def strang(self, a, e, tau):
        a, e = self.phi_e(a, e, 0.5 * tau)
        a, e = self.phi_a(a, e, tau)
        a, e = self.phi_e(a, e, 0.5 * tau)
        return a, e

    # -------------------------------------------------------------- (b, e) leapfrog
    def half_init(self, e0, b0, tau):
        """b_{-1/2} = b_0 + (tau/2) C Q1 e_0, so that the first step yields b_{1/2} = b_0 - (tau/2) C Q1 e_0."""
        return b0 + 0.5 * tau * (self.C @ (self.Q1 @ e0))

    def sync(self, e, b, tau):
        """b_n = b_{n-1/2} - (tau/2) C Q1 e_n."""
        return b - 0.5 * tau * (self.C @ (self.Q1 @ e))

    def step(self, e, b, tau, j=None):
        """One leapfrog step (e_n, b_{n-1/2}) -> (e_{n+1}, b_{n+1/2}); returns (e, b, x, b_old)."""
        x = self.Q1 @ e
        b_new = b - tau * (self.C @ x)
        y = self.CT @ (self.M2 @ b_new)
        e_new = e + tau * y
        if j is not None:
            e_new = e_new - tau * j
        return e_new, b_new, x, b

    def run(self, e, b, tau, nsteps, source=None, t_start=0, energy_every=0, record=None):
        """nsteps leapfrog steps from step index t_start; source(t) -> j vector (or None).

        Returns (e, b, energies) with energies the list of W_n at recorded steps."""
        W = []
        for n in range(nsteps):
            t_half = (t_start + n + 0.5) * tau
            j = source(t_half) if source is not None else None
            e_new, b_new, x, b_old = self.step(e, b, tau, j)
            if energy_every and (t_start + n) % energy_every == 0:
                W.append(0.5 * (e @ x) + 0.5 * (b_new @ (self.M2 @ b_old)))
            if record is not None:
                record(t_start + n, e, b_old, b_new, x)
            e, b = e_new, b_new
        return e, b, W

    # -------------------------------------------------------------- composed (higher-order) splittings
    def composed_step(self, e, b_sync, tau, weights, t0=0.0, source=None):
        """One step of a symmetric composition of Strang steps (the higher-order splittings the
        paper mentions after Eq. strangSplit): Strang maps of sizes w_1 tau, ..., w_m tau in turn,
        each in the (b, e) form  b -= (w tau / 2) C Q1 e;  e += w tau (C^T M2 b - j(t_mid));
        b -= (w tau / 2) C Q1 e,  with t_mid the midpoint of the sub-step.  From and to
        synchronised b."""
        t = t0
        for w in weights:
            h = w * tau
            b_sync = b_sync - 0.5 * h * (self.C @ (self.Q1 @ e))
            e = e + h * (self.CT @ (self.M2 @ b_sync))
            if source is not None:
                e = e - h * source(t + 0.5 * h)
            b_sync = b_sync - 0.5 * h * (self.C @ (self.Q1 @ e))
            t = t + h
        return e, b_sync

    def run_composed(self, e, b_sync, tau, nsteps, weights, source=None):
        for n in range(nsteps):
            e, b_sync = self.composed_step(e, b_sync, tau, weights, t0=n * tau, source=source)
        return e, b_sync

    def composed_jacobian(self, tau, weights):
        """Dense Jacobian of one composed step on (a, e) (products of Strang Jacobians)."""
        J = np.eye(2 * self.Q1.shape[0])
        for w in weights:
            J = self.strang_jacobian(w * tau) @ J
        return J

    def W(self, e, b, tau):
        """Conserved discrete energy of the state (e_n, b_{n-1/2})."""
        x = self.Q1 @ e
        b_new = b - tau * (self.C @ x)
        return 0.5 * (e @ x) + 0.5 * (b_new @ (self.M2 @ b))

    def H_tilde(self, e, b_sync):
        """The paper's modified Hamiltonian at synchronised time (Sec. 7, energy paragraph)."""
        return 0.5 * (e @ (self.Q1 @ e)) + 0.5 * (b_sync @ (self.M2 @ b_sync))

    # -------------------------------------------------------------- Jacobians (tiny meshes)
    def strang_jacobian(self, tau):
        """Dense Jacobian of the Strang map on (a, e) in R^{2 N1}."""
        n = self.Q1.shape[0]
        Q = self.Q1.toarray()
        P = self.P2.toarray()
        I = np.eye(n)
        Je = np.block([[I, -0.5 * tau * Q], [np.zeros((n, n)), I]])
        Ja = np.block([[I, np.zeros((n, n))], [tau * P, I]])
        return Je @ Ja @ Je


def yoshida4():
    """Weights of the fourth-order symmetric triple composition of a second-order symmetric map
    (Yoshida 1990): w1 = 1 / (2 - 2^(1/3)), w0 = -2^(1/3) / (2 - 2^(1/3)); (w1, w0, w1), sum 1."""
    c = 2.0 ** (1.0 / 3.0)
    w1 = 1.0 / (2.0 - c)
    return (w1, -c * w1, w1)


def pulse(t, amp, omega, t0, sigma):
    """Gaussian-modulated sinusoid s(t) (reading of the dipole envelope)."""
    return amp * np.exp(-((t - t0) / sigma) ** 2) * np.sin(omega * (t - t0))


class DipoleSource:
    """j(t) = sum_s s_s(t) d_s . Lambda1(x_s) restricted to the DoFs of the tet holding x_s."""

    def __init__(self, fem, sources, tau, n_rhs=1):
        self.N1 = fem.mesh.N1
        self.n_rhs = n_rhs
        self.items = []
        for s in sources:
            t = fem.mesh.locate(s["x"])
            vals = fem.point_values(t, s["x"]) @ np.asarray(s["d"], float)
            dofs = fem.dof1[t]
            ok = dofs >= 0
            sigma = s.get("width_steps", 20.0) * tau
            self.items.append(dict(dofs=dofs[ok], w=vals[ok], amp=s.get("amp", 1.0), omega=s["omega"],
                                   t0=s.get("t0_sigmas", 4.0) * sigma, sigma=sigma, rhs=s.get("rhs", 0), tet=t))

    def __call__(self, t):
        j = np.zeros((self.N1, self.n_rhs)) if self.n_rhs > 1 else np.zeros(self.N1)
        for it in self.items:
            a = pulse(t, it["amp"], it["omega"], it["t0"], it["sigma"])
            if self.n_rhs > 1:
                j[it["dofs"], it["rhs"]] += a * it["w"]
            else:
                j[it["dofs"]] += a * it["w"]
        return j
