/*
 * ygm.h -- C ABI of the GB300 (sm_103a) generalized Yee method (GYM) leapfrog library.
 *
 * The method (Glasser & Qin, "Generalized Yee methods"): Maxwell's equations on a
 * de Rham-conforming finite element complex, with the Hamiltonian
 *     H~ = 1/2 e^T Q1 e + 1/2 a^T C^T M2 C a            (Eq. discTildeHamilSystem)
 * where Q1 ~ M1^-1 is a sparse SPD approximate inverse (Sec. 5, Eq. NormalEqSolve)
 * and C is the integer curl of the complex (Eq. discreteDeRham).  Time stepping is the
 * Strang composition of the two exact shear maps (Eqs. shearMaps, strangSplit), run in
 * the staggered (b, e) form of Eq. preYeeFEECEqns / Eq. YeeLeapfrog:
 *     x         = Q1 e_n
 *     b_{n+1/2} = b_{n-1/2} - dt C x
 *     e_{n+1}   = e_n + dt (C^T M2 b_{n+1/2} - j_{n+1/2})
 * Units: eps0 = mu0 = c = 1.
 *
 * Domain: the PEC cube [0, side]^3 cut into n^3 cubes, each split into the 6 Kuhn
 * tetrahedra; tet index t = 6 (cx + n (cy + n cz)) + shape, shape in order of the vertex
 * chains (x,xy), (x,xz), (y,xy), (y,yz), (z,xz), (z,yz).  Order k = 1, 2, 3: trimmed
 * P_k^- Lambda^1 / P_k^- Lambda^2 in a hierarchical exact-sequence basis whose C, G, D
 * have entries in {0, +-1}.
 *
 * DoF layout (e, b, and every vector crossing this ABI): DoFs are grouped in classes
 * (entity shape, DoF index inside the entity); classes are ordered edges (7 shapes,
 * offsets x, y, xy, z, xz, yz, xyz), faces (12 shapes), tets (6 shapes), each shape with
 * its k (edge), k(k-1) (face), k(k-1)(k-2)/2 (tet) 1-form DoFs, or k(k+1)/2 (face),
 * (k-1)k(k+1)/2 (tet) 2-form DoFs.  Inside a class the anchors v (smallest vertex of the
 * entity, lattice coordinates) run x fastest over the interior box: along axis a,
 * v_a in [0, n-1] if the entity extends along a, else [1, n-1] (PEC removes entities
 * lying in the boundary).  With R right-hand sides, vectors are row-major [N][R]
 * (R contiguous).
 *
 * Conventions: every function returns 0 on success or a negative YGM_E* code; no
 * exception crosses the ABI; ygm_last_error() gives the message of the last failure of
 * that context.  Host pointers are read or written synchronously; device pointers
 * (on_device = 1) are read or written in stream order on the context's stream, which is
 * also where every kernel of this library runs.  The context owns all device memory it
 * allocates; inputs are copied, the caller keeps its buffers.
 */
#ifndef YGM_H
#define YGM_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define YGM_OK        0
#define YGM_EINVAL   -1   /* bad argument (sizes, NULL, NaN, non-positive eps/mu, ...) */
#define YGM_ECFL     -2   /* dt > tau_CFL (1 + 1e-12): refused, nothing is run (Prop. stability) */
#define YGM_ENOTSPD  -3   /* Q1 not SPD even after the allowed diagonal shift */
#define YGM_ENOMEM   -4   /* host or device allocation failed */
#define YGM_ECUDA    -5   /* a CUDA call failed (message carries cudaGetErrorString) */
#define YGM_ETIMEOUT -6   /* an iterative host solve (SPAI-OP PCG, cavity modes) reached its
                             iteration limit without converging, or a bounded device wait gave up:
                             the tensor-core MMA completion, or a stage of the bulk-copy Q1 apply
                             (reported by the next ygm_get_state / ygm_energy) */
#define YGM_ENODEV   -7   /* no CUDA device is available */

#define YGM_FP64 0        /* fields, Q1 and arithmetic in double */
#define YGM_FP32 1        /* fields, Q1 and arithmetic in float; diagnostics in double */
/* FP32 fields and kernels, with the one dense contraction of the batched mode -- C^T M2 of every
 * curl-carrying class at a batch of lattice points, (points x columns) x |U| times |U| x classes
 * (Eq. dTIsFiniteDiff with the merged constant stencil of a uniform mu) -- on the tcgen05 tensor
 * cores with FP32 accumulation.  Needs n_rhs = 32, 64 or 128, a uniform mu and order 1 or 2
 * (YGM_EINVAL otherwise).  Q1 e stays on FP32 SIMT: a TF32 Q1 would not stay positive definite
 * (its relative spacing 2^-11 exceeds lambda_min / lambda_max of Q1, e.g. 1.8e-4 at N = 32, k = 2). */
#define YGM_FP32_TC_TF32   2   /* operands truncated to TF32 (one pass): ~1e-3 relative per product */
#define YGM_FP32_TC_3XTF32 3   /* operands split hi + lo in TF32, three passes: ~2^-21 per product */

#define YGM_Q1_DEFAULT 0  /* k = 1: S(M1); k >= 2: S(M1^2) in the orthogonalised basis */
#define YGM_Q1_DIAG    1  /* S(1): q_l = M_ll / sum_k M_kl^2 */
#define YGM_Q1_SM1     2  /* S(M1): DoF pairs sharing a tetrahedron, plain basis */
#define YGM_Q1_SM1SQ   3  /* S(M1^2), orthogonalised basis for k >= 2 */

typedef struct ygm_ctx ygm_ctx;

typedef struct {
    int32_t n;       /* cubes per side, >= 1 */
    double side;     /* edge length of the cube, > 0 */
} ygm_mesh;

typedef struct {
    int32_t precision;     /* YGM_FP64, YGM_FP32, YGM_FP32_TC_TF32 or YGM_FP32_TC_3XTF32 */
    int32_t q1_pattern;    /* YGM_Q1_* */
    int32_t n_rhs;         /* R >= 1 right-hand sides (independent excitations) */
    int32_t energy_every;  /* record W_n every K steps inside ygm_step; 0 = off */
    int32_t threads;       /* host threads for the FP64 set-up; 0 = all cores */
    int32_t device;        /* CUDA device ordinal; -1 = host-only set-up (operators can be
                              inspected with ygm_sizes / ygm_export_q1 / ygm_local_blocks /
                              ygm_q1_info; every stepping call returns YGM_ENODEV) */
    void*   stream;        /* cudaStream_t to run on; NULL = the context creates its own
                              non-blocking stream.  cudaStreamLegacy is accepted, but a batch
                              whose first member runs on it cannot replay a CUDA graph (the
                              legacy stream cannot be captured: ygm_batch_step returns
                              YGM_ECUDA with use_graph = 1) */
} ygm_opts;

/* Point dipole J = d delta(x - x0) s(t), s(t) = amp exp(-((t - t0)/sigma)^2) sin(omega (t - t0)),
 * entering e through j_i = s(t) d . Lambda1_i(x0) (template: the current term of Eq. allEOM). */
typedef struct {
    double x[3];      /* position inside the cube */
    double d[3];      /* dipole moment direction and size */
    double amp, omega, t0, sigma;
    int32_t rhs;      /* which right-hand side column it drives, 0 <= rhs < n_rhs */
} ygm_source;

/* Build the mesh, bases, M1(eps), M2(mu), C, Q1 (SPAI, FP64, symmetrised, SPD-checked),
 * tau_CFL = 2 / sqrt(lambda_max(Q1 P2)) (Prop. stability) and upload the operators.
 * eps, mu: per-tet arrays of length 6 n^3 (host, copied) or NULL for 1.  The state starts at
 * e = 0, b = 0, t = 0.  Errors: YGM_EINVAL, YGM_ENOTSPD, YGM_ENOMEM, YGM_ECUDA, YGM_ENODEV;
 * on error *out is NULL. */
int ygm_create(const ygm_mesh* mesh, int order, const double* eps, const double* mu,
               const ygm_opts* opts, ygm_ctx** out);

/* A second context of the same discrete problem: the mesh, order, eps, mu and the current
 * operators of src (its Q1 included, also one installed by ygm_set_q1 or ygm_spai_op) are
 * copied from src's host set-up, so nothing of Sec. 5 is recomputed; precision, n_rhs,
 * energy_every, device and stream come from opts (q1_pattern and threads are ignored).  src is
 * only read and may be host-only.  The new state is e = 0, b = 0, t = 0.  Errors as ygm_create. */
int ygm_create_like(const ygm_ctx* src, const ygm_opts* opts, ygm_ctx** out);

/* Sizes: N1 (1-form DoFs), N2 (2-form DoFs), stored nonzeros of the symmetric Q1, and
 * tau_CFL.  Any pointer may be NULL. */
int ygm_sizes(const ygm_ctx* ctx, int64_t* n1, int64_t* n2, int64_t* q1_nnz, double* dt_cfl);

/* Copy a state in: e [N1][R], b [N2][R] in the context precision (double for YGM_FP64,
 * float for YGM_FP32), synchronised (b at the same time as e).  Resets the step count to 0
 * and the staggering (the next ygm_step starts with the initial half step). */
int ygm_set_state(ygm_ctx* ctx, const void* e, const void* b, int on_device);

/* Copy the state out.  synced = 1 returns b at the time of e (b_n = b_{n-1/2} - dt/2 C Q1 e_n,
 * the closing half step of Eq. strangSplit, computed into scratch, state untouched);
 * synced = 0 returns the staggered b_{n-1/2}.  Either pointer may be NULL. */
int ygm_get_state(ygm_ctx* ctx, void* e, void* b, int on_device, int synced);

/* e0 = M1 Pi E0: k = 1 the canonical Whitney interpolant (edge integrals, Eq. WhitneyFormDefn)
 * scaled by M1; k >= 2 the L2 load vector int E0 . Lambda1_i (= M1 times the L2 projection).
 * E0(x, out, user) is called on host points; the result is written to e for column `rhs`
 * and b is set to 0 (a state set: step count reset). */
int ygm_project_E(ygm_ctx* ctx, void (*E0)(const double x[3], double out[3], void* user),
                  void* user, int32_t rhs);

/* Advance n full steps of size dt (Eq. YeeLeapfrog), with the sources active.  dt must not
 * exceed tau_CFL (YGM_ECFL, nothing run).  The first step after a state set runs the initial
 * half step b_{-1/2} = b_0 + dt/2 C Q1 e_0.  A dt different from the previous call's is handled
 * by closing the old staggering with dt_old/2 and reopening it with dt/2 (exact Strang
 * composition).  Asynchronous on the context stream; returns after enqueueing. */
int ygm_step(ygm_ctx* ctx, int64_t n, double dt, const ygm_source* src, int32_t n_src);

/* One leapfrog step on caller-owned device buffers, with no device allocation (no cudaMalloc,
 * cudaFree or allocating library call).  The paper has no counterpart: this entry point exists
 * for callers that cannot allocate device memory -- e.g. a process whose device memory is
 * reserved up front by another allocator, or code under a latency budget that rules out
 * cudaMalloc, which may synchronise the device.
 * State (e_n, b_{n-1/2}) in the context precision: x = Q1 e (into a fixed 16 MiB file-scope
 * device scratch array, not into context memory), b_out = b_in - dt C x, e += dt C^T M2 b_out.
 * No source term, no half steps, no energy recording; the context's own state is untouched.
 * b_out may equal b_in; if it differs, its entries outside the range of C (the divergence part)
 * are not written.  Limit: N1 * n_rhs * sizeof(real) <= 16 MiB (2,097,152 DoFs in FP64,
 * 4,194,304 in FP32); larger contexts get YGM_EINVAL.  The first call on a device looks up the
 * scratch array's device address (cudaGetSymbolAddress) and should therefore come before any
 * stream capture.  All calls share the one scratch array, which keeps the last call's contents:
 * calls whose work overlaps on the GPU (other streams, other contexts) race on it.  Every element
 * of the scratch is written before it is read, so nothing needs clearing.  Asynchronous on the
 * context stream; errors YGM_EINVAL, YGM_ECFL, YGM_ENODEV, YGM_ECUDA. */
int ygm_step_noalloc(ygm_ctx* ctx, void* e, const void* b_in, void* b_out, double dt);

/* Splitting of one time step of ygm_step.  order 2 (default): the Strang leapfrog of Eq. strangSplit
 * / Eq. YeeLeapfrog.  order 4: the higher-order splitting the paper mentions after Eq. strangSplit,
 * taken as the symmetric triple composition of Strang steps of sizes w1 dt, w0 dt, w1 dt with
 * w1 = 1 / (2 - 2^(1/3)), w0 = 1 - 2 w1 (Yoshida's fourth-order weights; w0 < 0, so the CFL check is
 * |w0| dt <= tau_CFL).  The sub-steps reuse the leapfrog kernels with their own coefficients and
 * the sources are applied at each sub-step's midpoint; the staggered b lags by w1 dt / 2.  Must be
 * set before the first step (or after ygm_set_state / ygm_project_E); order 4 needs
 * energy_every = 0 (W_n is the Strang leapfrog's invariant) and is not available to ygm_adjoint
 * or the batch.  Errors: YGM_EINVAL. */
int ygm_set_splitting(ygm_ctx* ctx, int32_t order);

/* Conserved discrete energy of the current state (e_n, b_{n-1/2}), per right-hand side:
 *   W_n = 1/2 e_n^T Q1 e_n + 1/2 b_{n+1/2}^T M2 b_{n-1/2}
 * (telescoping invariant of the leapfrog; exact up to round-off without sources), and the
 * paper's H~ = 1/2 e^T Q1 e + 1/2 b_n^T M2 b_n at synchronised time.  FP64 compensated
 * (Neumaier) sums in a fixed order.  W, Htilde: host arrays of length R; Htilde may be NULL.
 * Synchronises the context stream. */
int ygm_energy(ygm_ctx* ctx, double* W, double* Htilde);

/* Energies W recorded by ygm_step every energy_every steps since the last state set:
 * copies up to max_count values (per RHS, [count][R]) to host `out` and returns the count in
 * *count.  Synchronises the context stream. */
int ygm_energy_history(ygm_ctx* ctx, double* out, int64_t max_count, int64_t* count);

/* Current time step index (full steps since the last state set) and time. */
int ygm_time(const ygm_ctx* ctx, int64_t* step, double* t);

/* The assembled symmetric Q1 in CSR over the global DoF numbering (FP64, as computed by the
 * set-up; columns sorted).  rowptr: N1 + 1 entries, colind / val: q1_nnz entries (host). */
int ygm_export_q1(const ygm_ctx* ctx, int64_t* rowptr, int64_t* colind, double* val);

/* Install a caller-supplied symmetric Q1 (CSR over the global numbering, FP64 host arrays,
 * columns sorted; rowptr has N1 + 1 entries) in place of the SPAI: any symmetric Q1 keeps the
 * map symplectic (Theorem symplecticity); it must be SPD for stability (Prop. stability).  Its
 * pattern must lie inside this context's stencil (S(1), S(M1) or S(M1^2) of q1_pattern).  The
 * SPD check and tau_CFL are recomputed; the state is kept.  Errors: YGM_EINVAL (pattern,
 * symmetry, sizes), YGM_ENOTSPD (the previous Q1 is kept), YGM_ECUDA (the device copies could
 * not be refreshed: destroy the context).  Synchronises the context stream. */
int ygm_set_q1(ygm_ctx* ctx, const int64_t* rowptr, const int64_t* colind, const double* val);

/* Operator-probed SPAI, SPAI-OP (Sec. 5.1): replace Q1 by the symmetric matrix on the current
 * Q1 pattern that minimises ||M1 Q1 - 1||_F^2 + lambda sum_k ||(M1 Q1 - 1) P2 v_k||^2
 * (Eq. SPAIOPobjective), i.e. solves the Sylvester system of Eq. SPAIOPSylvester by preconditioned
 * conjugate gradients with the diagonal preconditioner of Eq. diagonalPreconditioner, starting
 * from the current Q1 (the column-wise SPAI after ygm_create).  lambda = 0 gives the
 * symmetry-constrained SPAI.  Host FP64 set-up work; afterwards the SPD check and tau_CFL are
 * recomputed and the device copies refreshed, the state is kept.
 *   V        probe modes v_k (eigenmodes of M1^-1 P2 of interest), host, N1 x n_probe,
 *            column-major (mode k at V + k * N1), copied; may be NULL when n_probe = 0
 *   lambda   probing weight >= 0
 *   max_iter / tol  PCG stops when ||r|| <= tol ||r_0|| (relative residual of the system)
 *   iters, rel_residual  (may be NULL) PCG iterations run and the final relative residual
 * Where the SPAI is built in the entity-orthonormal basis (ygm_q1_info ortho = 1, orders >= 2),
 * the same system is solved for Q' = T^-T Q1 T^-1 with M' = T M1 T^T and probes T P2 v_k, and
 * Q1 = T^T Q' T keeps its pattern.  Errors: YGM_EINVAL (arguments), YGM_ETIMEOUT (PCG did not
 * converge within max_iter; Q1 unchanged), YGM_ENOTSPD (the previous Q1 is kept), YGM_ECUDA (the
 * device copies could not be refreshed: destroy the context).  Synchronises the context stream. */
int ygm_spai_op(ygm_ctx* ctx, const double* V, int32_t n_probe, double lambda, int32_t max_iter, double tol,
                int32_t* iters, double* rel_residual);

/* Probe modes for ygm_spai_op (Sec. 5.1: eigenmodes of K = M1^-1 P2 at the frequencies of
 * interest): the `count` lowest non-kernel eigenpairs of P2 v = omega^2 M1 v of this context's
 * exact FEEC operators (host FP64; the approximate Q1 is not involved).  Block shift-invert
 * subspace iteration in the M1 inner product, kept M1-orthogonal to ker C (interior vertex
 * gradients and the gradient 1-forms); each pair converges to
 * ||P2 v - omega^2 M1 v|| <= tol omega^2 ||M1 v||.
 *   V         host output, N1 x count column-major (mode k at V + k * N1), v^T M1 v = 1
 *   omega_sq  host output, count values, ascending
 *   iters     (may be NULL) outer iterations run
 * Degenerate eigenvalues return an M1-orthonormal basis of their eigenspace.  Cost: count + 4 or
 * more shifted CG solves per iteration, so it is meant for small and medium meshes.  Errors:
 * YGM_EINVAL (arguments, count above the number of non-kernel modes, an inner solve that failed),
 * YGM_ETIMEOUT (not converged within max_iter).  Does not touch the device. */
int ygm_cavity_modes(ygm_ctx* ctx, int32_t count, double* V, double* omega_sq, int32_t max_iter, double tol,
                     int32_t* iters);

/* Derivative of the column SPAI with respect to the per-tet permittivity (Eq. NormalEqSolve,
 * differentiated): given q1bar = dL/dQ1 for some scalar L, on the pattern of ygm_export_q1 (same
 * CSR order), returns grad_eps[t] = sum_ij q1bar_ij dQ1_ij / d eps_t for the 6 n^3 tets.
 * Q1 = (P + P^T) / 2 with P the column SPAI of M1(eps) = sum_T eps_T M1^T; per column l,
 * dq = (A^T A)^-1 (dA^T r - A^T dA q) with A = M1(:, I_l), r = 1_l - A q, dA = M1^T(:, I_l).
 * Dependences of L on eps other than through Q1 (e.g. an M1-weighted loss) are the caller's.
 * Orders >= 2 (ygm_q1_info ortho = 1) chain through the entity-orthonormal basis as well:
 * Q1 = T Q' T, Q' the column SPAI of M' = T M1 T, T = blockdiag (M1[g,g])^(-1/2) over the mesh
 * entities, its derivative taken in each block's eigenbasis.  Host FP64, reproducible for a given
 * thread count.  Q1 from ygm_set_q1 or ygm_spai_op is treated as if it were the column SPAI, which
 * it is not.  Errors: YGM_EINVAL, YGM_ENOTSPD. */
int ygm_q1_vjp(ygm_ctx* ctx, const double* q1bar, double* grad_eps);

/* Gradient of a probe-region field energy with respect to the per-tet permittivity, by the
 * discrete adjoint of the leapfrog (the transposed shear maps of Eq. shearMaps, newest step first)
 * on the device, chained through the SPAI derivative of ygm_q1_vjp on the host.  The paper defines
 * no loss; this one is
 *     L = dt sum_{n=0}^{nsteps-1} [1/2 x_n^T M1^R x_n + 1/2 b_{n+1/2}^T M2^R b_{n+1/2}],  x_n = Q1 e_n,
 * with M1^R, M2^R the mass matrices assembled over the tets t with region[t] != 0 only, for the
 * leapfrog run from rest (e_0 = 0, b = 0) under the given dipole sources (as ygm_step), dt fixed.
 * region: 6 n^3 bytes (tet order of ygm_create).  The forward run keeps the state every
 * checkpoint_every steps; the reverse sweep recomputes each segment from its checkpoint
 * (device memory: (nsteps / checkpoint_every) (N1 + N2) + checkpoint_every (2 N1 + N2) values,
 * plus one upper-triangle copy of Q1 for dL/dQ1).  Outputs: *loss; grad_eps[6 n^3] (may be NULL:
 * loss only, no host SPAI derivative).  Runs in the context precision.  Needs a one-column context
 * with uniform mu on the lattice path (YGM_EINVAL otherwise).  Overwrites the context state: it is
 * left at rest (e = b = 0, step 0).  Errors: YGM_EINVAL, YGM_ECFL, YGM_ECUDA, YGM_ENOMEM,
 * YGM_ENOTSPD (a normal matrix of the SPAI derivative). */
int ygm_adjoint(ygm_ctx* ctx, int64_t nsteps, double dt, const ygm_source* src, int32_t n_src, const uint8_t* region,
                int32_t checkpoint_every, double* loss, double* grad_eps);

/* ---- uneven batch: many independent cavities stepped by one persistent launch ----------------
 * The paper steps one field; batching independent cavities of different size n and order k is a
 * throughput pattern of this library.  Each member is a one-column context (its own mesh, eps,
 * Q1 and state, YGM_FP32 or YGM_FP64, all of one precision and device, uniform mu); the batch
 * holds pointers to them and they must outlive it.  One ygm_batch_step runs, for every member,
 * exactly the leapfrog of ygm_step (Eq. YeeLeapfrog in the form of Eq. preYeeFEECEqns, the
 * member's own dt and dipole), as a single cooperative kernel: per step three phases (Q1 e, the
 * b update, the e update with the source) over (cavity, block) work items separated by grid-wide
 * barriers whose waits have an iteration cap.  Members' states are read and written through the
 * usual per-context calls (ygm_set_state, ygm_get_state, ygm_energy).  Errors: YGM_EINVAL,
 * YGM_ENODEV, YGM_ECUDA, YGM_ENOMEM (creation messages via ygm_last_error(NULL)). */
typedef struct ygm_batch ygm_batch;
int ygm_batch_create(ygm_ctx* const* cavities, int32_t count, ygm_batch** out);
/* nsteps leapfrog steps of every member: dt[count] (each <= its tau_CFL, else YGM_ECFL and nothing
 * runs); src = NULL or one dipole per member (src[i].rhs ignored).  use_graph = 1 replays the
 * launch from a CUDA graph captured on first use (recaptured when nsteps or the launch shape
 * changes).  Asynchronous on the first member's stream, ordered after and before the members' own
 * streams; a barrier timeout is reported by ygm_batch_status. */
int ygm_batch_step(ygm_batch* batch, int64_t nsteps, const double* dt, const ygm_source* src, int32_t use_graph);
/* Synchronise and report a grid-barrier timeout of an earlier launch (YGM_ETIMEOUT; the flag stays
 * set until ygm_batch_status_clear).  After a timeout the members' states are invalid. */
int ygm_batch_status(ygm_batch* batch);
int ygm_batch_status_clear(ygm_batch* batch);
/* Polls (each ~0.1-1 us) a grid-barrier wait makes before it gives up; default 2^24.  0 makes every
 * wait that does not find the barrier already complete give up at once, which forces the timeout
 * path (used to test it). */
int ygm_batch_wait_limit(ygm_batch* batch, int64_t polls);
/* Autotuner: times trial_steps steps for every launch shape (1..4 CTAs per SM, within the
 * occupancy limit) and work order (0: cavity by cavity; 1: Q1 items longest stencil first, the
 * other phases interleaved across cavities), keeps the fastest, and restores every member's state
 * and time.  Outputs (may be NULL): the choice and its milliseconds per step. */
int ygm_batch_tune(ygm_batch* batch, int32_t trial_steps, const double* dt, const ygm_source* src, int32_t* ctas_per_sm,
                   int32_t* order, double* ms_per_step);
const char* ygm_batch_last_error(const ygm_batch* batch);
void ygm_batch_destroy(ygm_batch* batch);   /* NULL-safe; does not destroy the members */

/* ---- cubical Whitney GYM (the Yee scheme) on a periodic box: the structured-grid kernel family ----
 * Sec. 4: with cubical Whitney forms (average-normalised DoFs, Eq. WhitneyFormDefn), the curl of
 * Eq. dIsFiniteDiff (+-1/h), and diagonal Q1 and M2 (Eq. YeeMassMatrices: Q1 = Delta_V^-1 I,
 * M2 = Delta_V I), the GYM leapfrog is Yee's method.  Grid n[3] cubes with edge lengths h[3],
 * periodic; DoFs: x, y, z edges (e) and faces with x, y, z normals (b) anchored at each vertex
 * (i, j, k), index a * nc + i + n0 (j + n1 k), nc = n0 n1 n2.  q1, m2: 3 nc positive diagonal
 * values each (e.g. material weights or an S(1) SPAI), NULL for the lumped defaults.  The CFL bound
 * is the Gershgorin bound of lambda_max(Q1 C^T M2 C) (conservative; ygm_yee_sizes).  State and
 * staggering as for ygm_set_state / ygm_step / ygm_get_state; no sources.  Errors: YGM_EINVAL,
 * YGM_ECFL, YGM_ECUDA, YGM_ENOMEM; messages via ygm_yee_last_error (NULL for creation). */
typedef struct ygm_yee ygm_yee;
int ygm_yee_create(const int32_t n[3], const double h[3], const double* q1, const double* m2, int32_t precision,
                   int32_t device, void* stream, ygm_yee** out);
int ygm_yee_sizes(const ygm_yee* yee, int64_t* n1, int64_t* n2, double* dt_cfl);
int ygm_yee_set_state(ygm_yee* yee, const void* e, const void* b, int on_device);
int ygm_yee_step(ygm_yee* yee, int64_t n, double dt);
int ygm_yee_get_state(ygm_yee* yee, void* e, void* b, int on_device, int synced);
const char* ygm_yee_last_error(const ygm_yee* yee);
void ygm_yee_destroy(ygm_yee* yee);

/* SPD check of Q1 (Sec. 5.1, practical considerations): Lanczos estimates of the smallest and
 * largest eigenvalue before any shift, the diagonal shift applied (0 if none), lambda_max(Q1 P2),
 * and which pattern / basis was used (YGM_Q1_*, ortho = 1 for the orthogonalised basis). */
int ygm_q1_info(const ygm_ctx* ctx, double* lmin, double* lmax, double* shift, double* omega_max_sq,
                int32_t* pattern, int32_t* ortho);

/* Local reference blocks (FP64, identical for the 6 Kuhn shapes in local order):
 * M1 (n1 x n1), M2 restricted to the curl-carrying 2-forms (n2a x n2a), sizes in n1/n2a. */
int ygm_local_blocks(const ygm_ctx* ctx, int32_t* n1, int32_t* n2a, double* M1, double* M2a);

/* Q1 apply kernel of a one-column context (x = Q1 e of Eq. YeeLeapfrog on the upper-triangle
 * lattice: every value of the symmetric Q1 of Sec. 5 stored once per pair).  kernel: 0 = automatic
 * (per-thread loads, the faster of the two on GB300: 205 us against 284 us for one FP32 apply at
 * N = 32, k = 2), 1 = per-thread loads (k_qapply_s), 2 = bulk copies of each slot's run into
 * shared-memory stages by a producer warp (k_qapply_t; available where every run it copies lies
 * inside the stored lattice).
 * stages (kernel 0 or 2): 0 = as many as fit (at most 4), else 2..8.  Both kernels add the same
 * terms in the same order and give bit-identical x.  *blocks_per_sm (NULL allowed) receives the
 * selected kernel's resident blocks per SM.  Synchronises the context stream.  Errors: YGM_EINVAL
 * (kernel or stages out of range, kernel 2 unavailable, or a context with n_rhs > 1, which has
 * no upper-triangle path), YGM_ENODEV, YGM_ECUDA. */
int ygm_set_qapply(ygm_ctx* ctx, int32_t kernel, int32_t stages, int32_t* blocks_per_sm);

/* Launch mode of the one-column step's kernels (x = Q1 e, the b update, the e update of Eq.
 * YeeLeapfrog).  pdl = 1 (the default): each is launched with programmatic stream serialization,
 * so its blocks start and load their constant tables while the previous kernel finishes, then
 * wait for it before reading its output or writing anything; results are identical to pdl = 0,
 * ordinary stream-ordered launches.  Errors: YGM_EINVAL (pdl not 0 or 1), YGM_ENODEV. */
int ygm_set_launch(ygm_ctx* ctx, int32_t pdl);

/* Per-launch CUDA-event timing on the context stream: enable = 1 brackets every kernel launch
 * with a pair of events; ygm_kernel_times synchronises, returns the summed milliseconds and
 * launch counts of each kernel kind since the last query (kinds: 0 Q1 apply, 1 curl -> b,
 * 2 curl^T M2 -> e, 3 sources, 4 energy) into ms[5] / count[5], and clears the record. */
int ygm_kernel_timing(ygm_ctx* ctx, int enable);
int ygm_kernel_times(ygm_ctx* ctx, double* ms, int64_t* count);

/* Launch statistics: kernels launched by this context so far (all kernels of the library). */
int ygm_launch_count(const ygm_ctx* ctx, int64_t* count);

/* Sizes of one Q1 apply x = Q1 e, for roofline accounting (no compute, no device access).
 * all_rows = 1 describes the launch that computes every row (steps with an energy read-out and
 * ygm_energy); all_rows = 0 the launch of every other step, which computes only the rows of the
 * curl-carrying 1-forms: C has zero columns at the gradient 1-forms (Sec. 2, C G = 0), so C x
 * never reads the other rows.  rows: rows computed; unique_values: distinct Q1 values those rows
 * use, a symmetric pair counted once; stored_values: Q1 entries the kernel streams (full rows,
 * zeros at neighbours outside the mesh, plane padding).  NULL outputs are skipped.
 * Returns YGM_EINVAL for a NULL context, YGM_ENODEV for a host-only one. */
int ygm_qapply_counts(const ygm_ctx* ctx, int all_rows, int64_t* rows, int64_t* unique_values,
                      int64_t* stored_values);

/* Message of the last failure on this context (or of the last failed ygm_create when ctx is
 * NULL).  Valid until the next call on the same context. */
const char* ygm_last_error(const ygm_ctx* ctx);

/* Free the context and its device memory; NULL-safe.  Synchronises the stream. */
void ygm_destroy(ygm_ctx* ctx);

#ifdef __cplusplus
}
#endif

#endif /* YGM_H */
