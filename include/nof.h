/*
 * nof.h - C ABI of the GB300 library for the density-fitted PNOF JK step.
 *
 * The operation follows DoNOF 2.0 (Lew-Yee, Mitxelena, del Campo, Piris, arXiv 2512.13550):
 * a closed-shell natural-orbital-functional energy E[{n_p, phi_p}] (Theory section, Eq. ENOF)
 * in its JKL-only form (Eq. PNOF) over the electron-pairing structure of Eq. OmegaG / Fig. 1,
 * with occupations from the trigonometric gamma mapping (Occupation Number Optimization
 * subsection), the Lagrangian and orbital gradient g = 4(lambda - lambda^T) and the orbital
 * rotation C <- C exp(y) (Natural Orbital Optimization subsection), with the two-electron
 * integrals approximated by the resolution of the identity (ERITYP='RI', Single Point
 * Energy section).
 *
 * Conventions for every entry point:
 *  - Return value: NOF_OK (0) or a negative NOF_E* code. Nothing aborts or throws across the
 *    ABI; nof_last_error() returns a thread-local message for the last failure.
 *  - Array arguments are DEVICE pointers owned by the caller, FP64, row-major, unless the
 *    comment says "host". Calls are asynchronous on the stream given to nof_create; the
 *    caller synchronises (or calls nof_sync) before reading results.
 *  - Orbital coefficients: C is nbf x nbf, C[mu * nbf + p] = C_mu,p, so
 *    phi_p = sum_mu C_mu,p chi_mu. Columns are orbitals and must be S-orthonormal for the
 *    energy to be the functional's.
 *  - Orbitals 0 .. nact-1 are active (nonzero occupation); nact = (N/2)(ncwo + 1).
 *  - gamma has ngamma = (N/2) ncwo entries stored slot-major: gamma[i * (N/2) + g] is the
 *    variable of slot i of subspace g. Trigonometric mapping: slot 0 is the strong orbital's
 *    angle gamma_g and slot i the angle of weak orbital p_i. Softmax mapping: slot i is the
 *    variable of weak orbital p_{i+1}.
 *  - The library owns only its workspaces (allocated by nof_build_B, freed by nof_destroy).
 */
#ifndef NOF_H
#define NOF_H

#ifdef __cplusplus
extern "C" {
#endif

#define NOF_OK 0
#define NOF_EINVAL -1      /* bad argument: null pointer, size, option, unsupported system */
#define NOF_ENOMEM -2      /* device allocation failed */
#define NOF_ECUDA -3       /* a CUDA runtime call failed (message has the CUDA error) */
#define NOF_ETIMEOUT -4    /* a bounded device-side wait gave up */
#define NOF_ENONFINITE -5  /* NaN or Inf found in an input or a result */
#define NOF_EILLCOND -6    /* the aux Coulomb metric is numerically singular */
#define NOF_ENOTCONV -7    /* an iteration did not converge */
#define NOF_ESTATE -8      /* call out of order (e.g. nof_jk before nof_build_B) */

/* Arithmetic of the JK / Lagrangian contractions. */
#define NOF_PREC_FP64 0       /* plain FP64 SIMT kernels */
#define NOF_PREC_SPLIT_BF16 1 /* tcgen05 tensor cores on exact BF16 digit planes (4 or 5 base-256
                                 digits per element, about 32 or 40 significant bits; FP32 exact
                                 partial sums) */

typedef struct nof_ctx nof_ctx;

/* Functional and optimiser options. Field names follow the paper's input keywords where one
 * exists (IPNOF, ISOFTMAX, NCWO = N_g of Eq. OmegaG). */
typedef struct {
    int ipnof;        /* 7 = PNOF7 (default), 5 = PNOF5 */
    int isoftmax;     /* ON mapping (Occupation Number Optimization subsection): 0 = trigonometric
                         (default); 1 = softmax, n_g = 1 / (1 + sum_k exp(gamma_{p_k})) and
                         n_{p_i} = n_g exp(gamma_{p_i}), which does not keep n_g >= 1/2 */
    int ncwo;         /* N_g, weak orbitals per subspace (>= 1) */
    int precision;    /* NOF_PREC_FP64 or NOF_PREC_SPLIT_BF16 */
    int on_iters;     /* steepest-descent ON steps per nof_step (default 20) */
    double on_lr;     /* ON step length (default 0.3) */
    double lr;        /* ADAM learning rate for the orbital rotation (default 0.02) */
    double b1, b2;    /* ADAM moment decays (default 0.9, 0.999) */
    double eps;       /* ADAM epsilon (default 1e-8) */
    int digits;       /* NOF_PREC_SPLIT_BF16 only: BF16 digits per element, 4 or 5; 0 (default)
                         chooses 5 when naux * nact > 80000 (where the truncation error of 4
                         digits, accumulated over the naux * nact terms of the Lagrangian, nears
                         1e-6), else 4 */
    int graphs;       /* 1 (default): the second nof_energy_grad call with a set of pointers among
                         the last four sets of direct calls records its kernels as a CUDA graph on
                         the context's stream, and later calls with those pointers replay it (one
                         launch instead of about 20). Up to four graphs are kept (the least
                         recently used is replaced), so a caller may alternate between buffer
                         sets, e.g. to overlap its copies with the evaluations. A graph reads the
                         arrays, so their contents may change between calls. 0: every call
                         launches its kernels one by one.
                         No graph is recorded on the legacy default stream (stream 0), while
                         nof_profile is on, or while the caller is capturing the stream. */
} nof_options;

/* s-only contracted basis repeated on every atom (host arrays). Shell s has nprim[s]
 * primitives; exponents and contraction coefficients are concatenated over shells.
 * Primitives are normalised, then each contraction is renormalised. For an auxiliary
 * basis every primitive is its own (uncontracted) function and coefs are ignored. */
typedef struct {
    int nshell;
    const int* nprim;      /* host [nshell] */
    const double* exps;    /* host [sum nprim] */
    const double* coefs;   /* host [sum nprim] */
} nof_basis;

/* Fill opt with the defaults listed above. */
void nof_default_options(nof_options* opt);

/* Create a context on the current CUDA device. stream is a cudaStream_t (NULL = legacy
 * default stream); every kernel of this context runs on it. */
int nof_create(nof_ctx** out, const nof_options* opt, void* stream);

/* Free the context and all of its device workspaces. Safe on NULL. */
int nof_destroy(nof_ctx* ctx);

/* Set-up for one geometry (the integral / RI stage of the Single Point Energy section,
 * ERITYP='RI'): computes on the device S, H = T + V, V_nn, the three-centre integrals
 * (P|mu nu), the Coulomb metric (P|Q) and its Cholesky factor L, and stores
 * B^P_{mu nu} = sum_Q (L^{-1})_{PQ} (Q|mu nu) in the format the precision option needs.
 * xyz: host [natom][3] bohr; Z: host [natom] nuclear charges (NULL = all 1).
 * Only closed-shell singlets: mult must be 1 and sum(Z) - charge even and positive.
 * Returns NOF_EILLCOND if a pivot of the metric falls below 1e-14 of its largest diagonal. */
int nof_build_B(nof_ctx* ctx, int natom, const double* xyz, const double* Z, int charge,
                int mult, const nof_basis* orb, const nof_basis* aux);

/* Sizes of the built system (any pointer may be NULL). vnn is copied to the host
 * (synchronises the stream). */
int nof_query(nof_ctx* ctx, int* nbf, int* naux, int* nact, int* ngamma, double* vnn);

/* Copy S and H (nbf x nbf) into caller device buffers. */
int nof_get_SH(nof_ctx* ctx, double* S, double* H);

/* Copy the fitted tensor B as FP64 [naux][nbf][nbf] (reconstructed from the stored digit
 * planes under NOF_PREC_SPLIT_BF16). Used to check sum_P B^P B^P against exact ERIs. */
int nof_get_B(nof_ctx* ctx, double* B);

/* Launch shapes the autotuner chose at nof_build_B for the split path (no paper counterpart):
 * out[0..3] (host) = N-tile widths of the three digit GEMMs (half transform, full transform,
 * Lagrangian contraction) and the Lagrangian's split-K chunk in K atoms of 16.
 * NOF_EINVAL unless the context is built with NOF_PREC_SPLIT_BF16. */
int nof_tuned_tiles(nof_ctx* ctx, int* out);

/* Digits per element of the split path's operands (4 or 5: the option `digits`, or the automatic
 * choice at nof_build_B) into *nd (host); no paper counterpart. A digit GEMM then makes
 * nd (nd + 1) / 2 BF16 products per K atom and reads 2 nd bytes per operand element.
 * NOF_EINVAL unless the context is built with NOF_PREC_SPLIT_BF16. */
int nof_split_digits(nof_ctx* ctx, int* nd);

/* C = S^{-1/2} Q (Loewdin orthonormalisation, S^{-1/2} by a Newton-Schulz iteration on the
 * device). Q: nbf x nbf orthogonal. Gives S-orthonormal orbitals for any orthogonal Q. */
int nof_lowdin(nof_ctx* ctx, const double* Q, double* C);

/* Core-Hamiltonian starting orbitals: C0 = X U with X = S^{-1/2} (Newton-Schulz) and U the
 * eigenvectors of X^T H X in ascending order of the eigenvalues (cyclic Jacobi on the device).
 * eps (device, nbf; may be NULL) receives the eigenvalues. Columns of C0 are S-orthonormal.
 * Degenerate eigenvalues leave the basis of their subspace arbitrary. */
int nof_core_guess(nof_ctx* ctx, double* C0, double* eps);

/* J_pq = sum_P b^P_pp b^P_qq and K_pq = sum_P (b^P_pq)^2 over the active orbitals, with
 * b^P = C_a^T B^P C_a (the orbital transformation of the RI tensor; Eq. PNOF uses J and K,
 * and L = K for real orbitals). J, K: nact x nact. */
int nof_jk(nof_ctx* ctx, const double* C, double* J, double* K);

/* One energy+gradient evaluation at fixed (C, gamma):
 *   E       (1 double)      the PNOF energy of Eq. PNOF plus V_nn;
 *   g_orb   (nbf x nbf)     g_pq = dE/dy_pq = 4 (lambda_pq - lambda_qp) for C' = C exp(y);
 *   g_gamma (ngamma)        dE/dgamma through the trigonometric mapping.
 * Any output pointer may be NULL to skip copying it (E is always computed). */
int nof_energy_grad(nof_ctx* ctx, const double* C, const double* gamma, double* E,
                    double* g_orb, double* g_gamma);

/* One alternating optimisation step, in place:
 *   1. J, K, h_pp at C;  2. on_iters ON steps gamma -= on_lr dE/dgamma with J, K fixed;
 *   3. E, lambda, g at (C, gamma);  4. ADAM on g (moments m, v: nbf x nbf, step counter *t
 *   on the host, incremented);  5. C <- C exp(y) (Taylor-12 scaling and squaring).
 * out (device, 3 doubles): E at (C_old, gamma_new), ||g||_F, max |lambda - lambda^T|.
 * t == NULL selects a step that can be captured in a CUDA graph: the step counter is a device
 * integer owned by the context (zero after nof_build_B, advanced on the device), and exp(y) is
 * scaled by a fixed 2^-12 with 12 squarings instead of a scaling read back to the host. Such a
 * step makes no host synchronisation and no host-side state change; a rotation with
 * ||y||_F > 4096 is reported by nof_sync as NOF_ENOTCONV. */
int nof_step(nof_ctx* ctx, double* C, double* gamma, double* m, double* v, int* t, double* out);

/* ---- Converged optimisation loop --------------------------------------------------------- */

/* Parameters of nof_optimize (defaults from nof_default_opt_params). */
typedef struct {
    int maxit;        /* outer iterations at most (default 1000) */
    int maxloop;      /* ADAM orbital steps per outer iteration (default 10) */
    double gtol;      /* stop when ||g||_F < gtol ... (default 1e-5) */
    double etol;      /* ... and |E_k - E_{k-1}| < etol (default 1e-8 Ha) */
    double lr;        /* initial ADAM rate (default 0.02) */
    double lr_min;    /* also stop once the rate falls below this (default 1e-12) */
    double on_tol;    /* ON optimisation: max |dE/dgamma| at convergence (default 1e-8) */
    int on_maxit;     /* ON optimisation: BFGS steps at most per outer iteration (default 500) */
    double eps_rel;   /* ADAM's epsilon in a block is max(the context's eps, eps_rel ||g_k||_F) (default 0) */
    double lr_grow;   /* the rate is multiplied by this (>= 1) after a block that found better orbitals
                         (default 1) */
    int orbopt;       /* orbital steps: 0 ADAM blocks only; 1 L-BFGS only; 2 (default) ADAM blocks until
                         the rate falls below lr * lbfgs_after, then L-BFGS steps */
    int memory;       /* L-BFGS pairs kept (1..64, default 20) */
    double lbfgs_after; /* see orbopt (default 1/64) */
} nof_opt_params;

void nof_default_opt_params(nof_opt_params* p);

/* The converged ON / NO optimisation: the paper optimises the ONs and the orbitals separately
 * (Theory section, after Eq. sum1), the orbitals by rotations with ADAM on g = 4(lambda - lambda^T)
 * (Natural Orbital Optimization subsection), until the lambda-symmetry and energy thresholds hold
 * (NTHRESHL / NTHRESHE, Single Point Energy section). The ADAM details are delegated by the paper;
 * this loop is the reading the oracle implements. Outer iteration k:
 *   1. J, K, h_pp at C_k; the ONs converged at fixed J, K: BFGS on gamma with an Armijo step
 *      control to max |dE/dgamma| < on_tol (one CUDA block);
 *   2. E_k, lambda, g_k at (C_k, gamma_k); stop when ||g_k||_F < gtol and |E_k - E_{k-1}| < etol;
 *   3. maxloop ADAM steps on the orbitals from zero moments (the context's b1, b2, eps) with
 *      gamma_k fixed, each a full evaluation; the best orbitals (energy lower by more than etol,
 *      or equal within etol with ||g|| at most 0.9 of the best) become C_{k+1}; if no step is
 *      better than (E_k, ||g_k||) the rate halves, and the loop ends once the rate is below
 *      lr_min. With orbopt 2, once the rate is below lr * lbfgs_after (ADAM's normalised steps
 *      then make little progress), every outer iteration takes instead one L-BFGS step on the
 *      rotation generators (two-loop recursion over the last `memory` pairs, <A,B> = sum_{p<q}
 *      A_pq B_pq; step length halved from 1 until an Armijo decrease, or, where the predicted
 *      decrease is below etol, a smaller ||g|| with the energy within etol; a failed search
 *      retries from steepest descent, then halves the rate). orbopt 1 takes L-BFGS steps from
 *      the start (the first one -g lr / max|g|).
 * C (device, nbf x nbf) and gamma (device, ngamma) are the start and receive the final state.
 * history: host [maxit][3] of (E_k, ||g_k||_F, lr_k) per outer iteration, or NULL.
 * result: host [8]: final E, ||g||_F, max |lambda - lambda^T|, outer iterations, evaluations,
 * converged (1 or 0), final rate, total ON (BFGS) steps. Synchronises the context's stream after
 * every evaluation (three doubles read back). Workspaces (6 nbf^2 + ngamma^2 + 6 ngamma doubles)
 * are allocated on the first call and freed with the context. Errors: NOF_EINVAL (null pointer,
 * bad parameter), NOF_ESTATE, NOF_ENOMEM, NOF_ENONFINITE (a NaN or Inf energy or gradient; the
 * device status word is cleared, since the return value reports it). */
int nof_optimize(nof_ctx* ctx, double* C, double* gamma, const nof_opt_params* params, double* history,
                 double* result);

/* Batched evaluation (the batching of many geometries): `count` independent contexts, each built
 * with its own geometry and created on its own stream, evaluate nof_energy_grad concurrently.
 * The call forks from `stream` (a cudaStream_t) onto every context's stream with events and joins
 * back, so capturing `stream` in a CUDA graph captures the whole batch as one graph launch. The
 * pointer arrays are host arrays of `count` device pointers (C, gamma, E required; g_orb and
 * g_gamma may be NULL or hold NULL entries). Results equal those of the same instances evaluated
 * one by one. */
int nof_energy_grad_batch(nof_ctx* const* ctxs, int count, const double* const* C,
                          const double* const* gamma, double* const* E, double* const* g_orb,
                          double* const* g_gamma, void* stream);

/* ---- Nuclear gradient ----------------------------------------------------------------- */

/* dE/dR (atomic units, device array [natom][3]) of the RI-PNOF energy at the state (C, gamma),
 * for the geometry optimisation and dynamics the paper lists among DoNOF's capabilities (the
 * paper prints no formula). The orbitals follow the nuclei through the connection
 * C(x) = C (C^T S(x) C)^{-1/2}, which keeps them orthonormal:
 *   dE/dx = sum P h^x - 2 sum (C lambda C^T) S^x + sum_P sum Gamma^P (uv|P)^x - sum Z V^x + V_nn^x
 * with the one-particle density P = 2 C diag(n) C^T, the Lagrangian lambda of nof_energy_grad,
 * Gamma^P = C Y^P C^T and Z from the fitting coefficients c = V^-1 (Q|pq)
 * (Y^P_pq = 2 delta_pq sum_r A_pr c^P_rr - 2 B_pq c^P_pq, Z_PQ = sum A_pq c^P_pp c^Q_qq -
 * B_pq c^P_pq c^Q_pq). At a converged state this is the physical force (negated). Integral
 * derivatives of the s Gaussians are evaluated on the fly; the sums run in a fixed order.
 * NOF_PREC_FP64 contexts only. Workspaces (about X nbf^2 doubles) are allocated on the first
 * call. Stream-ordered. Errors: NOF_EINVAL (null pointer, split-precision context),
 * NOF_ESTATE, NOF_ENOMEM. */
int nof_nuclear_gradient(nof_ctx* ctx, const double* C, const double* gamma, double* grad);

/* ---- Finite-field polarizability and hyperpolarizabilities (NLOPs subsection) ------------ */

/* Static electric field F (atomic units, host array of 3: x, y, z), the EVEC input of the
 * NLOPs subsection. The Hamiltonian gains -mu.F with mu = -sum_i r_i + sum_A Z_A R_A: every
 * later evaluation and step of the context uses h + F.<mu|r|nu> and V_nn - F.sum_A Z_A R_A.
 * F = (0, 0, 0) restores the field-free values exactly. The dipole integrals (s Gaussians: the
 * product-centre times the overlap of each primitive pair) are computed on the first call.
 * Stream-ordered. Errors: NOF_EINVAL (null pointer, non-finite F), NOF_ESTATE (before
 * nof_build_B), NOF_ENOMEM. */
int nof_set_field(nof_ctx* ctx, const double* F);

/* Dipole moment of the state (C, gamma): mu_k = -2 sum_p n_p <phi_p|r_k|phi_p> + sum_A Z_A R_A,k
 * for k = x, y, z: the expectation value with the one-particle density matrix of the
 * functional, which is diagonal in the natural orbitals (NLOPs subsection). C, gamma: device
 * arrays as for nof_energy_grad; mu: device array of 3 doubles. Stream-ordered; the sums run in
 * a fixed order. Errors: NOF_EINVAL, NOF_ESTATE, NOF_ENOMEM. */
int nof_dipole(nof_ctx* ctx, const double* C, const double* gamma, double* mu);

/* Centred finite differences of order h^2 at the dyadic steps h_k = step 2^{k-1},
 * k = 1 .. npoint (NLOPs subsection), from dipoles at the 2 npoint + 3 distinct fields in the
 * order 0, h_1 .. h_{npoint+1}, -h_1 .. -h_{npoint+1} (2 h_k = h_{k+1}):
 *   alpha(h) = (mu(h) - mu(-h)) / (2h),  beta(h) = (mu(h) - 2 mu(0) + mu(-h)) / h^2,
 *   gamma(h) = (mu(2h) - 2 mu(h) + 2 mu(-h) - mu(-2h)) / (2 h^3).
 * Host arrays: mu [2 npoint + 3], alpha, beta, gamma [npoint]. No device work.
 * Errors: NOF_EINVAL (null pointer, npoint < 1, step <= 0). */
int nof_field_differences(const double* mu, int npoint, double step, double* alpha, double* beta,
                          double* gamma);

/* Romberg-Richardson triangle with p = 2 (NLOPs subsection) of D[k-1] = D(h_k), k = 1 .. npoint:
 * R(k, 1) = D(h_k), R(k, j) = R(k, j-1) + (R(k, j-1) - R(k+1, j-1)) / (4^{j-1} - 1) for
 * k <= npoint - j + 1. R: host [npoint][npoint], R[(k-1) npoint + j-1] = R(k, j), the other
 * entries NaN. Selection: over every column j and vertical pair (k, k+1) of it, the smallest
 * Delta = |R(k+1, j) - R(k, j)| selects R(k, j+1); equal Deltas go to the smaller |value|.
 * best[0] = value, best[1] = Delta; sel[0], sel[1] = the selecting pair's k and j (1-based).
 * With npoint = 1, best = (D[0], NaN) and sel = (1, 1). No device work.
 * Errors: NOF_EINVAL (null pointer, npoint < 1). */
int nof_romberg(const double* D, int npoint, double* R, double* best, int* sel);

/* ISOALPHA (NLOPs subsection): from the diagonal polarizabilities a[0..2] = alpha_xx, alpha_yy,
 * alpha_zz, out[0] = (axx + ayy + azz) / 3 and out[1] = sqrt(((axx - ayy)^2 + (ayy - azz)^2 +
 * (azz - axx)^2) / 2) (the anisotropy, Raman convention). Host arrays; no device work.
 * Errors: NOF_EINVAL (null pointer). */
int nof_polarizability_invariants(const double* a, double* out);

/* nof_step on `count` contexts at once (the independent field instances of the finite-field
 * workload): each context on its own stream, forked from `stream` and joined back with events,
 * as nof_energy_grad_batch. Host arrays of `count` pointers: C, gamma, m, v, out (device) and
 * t (host step counters); t itself may be NULL, selecting every context's device-side counter
 * (see nof_step), so that capturing `stream` captures the whole batched step as one CUDA graph.
 * Errors: as nof_step; NOF_EINVAL for a bad count or a null entry. */
int nof_step_batch(nof_ctx* const* ctxs, int count, double* const* C, double* const* gamma,
                   double* const* m, double* const* v, int* const* t, double* const* out, void* stream);

/* Learned starting guess (no counterpart in the paper, which only notes that its Python version
 * suits machine-learning workflows): a perceptron x (F) -> relu (H) -> relu (H) -> y (O) in FP32
 * with hand-written kernels. Parameters theta are packed W1 [H][F], b1 [H], W2 [H][H], b2 [H],
 * W3 [O][H], b3 [O] (nof_mlp_param_count floats). X: [B][F], Y and T: [B][O], all device FP32,
 * row-major. work: device scratch of nof_mlp_work_size(B, H, O) floats owned by the caller.
 * nof_mlp_loss_grad writes loss = mean over the batch of sum_o (y - t)^2 (device scalar, may be
 * NULL) and its gradient (packed like theta). nof_mlp_adam takes one bias-corrected Adam step
 * with decoupled weight decay wd (t >= 1 is the step count) on P parameters in place. */
/* BF16 inference on the tensor cores: nof_mlp_to_bf16 converts the P packed FP32 parameters to BF16
 * (theta_bf16: device, P 16-bit values, owned by the caller); nof_mlp_forward_bf16 then computes Y
 * like nof_mlp_forward with every layer a BF16 x BF16 product (mma.sync m16n8k16, FP32
 * accumulation; activations rounded to BF16 as each layer loads them, biases in FP32 from theta).
 * work: device scratch of 2 B H floats. */
int nof_mlp_to_bf16(long long P, const float* theta, void* theta_bf16, void* stream);
int nof_mlp_forward_bf16(int B, int F, int H, int O, const void* theta_bf16, const float* theta, const float* X,
                         float* Y, float* work, void* stream);
long long nof_mlp_param_count(int F, int H, int O);
long long nof_mlp_work_size(int B, int H, int O);
int nof_mlp_forward(int B, int F, int H, int O, const float* theta, const float* X, float* Y, float* work,
                    void* stream);
int nof_mlp_loss_grad(int B, int F, int H, int O, const float* theta, const float* X, const float* T,
                      float* loss, float* grad, float* work, void* stream);
int nof_mlp_adam(long long P, float* theta, const float* grad, float* m, float* v, int t, float lr, float b1,
                 float b2, float eps, float wd, void* stream);

/* Wait for the context's stream and report any device-side status word. */
int nof_sync(nof_ctx* ctx);

/* Measurement hooks (no paper counterpart; used by the benchmark):
 * nof_kernel_launches: number of kernels this library has launched in the process so far.
 * nof_profile: CUDA-event timing, on the context's stream, of one contraction of every later
 *   evaluation: enable = 1 the half transform T = B C (the default), 2 the full transform
 *   b = C^T T (split path), 3 the Lagrangian contraction sum_P T^P W^P (split path); 0 turns it
 *   off. Any call clears the accumulated record; other values are NOF_EINVAL.
 * nof_profile_read: synchronise and return the accumulated device time (ms) and launch count
 *   of the timed contraction, and its kernel's name (static string; may be NULL). */
long long nof_kernel_launches(void);
int nof_profile(nof_ctx* ctx, int enable);
int nof_profile_read(nof_ctx* ctx, double* ms, int* launches, const char** name);

/* Self-test of the exact BF16 digit-plane tensor-core GEMM (no paper counterpart): random
 * digit planes (M x K and N x K, K = 16 katoms, nd = 4 or 5 digits) multiplied on tcgen05 with
 * N tiles of `bn` columns (16, 32, 48, 64, 80 or 96) and K chunks of
 * `chunk_atoms` atoms (integer atomics when chunk_atoms < katoms; the last chunk may be
 * shorter), and by a SIMT integer reference; *max_abs_diff (host) receives the largest
 * difference of the exact fixed-point results (0 when correct). The same product then runs twice
 * more with tiles taken dynamically from a fetch-and-add counter (the second launch checks that
 * the first left the counter at zero), each entering the same comparison. With one K chunk and
 * an even N the product is also written in the scaled double-float mode (random row and column
 * exponents in [-6, 6]), and, when katoms is a multiple of digit_scale_part_atoms(nd), in the
 * per-part FP64 mode with every part's exponents equal to those: a scaled value further than
 * 2^-38 of the largest |V| the shape allows from the exact V sets *max_abs_diff to 2^62.
 * Allocates and frees its own buffers; synchronises the device. */
int nof_selftest_digit_gemm(int M, int N, int bn, int nd, int katoms, int chunk_atoms, unsigned int seed,
                            long long* max_abs_diff);

/* Device time of one launch of the digit GEMM on zero operands (no paper counterpart;
 * measurement only): M x N output, N tiles of bn, nd digits, K = 16 katoms in chunks of
 * chunk_atoms. mode 0: exact int64 output (split-K atomics when chunk_atoms < katoms);
 * 1: scaled double-float output (one chunk); 2: per-part scales with an FP64 partial per K chunk
 * (chunk_atoms a multiple of digit_scale_part_atoms: 20 atoms with 5 digits, 8 with 4). Flags
 * added to `mode`: 4 = each launch timed alone after a 256 MiB write (L2 flushed, operands from
 * HBM); 8 = tiles taken dynamically from a
 * fetch-and-add counter instead of round-robin. One warm-up, then the mean of `reps` launches
 * timed with CUDA events on the default stream into *us_per_launch (host). Allocates and frees
 * its own buffers (the flush buffer is kept for the life of the process). */
int nof_bench_digit_gemm(int M, int N, int bn, int nd, int katoms, int chunk_atoms, int mode, int reps,
                         double* us_per_launch);

/* Failure detection of the digit GEMM (no paper counterpart): one launch of the M x N x 16 katoms
 * product whose producer issues no copies, so that its consumers' bounded waits run out. Every
 * mbarrier wait of the kernel is bounded by limit_ms (0 < limit_ms <= 1000); on a timeout the
 * kernel sets its status word and returns, and nothing it issued is left in flight. Returns
 * NOF_ETIMEOUT when the kernel reported the timeout (the expected outcome), with the launch's
 * device time in *elapsed_ms (host). Allocates and frees its own buffers; synchronises. */
int nof_selftest_digit_gemm_timeout(int M, int N, int bn, int nd, int katoms, double limit_ms,
                                    double* elapsed_ms);

/* J and K exactly as nof_jk computes them in FP64, without a context and without allocating
 * any device memory (the paper has no counterpart; this is a deployment variant).
 * Some callers cannot call cudaMalloc: an application whose device memory is owned by another
 * allocator (a framework's caching pool that has reserved the GPU, or a fixed memory budget),
 * or code that must not stall or fail on an allocation mid-run. This entry point keeps its
 * scratch in a fixed 48 MiB device array inside the library and only launches kernels on
 * `stream` (a cudaStream_t; NULL = default).
 *   B: device FP64 [naux][nbf][nbf] RI tensor (e.g. from nof_get_B); C: device FP64
 *   [nbf][nbf] orbitals (first nact columns used); J, K: device FP64 [nact][nact] outputs.
 * Limits: naux*nbf*nact + naux*nact*(nact + 1) <= 6291456 doubles, naux <= 65535 and
 * naux*nbf <= 65535*64; beyond them NOF_EINVAL before anything is queued.
 * When the 48 MiB are reserved: CUDA loads the library's modules lazily by default, so the
 * array is reserved on a device by the first call made with that device current (with eager
 * module loading, when the library is loaded); it stays reserved until the process exits.
 * A caller that later hands the GPU to its own pool or budget should make one call first.
 * That first call also looks up the array's device address; make it before any stream
 * capture. The address is cached per device index: do not call this again on a device after
 * cudaDeviceReset (or another teardown of its primary context) in the same process.
 * Calls share the array: calls that overlap on the GPU race. Asynchronous like every other
 * call. */
int nof_jk_static(int naux, int nbf, int nact, const double* B, const double* C, double* J,
                  double* K, void* stream);

/* Thread-local description of the last error (never NULL). */
const char* nof_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* NOF_H */
