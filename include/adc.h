/*
 * adc.h -- C ABI of the GB300 spin-adapted, density-fitted EA/IP-ADC(n) library
 * (n = 2, 3): setup of the static blocks, the Davidson sigma-vector build
 * sigma = M X, and the Davidson eigensolver with spectroscopic factors.
 *
 * Method: Banerjee & Sokolov, single-reference ADC for charged excitations.
 *   - M and T matrices: Sec. II A, Eqs. M_ea, M_ip, T_ea, T_ip (orders k+l+m = n).
 *   - Algorithm steps (amplitudes -> 1p-1p/1h-1h block -> Davidson sigma loop ->
 *     spectroscopic factors): Sec. III A, step list and Table 1.
 *   - Spin adaptation (closed shells): Sec. III B, Eqs. M_ij ... sigma_jka_bab,
 *     with the renormalisation of the Appendix (Eqs. appendix_1..4).
 *   - Density fitting (pq|rs) = sum_Q B^Q_pq B^Q_rs: Sec. III C, Eq. 19.
 *
 * Conventions
 *   - Orbitals: nmo = nocc + nvir spatial orbitals, occupied first.
 *   - eps[nmo]: orbital energies (Eh), diagonal Fock operator (H(0) of the
 *     Moller-Plesset partitioning).
 *   - Bq[naux][nmo][nmo]: density-fitting factors, row-major, symmetric in the
 *     last two indices (only the symmetric part is meaningful).
 *   - kind: ADC_EA (+1) or ADC_IP (-1).  order: 2 or 3.
 *   - Spin-adapted vector layout (length adc_dim):
 *       EA  [ Y_a (nvir) | Y_iab (nocc*nvir*nvir, b fastest) ]
 *       IP  [ Y_i (nocc) | Y_ija (nocc*nocc*nvir, a fastest) ]
 *     The metric of this basis is S = diag(1, 2 - P) where P swaps the two
 *     like indices (Appendix norm); M is S-symmetric.
 *   - Energies are eigenvalues w of the matrix the library applies:
 *       EA  M_+ (w = E_{N+1} - E_N; the paper's electron affinity is -w),
 *       IP  -M_- (w = E_{N-1} - E_N, the ionisation energy).
 *   - Spectroscopic factors use the Appendix normalisation (P = 2 sum_p X_p^2,
 *     so a Koopmans state has P = 2), with T through the method's order n
 *     (transition_order selects second order also for ADC(3)).
 *
 * Ownership: all inputs are caller-owned and copied; the handle owns every
 * device allocation it makes and releases it in adc_destroy.  Pointers marked
 * "host" are host memory; with on_device = 1 the vector arguments of
 * adc_sigma are device pointers (current device, row-major [nvec][dim]).
 * Work is issued on the handle's stream (adc_set_stream; default stream 0)
 * and every call returns after its work has completed on that stream.
 *
 * Errors: every int-returning call returns ADC_OK (0) or a negative code; the
 * message of the last failure is available from adc_last_error.  No C++
 * exception crosses the ABI.  A failed handle stays valid for adc_destroy.
 */
#ifndef GB300_ADC_H
#define GB300_ADC_H

#ifdef __cplusplus
extern "C" {
#endif

#define ADC_OK 0
#define ADC_ERR_ARG (-1)            /* invalid argument or size               */
#define ADC_ERR_OOM (-2)            /* device allocation failed               */
#define ADC_ERR_CUDA (-3)           /* CUDA runtime / cuBLAS failure          */
#define ADC_ERR_NOT_CONVERGED (-4)  /* Davidson hit max_iter; outputs filled  */
                                    /* with the best estimates                */
#define ADC_ERR_TIMEOUT (-5)        /* a bounded device wait gave up; the     */
                                    /* kernel returned and the handle stays   */
                                    /* usable (the device flag is cleared at  */
                                    /* the start of the next call)            */
#define ADC_ERR_NONFINITE (-6)      /* a non-finite value: in a guess vector, */
                                    /* or a Ritz value / residual (non-finite */
                                    /* sigma, e.g. from non-finite inputs)    */

#define ADC_EA 1
#define ADC_IP (-1)

#define ADC_PREC_FP64 0   /* every contraction in FP64                              */
#define ADC_PREC_BF16X3 1 /* DF ladder on tcgen05 tensor cores with hi/lo BF16       */
                          /* operands (3 products), FP32 accumulation (partial sums */
                          /* promoted to round-to-nearest FP32 registers) within an */
                          /* auxiliary chunk, FP64 across chunks; the large other   */
                          /* contractions on the same kernel in sigma and FP32-     */
                          /* accurate (BF16x9 emulated GEMM) in setup; FP64 vectors,*/
                          /* subspace and accumulation; converged roots refined     */

typedef struct adc_handle adc_handle; /* opaque */

typedef struct {
    int precision;           /* ADC_PREC_FP64 (default) or ADC_PREC_BF16X3            */
    int max_space_per_root;  /* Davidson subspace limit per root (default 8)          */
    int max_iter;            /* Davidson iteration limit (default 100)                */
    int nguess_extra;        /* extra guess vectors beyond nroots (default 2)         */
    double res_tol;          /* S-norm residual tolerance; <= 0 means sqrt(tol)       */
    int aux_chunk;           /* auxiliary functions per chunk of the ladder and of    */
                             /* the t1(3) contraction; 0 = automatic                  */
    int keep_per_root;       /* Ritz vectors kept per root when the space is          */
                             /* collapsed (thick restart, default 2)                  */
    int contractions;        /* non-ladder contractions: -1 follow precision (default:*/
                             /* FP64 -> 0; BF16X3 -> 2 in sigma, 1 in setup and      */
                             /* refinement for EA, 0 in setup and refinement for IP), */
                             /* 0 FP64 DGEMM, 1 FP32-accurate emulated GEMM, 2 (sigma)*/
                             /* unbatched contractions of >= 1e8 flop on the tensor-  */
                             /* core split-BF16 GEMM of the ladder, unless a free     */
                             /* dimension is <= 8 and the large operand is not a      */
                             /* cached constant; the rest on the library's own FP64 / */
                             /* FP32-accurate kernels (setup and refinement use 1)    */
    int refine;              /* BF16X3 only: converged roots are re-evaluated once    */
                             /* with the accurate ladder (FP32 partial sums promoted  */
                             /* every 64-deep K block) and Rayleigh-Ritz in their     */
                             /* span; 1 (default): other contractions as in sigma     */
                             /* (FP32-accurate), 2: FP64 for every other contraction, */
                             /* 0: no refinement                                      */
    int transition_order;    /* order of T in the spectroscopic amplitudes (Eqs.      */
                             /* T_ea, T_ip): 0 (default) = n, the method's order;     */
                             /* 2 = second order also for ADC(3) (no t1(3), no t2(2)) */
    double refine_res_tol;   /* BF16X3 with refine >= 1: > 0 continues the Davidson   */
                             /* from the converged roots with the accurate operator   */
                             /* (the refine arithmetic) until the S-norm residual is  */
                             /* below this value (vectors and spectroscopic factors   */
                             /* converged under that operator); 0 (default): one      */
                             /* Rayleigh-Ritz step in the span of the converged roots */
    int m11_on_the_fly;      /* 1: the 1p-1p (EA) / 1h-1h (IP) block is not precomputed */
                             /* (step 3 skipped); every sigma applies it from small    */
                             /* intermediates (Sec. III A, the alternative to step 3;  */
                             /* EA keeps the ladder of t, o^2 v^2); the preconditioner */
                             /* then uses zeroth-order one-particle energies and      */
                             /* adc_get_tensor("M11") is unavailable.  0 (default)     */
    const char* tune_cache;  /* NULL (default): tile widths from the cost model; else a */
                             /* text file of measured tile choices: a tensor-core     */
                             /* problem not yet in it (the sigma ladder's GEMM2 tile  */
                             /* width per B^Q shape, a generic contraction's tile     */
                             /* width per shape) is timed once on the device with     */
                             /* each candidate, and the fastest is kept (file         */
                             /* rewritten; read at setup; one table per path, shared  */
                             /* by the process's handles)                             */
    int cuda_graphs;         /* 1: in adc_davidson the sigma of a mixed-precision      */
                             /* handle runs as a CUDA graph per block size (captured  */
                             /* once on fixed buffers, replayed as one launch; for    */
                             /* small systems, where launches dominate; needs a      */
                             /* stream of the handle's own: adc_setup_batch, or      */
                             /* adc_set_stream); 0 (default)                          */
    int lean;                /* memory layout of a closed-shell EA handle in BF16X3    */
                             /* precision: 1 lean -- the o^2 v^2 integrals and         */
                             /* amplitudes of sigma held in FP32 (every contraction   */
                             /* reading them is split-BF16 or FP32-accurate, so the   */
                             /* results are those of the plain layout up to rounding),*/
                             /* no tau / ring2 tensors (their contractions expanded),  */
                             /* operand copies made per call rather than cached,       */
                             /* setup's o^2 v^2 temporaries in FP32; about a third of  */
                             /* the plain layout's memory (e.g. nocc=68, nvir=960,     */
                             /* naux=3000 fits one GPU); needs m11_on_the_fly = 0.     */
                             /* 0 plain; -1 (default) lean when the plain layout's     */
                             /* setup would not fit the free device memory            */
} adc_options;

/* Fill *opt with the defaults listed above.  Returns ADC_OK or ADC_ERR_ARG (NULL). */
int adc_default_options(adc_options* opt);

/*
 * Set up one system (Sec. III A steps 1-3): copies eps and Bq to the device,
 * forms the o-containing integral blocks, the MP amplitudes t(1) (and t(2),
 * t1(2) for order 3), and the 1p-1p (EA) / 1h-1h (IP) block through order n.
 *   eps  host [nmo]; Bq host [naux][nmo][nmo] (or device pointers if on_device=1)
 *   nocc >= 1, nvir >= 1, naux >= 1, order in {2,3}, kind in {ADC_EA, ADC_IP}
 *   opt  NULL for defaults
 *   out  receives the new handle (NULL on failure)
 * Errors: ADC_ERR_ARG, ADC_ERR_OOM, ADC_ERR_CUDA.
 */
int adc_setup(const double* eps, const double* Bq, int nocc, int nvir, int naux, int order, int kind,
              const adc_options* opt, int on_device, adc_handle** out);

/*
 * Set up nmol independent systems at once (the batched workload of many
 * small molecules).  Arrays of length nmol: eps[i], Bq[i] (host, or device
 * if on_device = 1), nocc[i], nvir[i], naux[i]; order, kind and opt are shared.
 * Each handle gets its own CUDA stream (owned, destroyed with the handle).
 * The systems are set up one after another (setup fills the GPU); solve
 * them with adc_davidson_batch, which overlaps their small kernels on the
 * GPU (or with the single-system calls, which stay valid).  out receives nmol handles, each
 * released with adc_destroy.  On failure no handle is returned and
 * adc_last_error(NULL) names the failing system.
 * Errors: as adc_setup.
 */
int adc_setup_batch(int nmol, const double* const* eps, const double* const* Bq, const int* nocc, const int* nvir,
                    const int* naux, int order, int kind, const adc_options* opt, int on_device, adc_handle** out);

/* Replace the solver options of a handle (max_space_per_root, max_iter,
 * nguess_extra, res_tol, keep_per_root, refine, transition_order,
 * refine_res_tol, cuda_graphs); precision,
 * contractions and aux_chunk stay as set up.  Errors: ADC_ERR_ARG. */
int adc_set_options(adc_handle* h, const adc_options* opt);

/*
 * Set up an unrestricted (open-shell) reference for EA/IP-UADC(n) sigma
 * products (the paper's UADC, Sec. II; FP64 only).  Spin orbitals are ordered
 * occupied alpha, occupied beta, virtual alpha, virtual beta; with o = nocc_a +
 * nocc_b and v = 2 nmo - o spin orbitals the vector is
 *   EA  [Y_a (v) | Y_iab (i, a<b), i-major, pairs in lexicographic order]
 *   IP  [Y_i (o) | Y_ija (i<j, a), a-major, pairs in lexicographic order]
 * and adc_sigma applies M (EA) or -M_- (IP).  The two-electron integrals are
 * (p_s q_s | r_t s_t) = sum_Q B^Q_{s,pq} B^Q_{t,rs} (Eq. 19 per spin pair).
 *   eps_a, eps_b  host [nmo] alpha / beta orbital energies, occupied first
 *   Ba, Bb        host [naux][nmo][nmo] alpha / beta DF factors, symmetric in pq
 * opt: NULL for defaults.  precision ADC_PREC_FP64 or ADC_PREC_BF16X3 (setup and
 * the refinement of converged roots in FP64; the sigma's ladder on the tensor
 * cores per spin block -- alpha-alpha, beta-beta and alpha-beta, the beta-alpha
 * block by antisymmetry -- and its other contractions as in the closed-shell
 * mixed sigma); aux_chunk also sets the chunks of the IP third-order coupling
 * intermediate sum_e B^Q_ie t_jk^de (naux x o^3 x v; 0 = at most 2^27 elements);
 * the solver options as for adc_setup; m11_on_the_fly is not available here.
 * adc_get_tensor returns "t2", "t2_2", "t1_2", "t1_3" (third-order singles, made
 * on first use) and "M11" in these spin-orbital dimensions (M11: the paper's
 * M_+ / M_- one-particle block).  adc_davidson runs with metric S = 1 (the
 * antisymmetric pair basis is orthonormal) and a preconditioner of diag(M11)
 * and the zeroth-order pair energies; its spectroscopic factors are those of
 * one spin-orbital component, P = sum_p X_p^2 with T through order n (a
 * Koopmans state has P = 1).  adc_mp_energy is not available on these handles.
 * Errors: ADC_ERR_ARG, ADC_ERR_OOM, ADC_ERR_CUDA (message: adc_last_error(NULL)).
 */
int adc_setup_unrestricted(const double* eps_a, const double* eps_b, const double* Ba, const double* Bb, int nocc_a,
                           int nocc_b, int nmo, int naux, int order, int kind, const adc_options* opt, adc_handle** out);

/* Length of the spin-adapted vector (see layout above). */
int adc_dim(const adc_handle* h, long long* dim);

/*
 * Moller-Plesset correlation energy of the reference through order n
 * (Sec. III A step 2), from the setup's amplitudes:
 *   e[0] = E(2) = sum (ia|jb) (2 t_ij^ab - t_ij^ba)               (t = t2(1))
 *   e[1] = E(3) = sum (ia|jb) (2 t2_ij^ab - t2_ij^ba)  (ADC(3) only; t2 = t2(2))
 * E(1) = 0 for the normal-ordered perturbation.  n_out = number of doubles e
 * holds; min(n_out, order - 1) values are written.  Errors: ADC_ERR_ARG.
 */
int adc_mp_energy(const adc_handle* h, double* e, int n_out);

/* Issue subsequent work on this CUDA stream (cudaStream_t passed as void*). */
int adc_set_stream(adc_handle* h, void* stream);

/*
 * sigma = M X for nvec vectors (Sec. III A step 4; Eqs. sigma_i_adapted_3,
 * sigma_jka_bab and their EA analogue).  X and S are row-major [nvec][dim];
 * host pointers if on_device = 0 (copied in and out inside the call), device
 * pointers if on_device = 1.  X and S must not overlap.
 * Errors: ADC_ERR_ARG (nvec < 1, NULL), ADC_ERR_OOM, ADC_ERR_CUDA.
 */
int adc_sigma(adc_handle* h, const double* X, double* S, int nvec, int on_device);

/*
 * Lowest nroots roots by multi-root Davidson in the S inner product (Eq. eig,
 * Sec. III A step 4), then spectroscopic factors (Eq. spec_factors, Appendix)
 * from the transition moments T through order n (Eqs. T_ea, T_ip, k + l <= n;
 * for ADC(3) this includes the third-order singles t1(3)).
 *   tol       convergence threshold on the eigenvalue change (Eh)
 *   guess     NULL or host [nguess = nroots][dim] initial vectors
 *   energies  host [nroots], ascending
 *   specfac   host [nroots] or NULL
 *   vectors   host [nroots][dim] (S-normalised eigenvectors) or NULL
 *   stats     host double[8] or NULL: {iterations, sigma vectors, seconds,
 *             max S-norm residual, sigma seconds, max |energy change| of the
 *             final refinement, refinement seconds, roots that fell back from
 *             the learned to the diagonal preconditioner}; with refinement the
 *             residual is that of the refined pairs under the accurate sigma
 * Errors: ADC_ERR_ARG, ADC_ERR_OOM, ADC_ERR_CUDA, ADC_ERR_TIMEOUT,
 * ADC_ERR_NONFINITE (non-finite guess element, or a non-finite Ritz value or
 * residual), ADC_ERR_NOT_CONVERGED (max_iter reached, or no correction vector
 * survived orthonormalisation while roots were unconverged; energies,
 * specfac, vectors and stats are still filled with the best estimates).
 */
int adc_davidson(adc_handle* h, int nroots, double tol, const double* guess, double* energies, double* specfac,
                 double* vectors, double* stats);

/*
 * adc_davidson for nmol handles concurrently (host threads, one handle each,
 * work on each handle's stream), without guesses or vectors:
 *   energies  host [nmol][nroots];  specfac host [nmol][nroots] or NULL
 *   stats     host [nmol][8] or NULL;  status host [nmol] or NULL (each
 *             system's adc_davidson return code)
 * Returns ADC_OK if every system converged, else the first non-OK code other
 * than ADC_ERR_NOT_CONVERGED if any (ADC_ERR_NOT_CONVERGED otherwise); the
 * handles' adc_last_error hold the messages.
 */
int adc_davidson_batch(adc_handle* const* h, int nmol, int nroots, double tol, double* energies, double* specfac,
                       double* stats, int* status);

/*
 * Copy an intermediate to host memory.  name is one of "M11" [n1][n1],
 * "t2" [o][o][v][v] (first-order doubles), "t2_2" (second-order doubles),
 * "t1_2" [o][v], "t1_3" [o][v] (third-order singles, Eq. t_singles at k = 3;
 * ADC(3) only, computed on the first request or the first spectroscopic
 * factors), "diag" [dim], or "X" [nroots][nmo]: the spectroscopic
 * amplitudes X_{p,mu} = sum_nu T_{p,nu} (S Y~)_nu of the last adc_davidson
 * that computed spectroscopic factors (Eq. spec_amp with the Appendix
 * renormalisation, P_mu = 2 sum_p X_{p,mu}^2; occupied orbitals first), or
 * "setup_seconds" [8]: wall seconds of adc_setup's phases (restricted handles):
 * inputs and the ladder's operand planes, integrals, amplitudes and E(2), the
 * ladder of t, the rest of t2(2) with t1(2) and E(3), the one-particle block,
 * the transition moments' parts and the diagonal, and the total.
 * n = number of doubles the buffer holds.  Errors: ADC_ERR_ARG (unknown name,
 * buffer too small, or the intermediate does not exist at this order / yet).
 */
int adc_get_tensor(adc_handle* h, const char* name, double* out, long long n);

/*
 * Live timing of the tensor-core GEMM launches (for roofline reporting).
 * enable = 1 clears the record and starts bracketing every tensor-core GEMM
 * launch on the handle's stream with CUDA events; enable = 0 stops,
 * synchronises and, if out is non-NULL, writes out[9] = {launches, total
 * milliseconds of those launches, algorithmic flops (unpadded), tensor-core
 * flops issued (split products over padded tiles), all own kernels launched
 * meanwhile, and for the DF-ladder GEMMs alone: launches, milliseconds,
 * algorithmic flops (4 naux nocc nvir^3-type count), tensor-core flops}.
 * Errors: ADC_ERR_ARG, ADC_ERR_CUDA.
 */
int adc_kernel_timing(adc_handle* h, int enable, double* out);

/*
 * The launches recorded by the last adc_kernel_timing bracket, one by one (after
 * it was stopped).  out NULL: returns the number of launches.  Else out holds at
 * least 7 doubles per launch and receives, per launch: M, N, K (padded), tile
 * width, algorithmic flops, milliseconds (CUDA events on the launch's stream),
 * and 1 for the DF ladder's GEMMs, 0 for the other contractions; returns the
 * number of launches.  Errors: ADC_ERR_ARG (NULL handle, timing still running,
 * buffer too short), ADC_ERR_CUDA.
 */
long long adc_kernel_launches(adc_handle* h, double* out, long long n);

/*
 * Allocation-free density-fitted ladder: out[n] = sum_Q B^Q X[n] B^Q for nmat
 * nvir x nvir matrices, i.e. sum_cd (ac|bd) X[n][c][d] -- the dominant 2p1h
 * (EA) sigma term, computed by the same tensor-core kernel as adc_sigma.  The
 * paper has no counterpart: it exists for callers that cannot allocate device
 * memory during the call (a host framework that owns all device memory and
 * forbids cudaMalloc/cudaFree inside library calls, which may synchronise the
 * device).  It allocates nothing: its intermediates live in a fixed 64 MiB
 * device array.  The setup of a BF16X3 handle looks up that array's device
 * address on its device (once per device, with that device current), which
 * loads the array with its module; the GPU then holds the 64 MiB until process
 * exit, and this call performs no lookup or module load of its own.
 *   h    handle set up with precision ADC_PREC_BF16X3 (uses its split B^Q)
 *   X    device [nmat][nvir][nvir] FP64;  out  device [nmat][nvir][nvir] FP64,
 *        overwritten; X and out must not overlap
 * All calls share the one array and it keeps the last call's contents: calls
 * that overlap on the GPU (other streams, other threads) race.  Work runs on
 * the handle's stream; before returning, the call reads the kernels' timeout
 * flag back to the host and synchronises that stream.
 * Errors: ADC_ERR_ARG (NULL pointers, nmat < 0, handle not BF16X3, or nvir so
 * large that one matrix and one auxiliary function exceed the 64 MiB),
 * ADC_ERR_CUDA, ADC_ERR_TIMEOUT.
 */
int adc_ladder_noalloc(adc_handle* h, const double* X, double* out, long long nmat);

/*
 * Spectral function (density of states) of computed roots on a frequency grid
 * (Eqs. spec_function and PES): A(w) = -1/pi Im sum_mu P_mu / (w - w_mu + i eta)
 * = 1/pi sum_mu P_mu eta / ((w - w_mu)^2 + eta^2), on the axis of the energies
 * adc_davidson returns (EA: E_{N+1} - E_N; IP: ionisation energies).  With P
 * from adc_davidson (Appendix normalisation) A integrates to sum_mu P_mu and
 * counts both spin components.  Host arrays: energies, specfac [nroots];
 * omega, A [nomega].  Host computation (O(nroots * nomega)); no handle needed.
 * Errors: ADC_ERR_ARG (NULL arrays, negative counts, eta <= 0).
 */
int adc_spectrum(const double* energies, const double* specfac, int nroots, double eta, const double* omega, int nomega,
                 double* A);

/*
 * Learned Davidson preconditioner.  The paper uses the diagonal correction
 * t = r / (w - D) (Sec. III A, Davidson); this adds to its multiplier a small
 * network m(f) (3 -> 64 -> 64 -> 1, tanh, FP32) of per-element features
 * f = (d, sign(d)/max(|d|, 0.01), [element in the 1p/1h block]), d = D - w:
 *   t_x = r_x (1 / (w - D_x) + m(f_x)),
 * weights laid out W1[64][3], b1[64], W2[64][64], b2[64], W3[64], b3
 * (adc_mlp_nweights() floats; all zero = the diagonal preconditioner).
 * Training samples (host arrays of n): d = D_x - w, blk (1: 1p/1h block),
 * r = residual element, t = exact correction element (y_exact / <y, y_exact>_S
 * - y of a Davidson iterate y); loss = sum (r (p + m) - t)^2 / sum t^2.
 *   adc_mlp_loss_grad: loss and gradient (host grad [nweights]) at `weights`
 *   adc_mlp_train:     `steps` full-batch Adam steps of rate lr on the GPU;
 *                      weights host in/out; loss_hist host [steps] or NULL
 *   adc_set_mlp:       use these weights (host) in adc_davidson of this handle,
 *                      NULL for the diagonal preconditioner (default).  A root
 *                      whose residual does not fall below 0.9 x its best for 4
 *                      iterations falls back to the diagonal preconditioner.
 * Errors: ADC_ERR_ARG, ADC_ERR_CUDA (adc_last_error(NULL) for the first two).
 */
int adc_mlp_nweights(void);
int adc_mlp_loss_grad(const float* weights, const double* d, const unsigned char* blk, const double* r, const double* t,
                      long long n, float* grad, double* loss);
int adc_mlp_train(float* weights, const double* d, const unsigned char* blk, const double* r, const double* t, long long n,
                  int steps, float lr, double* loss_hist);
int adc_set_mlp(adc_handle* h, const float* weights);

/*
 * Training samples for the learned preconditioner from this handle's own plain
 * Davidson (closed-shell handles).  The roots are first converged tightly (to
 * exact_tol on the energies, S-norm residual 1e-6 or the handle's res_tol if
 * smaller); then for each k = iters[0 .. n_iters) the solver is stopped after k
 * iterations, and for each of the nroots iterates y (Ritz value w) the library
 * forms on the device the residual r = sigma(y) - w y and the exact correction
 * t = y_exact / <y_exact, y>_S - y, y_exact the converged root of largest
 * S-overlap (S = diag(1, 2 - P), Appendix norm).  Each sample is one element x:
 * d = D_x - w, blk = [x in the 1p/1h block], r_x, t_x; per (k, root) the samples
 * are every 1p/1h element followed by min(per_vector, dim - n1) distinct
 * 2p1h/2h1p elements drawn by a splitmix64 stream seeded by `seed`.
 * Host outputs d, r, t (double) and blk (bytes) of length n >= adc_mlp_nsamples;
 * the handle's solver options are restored on return.
 * adc_mlp_nsamples returns that count (n_iters * nroots * (n1 + min(per_vector,
 * dim - n1))), or -1 for invalid arguments.
 * Errors: ADC_ERR_ARG, ADC_ERR_OOM, ADC_ERR_CUDA, ADC_ERR_NONFINITE.
 */
long long adc_mlp_nsamples(const adc_handle* h, int nroots, int n_iters, long long per_vector);
int adc_mlp_samples(adc_handle* h, int nroots, const int* iters, int n_iters, long long per_vector,
                    unsigned long long seed, double exact_tol, double* d, unsigned char* blk, double* r, double* t,
                    long long n);

/* Message of the last error on this handle (or of the last failed adc_setup
 * when h is NULL).  Never NULL. */
const char* adc_last_error(const adc_handle* h);

/* Release the handle and all its device memory.  NULL is ignored. */
void adc_destroy(adc_handle* h);

#ifdef __cplusplus
}
#endif
#endif /* GB300_ADC_H */
