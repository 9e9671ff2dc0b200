/*
 * ccgf.h - C ABI of the GB300 periodic coupled-cluster Green's function library.
 *
 * The library computes the k-point CCGF of the paper (Eq. 9),
 *   G+_pq(k,w) = <Phi0|(1+Lambda) a_bar_{pk} [w - (H_bar - E) + i eta]^-1 a_bar+_{qk} |Phi0>,
 *   G-_pq(k,w) = <Phi0|(1+Lambda) a_bar+_{qk} [w + (H_bar - E) - i eta]^-1 a_bar_{pk} |Phi0>,
 * with the EOM-CCSD ansatz of Eq. 8 (1h + 2h1p for the removal part,
 * 1p + 2p1h for the addition part): the shifted linear systems of Eq. 6 are
 * solved by batched GMRES whose operator is the EOM-IP / EA-CCSD
 * similarity-transformed Hamiltonian (the sigma vector), and the solutions are
 * contracted with the left vectors as in Eq. 7.
 *
 * Conventions shared by every call
 *   - Complex numbers are interleaved pairs of double (re, im): a "complex
 *     array of n elements" is 2n doubles, 16-byte aligned.
 *   - k index = (k1*n2 + k2)*n3 + k3 on the (n1, n2, n3) mesh; momentum
 *     addition is modulo each mesh dimension.
 *   - Orbitals per k are ordered occupied first (nocc), then virtual (nvir);
 *     nmo = nocc + nvir. The reference Fock matrix is diag(mo_energy).
 *   - Closed-shell (restricted) reference; G_pq is the alpha-alpha block.
 *   - EOM vectors at total momentum K, spin-adapted:
 *       IP: r1[i] (nocc), then r2[ki][kj][i][j][a] with k_a = ki + kj - K;
 *       EA: r1[a] (nvir), then r2[kj][ka][j][a][b] with k_b = K + kj - ka.
 *     dim_ip = nocc + nk^2 nocc^2 nvir, dim_ea = nvir + nk^2 nocc nvir^2.
 *   - Every call is stream-ordered on the caller's CUDA stream (cudaStream_t
 *     passed as void*; NULL = the legacy default stream). A call synchronises
 *     the stream only where stated: ccgf_solve_gf reads the convergence flags
 *     once per Arnoldi step; a sigma call synchronises only when it first meets
 *     a new vector count or momentum (plan and workspace set-up, which may
 *     allocate) and, with CCGF_TF32X3 or CCGF_FP64_TC, once at its end to read
 *     the tensor-core error flag. Repeated FP64 / FP32 sigma calls of one shape
 *     allocate nothing and do not synchronise. Copies kept only for speed (FP32
 *     and sliced copies of the intermediates, cached right-hand sides and left
 *     vectors) are released when a call needs their memory and made again later.
 *   - Errors are returned as status codes; nothing aborts, throws or traps.
 *     ccgf_last_error() gives a message for the last failing call on this
 *     thread. One handle per host thread.
 */
#ifndef CCGF_H
#define CCGF_H

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    CCGF_OK = 0,
    CCGF_NOT_CONVERGED = 1,      /* warning: outputs written, some residuals above tol */
    CCGF_ERR_INVALID_ARG = -1,
    CCGF_ERR_OOM = -2,
    CCGF_ERR_CUDA = -3,
    CCGF_ERR_NAN = -4,
    CCGF_ERR_TIMEOUT = -5
} ccgf_status;

typedef enum {
    CCGF_FP64 = 0,       /* plain form: every step in FP64 */
    CCGF_FP32 = 1,       /* sigma contractions in FP32 (FP32 accumulate) inside FP64 refinement */
    CCGF_TF32X3 = 2      /* sigma contractions on the tensor cores (tcgen05): each FP32 operand split
                            into two TF32 parts, three products (hi*hi + hi*lo + lo*hi) accumulated
                            in FP32, inside FP64 refinement; contractions too small for a 128-row
                            tile run as in CCGF_FP32. A tensor-core wait that runs past its limit
                            (ccgf_options::device_wait_timeout_ms) makes the call return
                            CCGF_ERR_TIMEOUT. */,
    CCGF_FP64_TC = 3     /* FP64-accurate sigma on the tensor cores: each FP64 operand of a contraction
                            whose A block is a stored intermediate is cut into integer slices of 8
                            bits under a per-row (per-column) power of two; their products and
                            sums below 2^24 are exact in tcgen05.mma.kind::tf32, so the product
                            terms down to 2^-32 of the leading one are formed exactly, those down
                            to 2^-40 with FP32 rounding far below that, and smaller ones dropped
                            (error ~2^-41 of n max|a| max|b|). Partial sums are drained into double-word
                            FP32 accumulators and the result written in FP64. The other
                            contractions, and those whose sliced copy does not fit in device memory
                            (3.5 x the FP64 intermediate), run in FP64 SIMT. Treated as FP64 by the
                            solver (no refinement). Waits as in CCGF_TF32X3. */
} ccgf_precision;

typedef enum { CCGF_SECTOR_IP = 1, CCGF_SECTOR_EA = 2, CCGF_SECTOR_BOTH = 3 } ccgf_sector;

/* The problem of the paper's k-point CCGF section: orbital energies, integrals,
 * ground-state amplitudes and Lambda. All pointers are borrowed for the call
 * and copied; they are host pointers unless inputs_on_device != 0.          */
typedef struct {
    int kmesh[3];
    int nocc, nvir, naux;
    const double *mo_energy;  /* real [nk][nmo]                                           */
    const double *L;          /* complex [nk][nk][naux][nmo][nmo]: (p k1 q k2|r k3 s k4) =
                                 sum_Q L[k1,k2,Q,p,q] L[k3,k4,Q,r,s] if k1+k3 = k2+k4     */
    const double *t1;         /* complex [nk][nocc][nvir]                                 */
    const double *t2;         /* complex [nk][nk][nk][nocc][nocc][nvir][nvir],
                                 t2[ki,kj,ka][i,j,a,b], k_b = ki + kj - ka                */
    const double *l1;         /* complex, layout of t1; NULL => conj(t1)                  */
    const double *l2;         /* complex, layout of t2; NULL => conj(t2)                  */
    int inputs_on_device;
} ccgf_system;

typedef struct {
    ccgf_precision prec;      /* arithmetic of the inner sigma (see ccgf_precision)       */
    double tol;               /* relative residual ||b - M x|| / ||b|| per right-hand side */
    int restart_m;            /* GMRES restart length                                      */
    int max_iter;             /* cap on inner iterations per right-hand side              */
    int max_refine;           /* cap on GMRES cycles (restarts) per batch. With a low-
                                 precision inner sigma a cycle that stops at the restart
                                 length restarts from the low-precision residual; the FP64
                                 true residual is taken when the iteration meets the target
                                 (refinement step), and only it decides convergence; after
                                 a failed check the low-precision iteration aims at a tenth
                                 of the target                                            */
    int omega_chunk;          /* frequencies solved together per (sector, K) batch (at most;
                                 the solver splits batches that do not fit in device memory) */
    double device_wait_timeout_ms; /* bound of every tensor-core device wait, (0, 60000] ms;
                                      a wait that runs out makes the call return
                                      CCGF_ERR_TIMEOUT. Build: the handle's bound for sigma
                                      calls; solve: the bound during that solve.           */
    int warm_start;           /* 1: initial vectors from the trained warm-start network
                                 (ccgf_train_warmstart), kept per column only when their true
                                 residual is below the cold start's |b|                    */
    int kpoint;               /* solve: -1 all k-points (default), else only this total momentum
                                 (G of the other k-points is left zero)                     */
    int orbital_first;        /* solve: right-hand sides for orbitals [orbital_first,          */
    int orbital_count;        /*   orbital_first + orbital_count) only (count 0: all); G keeps
                                 IP rows p / EA columns q of those orbitals, zero elsewhere   */
    int direct_terms;         /* build only: 0 chooses by size; 1 stores every H_bar block;
                                 2 stores no O(nk^3 o v^3) block: the W_vvvo r1 term, the
                                 (2<am|ef> - <am|fe>) r2 term of the EA singles and the T2 part of
                                 the EA ladder are then formed in each sigma from the
                                 density-fitting factors (same operator, less memory)       */
    ccgf_precision refine_prec; /* solve with CCGF_FP32 / CCGF_TF32X3: the true residual's sigma,
                                 CCGF_FP64 (default) or CCGF_FP64_TC                        */
} ccgf_options;

typedef struct {
    long long rhs_solved;       /* right-hand sides solved                                */
    long long inner_iterations; /* sum over batches of GMRES iterations (batch-parallel)  */
    long long fp64_sigma_calls; /* FP64 sigma batches (true-residual recomputes)          */
    long long lowp_sigma_calls; /* low-precision sigma batches (iterations and restarts)   */
    double max_rel_residual;    /* largest final true relative residual                   */
    double sigma_ms;            /* device time of the sigma calls inside Arnoldi steps    */
    double total_ms;            /* device time of the whole solve                         */
    long long kernel_launches;  /* kernels launched by the solve                          */
    long long warm_columns;     /* right-hand sides that started from the network's x0    */
    long long warm_fallbacks;   /* right-hand sides where the cold start was kept         */
    double warm_val_loss;       /* ccgf_train_warmstart: validation loss of the network   */
    double warm_val_loss_baseline; /* ... of the baseline alone (zero correction)         */
    double warm_rel_residual;   /* mean |b - M x0| / |b| of the starts used (cold = 1)     */
    double warm_rel_residual_net;  /* ... of the network's prediction (0 when not used)   */
    double warm_rel_residual_base; /* ... of the baseline alone                           */
    long long restart_used;     /* GMRES restart length used (the requested one unless device
                                   memory made the solver shorten it, never below 10)      */
    long long columns_per_batch;/* largest number of right-hand sides solved together: all
                                   orbitals x omega_chunk frequencies when they fit in device
                                   memory, else orbital chunks of equal width             */
    double vector_ms;           /* device time of the Arnoldi vector steps after each sigma
                                   (shift, both CGS passes, norm, normalisation)           */
    double vector_bytes;        /* their algorithmic HBM traffic: 16 (4J + 12) D nv bytes per
                                   step with J basis vectors (vector_bytes / vector_ms: GB/s) */
    double refine_ms;           /* device time of the FP64 true-residual sigma calls       */
    double vector_flops;        /* FP64 flops of the vector steps timed in vector_ms: (32 J + 14)
                                   D nv per step (8 per complex multiply-add in both CGS passes,
                                   shift 8, norm 4, normalisation 2)                        */
} ccgf_stats;

typedef struct ccgf_handle ccgf_handle;

/* Default options: FP64, tol 1e-10, restart 30, max_iter 2000, max_refine 20, omega_chunk 1,
 * device waits bounded at 1000 ms, no warm start. */
void ccgf_default_options(ccgf_options *opt);

/* Build the similarity-transformed Hamiltonian blocks (Eq. 5) for the EOM-CCSD
 * sigma vectors: T1-dressed integrals, F_oo, F_vv, F_ov and the W blocks, all in
 * FP64 (plus FP32 copies), in GEMM-ready layouts; also the RHS / left-vector
 * ingredients (T, Lambda). The handle owns all device memory it allocates.
 * Errors: INVALID_ARG (sizes, NULL), OOM (cudaMalloc), CUDA, NAN (non-finite input). */
ccgf_status ccgf_build_intermediates(const ccgf_system *sys, const ccgf_options *opt,
                                     void *stream, ccgf_handle **out);

ccgf_status ccgf_dims(const ccgf_handle *h, int *nk, int *nocc, int *nvir,
                      long long *dim_ip, long long *dim_ea);

/* y = A_IP x (Eq. 8, removal part): the connected EOM-IP-CCSD operator H_bar - E
 * on nvec vectors at total momentum kshift. x, y: device complex [nvec][dim_ip],
 * caller-owned, must not alias. prec selects the arithmetic of the contractions
 * (inputs and outputs stay FP64). The handle keeps its transpose buffers, plans and
 * scratch between calls: the first call with a new nvec (or kshift) allocates and
 * synchronises, later calls of that shape only enqueue kernels (CCGF_TF32X3 then
 * synchronises once to read the tensor-core error flag). Errors: INVALID_ARG
 * (kshift, nvec, NULL), OOM (workspace), CUDA, TIMEOUT (CCGF_TF32X3 wait bound). */
ccgf_status ccgf_sigma_ip(ccgf_handle *h, int kshift, long long nvec, const double *x,
                          double *y, ccgf_precision prec, void *stream);

/* y = A_EA x (Eq. 8, addition part), as ccgf_sigma_ip with dim_ea. */
ccgf_status ccgf_sigma_ea(ccgf_handle *h, int kshift, long long nvec, const double *x,
                          double *y, ccgf_precision prec, void *stream);

/* Right-hand side b_p = P a_bar_p |Phi0> (IP) or b_q = P a_bar+_q |Phi0> (EA) and
 * left vector e_q = <Phi0|(1+Lambda) a_bar+_q|mu> (IP) or e_p = <..|a_bar_p|mu> (EA)
 * for orbital p at momentum K (Eq. 6-7); out: device complex [dim]. */
ccgf_status ccgf_rhs(ccgf_handle *h, int sector, int K, int p, double *out, void *stream);
ccgf_status ccgf_left(ccgf_handle *h, int sector, int K, int p, double *out, void *stream);

/* G_pq(k,w) = G+ + G- (Eq. 9) for all k, all p, q and the nomega frequencies,
 * sectors = CCGF_SECTOR_IP / EA / BOTH (the other part is left out of the sum).
 * IP: (w - i eta + A_IP) X_p = b_p, G-[p,q] = e_q . X_p;
 * EA: (w + i eta - A_EA) Y_q = b_q, G+[p,q] = e_p . Y_q.
 * G_out: complex [nk][nomega][nmo][nmo], caller-owned, host or device memory
 * (G_on_device). omega: host array. Returns NOT_CONVERGED (G still written) when
 * some right-hand side missed opt->tol within the caps. stats may be NULL. */
ccgf_status ccgf_solve_gf(ccgf_handle *h, int sectors, int nomega, const double *omega,
                          double eta, const ccgf_options *opt, double *G_out, int G_on_device,
                          ccgf_stats *stats, void *stream);

/* Model-order-reduction CCGF (the paper's MOR frequency interpolation): G_pq(k,w) of Eq. 9 on the
 * nomega grid frequencies from a reduced model per (sector, k). The shifted systems are solved (as in
 * ccgf_solve_gf, with opt) at the n_mor model frequencies omega_mor (1..64, host array) for every
 * orbital; an orthonormal basis V of the span of those solutions (Gram matrix diagonalised, directions
 * with singular value below 1e-7 of the largest dropped) projects the EOM operator, the right-hand
 * sides and the left vectors (A_r = V^H A V, b_r = V^H b, e_r = e V); the reduced systems of dimension
 * rank(V) <= nmo n_mor are then solved at every grid frequency. G is exact (up to the solver
 * tolerance) at the model frequencies. opt->kpoint selects one k (-1: all); the orbital slice and the
 * warm start of opt are ignored. stats: the model solves' counters, columns_per_batch = the largest
 * reduced dimension. G_out as ccgf_solve_gf. Synchronises. Errors as ccgf_solve_gf. */
ccgf_status ccgf_solve_gf_mor(ccgf_handle *h, int sectors, int n_mor, const double *omega_mor, int nomega, const double *omega,
                              double eta, const ccgf_options *opt, double *G_out, int G_on_device, ccgf_stats *stats,
                              void *stream);

/* Spectral function and density of states (Eq. 10): A(k,w) = -(1/pi) Im G(k,w); its trace over the
 * orbitals is the k-resolved density of states
 *   dos[k][w] = -(1/pi) Im sum_p G[k][w][p][p]                        (G_minus == NULL)
 *   dos[k][w] = -(1/pi) Im sum_p G[k][w][p][p] + (1/pi) Im sum_p G_minus[k][w][p][p]
 * G: complex [nk][nomega][nmo][nmo] as ccgf_solve_gf writes it (the time-ordered G = G+ + G-, whose
 * removal part gives negative -Im G / pi below the gap); with G_minus != NULL, G holds the addition
 * part G+ (a solve with CCGF_SECTOR_EA) and G_minus the removal part G- (CCGF_SECTOR_IP), which enters
 * with the opposite sign (the retarded convention: positive peaks on both sides of the gap).
 * dos: real [nk][nomega]; dos_total (NULL allowed): real [nomega], (1/nk) sum_k dos[k]. All device
 * pointers, caller-owned; stream-ordered, no synchronisation. Errors: INVALID_ARG, CUDA. */
ccgf_status ccgf_spectral_function(int nk, int nomega, int nmo, const double *G, const double *G_minus, double *dos,
                                   double *dos_total, void *stream);

/* Active-space self-energy correction (Eqs. 12-14), for every k and frequency:
 *   Sigma_CAS = G_GW,CAS^-1 - G_CC,CAS^-1,  Sigma_full = V Sigma_CAS V^+,  G_out = [G_GW^-1 - Sigma_full]^-1.
 * V: complex [nk][nmo][nact], natural-orbital coefficients of the nact active orbitals (Eq. 11);
 * G_gw: complex [nk][nomega][nmo][nmo] (GW, full space); G_gw_cas, G_cc_cas: complex
 * [nk][nomega][nact][nact] (GW and coupled cluster in the active space, e.g. ccgf_solve_gf on the
 * active-space system); G_out: complex [nk][nomega][nmo][nmo]. The GW Green's functions are inputs
 * (computing them is outside this library). Device pointers, caller-owned; one thread block per (k, w)
 * inverts in shared memory (nmo <= 110). Synchronises the stream to read the singularity flag.
 * Errors: INVALID_ARG (sizes, NULL, a singular matrix), CUDA. */
ccgf_status ccgf_self_energy_correction(int nk, int nomega, int nmo, int nact, const double *V, const double *G_gw,
                                        const double *G_gw_cas, const double *G_cc_cas, double *G_out, void *stream);

/* Learned warm start (no counterpart in the paper's method; it only changes the initial
 * vectors of the Eq. 6 solves): solves all sectors' right-hand sides at the n_train
 * training frequencies (ascending, >= 3) with opt (cold start), keeps their solutions in
 * the handle, then trains the per-element network (14 features -> 256 -> 256 -> 2, tanh,
 * bfloat16-rounded weights in the forward pass, FP32 accumulation) with Adam for `steps`
 * steps of rows_per_step random elements of interior training frequencies, each predicted
 * from its two neighbours. The network predicts a correction to a baseline (the neighbours'
 * solutions carried to the new frequency along each element's diagonal resolvent); after
 * training it is kept only if its validation loss beats the baseline's (steps = 0: baseline
 * only). Later solves with opt->warm_start = 1 use it. final_loss (the kept model's
 * validation loss) and stats may be NULL. Errors: INVALID_ARG, OOM, CUDA, NAN (diverged). */
ccgf_status ccgf_train_warmstart(ccgf_handle *h, int sectors, int n_train, const double *omega_train,
                                 double eta, const ccgf_options *opt, int steps,
                                 long long rows_per_step, double lr, unsigned seed,
                                 double *final_loss, ccgf_stats *stats, void *stream);

/* The warm-start network on its own (device pointers, float32): parameters theta =
 * W1 [F][H], b1 [H], W2 [H][H], b2 [H], W3 [H][2], b3 [2] (ccgf_mlp_param_count(F, H)
 * floats); X [rows][F]; T, Y [rows][2]. bf16 != 0 rounds W1, W2, W3 to bfloat16 first.
 * Loss = sum (Y - T)^2 / rows; grad (device, param count floats) is its gradient. */
long long ccgf_mlp_param_count(int F, int H);
ccgf_status ccgf_mlp_forward(int F, int H, long long rows, const float *theta, const float *X,
                             int bf16, float *Y, void *stream);
ccgf_status ccgf_mlp_loss_grad(int F, int H, long long rows, const float *theta, const float *X,
                               const float *T, int bf16, double *loss, float *grad, void *stream);

/* Measurement helper (no counterpart in the paper): runs one sigma call like
 * ccgf_sigma_ip / ccgf_sigma_ea (sector = CCGF_SECTOR_IP / EA) with a CUDA event
 * between consecutive launches of its plan, and returns per step the device time
 * (step_ms) and the algorithmic flops (step_flops: 8 per complex multiply-add of
 * the contraction, no padding) for up to max_steps steps; *nsteps receives the
 * number of plan steps. Synchronises the stream. Arrays are host memory owned
 * by the caller. Errors as ccgf_sigma_ip. */
ccgf_status ccgf_sigma_profile(ccgf_handle *h, int sector, int kshift, long long nvec, const double *x,
                               double *y, ccgf_precision prec, void *stream, int max_steps,
                               double *step_ms, double *step_flops, int *nsteps);
/* Label of plan step `step` of the (sector, kshift) sigma plan built by a previous
 * call with the current nvec ("" when absent). The string is owned by the library. */
const char *ccgf_sigma_step_name(const ccgf_handle *h, int sector, int kshift, int step);

/* ccgf_sigma_ip without device allocation (no counterpart in the paper): the same
 * FP64 EOM-IP sigma, for callers that must not call cudaMalloc during a call (a host
 * framework that owns all device memory through its own pool, a latency-critical
 * loop that cannot afford the synchronisation an allocation may imply, a process
 * whose device memory is already fully reserved). All scratch lives in one static
 * device array of 32 MiB per device (held until the process exits); a (dim_ip, nvec)
 * that does not fit returns CCGF_ERR_INVALID_ARG with the size it would need. The
 * first call on a device looks up the array's address. Calls share the array: calls
 * whose kernels overlap on the GPU race, so order them. x, y: device complex [nvec][dim_ip], as ccgf_sigma_ip; stream-ordered,
 * does not synchronise. */
ccgf_status ccgf_sigma_ip_noalloc(ccgf_handle *h, int kshift, long long nvec, const double *x,
                                  double *y, void *stream);

/* GEMM kernel selection (no counterpart in the paper). With autotuning on (the default; the
 * environment variable CCGF_AUTOTUNE=0 starts it off), the first run of a sigma plan times every
 * candidate kernel of each contraction (the SIMT tile shapes, each also with the K split that best
 * fills whole waves of the GPU, the few-row kernel where it applies, and, for CCGF_TF32X3, the three
 * tensor-core kernels) on the real operands and keeps the fastest; the choice is cached for the
 * process by shape, so it is measured once. Off: the launcher's model picks the SIMT tile and
 * CCGF_TF32X3 uses the tensor cores wherever the shape allows. Process-wide; affects plans built
 * after the call. */
void ccgf_set_autotune(int enable);
/* Kernel chosen for plan step `step` of the (sector, kshift) plan at precision prec:
 * -1 not a contraction (or no such step / plan), 0 not tuned (defaults apply), 1..99 the SIMT
 * kernel with the launcher's k-th tile shape, k + 1000 s the same kernel with K split over s
 * thread blocks (partial sums reduced by a second kernel), 200 the few-row kernel (one thread
 * per output column, for at most 8 rows and a short reduction), 100 the tensor-core kernel with A by TMA and B
 * staged by producer warps, 101 the register-fed tensor-core kernel, 102 the tensor-core kernel
 * with both operands by asynchronous copies (B from a pre-expanded image), 300 the register-fed
 * tensor-core kernel and 301 the tensor GEMM on a block kept only in FP64 (rounded as it is loaded),
 * 400 a tensor GEMM (pair index maps) of a term formed from the density-fitting factors. */
int ccgf_sigma_step_kernel(const ccgf_handle *h, int sector, int kshift, int step, ccgf_precision prec);

/* Self-test of the bounded device waits (no counterpart in the paper): one warp allocates
 * tensor memory, waits on an mbarrier that nothing arrives on for limit_ms (0 < limit_ms <= 2000),
 * records the timeout, frees the tensor memory and returns. Returns CCGF_ERR_TIMEOUT when the
 * wait gave up as designed (the CUDA context stays usable), CCGF_OK if it did not. Synchronises
 * the stream. */
ccgf_status ccgf_tensor_wait_selftest(double limit_ms, void *stream);

/* Failure injection for error-path tests (no counterpart in the paper): after `after` more
 * successful device allocations, every allocation of the library fails with CCGF_ERR_OOM
 * (without calling cudaMalloc) until the hook is reset with after = -1. Process-wide. */
void ccgf_inject_alloc_failure(long long after);

/* Number of kernels this handle has launched since it was built (build included). */
long long ccgf_launch_count(const ccgf_handle *h);

void ccgf_destroy(ccgf_handle *h);
const char *ccgf_status_string(ccgf_status s);
const char *ccgf_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* CCGF_H */
