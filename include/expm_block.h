/*
 * expm_block.h -- C ABI of the GB300 (sm_103a) preconditioned shifted block FOM library.
 *
 * Computes Z = r(tA) B, the Caratheodory-Fejer (CF) rational approximation of
 * e^{tA} B (Wu, Pang, Sun, "Preconditioning the restarted and shifted block FOM
 * algorithm for matrix exponential computation", arXiv:1405.0707):
 *
 *   r(x) = omega_0 + sum_{i=1..nu} omega_i / (x - tau_i)            (Section 2, eq. (11))
 *
 * The nu shifted systems (tA - tau_i I) X_i = B (eq. (3)) are solved together by the
 * restarted shifted block FOM with the right preconditioner (tA)^{-1} common to every
 * shift (Section 4.1, eq. (3188)): block Arnoldi on (tA)^{-1} (eq. (4.5)), projected
 * systems (I - tau_i H_m) Z_i = E_1 R_i (eq. (3236)), residual norms by eq. (49),
 * restart from V_{m+1} with the collinear residuals (Algorithm 2, k = 0).
 *
 * Conventions for every entry point
 *   - Matrices are column-major with an explicit leading dimension (ld >= rows).
 *   - "device" pointers are CUDA global-memory pointers on the plan's device; the
 *     caller owns them and keeps them valid until the call's stream work completes.
 *     "host" pointers are ordinary CPU memory, read or written before return.
 *   - All device work is issued on the plan's stream (given at plan creation).  Calls
 *     that return numbers to the host (info, residuals) synchronise that stream.
 *   - No entry point calls exit/abort or prints; every failure is a status code.
 *     After EXPM_CUDA_ERROR the plan should be destroyed.
 *   - Only real data (A and B real); the conjugate poles are folded
 *     (Section 2: "one only needs to solve nu/2 shifted linear systems").
 */
#ifndef EXPM_BLOCK_H
#define EXPM_BLOCK_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    EXPM_OK = 0,
    EXPM_INVALID_ARG = 1,      /* bad size, pointer, descriptor or option            */
    EXPM_NOT_CONVERGED = 2,    /* max_cycles reached; Z still written, info filled   */
    EXPM_BREAKDOWN = 3,        /* reserved: a breakdown of the block Arnoldi process
                                  is not an error (see expm_info.breakdown)         */
    EXPM_NUMERICAL = 4,        /* NaN/Inf, or a Cholesky pivot <= 0 in the block QR  */
    EXPM_CUDA_ERROR = 5,       /* a CUDA runtime call or kernel launch failed         */
    EXPM_NO_MEMORY = 6,        /* device allocation failed at plan creation           */
    EXPM_INTERNAL = 7,
    EXPM_TIMEOUT = 8           /* a bounded device-side wait ran out (the kernel returned
                                  without finishing; the device context stays usable)   */
} expm_status;

/* Operator families (the problem of Section 1: tA large, sparse, negative definite). */
typedef enum {
    /* t * (diff * Laplacian_h - vel . grad_h) on the unit interval/square/cube,
     * N_d interior points per axis, h_d = 1/(N_d + 1), homogeneous Dirichlet boundary,
     * second-order central differences, grid index x fastest.  Requires cell Peclet
     * |vel_d| h_d / (2 diff) < 1 on every axis (then tA is diagonally similar to a
     * symmetric negative definite matrix).  The 1-D case with vel = 0 and diff = 1 is
     * (n+1)^2 tridiag(1, -2, 1); the 2-D Laplacian is the paper's Example 5.1 matrix. */
    EXPM_OP_CONV_DIFF = 0,
    /* t * T, T the n x n symmetric Toeplitz matrix with first column (a_0, .., a_bw, 0, ..)
     * (Example 5.4).  Products by circulant embedding (size N = 2^k >= max(n + bw, 2n),
     * N <= 2^22) and a four-step FFT (FP64; double-float in mixed plans); the exact inverse
     * (Algorithm 2's preconditioner) by the Gohberg-Semencul formula (Section 4.1) from the
     * generator x = T^{-1} e_1, computed at plan creation by conjugate gradients with the FFT
     * product, preconditioned by T. Chan's optimal circulant when n is a power of two (the
     * large-norm operators of Example 5.4's regime, kappa ~ 1e9, need it).  Requires a_0 < 0
     * and T negative definite, certified either by a_0 + 2 sum_k |a_k| < 0 (compensated sum)
     * or, for bw <= 4096, by a bound of the symbol's largest value a_0 + 2 sum_k a_k cos(k theta)
     * (grid plus Bernstein's inequality) below 0. */
    EXPM_OP_TOEPLITZ_SYM = 1,
    /* t * A, A a general real n x n sparse matrix in CSR form (host arrays, copied at plan
     * creation; column indices need not be sorted).  The Krylov operator of Algorithm 1 is
     * the sparse product; Algorithm 2's (tA)^{-1} is applied INEXACTLY by an inner iterative
     * solve, the alternative Section 4.1 names for matrices too large for a direct solver:
     * BiCGStab with the Jacobi preconditioner on every column of the block at once, to the
     * relative residual opts.inner_tol.  Theorem 4.3 bounds what the inexact inverse costs:
     *   ||X_i - X~_i|| / ||X_i|| <~ kappa(A) ||(I - tau_i A^{-1})^{-1}|| ||A~^{-1} - A^{-1}|| / ||A^{-1}||,
     * so inner_tol must sit below the wanted accuracy by about kappa(A).  Requires every
     * diagonal entry negative and every row weakly diagonally dominant,
     * sum_{j != i} |a_ij| <= |a_ii| (a Gershgorin certificate that the spectrum of A lies in
     * the closed left half-plane, where the CF approximation of Section 2 applies, and that
     * the Jacobi-preconditioned inner solve is well posed).  Restart cycles of these plans are
     * not captured as CUDA graphs (the inner solve's stop test reads residual norms on the
     * host), and certify mode, the adjoint and the one-graph batch do not take them.
     * Block width p_max <= 16. */
    EXPM_OP_CSR = 2
} expm_op_kind;

typedef struct {
    int32_t kind;          /* expm_op_kind                                           */
    int32_t ndim;          /* CONV_DIFF: 1, 2 or 3                                   */
    int32_t side[3];       /* CONV_DIFF: interior grid points per axis (x, y, z); unused = 1 */
    double  diff;          /* CONV_DIFF: diffusion coefficient (> 0)                 */
    double  vel[3];        /* CONV_DIFF: convection velocity per axis                */
    int64_t n;             /* TOEPLITZ_SYM: order n >= 2                             */
    const double* toeplitz_col; /* TOEPLITZ_SYM: host, a_0 .. a_bw (read at plan creation) */
    int64_t toeplitz_bw;   /* TOEPLITZ_SYM: bandwidth, 0 <= bw <= n - 1              */
    const int64_t* csr_rowptr;  /* CSR: host, n + 1 offsets, rowptr[0] = 0, nondecreasing */
    const int32_t* csr_colind;  /* CSR: host, rowptr[n] column indices in [0, n)          */
    const double*  csr_val;     /* CSR: host, rowptr[n] values (n from the field n)       */
} expm_op_desc;

typedef enum {
    EXPM_PREC_FP64 = 0,    /* every step in FP64 (the plain path)                    */
    /* Mixed: bulk arithmetic on the FP32 pipe, data and small solves in FP64.
     * - The DST-I transforms of the exact inverse run in FP32, and the inverse is refined
     *   to FP64 accuracy (x += inv32(V - tA x), residual in FP64). Theorem 4.3 makes the
     *   inverse's accuracy the one that matters.
     * - Symmetric Toeplitz operators run their FFTs in double-float (float pairs, 2^-48).
     * - The CGS2 projections are FP32 products.
     * - The first Gram-Schmidt update, the application of each Cholesky-QR factor and the
     *   Z update run in double-float. Corrections of size O(eps_32) are formed in FP32. For
     *   blocks of p >= 12 against at least 64 basis columns the first update runs on the
     *   tensor cores instead, on exact bf16 digit slices with FP32 accumulation.
     * - Algorithm 1's operator tA (stencils) is applied in double-float; the refinement
     *   residual of the inverse stays FP64.
     * - The basis is stored in FP64, and the projected systems and the combination stay
     *   FP64.
     * So the Arnoldi relation and the collinear restart hold to ~1e-14 or better.
     * Results agree with EXPM_PREC_FP64 to ~1e-12 relative. */
    EXPM_PREC_MIXED = 1
} expm_precision;

/* Which of the paper's two algorithms runs.  Algorithm 2 (PSBFOM, Krylov operator
 * (tA)^{-1}) pays off when ||tA|| >> |tau_i| (eq. (43), Example 5.2); Algorithm 1 (SBFOM,
 * Krylov operator tA, Section 3) is the better choice when ||tA|| is comparable to the
 * poles.  AUTO picks Algorithm 2 iff the Gershgorin bound of ||tA|| is at least
 * EXPM_AUTO_RATIO * max_i |tau_i| (a build choice: the paper gives no rule).  The ratio is
 * where the two algorithms' measured times cross on the 3-D convection-diffusion instances
 * (n 2^16 .. 2^19, p 1 .. 16, m = 10): below ~30 Algorithm 1 was faster on every instance,
 * above ~40 Algorithm 2 on every one. */
typedef enum {
    EXPM_ALG_AUTO = 0,
    EXPM_ALG_SBFOM = 1,     /* Algorithm 1 */
    EXPM_ALG_PSBFOM = 2     /* Algorithm 2 */
} expm_algorithm;
#define EXPM_AUTO_RATIO 36.0

typedef struct {
    int32_t m;             /* block Arnoldi steps per cycle (restart length), >= 1   */
    int32_t max_cycles;    /* cap on restart cycles, >= 1                            */
    double  tol;           /* stop when max_i ||R_i||_F <= tol ||B||_F  (eq. (49) /
                              eq. (365) for Algorithm 1)                             */
    int32_t precision;     /* expm_precision                                         */
    int32_t fixed_cycles;  /* > 0: run exactly this many cycles, ignoring tol        */
    int32_t algorithm;     /* expm_algorithm                                         */
    int32_t certify;       /* 1: also accumulate every pole's X_i and report the true
                              FP64 residuals ||B - (tA - tau_i I) X_i||_F (eq. (3))   */
    int32_t nu_cf;         /* even CF degree nu, 2 <= nu <= 2*EXPM_MAX_POLES; 0 = 14, the
                              degree of the paper's experiments (Section 5)            */
    int32_t k_defl;        /* deflated restart (the restart of Algorithm 1 with
                              deflation, used by both algorithms): keep k Ritz vectors of H_m at every restart
                              (Algorithm 2: largest |mu|, Remark 4.1; Algorithm 1:
                              smallest |theta|); k is rounded up to a multiple of the
                              block width p and conjugate pairs are kept together (see
                              expm_ritz_basis); 0 = plain restart.  Requires
                              k_defl <= (m - 1) p_max.                                 */
    int32_t row_ctas_per_sm;  /* launch shape of the row-parallel passes (Cholesky-QR, Z
                                 update, reductions): CTAs per SM, 1..8; 0 = 2          */
    int32_t cgs_ctas_per_sm;  /* ... of the first Gram-Schmidt pass: 1..8; 0 = twice
                                 row_ctas_per_sm.  Both are what the autotuner of the
                                 Python package chooses per problem class.             */
    double  inner_tol;     /* CSR operators, Algorithm 2: relative residual of the inner
                              solve of A y = v, per column; 0 = 1e-12                  */
    int32_t inner_maxit;   /* ... and its iteration cap per application; 0 = 2000      */
    int32_t grid_sms;      /* SMs that the grids of the row-parallel passes after the
                              first Gram-Schmidt pass (Cholesky-QR, Z update, reductions)
                              are sized for: CTAs = row_ctas_per_sm x grid_sms; 0 = all of
                              the device's.  The first Gram-Schmidt pass always spans the
                              device.  Plans whose solves run at the same time
                              (expm_block_batched, expm_batch_*) can each take a share:
                              those passes are latency-bound (a serial p x p
                              factorisation in every CTA), and fewer CTAs with more rows
                              each leave SMs to the other instances' kernels.  Results do
                              not depend on it beyond the order of the row partial sums. */
} expm_opts;

#define EXPM_MAX_POLES 16

typedef struct {
    int32_t cycles;              /* restart cycles run                               */
    int32_t block_steps;         /* block applications of (tA)^{-1}                  */
    int64_t matvecs;             /* p * block_steps: the paper's Mat-Vec count (Sec. 5) */
    int32_t converged;           /* 1 if max_i resid[i] <= tol ||B||_F               */
    int32_t breakdown;           /* 1 if a block step found the block Krylov space
                                    invariant up to rounding (informational)         */
    int32_t npoles;              /* nu/2 poles with Im tau > 0                        */
    double  resid[EXPM_MAX_POLES]; /* eq. (49) norms ||R_i||_F after the last cycle   */
    double  normB;               /* ||B||_F                                          */
    int32_t algorithm;           /* 1 or 2: the algorithm that ran                   */
    double  normA_bound;         /* Gershgorin bound of ||tA|| used by AUTO          */
    double  true_resid[EXPM_MAX_POLES]; /* certify: ||B - (tA - tau_i I) X_i||_F in FP64 */
    int32_t kept;                /* deflated restart: Ritz vectors kept at the last restart */
    int64_t inner_iters;         /* CSR operators: inner solver iterations, summed over the
                                    block applications of the call                      */
} expm_info;

typedef struct expm_plan_s expm_plan;

/* ---------------------------------------------------------------------------------
 * expm_cf_coeffs -- the CF table of Section 2 for e^x on (-inf, 0].
 *   nu          : even degree, 2 <= nu <= 2*EXPM_MAX_POLES (the paper uses 14, Sec. 5)
 *   tau_re_im   : host, 2*(nu/2) doubles out: poles with Im tau > 0, (re, im) pairs,
 *                 ordered by decreasing Im
 *   omega_re_im : host, 2*(nu/2) doubles out: matching residues
 *   omega0      : host, 1 double out: r(-inf)
 *   sigma       : host, 1 double out (may be NULL): the CF error estimate (the
 *                 (nu+1)-st Hankel singular value)
 * Poles from the singular vector of the Hankel matrix of the Chebyshev coefficients of
 * e^x transplanted to [-1, 1]; residues by a least-squares fit with those poles.
 * Computed on the host in double-double arithmetic once per nu, then cached.
 * Errors: EXPM_INVALID_ARG (nu, NULL pointer), EXPM_INTERNAL (construction failed).
 * ------------------------------------------------------------------------------ */
expm_status expm_cf_coeffs(int nu, double* tau_re_im, double* omega_re_im,
                           double* omega0, double* sigma);

/* ---------------------------------------------------------------------------------
 * expm_ritz_basis -- the eigenproblem of the deflated restart (Algorithm 1's restart
 * with deflation; Algorithm 2 uses it with the Krylov operator A^{-1}): eigenpairs of the mp x mp real
 * matrix H_m, the wanted Ritz values (largest |mu| when largest != 0, Remark 4.1, else
 * smallest |theta|), eigenvectors of complex pairs split into real and imaginary parts,
 * orthonormalised -> P (mp x kept).  Host only (no device work).
 *   Hm      : host, mp x mp, column-major, leading dimension ldh >= mp (not modified)
 *   k       : wanted count, 1 <= k <= mp; rounded up to a multiple of align (>= 1)
 *   P       : host out, mp x kept, column-major, leading dimension ldp >= mp
 *   kept    : host out: the number of columns written, a multiple of align, <= the rounded k
 * Selection (a reading: the paper lets k "be increased or decreased"): Ritz values are
 * walked in wanted order, a conjugate pair as one group of two columns; a group is kept
 * when it still fits in the rounded k, a pair that does not fit is skipped in favour of
 * the next real value; if the count is then not a multiple of align, the least wanted
 * groups are dropped until it is.  Eigenvalues by the Francis double-shift QR algorithm
 * on the Hessenberg form, eigenvectors by back substitution on the real Schur form.
 * Errors: EXPM_INVALID_ARG, EXPM_NUMERICAL (no convergence, non-finite input).
 * ------------------------------------------------------------------------------ */
expm_status expm_ritz_basis(const double* Hm, int64_t ldh, int mp, int k, int largest,
                            int align, double* P, int64_t ldp, int* kept);

/* ---------------------------------------------------------------------------------
 * expm_plan_create -- "LU once and for all" (Section 4.1; Section 5): set up the exact
 * inverse of A (without t: (tA)^{-1} = A^{-1}/t) and allocate the workspace for block
 * width up to p_max and the options' m.  For EXPM_OP_TOEPLITZ_SYM the setup is the
 * spectrum of the circulant embedding (one FFT) and, unless opts.algorithm is
 * EXPM_ALG_SBFOM, the Gohberg-Semencul generator (conjugate gradients on the device;
 * EXPM_NOT_CONVERGED if its residual stays above 1e-12).  EXPM_PREC_MIXED on a Toeplitz
 * operator computes the spectra and the generator in FP64 and runs the later products
 * and inverses in double-float.
 *   op      : host descriptor (read during the call)
 *   p_max   : 1 <= p_max <= 32; m * p_max <= 512
 *   opts    : host options (copied)
 *   stream  : cudaStream_t (NULL = legacy default stream) used by every later call
 *   out     : host, receives the plan; owned by the caller, free with expm_plan_destroy
 * The plan owns all device memory it allocates (Krylov basis, Hessenberg matrix,
 * preconditioner tables).  Errors: EXPM_INVALID_ARG, EXPM_NO_MEMORY, EXPM_CUDA_ERROR,
 * EXPM_NOT_CONVERGED (Toeplitz generator).
 * ------------------------------------------------------------------------------ */
expm_status expm_plan_create(const expm_op_desc* op, int p_max, const expm_opts* opts,
                             void* stream, expm_plan** out);

void expm_plan_destroy(expm_plan* plan);

/* ---------------------------------------------------------------------------------
 * expm_block -- Z = r(tA) B by Algorithm 2 (PSBFOM, restart without deflation), or by
 * Algorithm 1 (SBFOM) when opts.algorithm asks for it or AUTO selects it.
 *   t      : time, t > 0 (t is folded into A as in Section 1)
 *   dB     : device, n x p, leading dimension ldb >= n (not modified)
 *   p      : 1 <= p <= p_max
 *   dZ     : device, n x p out, leading dimension ldz >= n; must not alias dB
 *   info   : host out (may be NULL)
 * Per cycle: m block steps of W = (tA)^{-1} V_j, block classical Gram-Schmidt with one
 * reorthogonalisation, Cholesky-QR of W; then the nu/2 projected systems of eq. (3236)
 * in one launch, the eq. (49) norms, and the update Z += V_{m+1} sum_i 2 Re(omega_i
 * H~_m Z_i), which equals sum_i 2 Re(omega_i (X_i - X_i^0)) because
 * (tA)^{-1} V_m = V_{m+1} H~_m (eq. (4.5)) and X_i = (tA)^{-1} Y_i.
 * Algorithm 1 instead applies W = tA V_j, solves (H_m - tau_i I) Z_i = E_1 S_i (eq. (3.3)),
 * restarts from S_i = -H_{m+1,m} E_m^T Z_i (eq. (35)) and adds V_m sum_i 2 Re(omega_i Z_i).
 * Returns EXPM_NOT_CONVERGED (Z holds the last iterate) if max_cycles is reached.
 * Synchronises the plan's stream once per cycle (residual norms to the host).
 * ------------------------------------------------------------------------------ */
expm_status expm_block(expm_plan* plan, double t, const double* dB, int64_t ldb, int p,
                       double* dZ, int64_t ldz, expm_info* info);

/* expm_block_host -- the same computation with HOST buffers: copies B (n x p, ldb) to
 * the plan's device staging buffer, runs expm_block, copies Z back (n x p, ldz).
 * B and Z are ordinary (preferably page-locked) host memory.  Same errors. */
expm_status expm_block_host(expm_plan* plan, double t, const double* hB, int64_t ldb,
                            int p, double* hZ, int64_t ldz, expm_info* info);

/* ---------------------------------------------------------------------------------
 * expm_block_batched -- count independent calls of expm_block in one call: instance i
 * computes dZ[i] = r(t[i] A_i) dB[i] with plans[i] (n_i x p[i], leading dimensions ldb[i],
 * ldz[i]).  Instances of different order, width, time and operator family may be mixed.
 * Each plan's restart cycles run on that plan's stream (as captured CUDA graphs when the
 * stream is not the legacy default stream); the host keeps every instance's next cycle
 * queued as soon as its stop test has been read, so instances on distinct streams overlap
 * on the GPU.  The paper solves one problem at a time; this is a serving variant.
 *   plans : host array of count distinct plans (one call per plan: the plan's workspace)
 *   t, ldb, p, ldz : host arrays of count entries; dB, dZ: host arrays of device pointers
 *   info  : host array of count expm_info (may be NULL)
 * Returns the first hard error of any instance, else EXPM_NOT_CONVERGED if any instance
 * stopped unconverged (its Z is still written), else EXPM_OK.  Synchronises every plan's
 * stream.  Errors: EXPM_INVALID_ARG (bad argument of any instance, a repeated plan) and
 * those of expm_block.
 * ------------------------------------------------------------------------------ */
expm_status expm_block_batched(expm_plan* const* plans, int count, const double* t,
                               const double* const* dB, const int64_t* ldb, const int* p,
                               double* const* dZ, const int64_t* ldz, expm_info* info);

/* expm_block_batched_host -- expm_block_batched with HOST buffers: hB[i] (n_i x p[i], ldb[i])
 * is copied to plans[i]'s device staging buffer on the plan's stream before the instance's
 * first cycle, and Z back to hZ[i] (ldz[i]) after its last, so one instance's copies overlap
 * with the others' cycles.  hB[i] and hZ[i] are ordinary (preferably page-locked) host
 * memory.  Same errors as expm_block_batched. */
expm_status expm_block_batched_host(expm_plan* const* plans, int count, const double* t,
                                    const double* const* hB, const int64_t* ldb, const int* p,
                                    double* const* hZ, const int64_t* ldz, expm_info* info);

/* ---------------------------------------------------------------------------------
 * expm_batch_create / expm_batch_run / expm_batch_destroy -- many independent solves as ONE
 * CUDA graph launch (a serving variant; the paper solves one problem at a time).  Instance i
 * computes dZ[i] = r(t[i] A_i) dB[i] with plans[i] as expm_block would; every instance is one
 * branch of the graph: its start, a device-side WHILE loop of restart cycles whose stop test
 * (eq. (49) / eq. (365), max_cycles, fixed_cycles) runs in a kernel and sets the loop's
 * condition, and its finish.  The branches run concurrently and no host work happens between
 * cycles.  The graph is built once (create) and replayed by every run with the same
 * arguments; the buffers dB, dZ must stay valid and in place for the batch's lifetime.
 *   plans  : distinct plans, each with a stream other than the legacy default stream, no
 *            deflated restart (opts.k_defl = 0: its eigenproblem runs on the host) and no
 *            certify mode
 *   t, dB, ldb, p, dZ, ldz : as expm_block_batched
 *   stream : cudaStream_t on which expm_batch_run launches the graph
 *   out    : host, receives the batch (free with expm_batch_destroy)
 * expm_batch_run launches the graph, synchronises the stream and fills info[i] (may be NULL);
 * it returns the first hard error, else EXPM_NOT_CONVERGED if any instance stopped
 * unconverged, else EXPM_OK.  While a batch runs, its plans must not be used by other calls.
 * Errors: EXPM_INVALID_ARG, EXPM_NO_MEMORY, EXPM_CUDA_ERROR, and those of expm_block. */
typedef struct expm_batch_s expm_batch;
expm_status expm_batch_create(expm_plan* const* plans, int count, const double* t,
                              const double* const* dB, const int64_t* ldb, const int* p,
                              double* const* dZ, const int64_t* ldz, void* stream, expm_batch** out);
expm_status expm_batch_run(expm_batch* batch, expm_info* info);
void expm_batch_destroy(expm_batch* batch);

/* ---------------------------------------------------------------------------------
 * expm_block_adjoint -- the adjoint of Z = r(tA) B for a loss L with G = dL/dZ:
 *   dGB = dL/dB = r(tA)^T G = r(tA^T) G  (r has real coefficients), computed by the same
 *         method on A^T: for EXPM_OP_CONV_DIFF the stencil with the velocity negated
 *         (central differences), held in a companion plan created on the first call with
 *         the plan's options (it allocates); a Toeplitz operator is its own transpose;
 *   hGt = dL/dt = <G, A Z>  (d/dt e^{tA} B = A e^{tA} B; the derivative of the exponential
 *         that r approximates), from the forward result Z.
 * Nothing of the forward Krylov bases is kept: the backward solve recomputes its own.
 *   dG  : device n x p (ldg), not modified;  1 <= p <= p_max
 *   dZ  : device n x p (ldz), the forward result (needed only when hGt != NULL)
 *   dGB : device n x p out (ldgb), or NULL to skip dL/dB; must not alias dG or dZ
 *   hGt : host, 1 double out, or NULL to skip dL/dt
 *   info: host out (may be NULL): the A^T solve's info
 * Synchronises the plan's stream.  Errors: those of expm_block, EXPM_INVALID_ARG when both
 * outputs are NULL.
 * ------------------------------------------------------------------------------ */
expm_status expm_block_adjoint(expm_plan* plan, double t, const double* dG, int64_t ldg, int p,
                               const double* dZ, int64_t ldz, double* dGB, int64_t ldgb,
                               double* hGt, expm_info* info);

/* ---------------------------------------------------------------------------------
 * Component entry points (the hot path's kernels, exposed for parity tests and
 * measurement).  All are stream-ordered on the plan's stream and do not synchronise.
 *
 * expm_op_apply   : W = tA V  (the operator of Algorithm 1 and of the residual
 *                   B - (tA - tau I) X; Section 1 / eq. (3)).
 * expm_prec_apply : W = (tA)^{-1} V, the exact inner solve that replaces the paper's
 *                   sparse LU (Section 4.1, "U \ (L \ w)"): a transform along every
 *                   axis but x with the axis' eigenvectors (diagonal similarity + DST-I),
 *                   then tridiagonal solves along x for each transformed mode; for a
 *                   Toeplitz operator the Gohberg-Semencul formula (six FFTs per column
 *                   pair; EXPM_INVALID_ARG if the plan was created for EXPM_ALG_SBFOM).
 *   dV, dW : device, n x p (ld >= n), must not alias; 1 <= p <= p_max.
 * Errors: EXPM_INVALID_ARG, EXPM_CUDA_ERROR (launch failure).
 * ------------------------------------------------------------------------------ */
expm_status expm_op_apply(expm_plan* plan, double t, const double* dV, int64_t ldv, int p,
                          double* dW, int64_t ldw);
expm_status expm_prec_apply(expm_plan* plan, double t, const double* dV, int64_t ldv, int p,
                            double* dW, int64_t ldw);

/* expm_prec_apply_noalloc -- W = (tA)^{-1} V like expm_prec_apply, for callers that cannot
 * call cudaMalloc (for example a host application whose own pool allocator owns all device
 * memory and forbids raw allocations by libraries, or a latency-critical loop that must not
 * enter the CUDA allocator).  The paper has no counterpart: this is a deployment variant.
 * It needs no plan and allocates nothing: the transform tables, the Thomas factors and the
 * transform temporary live in one fixed 8 MiB device array inside the library (held by every
 * GPU that loads the library until the process exits).  Each call rebuilds what it reads.
 *   op        : host descriptor, EXPM_OP_CONV_DIFF with ndim 1 or 2
 *   dV, dW    : device, n x p (ld >= n), must not alias; 1 <= p <= 32
 *   stream    : cudaStream_t (NULL = legacy default stream); the call is stream-ordered
 * Size limit: 1-D needs 2n doubles, 2-D needs 2 N_y^2 + N_y + 2n + n p doubles (each
 * region rounded up to 32) within 2^20 doubles; larger problems return EXPM_INVALID_ARG.
 * The first call on a device looks up the array's device address (cudaGetSymbolAddress)
 * with that device current; make that first call before any stream capture.  All calls
 * share the array, so calls that overlap on the GPU (different streams or host threads on
 * one device) race: order them.  Errors: EXPM_INVALID_ARG, EXPM_CUDA_ERROR. */
expm_status expm_prec_apply_noalloc(const expm_op_desc* op, double t, const double* dV,
                                    int64_t ldv, int p, double* dW, int64_t ldw, void* stream);

/* expm_arnoldi -- one block Arnoldi pass (eq. (4.5)) from an orthonormal V_1:
 *   dV1 : device n x p (ldv1), orthonormal start block (copied into the basis)
 *   dVout : device n x (m+1)p out (ldvo), the basis V_{m+1}
 *   dHout : device (m+1)p x mp out (ldh), the band Hessenberg H~_m
 * With Cholesky-QR the new blocks' R factors have a positive diagonal, so the basis
 * equals Ruhe's variant's (Section 3) in exact arithmetic.  Synchronises the stream
 * (status flags).  Errors: EXPM_INVALID_ARG, EXPM_NUMERICAL, EXPM_CUDA_ERROR. */
expm_status expm_arnoldi(expm_plan* plan, double t, const double* dV1, int64_t ldv1, int p,
                         double* dVout, int64_t ldvo, double* dHout, int64_t ldh);

/* ---------------------------------------------------------------------------------
 * Profiling (not part of the paper: measurement support).  Kernel launches are always
 * counted; with profiling enabled, CUDA events on the plan's stream bracket every launch
 * and their durations are accumulated per kernel class at each stream synchronisation.
 * expm_plan_profile(plan, 1) resets the counters and enables timing, (plan, 0) disables.
 * expm_plan_get_profile copies min(nstages, EXPM_NSTAGES) entries (host arrays, either may
 * be NULL) and the total launch count.  Errors: EXPM_INVALID_ARG, EXPM_CUDA_ERROR.
 * ------------------------------------------------------------------------------ */
typedef enum {
    EXPM_STAGE_GEMM = 0,      /* DST-I transforms of the exact inverse (batched FP64 GEMM) */
    EXPM_STAGE_TRIDIAG = 1,   /* tridiagonal line solves of the exact inverse            */
    EXPM_STAGE_CGS = 2,       /* block CGS2 row passes (projection / update)             */
    EXPM_STAGE_REDUCE = 3,    /* partial-sum reductions of the projections                */
    EXPM_STAGE_QR = 4,        /* Cholesky-QR (Gram/Cholesky/triangular solve)             */
    EXPM_STAGE_POLES = 5,     /* projected shifted systems (eq. (3236)) + combination     */
    EXPM_STAGE_UPDATE = 6,    /* Z += V_{m+1} Wc and restart copy                          */
    EXPM_STAGE_OTHER = 7,     /* copies, initialisation, final Z = omega_0 B + Z_acc       */
    EXPM_STAGE_STENCIL = 8,   /* W = tA V                                                  */
    EXPM_NSTAGES = 9
} expm_stage;

expm_status expm_plan_profile(expm_plan* plan, int enable);
expm_status expm_plan_get_profile(expm_plan* plan, double* stage_ms, int64_t* stage_launches,
                                  int nstages, int64_t* total_launches);

/* expm_peak_fma -- measurement support for the roofline denominators (not part of the
 * paper's method): the device's FMA throughput, kind 0 = FP64, 1 = FP32, from one launch of
 * eight independent FMA chains per thread on every SM (iters FMAs per chain), timed with
 * CUDA events on the stream.  tflops: host out, 2 flops per FMA.  Synchronises the stream.
 * Errors: EXPM_INVALID_ARG, EXPM_CUDA_ERROR. */
expm_status expm_peak_fma(int kind, int64_t iters, double* tflops, void* stream);

const char* expm_status_str(expm_status s);

#ifdef __cplusplus
}
#endif

#endif /* EXPM_BLOCK_H */
