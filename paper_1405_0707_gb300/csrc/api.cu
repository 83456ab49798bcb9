// api.cu -- C ABI entry points and the restart-cycle driver of Algorithm 2 (PSBFOM, k = 0).
//
// Host side of one call to expm_block:
//   start (Algorithms 1 and 2 alike): X_i^0 = 0, R_i^0 = B = V_1 R  (Cholesky QR)
//   per cycle:
//     block Arnoldi: m block steps W = (tA)^{-1} V_j -> CGS2 -> Cholesky QR -> V_{j+1}, H~_m (eq. (4.5))
//     projected systems: all poles in one launch (eq. (3236)), norms by eq. (49),
//             Z += V_{m+1} sum_i 2 Re(omega_i H~_m Z_i); restart V_1 <- V_{m+1}
//     one device->host copy of the nu/2 residual norms + status flags, then the stop test
//   Z = omega_0 B + Z_acc   (eq. (11) with the conjugate pairs folded)
#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <new>
#include <thread>

#include "internal.h"

using namespace expm;

namespace {

#define CK(call)                                          \
    do {                                                  \
        if ((call) != cudaSuccess) return EXPM_CUDA_ERROR; \
    } while (0)

constexpr int kNu = 14;
constexpr int kStatDoubles = 32;   // res[0..15], normsq at [16], int flags at doubles [24..25]

// small scratch map (in doubles)
constexpr size_t kOffH = 0;                                        // h: kMaxMP x kMaxP
constexpr size_t kOffR = kOffH + (size_t)kMaxMP * kMaxP;           // R
constexpr size_t kOffRi = kOffR + kMaxP * kMaxP;                   // R^{-1}
constexpr size_t kOffRt = kOffRi + kMaxP * kMaxP;                  // product of R factors
constexpr size_t kOffWc = kOffRt + kMaxP * kMaxP;                  // (kMaxMP + kMaxP) x kMaxP
constexpr size_t kOffTau = kOffWc + (size_t)(kMaxMP + kMaxP) * kMaxP;   // 4 x 16
constexpr size_t kOffG = kOffTau + 4 * EXPM_MAX_POLES;               // reduced Gram matrix
constexpr size_t kOffRt2 = kOffG + kMaxP * kMaxP;                    // Rtot after pass 2
constexpr size_t kOffRt3 = kOffRt2 + kMaxP * kMaxP;                  // Rtot after pass 3
constexpr size_t kSmallDoubles = kOffRt3 + kMaxP * kMaxP;

inline int64_t round_up(int64_t a, int64_t b) { return (a + b - 1) / b * b; }
inline int* flags_of(double* stat) { return reinterpret_cast<int*>(stat + 24); }

double* sm(expm_plan* P, size_t off) { return P->small + off; }

// ---- profiling: count every launch; with profiling on, bracket it with events
constexpr int kEventPool = 2048;
int prof_begin(expm_plan* P) {
    if (!P->prof || P->ev_used + 2 > (int)P->ev.size()) return -1;
    const int e = P->ev_used;
    P->ev_used += 2;
    cudaEventRecord(P->ev[e], P->stream);
    return e;
}
void prof_end(expm_plan* P, int stage, int e, int nlaunch) {
    P->launches += nlaunch;
    P->stage_launches[stage] += nlaunch;
    if (e < 0) return;
    cudaEventRecord(P->ev[e + 1], P->stream);
    P->pend_stage.push_back(stage);
}
// after a stream synchronisation: fold the pending event pairs into the stage totals
void prof_flush(expm_plan* P) {
    for (size_t k = 0; k < P->pend_stage.size(); ++k) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, P->ev[2 * k], P->ev[2 * k + 1]) == cudaSuccess)
            P->stage_ms[P->pend_stage[k]] += ms;
    }
    P->pend_stage.clear();
    P->ev_used = 0;
}

#define LAUNCH(stage, call)                          \
    do {                                             \
        const int e_ = prof_begin(P);                \
        if ((call) != cudaSuccess) return EXPM_CUDA_ERROR; \
        prof_end(P, (stage), e_, 1);                 \
    } while (0)

// The mixed path with p <= 8 runs the Cholesky QR with FP32 factorisations fused into the
// triangular solves (k_qr_mixed_rows); everything else uses k_chol + k_trsm.
inline bool fused_qr(const expm_plan* P, int p) {
    return p <= kRowsMaxP && P->opts.precision == EXPM_PREC_MIXED;
}

// cgs_cols > 0 (mixed path, after the row-chunk CGS kernels): the first pass also applies
// the second CGS pass's correction W -= V[:, 0:cgs_cols] h, with h followed by the Gram
// matrix of W before it (k_qr_mixed_rows<3>).
expm_status qr_block(expm_plan* P, int p, double* out, int64_t ldo, bool withH, int hrow, int hcol,
                     double* normsq, bool gram_done, int cgs_cols = 0) {
    cudaStream_t s = P->stream;
    const int64_t n = P->n, ld = P->ld;
    const double shift = 11.0 * ((double)n * p + (double)p * (p + 1)) * std::ldexp(1.0, -53);
    int* flags = flags_of(P->stat);
    if (fused_qr(P, p)) {
        // mixed path: three passes with FP32 factorisations fused into the triangular solves;
        // the Gram matrix arrives reduced in G (from the last Gram-Schmidt pass, or here)
        double* G = sm(P, kOffG);
        double* Hq = withH ? P->H : nullptr;
        if (!gram_done) {
            LAUNCH(EXPM_STAGE_QR, launch_proj_partial(P->W, ld, p, P->W, ld, p, n, P->part, P->nblk, s));
            LAUNCH(EXPM_STAGE_QR, launch_reduce_h(P->part, P->nblk, p, p, G, nullptr, 0, 0, 0, 0, s));
        }
        LAUNCH(EXPM_STAGE_QR, launch_qr_mixed_rows(P->W, ld, p, n, P->nblk, G, P->part, P->ctr, 0, sm(P, kOffR),
                                                   sm(P, kOffRi), nullptr, sm(P, kOffRt), Hq, P->ldH, hrow, hcol,
                                                   normsq, flags, P->W, ld, s, cgs_cols ? P->V : nullptr, ld,
                                                   cgs_cols, cgs_cols ? sm(P, kOffH) : nullptr,
                                                   (cgs_cols && P->qr_single) ? out : nullptr, ldo));
        LAUNCH(EXPM_STAGE_QR, launch_qr_mixed_rows(P->W, ld, p, n, P->nblk, G, P->part, P->ctr, 1, sm(P, kOffR),
                                                   sm(P, kOffRi), sm(P, kOffRt), sm(P, kOffRt2), Hq, P->ldH, hrow,
                                                   hcol, nullptr, flags, out, ldo, s));
        LAUNCH(EXPM_STAGE_QR, launch_qr_mixed_rows(P->W, ld, p, n, P->nblk, G, P->part, P->ctr, 2, sm(P, kOffR),
                                                   sm(P, kOffRi), sm(P, kOffRt2), sm(P, kOffRt3), Hq, P->ldH, hrow,
                                                   hcol, nullptr, flags, out, ldo, s));
        return EXPM_OK;
    }
    if (!gram_done) LAUNCH(EXPM_STAGE_QR, launch_proj_partial(P->W, ld, p, P->W, ld, p, n, P->part, P->nblk, s));
    double* Hq = withH ? P->H : nullptr;
    const int* extra = flags + 2;
    // pass 1: unshifted Cholesky, shifted when W is ill-conditioned (sets the third-pass flag)
    LAUNCH(EXPM_STAGE_QR, launch_chol(P->part, P->nblk, p, shift, sm(P, kOffR), sm(P, kOffRi),
                                      sm(P, kOffRt), 0, Hq, P->ldH, hrow, hcol, normsq, flags, s));
    LAUNCH(EXPM_STAGE_QR, launch_trsm(P->W, ld, p, n, sm(P, kOffRi), P->W, ld, P->part, P->nblk, 1, extra, 0, s));
    // pass 2: the last one for a well-conditioned block (writes the final block directly)
    LAUNCH(EXPM_STAGE_QR, launch_chol(P->part, P->nblk, p, 0.0, sm(P, kOffR), sm(P, kOffRi),
                                      sm(P, kOffRt), 1, Hq, P->ldH, hrow, hcol, nullptr, flags, s));
    LAUNCH(EXPM_STAGE_QR, launch_trsm(P->W, ld, p, n, sm(P, kOffRi), out, ldo, P->part, P->nblk, 1, extra, 1, s));
    // pass 3: only when pass 1 needed the shift (no-op otherwise)
    LAUNCH(EXPM_STAGE_QR, launch_chol(P->part, P->nblk, p, 0.0, sm(P, kOffR), sm(P, kOffRi),
                                      sm(P, kOffRt), 2, Hq, P->ldH, hrow, hcol, nullptr, flags, s));
    LAUNCH(EXPM_STAGE_QR, launch_trsm(P->W, ld, p, n, sm(P, kOffRi), out, ldo, nullptr, P->nblk, 0, extra, 2, s));
    return EXPM_OK;
}

// One FP32 application of (tA)^{-1} to R (FP64 in), written (acc = 0) or added (acc = 1)
// to X (FP64).  Same transforms and layouts as the FP64 path.
expm_status inv32_apply(expm_plan* P, double t, const void* R, int64_t ldr, int p, double* X,
                        int64_t ldx, int acc, int r_f64 = 1) {
    cudaStream_t s = P->stream;
    const int nx = P->ax[0].N, ny = P->ax[1].N, nz = P->ax[2].N;
    const int64_t ld = P->ld;
    const float lsub = (float)P->ax[0].l, inv_t = (float)(1.0 / t);
    if (P->ndim == 2) {
        GemmArgsMixed g1{R, P->Qf32[1], P->T1f, nx, ny, ny, 1, nx, ldr, 0, ny, 1, ld, 0, ny, p, 1, r_f64, 0, 0};
        LAUNCH(EXPM_STAGE_GEMM, launch_gemm32(g1, s));
        LAUNCH(EXPM_STAGE_TRIDIAG, launch_tridiag_lines32(P->T1f, ld, p, nx, ny, lsub, P->th_m32, P->th_c32, inv_t, s));
        GemmArgsMixed g2{P->T1f, P->Qi32[1], X, nx, ny, ny, ny, 1, ld, 0, 1, nx, ldx, 0, ny, p, 1, 0, 1, acc};
        LAUNCH(EXPM_STAGE_GEMM, launch_gemm32(g2, s));
        return EXPM_OK;
    }
    const int64_t nxy = (int64_t)nx * ny;
    GemmArgsMixed g1{R, P->Qf32[2], P->T2f, (int)nxy, nz, nz, 1, nxy, ldr, 0, 1, nxy, ld, 0, nz, p, 1, r_f64, 0, 0};
    LAUNCH(EXPM_STAGE_GEMM, launch_gemm32(g1, s));
    // the y transforms take (x, z) as one row index of nx nz rows (no padding per x line)
    GemmArgsMixed g2{P->T2f, P->Qf32[1], P->T1f, nx * nz, ny, ny, 1, nx, ld, 0, (int64_t)ny * nz, 1, ld, 0, ny, p, 1,
                     0, 0, 0, nx, nxy, ny};
    LAUNCH(EXPM_STAGE_GEMM, launch_gemm32(g2, s));
    LAUNCH(EXPM_STAGE_TRIDIAG, launch_tridiag_lines32(P->T1f, ld, p, nx, (int64_t)ny * nz, lsub, P->th_m32,
                                                      P->th_c32, inv_t, s));
    GemmArgsMixed g3{P->T1f, P->Qi32[1], P->T2f, nx * nz, ny, ny, (int64_t)ny * nz, 1, ld, 0, 1, nx, ld, 0, ny, p, 1,
                     0, 0, 0, nx, ny, nxy};
    LAUNCH(EXPM_STAGE_GEMM, launch_gemm32(g3, s));
    GemmArgsMixed g4{P->T2f, P->Qi32[2], X, (int)nxy, nz, nz, 1, nxy, ld, 0, 1, nxy, ldx, 0, nz, p, 1, 0, 1, acc};
    LAUNCH(EXPM_STAGE_GEMM, launch_gemm32(g4, s));
    return EXPM_OK;
}

// Mixed precision: W = (tA)^{-1} V to FP64 accuracy by iterative refinement of the FP32
// inverse: x_0 = inv32(V), x_{k+1} = x_k + inv32(V - tA x_k) with the residual in FP64
// (Theorem 4.3: the inverse's accuracy is what the shifted solutions inherit).  Each step
// multiplies the backward error by about eps_32 * rho^-N (diagonal similarity).
expm_status prec_apply_mixed(expm_plan* P, double t, const double* V, int64_t ldv, int p,
                             double* W, int64_t ldw) {
    cudaStream_t s = P->stream;
    expm_status st = inv32_apply(P, t, V, ldv, p, W, ldw, 0);
    if (st != EXPM_OK) return st;
    for (int k = 0; k < P->refine; ++k) {
        // the residual V - tA x in FP64, stored in FP32 (the R64 buffer): the transforms read
        // it as FP32 either way
        float* R32 = reinterpret_cast<float*>(P->R64);
        LAUNCH(EXPM_STAGE_STENCIL, launch_cd_apply(W, ldw, nullptr, P->ld, p, P->ndim, P->ax[0].N, P->ax[1].N,
                                                   P->ax[2].N, P->ax, -t, s, V, ldv, 1.0, R32, P->stencil_df & 2));
        st = inv32_apply(P, t, R32, P->ld, p, W, ldw, 1, 0);
        if (st != EXPM_OK) return st;
    }
    return EXPM_OK;
}

// ---- symmetric Toeplitz operator (k_fft.cu): products and the Gohberg-Semencul inverse
int toeplitz_nseq_max(const expm_plan* P) { return std::max(2, (P->p_max + 1) / 2); }

FftArgs fft_args(const expm_plan* P) {
    const ToeplitzOp& z = P->tz;
    FftArgs a;
    a.f = z.f;
    a.nreal = z.n;
    a.tw1 = z.tw1;
    a.tw2 = z.tw2;
    a.thi = z.thi;
    a.tlo = z.tlo;
    a.tw1f = z.tw1f;
    a.tw2f = z.tw2f;
    a.thif = z.thif;
    a.tlof = z.tlof;
    a.df = z.use_df ? 1 : 0;
    a.lam = z.lam;
    a.mu1 = z.mu1;
    a.mu2 = z.mu2;
    return a;
}

// W = tT V: per group of up to 2 nseq_max columns, the forward column pass (pairs of real
// columns packed as one complex sequence), the fused row pass (forward, times t lambda / N,
// inverse) and the inverse column pass (real and imaginary parts to the two columns).
expm_status toeplitz_matvec(expm_plan* P, double t, const double* V, int64_t ldv, int p, double* W,
                            int64_t ldw, int stage) {
    cudaStream_t s = P->stream;
    const int maxcols = 2 * toeplitz_nseq_max(P);
    for (int c0 = 0; c0 < p; c0 += maxcols) {
        const int pc = std::min(maxcols, p - c0), nseq = (pc + 1) / 2;
        FftArgs a = fft_args(P);
        a.V = V + (int64_t)c0 * ldv;
        a.ldv = ldv;
        a.W = W + (int64_t)c0 * ldw;
        a.ldw = ldw;
        a.p = pc;
        a.in = a.out = P->tz.Ua;
        a.scale = t / (double)P->tz.f.N;
        LAUNCH(stage, launch_fft_cols(a, FFT_COL_FWD_REAL, nseq, s));
        LAUNCH(stage, launch_fft_rows(a, FFT_ROW_MATVEC, nseq, s));
        a.scale = 1.0;
        LAUNCH(stage, launch_fft_cols(a, FFT_COL_INV_REAL, nseq, s));
    }
    return EXPM_OK;
}

// W = (tT)^{-1} V by the Gohberg-Semencul formula: five passes per column group (six
// transforms per sequence; see k_fft.cu).
expm_status toeplitz_inverse(expm_plan* P, double t, const double* V, int64_t ldv, int p, double* W,
                             int64_t ldw, int stage) {
    cudaStream_t s = P->stream;
    const ToeplitzOp& z = P->tz;
    const int maxcols = 2 * toeplitz_nseq_max(P);
    const int64_t N = z.f.N;
    for (int c0 = 0; c0 < p; c0 += maxcols) {
        const int pc = std::min(maxcols, p - c0), nseq = (pc + 1) / 2;
        FftArgs a = fft_args(P);
        a.V = V + (int64_t)c0 * ldv;
        a.ldv = ldv;
        a.W = W + (int64_t)c0 * ldw;
        a.ldw = ldw;
        a.p = pc;
        a.out = z.Ua;
        LAUNCH(stage, launch_fft_cols(a, FFT_COL_FWD_REAL, nseq, s));                  // F v
        a.in = z.Ua;
        a.out = z.Ub;
        a.out2 = z.Ub + 2 * N * nseq;
        a.scale = 1.0 / (double)N;
        LAUNCH(stage, launch_fft_rows(a, FFT_ROW_GSF_A, nseq, s));                     // conj(mu_k) F v, inverse rows
        a.in = a.out = z.Ub;
        LAUNCH(stage, launch_fft_cols(a, FFT_COL_INV_TRUNC_FWD, 2 * nseq, s));         // u_k, truncated, forward
        a.in = z.Ub;
        a.in2 = z.Ub + 2 * N * nseq;
        a.out = z.Ua;
        a.scale = 1.0 / ((double)N * t * z.x0);
        LAUNCH(stage, launch_fft_rows(a, FFT_ROW_GSF_B, nseq, s));                     // mu_1 F u_1 - mu_2 F u_2
        a.in = z.Ua;
        a.scale = 1.0;
        LAUNCH(stage, launch_fft_cols(a, FFT_COL_INV_REAL, nseq, s));                  // first n entries
    }
    return EXPM_OK;
}

// W = tA V for either operator family
expm_status op_apply_internal(expm_plan* P, double t, const double* V, int64_t ldv, int p, double* W,
                              int64_t ldw) {
    if (P->toeplitz) return toeplitz_matvec(P, t, V, ldv, p, W, ldw, EXPM_STAGE_STENCIL);
    if (P->csr) {
        LAUNCH(EXPM_STAGE_STENCIL, launch_csr_spmm(P->cs, t, V, ldv, p, W, ldw, P->stream));
        return EXPM_OK;
    }
    LAUNCH(EXPM_STAGE_STENCIL, launch_cd_apply(V, ldv, W, ldw, p, P->ndim, P->ax[0].N, P->ax[1].N, P->ax[2].N,
                                               P->ax, t, P->stream, nullptr, 0, 0.0, nullptr, P->stencil_df & 1));
    return EXPM_OK;
}

expm_status prec_apply_internal(expm_plan* P, double t, const double* V, int64_t ldv, int p,
                                double* W, int64_t ldw) {
    cudaStream_t s = P->stream;
    if (P->toeplitz) {
        if (!P->tz.gsf) return EXPM_INVALID_ARG;
        return toeplitz_inverse(P, t, V, ldv, p, W, ldw, EXPM_STAGE_GEMM);
    }
    if (P->csr) {
        // the inexact inverse of Section 4.1 (inner BiCGStab to opts.inner_tol, k_csr.cu);
        // its stop test synchronises the stream, so these plans run without cycle graphs
        int iters = 0, conv = 0;
        const double eta = P->opts.inner_tol > 0.0 ? P->opts.inner_tol : 1e-12;
        const int maxit = P->opts.inner_maxit > 0 ? P->opts.inner_maxit : 2000;
        ++P->launches;
        CK(csr_inverse(P->cs, t, V, ldv, p, W, ldw, eta, maxit, s, &iters, &conv));
        P->inner_iters += iters;
        return conv ? EXPM_OK : EXPM_NOT_CONVERGED;
    }
    if (P->opts.precision == EXPM_PREC_MIXED && P->ndim > 1) return prec_apply_mixed(P, t, V, ldv, p, W, ldw);
    const double inv_t = 1.0 / t;
    const int nx = P->ax[0].N, ny = P->ax[1].N, nz = P->ax[2].N;
    const int64_t ld = P->ld;
    const double lsub = P->ax[0].l;
    if (P->ndim == 1) {
        LAUNCH(EXPM_STAGE_TRIDIAG, launch_tridiag_lines(V, ldv, W, ldw, p, nx, 1, lsub, P->th_m, P->th_c, inv_t, s));
        return EXPM_OK;
    }
    if (P->ndim == 2) {
        GemmArgs g1{V, P->Qf[1], P->T1, nx, ny, ny, 1, nx, ldv, 0, ny, 1, ld, 0, ny, p, 1};
        LAUNCH(EXPM_STAGE_GEMM, launch_gemm(g1, s));
        LAUNCH(EXPM_STAGE_TRIDIAG, launch_tridiag_lines(P->T1, ld, P->T1, ld, p, nx, ny, lsub, P->th_m, P->th_c, inv_t, s));
        GemmArgs g2{P->T1, P->Qi[1], W, nx, ny, ny, ny, 1, ld, 0, 1, nx, ldw, 0, ny, p, 1};
        LAUNCH(EXPM_STAGE_GEMM, launch_gemm(g2, s));
        return EXPM_OK;
    }
    const int64_t nxy = (int64_t)nx * ny;
    GemmArgs g1{V, P->Qf[2], P->T2, (int)nxy, nz, nz, 1, nxy, ldv, 0, 1, nxy, ld, 0, nz, p, 1};
    LAUNCH(EXPM_STAGE_GEMM, launch_gemm(g1, s));
    GemmArgs g2{P->T2, P->Qf[1], P->T1, nx, ny, ny, 1, nx, ld, nxy, (int64_t)ny * nz, 1, ld, ny, ny, p, nz};
    LAUNCH(EXPM_STAGE_GEMM, launch_gemm(g2, s));
    LAUNCH(EXPM_STAGE_TRIDIAG, launch_tridiag_lines(P->T1, ld, P->T1, ld, p, nx, (int64_t)ny * nz, lsub,
                                                    P->th_m, P->th_c, inv_t, s));
    GemmArgs g3{P->T1, P->Qi[1], P->T2, nx, ny, ny, (int64_t)ny * nz, 1, ld, ny, 1, nx, ld, nxy, ny, p, nz};
    LAUNCH(EXPM_STAGE_GEMM, launch_gemm(g3, s));
    GemmArgs g4{P->T2, P->Qi[2], W, (int)nxy, nz, nz, 1, nxy, ld, 0, 1, nxy, ldw, 0, nz, p, 1};
    LAUNCH(EXPM_STAGE_GEMM, launch_gemm(g4, s));
    return EXPM_OK;
}

// Block step j (0-based): V_j -> W = Op V_j -> V_{j+1}, H column block j.
// Op = (tA)^{-1} (Algorithm 2) or tA (Algorithm 1).
expm_status block_step(expm_plan* P, double t, int j, int p, int alg) {
    cudaStream_t s = P->stream;
    const int64_t n = P->n, ld = P->ld;
    double* h = sm(P, kOffH);
    const double* Vj = P->V + (int64_t)j * p * ld;
    if (alg == 2) {
        expm_status st = prec_apply_internal(P, t, Vj, ld, p, P->W, ld);
        if (st != EXPM_OK) return st;
    } else {
        expm_status st = op_apply_internal(P, t, Vj, ld, p, P->W, ld);
        if (st != EXPM_OK) return st;
    }
    const int cols = (j + 1) * p;
    const int f32 = P->opts.precision == EXPM_PREC_MIXED ? 1 : 0;
    const int nbc = P->nblk_cgs;
    // first pass: FP64, or in the mixed path FP32 projection and double-float update (the
    // row-chunk kernels for p <= 16, else the tile kernels)
    const bool rows = f32 && cgs_rows_fit(cols, p);
    // the projection on the tensor cores (TF32 hi/lo products) when the plan chose it: by
    // default for p >= 8 and 48 <= cols <= 128 (one M tile), where it measured faster than
    // the FP32 kernel (whose cost grows with p; the tensor-core pass has a fixed cost per
    // 16-row chunk), and with at least one 256-row tile per CTA of the plan's CGS grid (its
    // set-up and per-tile read-back are amortised only then: on 256 x 256 it was slower)
    const bool ptc = rows && P->proj_tc && proj_tc_fit(cols, p) &&
                     (P->proj_tc == 1 || (p >= 8 && cols >= 48 && cols <= 128 && n >= (int64_t)256 * nbc));
    const int nb1 = ptc ? proj_tc_blocks(n, cols, nbc) : nbc;
    if (ptc)
        LAUNCH(EXPM_STAGE_CGS, launch_proj_tc(P->V, ld, cols, P->W, ld, p, n, P->part, nb1, flags_of(P->stat),
                                              P->tc_spin, s));
    else if (rows) LAUNCH(EXPM_STAGE_CGS, launch_cgs_rows(0, P->V, ld, cols, P->W, ld, p, n, nullptr, P->part, nbc, 0, s));
    else LAUNCH(EXPM_STAGE_CGS, launch_proj_partial(P->V, ld, cols, P->W, ld, p, n, P->part, nbc, s, f32));
    LAUNCH(EXPM_STAGE_REDUCE, launch_reduce_h(P->part, nb1, cols, p, h, P->H, P->ldH, 0, j * p, 0, s));
    if (rows && fused_qr(P, p)) {
        // update, second projection and the Gram matrix of W; the second pass's correction is
        // applied by the first Cholesky-QR pass.  The update on the tensor cores (exact bf16
        // slicing, k_cgs_tc) when the plan chose it, followed by the FP32 projection kernel with
        // the Gram outputs; else all three in one double-float pass on the FP32 pipe
        if (P->cgs_tc && cgs_tc_fit(cols, p) && (P->cgs_tc == 1 || (p >= 12 && cols >= 64))) {
            LAUNCH(EXPM_STAGE_CGS, launch_cgs_tc(P->V, ld, cols, P->W, ld, p, n, h, flags_of(P->stat), P->tc_spin, s));
            LAUNCH(EXPM_STAGE_CGS, launch_cgs_rows(0, P->V, ld, cols, P->W, ld, p, n, nullptr, P->part, nbc, 1, s));
            LAUNCH(EXPM_STAGE_REDUCE, launch_reduce_h(P->part, nbc, cols + p, p, h, P->H, P->ldH, 0, j * p, 1, s, cols));
        } else {
            LAUNCH(EXPM_STAGE_CGS, launch_cgs_rows(1, P->V, ld, cols, P->W, ld, p, n, h, P->part, nbc, 1, s));
            LAUNCH(EXPM_STAGE_REDUCE, launch_reduce_h(P->part, nbc, cols + p, p, h, P->H, P->ldH, 0, j * p, 1, s, cols));
        }
        return qr_block(P, p, P->V + (int64_t)(j + 1) * p * ld, ld, true, (j + 1) * p, j * p, nullptr, true, cols);
    }
    if (rows) LAUNCH(EXPM_STAGE_CGS, launch_cgs_rows(1, P->V, ld, cols, P->W, ld, p, n, h, P->part, nbc, 0, s));
    else LAUNCH(EXPM_STAGE_CGS, launch_update_proj(P->V, ld, cols, P->W, ld, p, n, h, P->part, nbc, 0, s,
                                                   f32 ? 2 : 0));
    LAUNCH(EXPM_STAGE_REDUCE, launch_reduce_h(P->part, nbc, cols, p, h, P->H, P->ldH, 0, j * p, 1, s));
    // second pass: in the mixed path the update is an O(eps_32) correction, formed in FP32;
    // with the fused QR its last CTA also reduces the Gram partials
    const bool fused = fused_qr(P, p);
    LAUNCH(EXPM_STAGE_CGS, launch_update_proj(P->V, ld, cols, P->W, ld, p, n, h, P->part, P->nblk, 1, s, 0, f32,
                                              fused ? sm(P, kOffG) : nullptr, fused ? P->ctr : nullptr));
    return qr_block(P, p, P->V + (int64_t)(j + 1) * p * ld, ld, true, (j + 1) * p, j * p, nullptr, true);
}

expm_status check_flags(const double* hstat) {
    const int* f = reinterpret_cast<const int*>(hstat + 24);
    if (f[0] & 16) return EXPM_TIMEOUT;   // a bounded device-side wait ran out
    if (f[0]) return EXPM_NUMERICAL;
    return EXPM_OK;
}

expm_status validate_block_args(expm_plan* P, double t, const void* B, int64_t ldb, int p,
                                const void* Z, int64_t ldz) {
    if (!P || !B || !Z) return EXPM_INVALID_ARG;
    if (!(t > 0.0) || !std::isfinite(t)) return EXPM_INVALID_ARG;
    if (p < 1 || p > P->p_max) return EXPM_INVALID_ARG;
    if (ldb < P->n || ldz < P->n) return EXPM_INVALID_ARG;
    if (B == Z) return EXPM_INVALID_ARG;
    return EXPM_OK;
}

// Gershgorin bound of ||tA||_inf for the convection-diffusion operator.
double norm_bound(const expm_plan* P, double t) {
    if (P->toeplitz) return t * P->tz.abs_rowsum;
    if (P->csr) return t * P->cs.abs_rowsum;
    double s = 0.0;
    for (int d = 0; d < P->ndim; ++d) s += std::fabs(P->ax[d].l) + std::fabs(P->ax[d].c) + std::fabs(P->ax[d].u);
    return t * s;
}

int choose_algorithm(const expm_plan* P, double t) {
    if (P->opts.algorithm == EXPM_ALG_SBFOM || P->opts.algorithm == EXPM_ALG_PSBFOM) return P->opts.algorithm;
    if (P->toeplitz && !P->tz.gsf) return EXPM_ALG_SBFOM;
    double tmax = 0.0;
    for (int i = 0; i < P->npoles; ++i) tmax = std::max(tmax, std::hypot(P->tau_re[i], P->tau_im[i]));
    return norm_bound(P, t) >= EXPM_AUTO_RATIO * tmax ? EXPM_ALG_PSBFOM : EXPM_ALG_SBFOM;
}

// Restart prologue of a plan with deflation (the restart copy is then not fused into the
// Z update): prologue 1 is the plain restart V_1 <- V_{m+1}; prologue 2 the deflated one,
// V_new = V_{m+1} blkdiag(P_k, I_p): columns 0..kk-1 <- V_m P_k (FP64, in chunks of 16
// columns), columns kk..kk+p-1 <- V_{m+1}, and H~ <- 0 with the host-formed leading block
// P_{k+1}^T H~ P_k ((kk + p) x kk) in place.  P_k and that block come from pinned host buffers
// filled after the previous cycle.
expm_status restart_prologue(expm_plan* P, int p, int kk, int prologue) {
    cudaStream_t s = P->stream;
    const int mp = P->opts.m * p;
    const int64_t n = P->n, ld = P->ld;
    double* Vnext = P->V + (int64_t)mp * ld;
    if (prologue == 1) {
        LAUNCH(EXPM_STAGE_UPDATE, launch_copy(Vnext, ld, P->V, ld, n, p, s));
        return EXPM_OK;
    }
    CK(cudaMemcpyAsync(P->Pkd, P->hPk, sizeof(double) * (size_t)mp * kk, cudaMemcpyHostToDevice, s));
    LAUNCH(EXPM_STAGE_UPDATE, launch_zero(P->Vk, ld, n, kk, s));
    for (int c0 = 0; c0 < kk; c0 += kRowsMaxP) {
        const int pc = std::min(kRowsMaxP, kk - c0);
        LAUNCH(EXPM_STAGE_UPDATE, launch_update_z(P->V, ld, mp, pc, n, P->Pkd + (size_t)mp * c0, P->Vk + (int64_t)c0 * ld,
                                                  ld, 0, s, P->nblk, 0));
    }
    LAUNCH(EXPM_STAGE_UPDATE, launch_copy(Vnext, ld, P->V + (int64_t)kk * ld, ld, n, p, s));
    LAUNCH(EXPM_STAGE_UPDATE, launch_copy(P->Vk, ld, P->V, ld, n, kk, s));
    CK(cudaMemsetAsync(P->H, 0, sizeof(double) * (size_t)P->ldH * P->opts.m * P->p_max, s));
    CK(cudaMemcpy2DAsync(P->H, sizeof(double) * P->ldH, P->hHnew, sizeof(double) * P->ldH,
                         sizeof(double) * (size_t)(kk + p), kk, cudaMemcpyHostToDevice, s));
    return EXPM_OK;
}

// One restart cycle: the restart prologue (plans with deflation), the block steps, the
// projected systems, the update and the restart copy, then the device->host copy of the
// residual norms and flags (and of H~ when the next restart may deflate); no synchronisation.
// kk > 0: the basis starts with kk kept Ritz vectors and the block steps begin at block kk/p.
expm_status issue_cycle(expm_plan* P, double t, int p, int alg, int kk = 0, int prologue = 0, bool d2h = true) {
    cudaStream_t s = P->stream;
    const int m = P->opts.m, mp = m * p;
    const int64_t n = P->n, ld = P->ld;
    if (prologue) {
        expm_status st = restart_prologue(P, p, kk, prologue);
        if (st != EXPM_OK) return st;
    }
    for (int j = kk / p; j < m; ++j) {
        expm_status st = block_step(P, t, j, p, alg);
        if (st != EXPM_OK) return st;
    }
    double* tau_re = sm(P, kOffTau);
    LAUNCH(EXPM_STAGE_POLES, launch_poles(P->H, P->ldH, mp, p, P->npoles, tau_re, tau_re + EXPM_MAX_POLES,
                                          tau_re + 2 * EXPM_MAX_POLES, tau_re + 3 * EXPM_MAX_POLES,
                                          P->S, P->poles, P->Wc_slots, P->stat, flags_of(P->stat), alg, s,
                                          P->opts.certify ? P->Zcert : nullptr, kk));
    LAUNCH(EXPM_STAGE_POLES, launch_combine2(P->H, P->ldH, mp, p, P->npoles, P->Wc_slots, sm(P, kOffWc), alg, s, kk));
    if (P->opts.certify) {
        // every pole's X_i (real and imaginary columns) += V_{m+1} C, before the restart copy
        LAUNCH(EXPM_STAGE_OTHER, launch_certify_coeffs(P->H, P->ldH, mp, p, P->npoles, P->Zcert, P->Ccert, alg, s, kk));
        LAUNCH(EXPM_STAGE_OTHER, launch_update_z(P->V, ld, mp + p, 2 * P->npoles * p, n, P->Ccert, P->Xcert, ld, 0,
                                                 s, P->nblk));
    }
    // mixed path: the product V Wc in double-float on the FP32 pipe (FP64 accumulation into Z)
    // (with deflation the restart happens in the next cycle's prologue, after V_m P_k)
    const bool defl = P->opts.k_defl > 0;
    LAUNCH(EXPM_STAGE_UPDATE, launch_update_z(P->V, ld, mp + p, p, n, sm(P, kOffWc), P->Zacc, ld, defl ? 0 : 1, s,
                                              P->nblk, P->opts.precision == EXPM_PREC_MIXED ? 1 : 0));
    if (!d2h) return EXPM_OK;   // the batch graph's stop test reads the status on the device
    CK(cudaMemcpyAsync(P->hpin, P->stat, sizeof(double) * kStatDoubles, cudaMemcpyDeviceToHost, s));
    if (defl) CK(cudaMemcpyAsync(P->hH, P->H, sizeof(double) * (size_t)P->ldH * mp, cudaMemcpyDeviceToHost, s));
    return EXPM_OK;
}

// Capture (once) and return the graph of one cycle for (alg, p, t); nullptr if capture is
// not possible, in which case the caller launches directly.
GraphEntry* graph_for(expm_plan* P, double t, int p, int alg, int kk = 0, int prologue = 0) {
    for (auto& g : P->graphs)
        if (g.alg == alg && g.p == p && g.t == t && g.kk == kk && g.prologue == prologue) return &g;
    if (P->graphs.size() >= 16) return nullptr;
    cudaStream_t s = P->stream;
    const int64_t l0 = P->launches;
    int64_t sl0[EXPM_NSTAGES];
    for (int k = 0; k < EXPM_NSTAGES; ++k) sl0[k] = P->stage_launches[k];
    if (cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    expm_status st = issue_cycle(P, t, p, alg, kk, prologue);
    cudaGraph_t graph = nullptr;
    cudaError_t ec = cudaStreamEndCapture(s, &graph);
    GraphEntry e;
    e.alg = alg;
    e.p = p;
    e.t = t;
    e.kk = kk;
    e.prologue = prologue;
    e.launches = P->launches - l0;
    for (int k = 0; k < EXPM_NSTAGES; ++k) {
        e.stage_launches[k] = P->stage_launches[k] - sl0[k];
        P->stage_launches[k] = sl0[k];
    }
    P->launches = l0;
    if (st != EXPM_OK || ec != cudaSuccess || !graph) {
        if (graph) cudaGraphDestroy(graph);
        cudaGetLastError();
        return nullptr;
    }
    cudaError_t ei = cudaGraphInstantiate(&e.exec, graph, 0);
    cudaGraphDestroy(graph);
    if (ei != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    P->graphs.push_back(e);
    return &P->graphs.back();
}

// State of one expm_block call between restart cycles.  run_block drives one call to the
// end; expm_block_batched interleaves several calls on their plans' streams.
struct RunState {
    double t = 0.0;
    const double* dB = nullptr;
    int64_t ldb = 0;
    int p = 0;
    double* dZ = nullptr;
    int64_t ldz = 0;
    int alg = 0;
    int cycles = 0;
    bool converged = false;
    bool done = false;
    double normB = 0.0;
    expm_status result = EXPM_OK;
    GraphEntry* ge = nullptr;
    int kk = 0;          // deflated restart: Ritz vectors kept for the next cycle
    int prologue = 0;    // 0 first cycle, 1 plain restart, 2 deflated restart (plans with k_defl)
    int steps = 0;       // block applications of the operator so far
};

// Start of the algorithm: R_i^0 = B = V_1 R for every pole; the cycle graph.
expm_status run_begin(expm_plan* P, RunState& r) {
    cudaStream_t s = P->stream;
    r.alg = choose_algorithm(P, r.t);
    const int m = P->opts.m, p = r.p;
    const int64_t n = P->n, ld = P->ld;
    CK(cudaMemsetAsync(P->stat, 0, sizeof(double) * kStatDoubles, s));
    CK(cudaMemsetAsync(P->ctr, 0, sizeof(unsigned) * 4, s));
    CK(cudaMemsetAsync(P->H, 0, sizeof(double) * (size_t)P->ldH * m * P->p_max, s));
    LAUNCH(EXPM_STAGE_OTHER, launch_zero(P->Zacc, ld, n, p, s));
    if (P->opts.certify) LAUNCH(EXPM_STAGE_OTHER, launch_zero(P->Xcert, ld, n, 2 * P->npoles * p, s));
    LAUNCH(EXPM_STAGE_OTHER, launch_copy(r.dB, r.ldb, P->W, ld, n, p, s));
    expm_status st = qr_block(P, p, P->V, ld, false, 0, 0, P->stat + 16, false);
    if (st != EXPM_OK) return st;
    if (fused_qr(P, p))   // the fused QR leaves R in Rt2, or in Rt3 when its third pass ran
        LAUNCH(EXPM_STAGE_OTHER, launch_init_S(sm(P, kOffRt2), p, P->npoles, P->S, s, sm(P, kOffRt3),
                                               flags_of(P->stat) + 2));
    else
        LAUNCH(EXPM_STAGE_OTHER, launch_init_S(sm(P, kOffRt), p, P->npoles, P->S, s));
    r.kk = 0;
    r.prologue = 0;
    return EXPM_OK;
}

// Issue one restart cycle (graph or direct launches) and mark its end with the plan's event.
expm_status run_issue(expm_plan* P, RunState& r) {
    cudaStream_t s = P->stream;
    ++r.cycles;
    r.steps += P->opts.m - r.kk / r.p;
    // graph of one restart cycle, cached per (algorithm, p, t, restart kind)
    r.ge = nullptr;
    if (P->use_graphs && !P->prof && P->stream != nullptr) r.ge = graph_for(P, r.t, r.p, r.alg, r.kk, r.prologue);
    if (r.ge) {
        CK(cudaGraphLaunch(r.ge->exec, s));
        P->launches += r.ge->launches;
        for (int k = 0; k < EXPM_NSTAGES; ++k) P->stage_launches[k] += r.ge->stage_launches[k];
    } else {
        expm_status st = issue_cycle(P, r.t, r.p, r.alg, r.kk, r.prologue);
        if (st != EXPM_OK) return st;
    }
    CK(cudaEventRecord(P->cycle_ev, s));
    return EXPM_OK;
}

// The deflated restart's small dense work, on the host after a cycle (H~ is in hH): the
// orthonormal Ritz basis P_k of H_m (expm_ritz_basis: Algorithm 2 keeps the largest |mu|,
// Remark 4.1; Algorithm 1 the smallest |theta|; a multiple of p), the new leading block
// P_{k+1}^T H~ P_k with P_{k+1} = blkdiag(P_k, I_p), and P_k in the chunked layout of the
// device product.  Without a usable basis the next restart is the plain one.
void prepare_deflation(expm_plan* P, RunState& r) {
    const int m = P->opts.m, p = r.p, mp = m * p, ldH = P->ldH;
    r.kk = 0;
    r.prologue = 1;
    const int kreq = std::min(P->opts.k_defl, (m - 1) * p);
    if (kreq < 1) return;
    std::vector<double> Pk((size_t)mp * mp);
    int kept = 0;
    if (expm_ritz_basis(P->hH, ldH, mp, kreq, r.alg == EXPM_ALG_PSBFOM ? 1 : 0, p, Pk.data(), mp, &kept) != EXPM_OK ||
        kept < 1 || kept > std::min(P->kdefl_max, (m - 1) * p))
        return;
    // T = H~ P_k ((mp + p) x kept), then the leading block: rows < kept are P_k^T T, rows
    // kept.. kept+p-1 the last block row of T
    const int rows = mp + p;
    std::vector<double> T((size_t)rows * kept, 0.0);
    for (int j = 0; j < kept; ++j)
        for (int b = 0; b < mp; ++b) {
            const double pb = Pk[(size_t)j * mp + b];
            if (pb == 0.0) continue;
            const double* hc = P->hH + (size_t)b * ldH;
            for (int a = 0; a < rows; ++a) T[(size_t)j * rows + a] += hc[a] * pb;
        }
    for (int j = 0; j < kept; ++j) {
        double* out = P->hHnew + (size_t)j * ldH;
        for (int i = 0; i < kept; ++i) {
            double acc = 0.0;
            for (int a = 0; a < mp; ++a) acc += Pk[(size_t)i * mp + a] * T[(size_t)j * rows + a];
            out[i] = acc;
        }
        for (int q = 0; q < p; ++q) out[kept + q] = T[(size_t)j * rows + mp + q];
    }
    for (int c0 = 0; c0 < kept; c0 += kRowsMaxP) {
        const int pc = std::min(kRowsMaxP, kept - c0);
        double* dst = P->hPk + (size_t)mp * c0;
        for (int a = 0; a < mp; ++a)
            for (int c = 0; c < pc; ++c) dst[(size_t)a * pc + c] = Pk[(size_t)(c0 + c) * mp + a];
    }
    r.kk = kept;
    r.prologue = 2;
}

// After a cycle's work has completed: flags, eq. (49) norms, the stop test.
void run_check(expm_plan* P, RunState& r) {
    prof_flush(P);
    const expm_status st = check_flags(P->hpin);
    if (st != EXPM_OK) {
        r.result = st;
        r.done = true;
        return;
    }
    r.normB = std::sqrt(P->hpin[16]);
    double mx = 0.0;
    for (int i = 0; i < P->npoles; ++i) mx = std::max(mx, P->hpin[i]);
    r.converged = mx <= P->opts.tol * r.normB;
    r.done = (P->opts.fixed_cycles > 0) ? r.cycles >= P->opts.fixed_cycles
                                        : (r.converged || r.cycles >= P->opts.max_cycles);
    if (!r.done && P->opts.k_defl > 0) prepare_deflation(P, r);
}

// Z = omega_0 B + Z_acc (eq. (11) with the conjugate pairs folded), certify, info.
expm_status run_finish(expm_plan* P, RunState& r, expm_info* info) {
    cudaStream_t s = P->stream;
    const int p = r.p;
    const int64_t n = P->n, ld = P->ld;
    LAUNCH(EXPM_STAGE_OTHER, launch_axpby(P->omega0, r.dB, r.ldb, 1.0, P->Zacc, ld, r.dZ, r.ldz, n, p, s));
    double true_res[EXPM_MAX_POLES] = {0};
    if (P->opts.certify) {
        // the true FP64 residuals ||B - (tA - tau_i I) X_i||_F of every pole (eq. (3))
        double* tau = sm(P, kOffTau);
        const double* AX = nullptr;
        if (P->toeplitz) {
            // tA X_i for the real and imaginary columns of every pole by FFT products
            expm_status st = toeplitz_matvec(P, r.t, P->Xcert, ld, 2 * P->npoles * p, P->Acert, ld, EXPM_STAGE_OTHER);
            if (st != EXPM_OK) return st;
            AX = P->Acert;
        }
        const int nx = P->toeplitz ? (int)n : P->ax[0].N;
        LAUNCH(EXPM_STAGE_OTHER, launch_true_resid(P->Xcert, ld, r.dB, r.ldb, p, P->npoles, P->ndim, nx, P->ax[1].N,
                                                   P->ax[2].N, P->ax, r.t, tau, tau + EXPM_MAX_POLES, P->rcert, s,
                                                   AX, ld));
        const int nb = true_resid_blocks(n);
        CK(cudaMemcpyAsync(P->hcert, P->rcert, sizeof(double) * (size_t)P->npoles * nb, cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
        for (int i = 0; i < P->npoles; ++i) {
            double s2 = 0.0;
            for (int b = 0; b < nb; ++b) s2 += P->hcert[(size_t)i * nb + b];
            true_res[i] = std::sqrt(s2);
        }
    }
    if (info) {
        std::memset(info, 0, sizeof(*info));
        info->cycles = r.cycles;
        info->converged = r.converged ? 1 : 0;
        info->npoles = P->npoles;
        info->breakdown = reinterpret_cast<const int*>(P->hpin + 24)[1] ? 1 : 0;
        for (int i = 0; i < P->npoles; ++i) info->resid[i] = P->hpin[i];
        info->normB = r.normB;
        info->algorithm = r.alg;
        info->normA_bound = norm_bound(P, r.t);
        for (int i = 0; i < P->npoles; ++i) info->true_resid[i] = true_res[i];
        info->kept = r.kk;
        info->inner_iters = P->inner_iters;
        // block applications of the operator: a deflated cycle starts at block kk / p
        info->block_steps = r.steps;
        info->matvecs = (int64_t)r.steps * p;
    }
    if (r.result != EXPM_OK) return r.result;
    if (P->opts.fixed_cycles > 0) return EXPM_OK;
    return r.converged ? EXPM_OK : EXPM_NOT_CONVERGED;
}

expm_status run_block(expm_plan* P, double t, const double* dB, int64_t ldb, int p, double* dZ,
                      int64_t ldz, expm_info* info) {
    RunState r;
    r.t = t;
    r.dB = dB;
    r.ldb = ldb;
    r.p = p;
    r.dZ = dZ;
    r.ldz = ldz;
    P->inner_iters = 0;
    expm_status st = run_begin(P, r);
    if (st != EXPM_OK) return st;
    while (!r.done) {
        if ((st = run_issue(P, r)) != EXPM_OK) return st;
        CK(cudaStreamSynchronize(P->stream));
        run_check(P, r);
    }
    return run_finish(P, r, info);
}

void free_plan(expm_plan* P) {
    if (!P) return;
    for (int d = 0; d < 3; ++d) {
        cudaFree(P->Qf[d]);
        cudaFree(P->Qi[d]);
        cudaFree(P->lam[d]);
    }
    cudaFree(P->th_m);
    cudaFree(P->th_c);
    for (int d = 0; d < 3; ++d) {
        cudaFree(P->Qf32[d]);
        cudaFree(P->Qi32[d]);
    }
    cudaFree(P->th_m32);
    cudaFree(P->th_c32);
    cudaFree(P->T1f);
    cudaFree(P->T2f);
    cudaFree(P->R64);
    cudaFree(P->V);
    cudaFree(P->W);
    cudaFree(P->T1);
    cudaFree(P->T2);
    cudaFree(P->Zacc);
    cudaFree(P->Bst);
    cudaFree(P->Zst);
    cudaFree(P->Xcert);
    cudaFree(P->Acert);
    cudaFree(P->cs.rowptr);
    cudaFree(P->cs.colind);
    cudaFree(P->cs.val);
    cudaFree(P->cs.dinv);
    cudaFree(P->cs.work);
    cudaFree(P->cs.part);
    cudaFree(P->cs.scal);
    cudaFree(P->cs.norms);
    if (P->cs.hnorms) cudaFreeHost(P->cs.hnorms);
    cudaFree(P->tz.col);
    cudaFree(P->tz.tw1);
    cudaFree(P->tz.tw2);
    cudaFree(P->tz.thi);
    cudaFree(P->tz.tlo);
    cudaFree(P->tz.tw1f);
    cudaFree(P->tz.tw2f);
    cudaFree(P->tz.thif);
    cudaFree(P->tz.tlof);
    cudaFree(P->tz.lam);
    cudaFree(P->tz.Ua);
    cudaFree(P->tz.Ub);
    cudaFree(P->tz.mu1);
    cudaFree(P->tz.mu2);
    cudaFree(P->Zcert);
    cudaFree(P->Ccert);
    cudaFree(P->rcert);
    delete[] P->hcert;
    cudaFree(P->H);
    cudaFree(P->part);
    cudaFree(P->small);
    cudaFree(P->poles);
    cudaFree(P->S);
    cudaFree(P->Wc_slots);
    cudaFree(P->stat);
    cudaFree(P->ctr);
    cudaFree(P->dotpart);
    cudaFree(P->Vk);
    cudaFree(P->Pkd);
    if (P->hH) cudaFreeHost(P->hH);
    if (P->hPk) cudaFreeHost(P->hPk);
    if (P->hHnew) cudaFreeHost(P->hHnew);
    if (P->hpin) cudaFreeHost(P->hpin);
    if (P->hdot) cudaFreeHost(P->hdot);
    if (P->cycle_ev) cudaEventDestroy(P->cycle_ev);
    if (P->adj) free_plan(P->adj);
    for (auto& e : P->ev) cudaEventDestroy(e);
    for (auto& g : P->graphs) cudaGraphExecDestroy(g.exec);
    delete P;
}

template <class T>
bool dalloc(T** p, size_t count) {
    if (count == 0) count = 1;
    return cudaMalloc(reinterpret_cast<void**>(p), sizeof(T) * count) == cudaSuccess;
}

// ---- Toeplitz plan setup
constexpr int64_t kToeplitzMaxN = int64_t(1) << 21;   // FFT size N <= 2^22 (see k_fft.cu)

// Upper bound of max_theta f(theta), f(theta) = a_0 + 2 sum_k a_k cos(k theta): the largest
// value on a grid of M points in [0, pi] plus (pi / 2M) max|f'|, max|f'| <= bw max|f|
// (Bernstein's inequality for trigonometric polynomials of degree bw).  The grid is refined
// while the bound is inconclusive (grid maximum < 0 <= bound), up to ~1e9 cosines.
double toeplitz_symbol_max_bound(const double* a, int64_t bw, double abs_rowsum) {
    if (bw == 0) return a[0];
    const double pi = 3.141592653589793238462643383279502884;
    double bound = 0.0;
    for (int64_t M = 64 * bw + 64;; M *= 4) {
        double mx = -1e300;
        for (int64_t j = 0; j <= M; ++j) {
            const double th = pi * (double)j / (double)M;
            double f = a[0];
            for (int64_t k = 1; k <= bw; ++k) f += 2.0 * a[k] * std::cos((double)k * th);
            mx = std::max(mx, f);
        }
        bound = mx + pi / (2.0 * (double)M) * (double)bw * abs_rowsum;
        if (mx >= 0.0 || bound < 0.0 || 4 * M * bw > 1000000000) break;
    }
    return bound;
}

// A general sparse operator's descriptor: the CSR structure (offsets from 0, nondecreasing,
// column indices in range, finite values) and the Gershgorin certificate of the operator
// kind's contract: every diagonal entry negative (duplicates summed) and every row weakly
// diagonally dominant, so the spectrum lies in the closed left half-plane.  abs_rowsum:
// max_i sum_j |a_ij|, the bound of ||A||_inf behind AUTO.
expm_status csr_validate(const expm_op_desc* op, double* abs_rowsum) {
    const int64_t n = op->n;
    if (n < 1 || n > INT32_MAX || !op->csr_rowptr) return EXPM_INVALID_ARG;
    const int64_t* rp = op->csr_rowptr;
    if (rp[0] != 0) return EXPM_INVALID_ARG;
    for (int64_t i = 0; i < n; ++i)
        if (rp[i + 1] < rp[i]) return EXPM_INVALID_ARG;
    const int64_t nnz = rp[n];
    if (nnz > 0 && (!op->csr_colind || !op->csr_val)) return EXPM_INVALID_ARG;
    double mx = 0.0;
    for (int64_t i = 0; i < n; ++i) {
        double dg = 0.0, off = 0.0, tot = 0.0;
        for (int64_t k = rp[i]; k < rp[i + 1]; ++k) {
            const int64_t j = op->csr_colind[k];
            const double a = op->csr_val[k];
            if (j < 0 || j >= n || !std::isfinite(a)) return EXPM_INVALID_ARG;
            if (j == i) dg += a;
            else off += std::fabs(a);
            tot += std::fabs(a);
        }
        if (!(dg < 0.0) || off > -dg * (1.0 + 1e-12)) return EXPM_INVALID_ARG;
        mx = std::max(mx, tot);
    }
    *abs_rowsum = mx;
    return EXPM_OK;
}

expm_status toeplitz_validate(const expm_op_desc* op, double* abs_rowsum) {
    if (op->n < 2 || op->n > kToeplitzMaxN) return EXPM_INVALID_ARG;
    if (op->toeplitz_bw < 0 || op->toeplitz_bw > op->n - 1 || !op->toeplitz_col) return EXPM_INVALID_ARG;
    const double* a = op->toeplitz_col;
    const int64_t bw = op->toeplitz_bw;
    // rs = |a_0| + 2 sum |a_k| and the Gershgorin bound a_0 + 2 sum |a_k|, both with
    // compensated (Neumaier) sums: for the fractional-diffusion operators the bound is a few
    // units against terms of 1e10, beyond what a plain sum resolves
    double rs = 0.0, rc = 0.0, gs = 0.0, gc = 0.0;
    auto add = [](double& sum, double& comp, double v) {
        const double t = sum + v;
        comp += (std::fabs(sum) >= std::fabs(v)) ? (sum - t) + v : (v - t) + sum;
        sum = t;
    };
    for (int64_t k = 0; k <= bw; ++k) {
        if (!std::isfinite(a[k])) return EXPM_INVALID_ARG;
        add(rs, rc, k > 0 ? 2.0 * std::fabs(a[k]) : std::fabs(a[k]));
        add(gs, gc, k > 0 ? 2.0 * std::fabs(a[k]) : a[k]);
    }
    rs += rc;
    gs += gc;
    if (!(a[0] < 0.0)) return EXPM_INVALID_ARG;
    // negative definite if either certificate holds: Gershgorin (a_0 + 2 sum |a_k| < 0, tight
    // for dense decaying columns such as the fractional-diffusion ones), or, for bw <= 4096,
    // the bound of the symbol's largest value (tight for short bands with mixed signs)
    const bool gersh = gs < 0.0;
    if (!gersh && !(bw <= 4096 && toeplitz_symbol_max_bound(a, bw, rs) < 0.0)) return EXPM_INVALID_ARG;
    *abs_rowsum = rs;
    return EXPM_OK;
}

// fixed-order sum of the dot-product partials
expm_status dot_host(expm_plan* P, const double* x, const double* y, double* part, double* hpart, double* out) {
    cudaStream_t s = P->stream;
    LAUNCH(EXPM_STAGE_OTHER, launch_dot_partial(x, y, P->n, part, s));
    CK(cudaMemcpyAsync(hpart, part, sizeof(double) * dot_blocks(), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    double acc = 0.0;
    for (int b = 0; b < dot_blocks(); ++b) acc += hpart[b];
    *out = acc;
    return EXPM_OK;
}

// T. Chan's optimal circulant preconditioner of the generator solve (the circulant C that
// minimises ||C - T||_F: first column c_k = ((n - k) a_k + k a_{n-k}) / n), applied by FFTs of
// length n; only when n is a power of two (the four-step FFT's lengths) and C is negative
// definite.  Owns its device buffers for the duration of the plan's setup.
struct CircPre {
    FftPlan f{};
    double *tw1 = nullptr, *tw2 = nullptr, *thi = nullptr, *tlo = nullptr;
    double *col = nullptr, *lam = nullptr, *U = nullptr;
    bool ok = false;
    ~CircPre() {
        cudaFree(tw1);
        cudaFree(tw2);
        cudaFree(thi);
        cudaFree(tlo);
        cudaFree(col);
        cudaFree(lam);
        cudaFree(U);
    }
};

FftArgs circ_args(const CircPre& c, int64_t n) {
    FftArgs a;
    a.f = c.f;
    a.nreal = n;
    a.tw1 = c.tw1;
    a.tw2 = c.tw2;
    a.thi = c.thi;
    a.tlo = c.tlo;
    a.lam = c.lam;
    a.in = a.out = c.U;
    a.p = 1;
    return a;
}

// z = C^{-1} r (one column): forward column pass, row pass times 1 / sigma, inverse column pass
expm_status circ_apply(expm_plan* P, const CircPre& c, const double* r, double* z) {
    cudaStream_t s = P->stream;
    FftArgs a = circ_args(c, P->n);
    a.V = r;
    a.ldv = P->ld;
    a.W = z;
    a.ldw = P->ld;
    a.scale = 1.0 / (double)c.f.N;
    if (launch_fft_cols(a, FFT_COL_FWD_REAL, 1, s) != cudaSuccess || launch_fft_rows(a, FFT_ROW_MATVEC, 1, s) != cudaSuccess)
        return EXPM_CUDA_ERROR;
    a.scale = 1.0;
    if (launch_fft_cols(a, FFT_COL_INV_REAL, 1, s) != cudaSuccess) return EXPM_CUDA_ERROR;
    return EXPM_OK;
}

expm_status circ_setup(expm_plan* P, const double* hcol, CircPre& c) {
    const int64_t n = P->n, bw = P->tz.bw;
    if (n < 64 || (n & (n - 1)) != 0) return EXPM_OK;       // not a power of two: no preconditioner
    c.f = fft_geometry(n);
    if (c.f.N != n || !fft_geometry_ok(c.f)) return EXPM_OK;
    cudaStream_t s = P->stream;
    const int64_t N = c.f.N;
    if (!(dalloc(&c.tw1, 2 * (size_t)c.f.N1) && dalloc(&c.tw2, 2 * (size_t)c.f.N2) && dalloc(&c.thi, 2 * (size_t)(N / 64)) &&
          dalloc(&c.tlo, 128) && dalloc(&c.col, (size_t)P->ld) && dalloc(&c.lam, (size_t)N) && dalloc(&c.U, 2 * (size_t)N))) {
        cudaGetLastError();
        return EXPM_NO_MEMORY;
    }
    std::vector<double> cc((size_t)n, 0.0), sig((size_t)N);
    auto at = [&](int64_t k) { return k <= bw ? hcol[k] : 0.0; };
    for (int64_t k = 0; k < n; ++k) cc[k] = ((double)(n - k) * at(k) + (double)k * (k ? at(n - k) : 0.0)) / (double)n;
    FftArgs a = circ_args(c, n);
    a.V = c.col;
    a.ldv = P->ld;
    if (cudaMemcpyAsync(c.col, cc.data(), sizeof(double) * n, cudaMemcpyHostToDevice, s) != cudaSuccess ||
        launch_fft_tables(c.f, c.tw1, c.tw2, c.thi, c.tlo, s) != cudaSuccess ||
        launch_fft_cols(a, FFT_COL_FWD_REAL, 1, s) != cudaSuccess || launch_fft_rows(a, FFT_ROW_FWD, 1, s) != cudaSuccess ||
        launch_real_part(c.U, c.lam, N, s) != cudaSuccess ||
        cudaMemcpyAsync(sig.data(), c.lam, sizeof(double) * N, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
        return EXPM_CUDA_ERROR;
    for (int64_t k = 0; k < N; ++k) {
        if (!(sig[k] < 0.0) || !std::isfinite(sig[k])) return EXPM_OK;   // not definite: plain CG
        sig[k] = 1.0 / sig[k];
    }
    if (cudaMemcpyAsync(c.lam, sig.data(), sizeof(double) * N, cudaMemcpyHostToDevice, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
        return EXPM_CUDA_ERROR;
    c.ok = true;
    return EXPM_OK;
}

// Generator x = T^{-1} e_1 of the Gohberg-Semencul formula by conjugate gradients with the
// FFT product (T is symmetric definite), preconditioned by T. Chan's circulant when n is a
// power of two (the large-norm operators of Example 5.4's regime have kappa ~ 1e9, where
// plain CG stalls), then mu_1 = F[x; 0], mu_2 = F[xh; 0].  Stop when the backward error
// ||e_1 - T x|| / (||T||_1 ||x|| + 1) reaches 1e-14; fail above 1e-12.
expm_status toeplitz_generator(expm_plan* P, const double* hcol) {
    cudaStream_t s = P->stream;
    ToeplitzOp& z = P->tz;
    const int64_t n = P->n, ld = P->ld, N = z.f.N;
    double *buf = nullptr, *part = nullptr;
    if (cudaMalloc(reinterpret_cast<void**>(&buf), sizeof(double) * 5 * ld) != cudaSuccess) return EXPM_NO_MEMORY;
    if (cudaMalloc(reinterpret_cast<void**>(&part), sizeof(double) * dot_blocks()) != cudaSuccess) {
        cudaFree(buf);
        return EXPM_NO_MEMORY;
    }
    std::vector<double> hpart(dot_blocks());
    double* x = buf;
    double* r = buf + ld;
    double* pp = buf + 2 * ld;
    double* w = buf + 3 * ld;
    double* zz = buf + 4 * ld;
    expm_status st = EXPM_OK;
    auto fail = [&](expm_status e) {
        cudaStreamSynchronize(s);
        cudaFree(buf);
        cudaFree(part);
        return e;
    };
    CircPre pre;
    if ((st = circ_setup(P, hcol, pre)) != EXPM_OK) return fail(st);
    auto precond = [&](const double* in, double* out) -> expm_status {
        if (pre.ok) return circ_apply(P, pre, in, out);
        return launch_copy(in, ld, out, ld, n, 1, s) == cudaSuccess ? EXPM_OK : EXPM_CUDA_ERROR;
    };
    if (cudaMemsetAsync(x, 0, sizeof(double) * ld, s) != cudaSuccess) return fail(EXPM_CUDA_ERROR);
    if (launch_unit(r, n, s) != cudaSuccess) return fail(EXPM_CUDA_ERROR);
    if ((st = precond(r, zz)) != EXPM_OK) return fail(st);
    if (launch_copy(zz, ld, pp, ld, n, 1, s) != cudaSuccess) return fail(EXPM_CUDA_ERROR);
    double rz = 0.0, xx = 0.0;
    if ((st = dot_host(P, r, zz, part, hpart.data(), &rz)) != EXPM_OK) return fail(st);
    const double rs = z.abs_rowsum;
    int it = 0;
    for (; it < 5000; ++it) {
        if ((st = toeplitz_matvec(P, 1.0, pp, ld, 1, w, ld, EXPM_STAGE_OTHER)) != EXPM_OK) return fail(st);
        double pw = 0.0;
        if ((st = dot_host(P, pp, w, part, hpart.data(), &pw)) != EXPM_OK) return fail(st);
        if (!(pw < 0.0) || !std::isfinite(pw)) return fail(EXPM_NUMERICAL);   // T negative definite
        const double alpha = rz / pw;
        if (launch_cg_step(x, r, pp, w, alpha, n, s) != cudaSuccess) return fail(EXPM_CUDA_ERROR);
        double rr = 0.0;
        if ((st = dot_host(P, r, r, part, hpart.data(), &rr)) != EXPM_OK) return fail(st);
        if (it % 8 == 0 && (st = dot_host(P, x, x, part, hpart.data(), &xx)) != EXPM_OK) return fail(st);
        if (std::sqrt(rr) <= 1e-14 * (rs * std::sqrt(xx) + 1.0)) break;
        if ((st = precond(r, zz)) != EXPM_OK) return fail(st);
        double rz_new = 0.0;
        if ((st = dot_host(P, r, zz, part, hpart.data(), &rz_new)) != EXPM_OK) return fail(st);
        if (launch_cg_dir(pp, zz, rz_new / rz, n, s) != cudaSuccess) return fail(EXPM_CUDA_ERROR);
        rz = rz_new;
    }
    // true residual ||e_1 - T x||
    if ((st = toeplitz_matvec(P, 1.0, x, ld, 1, w, ld, EXPM_STAGE_OTHER)) != EXPM_OK) return fail(st);
    if (launch_unit(pp, n, s) != cudaSuccess ||
        launch_axpby(1.0, pp, ld, -1.0, w, ld, r, ld, n, 1, s) != cudaSuccess)
        return fail(EXPM_CUDA_ERROR);
    double res2 = 0.0;
    if ((st = dot_host(P, r, r, part, hpart.data(), &res2)) != EXPM_OK) return fail(st);
    if ((st = dot_host(P, x, x, part, hpart.data(), &xx)) != EXPM_OK) return fail(st);
    z.cg_iters = it;
    z.cg_resid = std::sqrt(res2) / (rs * std::sqrt(xx) + 1.0);
    if (!(z.cg_resid <= 1e-12)) return fail(EXPM_NOT_CONVERGED);
    if (cudaMemcpyAsync(&z.x0, x, sizeof(double), cudaMemcpyDeviceToHost, s) != cudaSuccess)
        return fail(EXPM_CUDA_ERROR);
    // spectra of [x; 0] and [xh; 0] (transposed order)
    FftArgs a = fft_args(P);
    a.in = a.out = z.Ua;
    if (launch_embed_gsf(x, n, N, z.Ua, s) != cudaSuccess || launch_fft_cols(a, FFT_COL_FWD_CPLX, 2, s) != cudaSuccess ||
        launch_fft_rows(a, FFT_ROW_FWD, 2, s) != cudaSuccess ||
        cudaMemcpyAsync(z.mu1, z.Ua, sizeof(double) * 2 * N, cudaMemcpyDeviceToDevice, s) != cudaSuccess ||
        cudaMemcpyAsync(z.mu2, z.Ua + 2 * N, sizeof(double) * 2 * N, cudaMemcpyDeviceToDevice, s) != cudaSuccess)
        return fail(EXPM_CUDA_ERROR);
    if (cudaStreamSynchronize(s) != cudaSuccess) return fail(EXPM_CUDA_ERROR);
    if (!(z.x0 < 0.0) || !std::isfinite(z.x0)) return fail(EXPM_NUMERICAL);
    z.gsf = true;
    z.pcg = pre.ok;
    return fail(EXPM_OK);
}

// Allocations and spectra of the Toeplitz operator (after the common workspace).
expm_status toeplitz_setup(expm_plan* P, const expm_op_desc* op, bool want_inverse) {
    cudaStream_t s = P->stream;
    ToeplitzOp& z = P->tz;
    z.f = fft_geometry(std::max(z.n + z.bw, 2 * z.n));
    if (!fft_geometry_ok(z.f)) return EXPM_INVALID_ARG;
    const int64_t N = z.f.N;
    const size_t nseq = (size_t)toeplitz_nseq_max(P);
    bool ok = dalloc(&z.col, (size_t)z.bw + 1) && dalloc(&z.tw1, 2 * (size_t)z.f.N1) &&
              dalloc(&z.tw2, 2 * (size_t)z.f.N2) && dalloc(&z.thi, 2 * (size_t)(N / 64)) && dalloc(&z.tlo, 128) &&
              dalloc(&z.lam, (size_t)N) && dalloc(&z.Ua, 2 * (size_t)N * nseq);
    if (want_inverse)
        ok = ok && dalloc(&z.Ub, 4 * (size_t)N * nseq) && dalloc(&z.mu1, 2 * (size_t)N) && dalloc(&z.mu2, 2 * (size_t)N);
    if (!ok) {
        cudaGetLastError();
        return EXPM_NO_MEMORY;
    }
    if (fft_set_smem_limits() != cudaSuccess) return EXPM_CUDA_ERROR;
    FftArgs a = fft_args(P);
    a.in = a.out = z.Ua;
    if (cudaMemcpyAsync(z.col, op->toeplitz_col, sizeof(double) * (size_t)(z.bw + 1), cudaMemcpyHostToDevice, s) !=
            cudaSuccess ||
        launch_fft_tables(z.f, z.tw1, z.tw2, z.thi, z.tlo, s) != cudaSuccess ||
        launch_embed_toeplitz(z.col, z.bw, N, z.Ua, s) != cudaSuccess ||
        launch_fft_cols(a, FFT_COL_FWD_CPLX, 1, s) != cudaSuccess || launch_fft_rows(a, FFT_ROW_FWD, 1, s) != cudaSuccess ||
        launch_real_part(z.Ua, z.lam, N, s) != cudaSuccess || cudaStreamSynchronize(s) != cudaSuccess)
        return EXPM_CUDA_ERROR;
    if (want_inverse) {
        const expm_status st = toeplitz_generator(P, op->toeplitz_col);
        if (st != EXPM_OK) return st;
    }
    // Mixed precision: later products and inverses run their transforms in double-float
    // (FP32 pairs, ~2^-48 per operation); the spectra and the generator above stay FP64.
    if (P->opts.precision == EXPM_PREC_MIXED) {
        const int64_t N = z.f.N;
        if (!(dalloc(&z.tw1f, 4 * (size_t)z.f.N1) && dalloc(&z.tw2f, 4 * (size_t)z.f.N2) &&
              dalloc(&z.thif, 4 * (size_t)(N / 64)) && dalloc(&z.tlof, 4 * 64))) {
            cudaGetLastError();
            return EXPM_NO_MEMORY;
        }
        if (launch_fft_tables_df(z.tw1, z.tw1f, z.f.N1, s) != cudaSuccess ||
            launch_fft_tables_df(z.tw2, z.tw2f, z.f.N2, s) != cudaSuccess ||
            launch_fft_tables_df(z.thi, z.thif, N / 64, s) != cudaSuccess ||
            launch_fft_tables_df(z.tlo, z.tlof, 64, s) != cudaSuccess || cudaStreamSynchronize(s) != cudaSuccess)
            return EXPM_CUDA_ERROR;
        z.use_df = true;
    }
    return EXPM_OK;
}


}  // namespace

// A batch: the instances' arguments and the instantiated graph (see expm_batch_create).
struct expm_batch_s {
    std::vector<expm_plan*> plans;
    std::vector<RunState> rs;
    cudaStream_t stream = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    int* dctl = nullptr;              // per instance: cycles run, converged
    int* hctl = nullptr;              // pinned host mirror
    std::vector<int64_t> fixed_launches, cycle_launches;
};

namespace {

void batch_free(expm_batch* b) {
    if (!b) return;
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    cudaFree(b->dctl);
    if (b->hctl) cudaFreeHost(b->hctl);
    delete b;
}

// capture fn's stream work on P's stream into a child graph node of G with the given dependency
template <class F>
expm_status capture_child(expm_plan* P, cudaGraph_t G, const cudaGraphNode_t* dep, cudaGraphNode_t* out, F fn) {
    cudaGraph_t g = nullptr;
    if (cudaStreamBeginCapture(P->stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) return EXPM_CUDA_ERROR;
    const expm_status st = fn();
    const cudaError_t ec = cudaStreamEndCapture(P->stream, &g);
    if (st != EXPM_OK || ec != cudaSuccess || !g) {
        if (g) cudaGraphDestroy(g);
        cudaGetLastError();
        return st != EXPM_OK ? st : EXPM_CUDA_ERROR;
    }
    const cudaError_t ea = cudaGraphAddChildGraphNode(out, G, dep, dep ? 1 : 0, g);
    cudaGraphDestroy(g);
    return ea == cudaSuccess ? EXPM_OK : EXPM_CUDA_ERROR;
}

}  // namespace

extern "C" {

const char* expm_status_str(expm_status s) {
    switch (s) {
        case EXPM_OK: return "ok";
        case EXPM_INVALID_ARG: return "invalid argument";
        case EXPM_NOT_CONVERGED: return "not converged within max_cycles";
        case EXPM_BREAKDOWN: return "block Arnoldi breakdown";
        case EXPM_NUMERICAL: return "numerical failure (NaN/Inf or non-positive Cholesky pivot)";
        case EXPM_CUDA_ERROR: return "CUDA error";
        case EXPM_NO_MEMORY: return "device allocation failed";
        case EXPM_TIMEOUT: return "a bounded device-side wait ran out";
        default: return "internal error";
    }
}

expm_status expm_cf_coeffs(int nu, double* tau_re_im, double* omega_re_im, double* omega0,
                           double* sigma) {
    if (nu < 2 || nu > 2 * EXPM_MAX_POLES || (nu % 2) != 0) return EXPM_INVALID_ARG;
    if (!tau_re_im || !omega_re_im || !omega0) return EXPM_INVALID_ARG;
    std::vector<std::complex<double>> tau, om;
    double w0 = 0, sg = 0;
    if (!expm_internal_cf_table(nu, tau, om, w0, sg)) return EXPM_INTERNAL;
    for (size_t i = 0; i < tau.size(); ++i) {
        tau_re_im[2 * i] = tau[i].real();
        tau_re_im[2 * i + 1] = tau[i].imag();
        omega_re_im[2 * i] = om[i].real();
        omega_re_im[2 * i + 1] = om[i].imag();
    }
    *omega0 = w0;
    if (sigma) *sigma = sg;
    return EXPM_OK;
}

expm_status expm_plan_create(const expm_op_desc* op, int p_max, const expm_opts* opts,
                             void* stream, expm_plan** out) {
    if (!op || !opts || !out) return EXPM_INVALID_ARG;
    *out = nullptr;
    const bool toeplitz = op->kind == EXPM_OP_TOEPLITZ_SYM;
    const bool csr = op->kind == EXPM_OP_CSR;
    double abs_rowsum = 0.0;
    if (toeplitz) {
        const expm_status vs = toeplitz_validate(op, &abs_rowsum);
        if (vs != EXPM_OK) return vs;
    } else if (csr) {
        const expm_status vs = csr_validate(op, &abs_rowsum);
        if (vs != EXPM_OK) return vs;
        if (opts->certify || p_max > 16) return EXPM_INVALID_ARG;   // the sparse kernels take p <= 16
    } else {
        if (op->kind != EXPM_OP_CONV_DIFF) return EXPM_INVALID_ARG;
        if (op->ndim < 1 || op->ndim > 3) return EXPM_INVALID_ARG;
        if (!(op->diff > 0.0) || !std::isfinite(op->diff)) return EXPM_INVALID_ARG;
    }
    if (p_max < 1 || p_max > kMaxP) return EXPM_INVALID_ARG;
    if (opts->m < 1 || (int64_t)opts->m * p_max > kMaxMP) return EXPM_INVALID_ARG;
    if (opts->max_cycles < 1 || !(opts->tol >= 0.0)) return EXPM_INVALID_ARG;
    if (opts->precision != EXPM_PREC_FP64 && opts->precision != EXPM_PREC_MIXED) return EXPM_INVALID_ARG;
    // shared memory of the fused update + FP32 projection at the largest block step
    {
        const size_t cols = (size_t)opts->m * p_max, cs = cols | 1;
        size_t shm = 8 * (cols * p_max + 16 * cs + 16 * (size_t)p_max);
        if (opts->precision == EXPM_PREC_MIXED) shm += 4 * (16 * cs + 16 * (size_t)p_max + cols * p_max);
        if (shm > 225 * 1024) return EXPM_INVALID_ARG;   // 227 KB opt-in minus static memory
    }
    if (opts->algorithm < EXPM_ALG_AUTO || opts->algorithm > EXPM_ALG_PSBFOM) return EXPM_INVALID_ARG;
    if (opts->nu_cf != 0 && (opts->nu_cf < 2 || opts->nu_cf > 2 * EXPM_MAX_POLES || opts->nu_cf % 2 != 0))
        return EXPM_INVALID_ARG;
    if (opts->k_defl < 0 || (int64_t)opts->k_defl > (int64_t)(opts->m - 1) * p_max) return EXPM_INVALID_ARG;
    if (opts->row_ctas_per_sm < 0 || opts->row_ctas_per_sm > 8 || opts->cgs_ctas_per_sm < 0 || opts->cgs_ctas_per_sm > 8 ||
        opts->grid_sms < 0)
        return EXPM_INVALID_ARG;
    expm_plan* P = new (std::nothrow) expm_plan_s();
    if (!P) return EXPM_NO_MEMORY;
    P->op = *op;
    P->op.toeplitz_col = nullptr;   // host memory of the caller: not kept
    P->op.csr_rowptr = nullptr;
    P->op.csr_colind = nullptr;
    P->op.csr_val = nullptr;
    P->opts = *opts;
    P->toeplitz = toeplitz;
    P->csr = csr;
    P->ndim = (toeplitz || csr) ? 1 : op->ndim;
    P->p_max = p_max;
    P->stream = reinterpret_cast<cudaStream_t>(stream);
    {
        const char* ng = std::getenv("EXPM_DISABLE_GRAPHS");   // debugging switch
        P->use_graphs = !(ng && ng[0] == '1') && !csr;
        // test switch: "0" keeps the mixed path on the three-pass FP32 Cholesky-QR for every
        // block (the fallback of the single accurate pass)
        const char* sq = std::getenv("EXPM_QR_SINGLE_PASS");
        P->qr_single = !(sq && sq[0] == '0');
        // the first CGS pass's update on the tensor cores (k_cgs_tc, then the projection kernel
        // for the second pass and the Gram matrix) for mixed plans: by default for block
        // steps with p >= 12 and at least 64 basis columns, where it measured faster than the
        // double-float pass (whose cost grows with p, the tensor-core pass's with the basis
        // alone).  Test switch: "1" for every block step it fits, "0" never
        const char* tc = std::getenv("EXPM_CGS_TC");
        P->cgs_tc = opts->precision != EXPM_PREC_MIXED ? 0 : !tc ? 2 : tc[0] == '1' ? 1 : 0;
        // the first CGS pass's projection on the tensor cores (k_proj_tc) for mixed plans, by
        // shape (see block_step).  Test switch: "1" for every block step it fits, "0" never
        const char* ptc = std::getenv("EXPM_PROJ_TC");
        P->proj_tc = opts->precision != EXPM_PREC_MIXED ? 0 : !ptc ? 2 : ptc[0] == '1' ? 1 : 0;
        // test switch: the bound of the tensor-core kernel's waits (0 makes every wait run out)
        const char* sl = std::getenv("EXPM_TC_SPIN_LIMIT");
        if (sl) P->tc_spin = std::strtol(sl, nullptr, 10);
        // mixed plans apply Algorithm 1's operator tA in double-float (bit 0).  The refinement
        // residual of the FP32 inverse stays FP64: in double-float (bit 1) it limits the
        // refined inverse to ~2^-45 |tA| |x|, measured 3-4e-13 against the FP64 inverse on 3-D
        // grids instead of ~1e-13.  Test switch: "1" keeps both on the FP64 stencil, "3" puts
        // both in double-float
        const char* sf = std::getenv("EXPM_STENCIL_FP64");
        P->stencil_df = opts->precision != EXPM_PREC_MIXED ? 0 : !sf ? 1 : sf[0] == '1' ? 0 : sf[0] == '3' ? 3 : 1;
    }
    int64_t n = 1;
    if (toeplitz) {
        n = op->n;
        P->tz.n = op->n;
        P->tz.bw = op->toeplitz_bw;
        P->tz.abs_rowsum = abs_rowsum;
    } else if (csr) {
        n = op->n;
        P->cs.n = op->n;
        P->cs.nnz = op->csr_rowptr[op->n];
        P->cs.abs_rowsum = abs_rowsum;
    } else {
        for (int d = 0; d < 3; ++d) {
            Axis& a = P->ax[d];
            if (d < op->ndim) {
                const int N = op->side[d];
                if (N < 1 || N > (1 << 20)) { delete P; return EXPM_INVALID_ARG; }
                const double h = 1.0 / (N + 1);
                a.N = N;
                a.l = op->diff / (h * h) + op->vel[d] / (2.0 * h);
                a.c = -2.0 * op->diff / (h * h);
                a.u = op->diff / (h * h) - op->vel[d] / (2.0 * h);
                if (!(a.l * a.u > 0.0)) { delete P; return EXPM_INVALID_ARG; }   // cell Peclet >= 1
                n *= N;
            } else {
                a = Axis{};
            }
        }
        if (op->ndim > 1 && (int64_t)P->ax[1].N * P->ax[2].N * P->ax[0].N != n) { delete P; return EXPM_INVALID_ARG; }
    }
    P->n = n;
    P->ld = round_up(n, 32);
    // CF table (Section 2): degree opts.nu_cf, by default nu = 14 as in the paper's
    // experiments (Section 5)
    {
        std::vector<std::complex<double>> tau, om;
        double w0 = 0, sg = 0;
        const int nu = opts->nu_cf ? opts->nu_cf : kNu;
        if (!expm_internal_cf_table(nu, tau, om, w0, sg)) { delete P; return EXPM_INTERNAL; }
        P->npoles = (int)tau.size();
        for (int i = 0; i < P->npoles; ++i) {
            P->tau_re[i] = tau[i].real();
            P->tau_im[i] = tau[i].imag();
            P->om_re[i] = om[i].real();
            P->om_im[i] = om[i].imag();
        }
        P->omega0 = w0;
    }
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
        delete P;
        return EXPM_CUDA_ERROR;
    }
    {
        // CTAs of the row-parallel passes: blocks_per_sm x SMs, at least 64 rows each (the
        // plan options, as an autotuner picks them; else 2, and twice that for the first CGS
        // pass, measured best on the 256 x 256 workload).  SMs = the device's count for the
        // first CGS pass; for the other row passes, the share of it that the plan was given.
        int per_sm = opts->row_ctas_per_sm > 0 ? opts->row_ctas_per_sm : 2;
        const int sms_rows = opts->grid_sms > 0 ? std::min(sms, (int)opts->grid_sms) : sms;
        P->nblk = consistent_blocks(n, std::max(1, std::min<int>(per_sm * sms_rows, (int)((n + 63) / 64))));
        // the first CGS pass (projection, update) may use more CTAs than the other row passes
        const int per_sm_cgs = opts->cgs_ctas_per_sm > 0 ? opts->cgs_ctas_per_sm : 2 * per_sm;
        P->nblk_cgs = consistent_blocks(n, std::max(1, std::min<int>(per_sm_cgs * sms, (int)((n + 63) / 64))));
    }
    const int m = opts->m;
    const int64_t ld = P->ld;
    P->ldH = (m + 1) * p_max;
    const int mpm = m * p_max;
    bool ok = true;
    ok = ok && dalloc(&P->V, (size_t)ld * (m + 1) * p_max);
    ok = ok && dalloc(&P->W, (size_t)ld * p_max);
    ok = ok && dalloc(&P->T1, (size_t)ld * p_max);
    ok = ok && dalloc(&P->T2, (size_t)ld * p_max);
    ok = ok && dalloc(&P->Zacc, (size_t)ld * p_max);
    ok = ok && dalloc(&P->Bst, (size_t)ld * p_max);
    ok = ok && dalloc(&P->Zst, (size_t)ld * p_max);
    ok = ok && dalloc(&P->H, (size_t)P->ldH * mpm);
    ok = ok && dalloc(&P->part, (size_t)std::max(P->nblk, P->nblk_cgs) * (mpm + p_max) * p_max);
    ok = ok && dalloc(&P->small, kSmallDoubles);
    ok = ok && dalloc(&P->S, (size_t)P->npoles * p_max * p_max * 2);
    ok = ok && dalloc(&P->Wc_slots, (size_t)P->npoles * (mpm + p_max) * p_max);
    ok = ok && dalloc(&P->stat, kStatDoubles);
    ok = ok && dalloc(&P->ctr, 4) && cudaMemset(P->ctr, 0, sizeof(unsigned) * 4) == cudaSuccess;
    if (opts->certify) {
        const size_t w = 2 * (size_t)P->npoles * p_max, rows = (size_t)mpm + p_max;
        if (8 * (rows * w + 16 * (rows | 1)) > 225 * 1024) { free_plan(P); return EXPM_INVALID_ARG; }
        ok = ok && dalloc(&P->Xcert, (size_t)ld * w) && dalloc(&P->Zcert, (size_t)P->npoles * mpm * p_max * 2) &&
             dalloc(&P->Ccert, rows * w) && dalloc(&P->rcert, (size_t)P->npoles * true_resid_blocks(n));
        if (toeplitz) ok = ok && dalloc(&P->Acert, (size_t)ld * w);
        P->hcert = new (std::nothrow) double[(size_t)P->npoles * true_resid_blocks(n)];
        ok = ok && P->hcert != nullptr;
    }
    if (poles_smem_bytes(mpm, p_max) == 0)   // elimination does not fit in shared memory
        ok = ok && dalloc(&P->poles, (size_t)P->npoles * ((size_t)mpm * mpm + 2 * (size_t)mpm * p_max) * 2);
    ok = ok && cudaMallocHost(reinterpret_cast<void**>(&P->hpin), sizeof(double) * kStatDoubles) == cudaSuccess;
    ok = ok && dalloc(&P->dotpart, (size_t)dot_blocks() * p_max) &&
         cudaMallocHost(reinterpret_cast<void**>(&P->hdot), sizeof(double) * dot_blocks() * p_max) == cudaSuccess;
    ok = ok && cudaEventCreateWithFlags(&P->cycle_ev, cudaEventDisableTiming) == cudaSuccess;
    if (opts->k_defl > 0) {
        // the kept count never exceeds k_defl rounded up to a multiple of p, nor (m - 1) p
        P->kdefl_max = std::min(opts->k_defl + p_max - 1, (m - 1) * p_max);
        const size_t kd = (size_t)P->kdefl_max;
        ok = ok && dalloc(&P->Vk, (size_t)ld * kd) && dalloc(&P->Pkd, (size_t)mpm * kd);
        ok = ok && cudaMallocHost(reinterpret_cast<void**>(&P->hH), sizeof(double) * (size_t)P->ldH * mpm) == cudaSuccess;
        ok = ok && cudaMallocHost(reinterpret_cast<void**>(&P->hPk), sizeof(double) * (size_t)mpm * kd) == cudaSuccess;
        ok = ok && cudaMallocHost(reinterpret_cast<void**>(&P->hHnew), sizeof(double) * (size_t)P->ldH * kd) == cudaSuccess;
    }
    const bool mixed = opts->precision == EXPM_PREC_MIXED;
    if (csr) {
        CsrOp& c = P->cs;
        c.ld = ld;
        c.pmax = p_max;
        const size_t nb = (size_t)csr_blocks(n);
        ok = ok && cudaMalloc(reinterpret_cast<void**>(&c.rowptr), sizeof(int64_t) * (size_t)(n + 1)) == cudaSuccess;
        ok = ok && cudaMalloc(reinterpret_cast<void**>(&c.colind), sizeof(int) * (size_t)std::max<int64_t>(c.nnz, 1)) == cudaSuccess;
        ok = ok && dalloc(&c.val, (size_t)std::max<int64_t>(c.nnz, 1)) && dalloc(&c.dinv, (size_t)n);
        ok = ok && dalloc(&c.work, (size_t)9 * ld * p_max) && dalloc(&c.part, 2 * nb * p_max);
        ok = ok && dalloc(&c.scal, 8 * (size_t)p_max);
        ok = ok && dalloc(&c.norms, 2 * (size_t)p_max);
        ok = ok && cudaMallocHost(reinterpret_cast<void**>(&c.hnorms), sizeof(double) * 2 * (size_t)p_max) == cudaSuccess;
    } else if (!toeplitz) {
        // preconditioner tables: every axis but x is transformed
        int64_t nmodes = 1;
        for (int d = 1; d < P->ndim; ++d) {
            const int N = P->ax[d].N;
            ok = ok && dalloc(&P->Qf[d], (size_t)N * N) && dalloc(&P->Qi[d], (size_t)N * N) &&
                 dalloc(&P->lam[d], (size_t)N);
            nmodes *= N;
        }
        P->nmodes = nmodes;
        ok = ok && dalloc(&P->th_m, (size_t)P->ax[0].N * nmodes) && dalloc(&P->th_c, (size_t)P->ax[0].N * nmodes);
        if (mixed) {
            for (int d = 1; d < P->ndim; ++d) {
                const int N = P->ax[d].N;
                ok = ok && dalloc(&P->Qf32[d], (size_t)N * N) && dalloc(&P->Qi32[d], (size_t)N * N);
            }
            ok = ok && dalloc(&P->th_m32, (size_t)P->ax[0].N * nmodes) &&
                 dalloc(&P->th_c32, (size_t)P->ax[0].N * nmodes);
            ok = ok && dalloc(&P->T1f, (size_t)ld * p_max) && dalloc(&P->T2f, (size_t)ld * p_max);
            ok = ok && dalloc(&P->R64, (size_t)ld * p_max);
        }
    }
    if (!ok) {
        cudaGetLastError();
        free_plan(P);
        return EXPM_NO_MEMORY;
    }
    cudaStream_t s = P->stream;
    bool cuda_ok = krylov_set_smem_limits() == cudaSuccess && poles_set_smem_limits() == cudaSuccess &&
                   operator_set_smem_limits() == cudaSuccess && cgs_tc_set_smem_limits() == cudaSuccess;
    if (csr && cuda_ok) {
        CsrOp& c = P->cs;
        cuda_ok = cudaMemcpyAsync(c.rowptr, op->csr_rowptr, sizeof(int64_t) * (size_t)(n + 1), cudaMemcpyHostToDevice, s) == cudaSuccess &&
                  (c.nnz == 0 || (cudaMemcpyAsync(c.colind, op->csr_colind, sizeof(int) * (size_t)c.nnz, cudaMemcpyHostToDevice, s) == cudaSuccess &&
                                  cudaMemcpyAsync(c.val, op->csr_val, sizeof(double) * (size_t)c.nnz, cudaMemcpyHostToDevice, s) == cudaSuccess)) &&
                  launch_csr_dinv(c, s) == cudaSuccess;
    }
    if (!toeplitz && !csr) {
        const int64_t nmodes = P->nmodes;
        for (int d = 1; d < P->ndim && cuda_ok; ++d)
            cuda_ok = launch_axis_setup(P->Qf[d], P->Qi[d], P->lam[d], P->ax[d].N, P->ax[d].l,
                                        P->ax[d].c, P->ax[d].u, s) == cudaSuccess;
        if (cuda_ok)
            cuda_ok = launch_thomas_setup(P->th_m, P->th_c, P->ax[0].N, nmodes, P->ax[0].l, P->ax[0].c,
                                          P->ax[0].u, P->ndim > 1 ? P->lam[1] : nullptr, P->ax[1].N,
                                          P->ndim > 2 ? P->lam[2] : nullptr, P->ax[2].N, s) == cudaSuccess;
        if (cuda_ok && mixed) {
            for (int d = 1; d < P->ndim && cuda_ok; ++d) {
                const int64_t NN = (int64_t)P->ax[d].N * P->ax[d].N;
                cuda_ok = launch_d2f(P->Qf[d], P->Qf32[d], NN, s) == cudaSuccess &&
                          launch_d2f(P->Qi[d], P->Qi32[d], NN, s) == cudaSuccess;
            }
            const int64_t nt = (int64_t)P->ax[0].N * nmodes;
            if (cuda_ok)
                cuda_ok = launch_d2f(P->th_m, P->th_m32, nt, s) == cudaSuccess &&
                          launch_d2f(P->th_c, P->th_c32, nt, s) == cudaSuccess;
        }
    }
    if (cuda_ok) {
        double taus[4 * EXPM_MAX_POLES] = {0};
        for (int i = 0; i < P->npoles; ++i) {
            taus[i] = P->tau_re[i];
            taus[EXPM_MAX_POLES + i] = P->tau_im[i];
            taus[2 * EXPM_MAX_POLES + i] = P->om_re[i];
            taus[3 * EXPM_MAX_POLES + i] = P->om_im[i];
        }
        cuda_ok = cudaMemcpyAsync(P->small + kOffTau, taus, sizeof(taus), cudaMemcpyHostToDevice, s) == cudaSuccess;
    }
    if (cuda_ok) cuda_ok = cudaStreamSynchronize(s) == cudaSuccess && cudaGetLastError() == cudaSuccess;
    if (!cuda_ok) {
        free_plan(P);
        return EXPM_CUDA_ERROR;
    }
    if (toeplitz) {
        const expm_status ts = toeplitz_setup(P, op, opts->algorithm != EXPM_ALG_SBFOM);
        if (ts != EXPM_OK) {
            cudaGetLastError();
            free_plan(P);
            return ts;
        }
    }
    *out = P;
    return EXPM_OK;
}

void expm_plan_destroy(expm_plan* plan) {
    if (plan && plan->stream) cudaStreamSynchronize(plan->stream);
    free_plan(plan);
}

expm_status expm_block(expm_plan* plan, double t, const double* dB, int64_t ldb, int p,
                       double* dZ, int64_t ldz, expm_info* info) {
    expm_status st = validate_block_args(plan, t, dB, ldb, p, dZ, ldz);
    if (st != EXPM_OK) return st;
    return run_block(plan, t, dB, ldb, p, dZ, ldz, info);
}

expm_status expm_block_host(expm_plan* plan, double t, const double* hB, int64_t ldb, int p,
                            double* hZ, int64_t ldz, expm_info* info) {
    expm_status st = validate_block_args(plan, t, hB, ldb, p, hZ, ldz);
    if (st != EXPM_OK) return st;
    cudaStream_t s = plan->stream;
    const int64_t n = plan->n, ld = plan->ld;
    CK(cudaMemcpy2DAsync(plan->Bst, ld * sizeof(double), hB, ldb * sizeof(double), n * sizeof(double), p,
                         cudaMemcpyHostToDevice, s));
    st = run_block(plan, t, plan->Bst, ld, p, plan->Zst, ld, info);
    if (st != EXPM_OK && st != EXPM_NOT_CONVERGED) return st;
    CK(cudaMemcpy2DAsync(hZ, ldz * sizeof(double), plan->Zst, ld * sizeof(double), n * sizeof(double), p,
                         cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    return st;
}

}  // extern "C"

namespace {

// The batched driver behind expm_block_batched and expm_block_batched_host.  With host
// buffers, instance i's B is copied to its plan's staging buffer on the plan's stream before
// its first cycle and its Z copied back after its last, so the copies of one instance overlap
// with the other instances' cycles.
expm_status batched_run(expm_plan* const* plans, int count, const double* t, const double* const* B,
                        const int64_t* ldb, const int* p, double* const* Z, const int64_t* ldz, expm_info* info,
                        bool host) {
    if (count < 1 || !plans || !t || !B || !ldb || !p || !Z || !ldz) return EXPM_INVALID_ARG;
    for (int i = 0; i < count; ++i) {
        const expm_status st = validate_block_args(plans[i], t[i], B[i], ldb[i], p[i], Z[i], ldz[i]);
        if (st != EXPM_OK) return st;
        for (int j = 0; j < i; ++j)
            if (plans[j] == plans[i]) return EXPM_INVALID_ARG;   // one call per plan (its workspace)
    }
    std::vector<RunState> rs(count);
    std::vector<char> active(count, 0);
    std::vector<expm_status> status(count, EXPM_OK);
    int left = 0;
    for (int i = 0; i < count; ++i) {
        expm_plan* P = plans[i];
        RunState& r = rs[i];
        r.t = t[i];
        r.p = p[i];
        if (host) {
            if (cudaMemcpy2DAsync(P->Bst, P->ld * sizeof(double), B[i], ldb[i] * sizeof(double), P->n * sizeof(double),
                                  p[i], cudaMemcpyHostToDevice, P->stream) != cudaSuccess) {
                status[i] = EXPM_CUDA_ERROR;
                continue;
            }
            r.dB = P->Bst;
            r.ldb = P->ld;
            r.dZ = P->Zst;
            r.ldz = P->ld;
        } else {
            r.dB = B[i];
            r.ldb = ldb[i];
            r.dZ = Z[i];
            r.ldz = ldz[i];
        }
        expm_status st = run_begin(P, r);
        if (st == EXPM_OK) st = run_issue(P, r);
        if (st != EXPM_OK) {
            status[i] = st;
            continue;
        }
        active[i] = 1;
        ++left;
    }
    // every plan's cycles run on its own stream; poll the cycle events and keep each
    // instance's next cycle queued as soon as its stop test has been read
    while (left > 0) {
        bool progress = false;
        for (int i = 0; i < count; ++i) {
            if (!active[i]) continue;
            expm_plan* P = plans[i];
            const cudaError_t q = cudaEventQuery(P->cycle_ev);
            if (q == cudaErrorNotReady) continue;
            progress = true;
            expm_status st = EXPM_OK;
            if (q != cudaSuccess) {
                st = EXPM_CUDA_ERROR;
            } else {
                run_check(P, rs[i]);
                if (!rs[i].done) {
                    st = run_issue(P, rs[i]);
                    if (st == EXPM_OK) continue;
                } else {
                    st = run_finish(P, rs[i], info ? &info[i] : nullptr);
                    if (host && (st == EXPM_OK || st == EXPM_NOT_CONVERGED) &&
                        cudaMemcpy2DAsync(Z[i], ldz[i] * sizeof(double), P->Zst, P->ld * sizeof(double),
                                          P->n * sizeof(double), p[i], cudaMemcpyDeviceToHost, P->stream) != cudaSuccess)
                        st = EXPM_CUDA_ERROR;
                }
            }
            status[i] = st;
            active[i] = 0;
            --left;
        }
        if (!progress) std::this_thread::yield();
    }
    for (int i = 0; i < count; ++i)
        if (cudaStreamSynchronize(plans[i]->stream) != cudaSuccess && status[i] == EXPM_OK) status[i] = EXPM_CUDA_ERROR;
    // first hard error, else NOT_CONVERGED if any instance stopped unconverged
    expm_status worst = EXPM_OK;
    for (int i = 0; i < count; ++i) {
        if (status[i] != EXPM_OK && status[i] != EXPM_NOT_CONVERGED) return status[i];
        if (status[i] == EXPM_NOT_CONVERGED) worst = EXPM_NOT_CONVERGED;
    }
    return worst;
}

// ---- the batched form as one CUDA graph with device-side stop tests
//
// Every instance is one branch of the graph: its start (R^0 = B = V_1 R for every pole), a
// WHILE conditional node whose body is one restart cycle followed by k_stop, and its finish
// (Z = omega_0 B + Z_acc and the status back to the host).  k_stop applies the stop test of
// eq. (49) / eq. (365) on the device and sets the loop's condition, so the whole batched solve
// is a single graph launch with no host round trip per cycle; the branches run concurrently.
__global__ void k_stop(const double* __restrict__ stat, int npoles, double tol, int fixed, int max_cycles,
                       int* ctl, cudaGraphConditionalHandle h) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    const int c = ctl[0] + 1;
    ctl[0] = c;
    double mx = 0.0;
    for (int i = 0; i < npoles; ++i) mx = fmax(mx, stat[i]);
    const int flags = reinterpret_cast<const int*>(stat + 24)[0];
    const bool conv = mx <= tol * sqrt(stat[16]);
    ctl[1] = conv ? 1 : 0;
    const bool more = flags == 0 && (fixed > 0 ? c < fixed : (!conv && c < max_cycles));
    cudaGraphSetConditional(h, more ? 1u : 0u);
}

}  // namespace

extern "C" {

expm_status expm_block_batched(expm_plan* const* plans, int count, const double* t, const double* const* dB,
                               const int64_t* ldb, const int* p, double* const* dZ, const int64_t* ldz,
                               expm_info* info) {
    return batched_run(plans, count, t, dB, ldb, p, dZ, ldz, info, false);
}

expm_status expm_block_batched_host(expm_plan* const* plans, int count, const double* t, const double* const* hB,
                                    const int64_t* ldb, const int* p, double* const* hZ, const int64_t* ldz,
                                    expm_info* info) {
    return batched_run(plans, count, t, hB, ldb, p, hZ, ldz, info, true);
}

expm_status expm_batch_create(expm_plan* const* plans, int count, const double* t, const double* const* dB,
                              const int64_t* ldb, const int* p, double* const* dZ, const int64_t* ldz, void* stream,
                              expm_batch** out) {
    if (!out || count < 1 || !plans || !t || !dB || !ldb || !p || !dZ || !ldz) return EXPM_INVALID_ARG;
    *out = nullptr;
    for (int i = 0; i < count; ++i) {
        const expm_status st = validate_block_args(plans[i], t[i], dB[i], ldb[i], p[i], dZ[i], ldz[i]);
        if (st != EXPM_OK) return st;
        const expm_plan* P = plans[i];
        // the device-side loop needs no host work between cycles: no deflated restart (host
        // eigenproblem), no certify accumulation, a capturable stream
        if (P->opts.k_defl > 0 || P->opts.certify || P->csr || !P->stream) return EXPM_INVALID_ARG;
        for (int j = 0; j < i; ++j)
            if (plans[j] == plans[i]) return EXPM_INVALID_ARG;
    }
    expm_batch* b = new (std::nothrow) expm_batch_s();
    if (!b) return EXPM_NO_MEMORY;
    b->plans.assign(plans, plans + count);
    b->rs.resize(count);
    b->stream = reinterpret_cast<cudaStream_t>(stream);
    b->fixed_launches.assign(count, 0);
    b->cycle_launches.assign(count, 0);
    if (cudaMalloc(reinterpret_cast<void**>(&b->dctl), sizeof(int) * 2 * count) != cudaSuccess ||
        cudaMallocHost(reinterpret_cast<void**>(&b->hctl), sizeof(int) * 2 * count) != cudaSuccess ||
        cudaGraphCreate(&b->graph, 0) != cudaSuccess) {
        cudaGetLastError();
        batch_free(b);
        return EXPM_NO_MEMORY;
    }
    for (int i = 0; i < count; ++i) {
        expm_plan* P = plans[i];
        RunState& r = b->rs[i];
        r.t = t[i];
        r.dB = dB[i];
        r.ldb = ldb[i];
        r.p = p[i];
        r.dZ = dZ[i];
        r.ldz = ldz[i];
        int* ctl = b->dctl + 2 * i;
        const int64_t l0 = P->launches;
        cudaGraphNode_t nb = nullptr, nc = nullptr, nf = nullptr;
        expm_status st = capture_child(P, b->graph, nullptr, &nb, [&]() -> expm_status {
            CK(cudaMemsetAsync(ctl, 0, sizeof(int) * 2, P->stream));
            return run_begin(P, r);
        });
        const int64_t l1 = P->launches;
        cudaGraphConditionalHandle hdl;
        cudaGraphNodeParams cp = {};
        if (st == EXPM_OK) {
            if (cudaGraphConditionalHandleCreate(&hdl, b->graph, 1, cudaGraphCondAssignDefault) != cudaSuccess) {
                st = EXPM_CUDA_ERROR;
            } else {
                cp.type = cudaGraphNodeTypeConditional;
                cp.conditional.handle = hdl;
                cp.conditional.type = cudaGraphCondTypeWhile;
                cp.conditional.size = 1;
                if (cudaGraphAddNode(&nc, b->graph, &nb, nullptr, 1, &cp) != cudaSuccess) st = EXPM_CUDA_ERROR;
            }
        }
        if (st == EXPM_OK) {
            cudaGraph_t body = cp.conditional.phGraph_out[0];
            if (cudaStreamBeginCaptureToGraph(P->stream, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal) !=
                cudaSuccess) {
                st = EXPM_CUDA_ERROR;
            } else {
                st = issue_cycle(P, r.t, r.p, r.alg, 0, 0, false);
                if (st == EXPM_OK) {
                    k_stop<<<1, 32, 0, P->stream>>>(P->stat, P->npoles, P->opts.tol, P->opts.fixed_cycles,
                                                     P->opts.max_cycles, ctl, hdl);
                    if (cudaGetLastError() != cudaSuccess) st = EXPM_CUDA_ERROR;
                }
                cudaGraph_t g2 = body;
                if (cudaStreamEndCapture(P->stream, &g2) != cudaSuccess && st == EXPM_OK) st = EXPM_CUDA_ERROR;
            }
        }
        const int64_t l2 = P->launches;
        if (st == EXPM_OK)
            st = capture_child(P, b->graph, &nc, &nf, [&]() -> expm_status {
                LAUNCH(EXPM_STAGE_OTHER, launch_axpby(P->omega0, r.dB, r.ldb, 1.0, P->Zacc, P->ld, r.dZ, r.ldz, P->n,
                                                      r.p, P->stream));
                CK(cudaMemcpyAsync(P->hpin, P->stat, sizeof(double) * kStatDoubles, cudaMemcpyDeviceToHost, P->stream));
                CK(cudaMemcpyAsync(b->hctl + 2 * i, ctl, sizeof(int) * 2, cudaMemcpyDeviceToHost, P->stream));
                return EXPM_OK;
            });
        // launch accounting: the start and the finish once, the cycle body once per cycle
        b->fixed_launches[i] = (l1 - l0) + (P->launches - l2);
        b->cycle_launches[i] = (l2 - l1) + 1;
        P->launches = l0;
        if (st != EXPM_OK) {
            cudaGetLastError();
            batch_free(b);
            return st;
        }
    }
    if (cudaGraphInstantiate(&b->exec, b->graph, 0) != cudaSuccess) {
        cudaGetLastError();
        batch_free(b);
        return EXPM_CUDA_ERROR;
    }
    *out = b;
    return EXPM_OK;
}

expm_status expm_batch_run(expm_batch* b, expm_info* info) {
    if (!b || !b->exec) return EXPM_INVALID_ARG;
    CK(cudaGraphLaunch(b->exec, b->stream));
    CK(cudaStreamSynchronize(b->stream));
    expm_status worst = EXPM_OK;
    for (size_t i = 0; i < b->plans.size(); ++i) {
        expm_plan* P = b->plans[i];
        RunState& r = b->rs[i];
        r.cycles = b->hctl[2 * i];
        r.steps = r.cycles * P->opts.m;
        r.converged = b->hctl[2 * i + 1] != 0;
        r.normB = std::sqrt(P->hpin[16]);
        r.result = check_flags(P->hpin);
        P->launches += b->fixed_launches[i] + (int64_t)r.cycles * b->cycle_launches[i];
        if (info) {
            expm_info& f = info[i];
            std::memset(&f, 0, sizeof(f));
            f.cycles = r.cycles;
            f.block_steps = r.steps;
            f.matvecs = (int64_t)r.steps * r.p;
            f.converged = r.converged ? 1 : 0;
            f.npoles = P->npoles;
            f.breakdown = reinterpret_cast<const int*>(P->hpin + 24)[1] ? 1 : 0;
            for (int k = 0; k < P->npoles; ++k) f.resid[k] = P->hpin[k];
            f.normB = r.normB;
            f.algorithm = r.alg;
            f.normA_bound = norm_bound(P, r.t);
        }
        expm_status st = r.result;
        if (st == EXPM_OK && P->opts.fixed_cycles == 0 && !r.converged) st = EXPM_NOT_CONVERGED;
        if (st != EXPM_OK && st != EXPM_NOT_CONVERGED) return st;
        if (st == EXPM_NOT_CONVERGED) worst = st;
    }
    return worst;
}

void expm_batch_destroy(expm_batch* b) {
    if (b && b->stream) cudaStreamSynchronize(b->stream);
    batch_free(b);
}

expm_status expm_block_adjoint(expm_plan* plan, double t, const double* dG, int64_t ldg, int p,
                               const double* dZ, int64_t ldz, double* dGB, int64_t ldgb, double* hGt,
                               expm_info* info) {
    if (!plan || !dG || (!dGB && !hGt) || (hGt && !dZ)) return EXPM_INVALID_ARG;
    expm_status st = validate_block_args(plan, t, dG, ldg, p, dGB ? (const void*)dGB : (const void*)dZ,
                                         dGB ? ldgb : ldz);
    if (st != EXPM_OK) return st;
    if (hGt && (ldz < plan->n || dZ == dGB)) return EXPM_INVALID_ARG;
    if (plan->csr) return EXPM_INVALID_ARG;   // the adjoint needs A^T's plan (stencils, Toeplitz)
    expm_plan* P = plan;
    cudaStream_t s = P->stream;
    const int64_t n = P->n, ld = P->ld;
    if (hGt) {
        // dL/dt = <G, A Z> (t folded out): A Z into T1, then per-column dot products with
        // fixed-order partial sums
        if ((st = op_apply_internal(P, 1.0, dZ, ldz, p, P->T1, ld)) != EXPM_OK) return st;
        const int nb = dot_blocks();
        for (int c = 0; c < p; ++c)
            LAUNCH(EXPM_STAGE_OTHER, launch_dot_partial(dG + (int64_t)c * ldg, P->T1 + (int64_t)c * ld, n,
                                                        P->dotpart + (int64_t)c * nb, s));
        CK(cudaMemcpyAsync(P->hdot, P->dotpart, sizeof(double) * (size_t)nb * p, cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
        double acc = 0.0;
        for (int c = 0; c < p; ++c) {
            double sc = 0.0;
            for (int b = 0; b < nb; ++b) sc += P->hdot[(size_t)c * nb + b];
            acc += sc;
        }
        *hGt = acc;
    }
    if (!dGB) {
        if (info) std::memset(info, 0, sizeof(*info));
        return EXPM_OK;
    }
    // dL/dB = r(tA)^T G = r(tA^T) G by the same method on A^T
    expm_plan* PT = P;
    if (!P->toeplitz) {
        if (!P->adj) {
            expm_op_desc opT = P->op;
            for (int d = 0; d < 3; ++d) opT.vel[d] = -opT.vel[d];
            st = expm_plan_create(&opT, P->p_max, &P->opts, P->stream, &P->adj);
            if (st != EXPM_OK) {
                P->adj = nullptr;
                return st;
            }
        }
        PT = P->adj;
    }
    return run_block(PT, t, dG, ldg, p, dGB, ldgb, info);
}

expm_status expm_op_apply(expm_plan* plan, double t, const double* dV, int64_t ldv, int p,
                          double* dW, int64_t ldw) {
    expm_status st = validate_block_args(plan, t, dV, ldv, p, dW, ldw);
    if (st != EXPM_OK) return st;
    return op_apply_internal(plan, t, dV, ldv, p, dW, ldw);
}

expm_status expm_prec_apply(expm_plan* plan, double t, const double* dV, int64_t ldv, int p,
                            double* dW, int64_t ldw) {
    expm_status st = validate_block_args(plan, t, dV, ldv, p, dW, ldw);
    if (st != EXPM_OK) return st;
    return prec_apply_internal(plan, t, dV, ldv, p, dW, ldw);
}

expm_status expm_arnoldi(expm_plan* plan, double t, const double* dV1, int64_t ldv1, int p,
                         double* dVout, int64_t ldvo, double* dHout, int64_t ldh) {
    expm_status st = validate_block_args(plan, t, dV1, ldv1, p, dVout, ldvo);
    if (st != EXPM_OK) return st;
    if (!dHout) return EXPM_INVALID_ARG;
    const int m = plan->opts.m;
    if (ldh < (int64_t)(m + 1) * p) return EXPM_INVALID_ARG;
    cudaStream_t s = plan->stream;
    const int64_t n = plan->n, ld = plan->ld;
    CK(cudaMemsetAsync(plan->stat, 0, sizeof(double) * kStatDoubles, s));
    CK(cudaMemsetAsync(plan->ctr, 0, sizeof(unsigned) * 4, s));
    CK(cudaMemsetAsync(plan->H, 0, sizeof(double) * (size_t)plan->ldH * m * plan->p_max, s));
    expm_plan* P = plan;
    LAUNCH(EXPM_STAGE_OTHER, launch_copy(dV1, ldv1, plan->V, ld, n, p, s));
    for (int j = 0; j < m; ++j) {
        st = block_step(plan, t, j, p, EXPM_ALG_PSBFOM);
        if (st != EXPM_OK) return st;
    }
    LAUNCH(EXPM_STAGE_OTHER, launch_copy(plan->V, ld, dVout, ldvo, n, (m + 1) * p, s));
    CK(cudaMemcpy2DAsync(dHout, ldh * sizeof(double), plan->H, plan->ldH * sizeof(double),
                         (size_t)(m + 1) * p * sizeof(double), (size_t)m * p, cudaMemcpyDeviceToDevice, s));
    CK(cudaMemcpyAsync(plan->hpin, plan->stat, sizeof(double) * kStatDoubles, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    prof_flush(plan);
    return check_flags(plan->hpin);
}

expm_status expm_plan_profile(expm_plan* plan, int enable) {
    if (!plan) return EXPM_INVALID_ARG;
    if (plan->stream) CK(cudaStreamSynchronize(plan->stream));
    prof_flush(plan);
    if (enable && plan->ev.empty()) {
        plan->ev.resize(kEventPool);
        for (auto& e : plan->ev) CK(cudaEventCreate(&e));
    }
    if (enable) {
        plan->launches = 0;
        for (int k = 0; k < EXPM_NSTAGES; ++k) {
            plan->stage_launches[k] = 0;
            plan->stage_ms[k] = 0.0;
        }
    }
    plan->prof = enable != 0;
    return EXPM_OK;
}

expm_status expm_plan_get_profile(expm_plan* plan, double* stage_ms, int64_t* stage_launches,
                                  int nstages, int64_t* total_launches) {
    if (!plan || nstages < 0) return EXPM_INVALID_ARG;
    if (plan->stream) CK(cudaStreamSynchronize(plan->stream));
    prof_flush(plan);
    for (int k = 0; k < nstages && k < EXPM_NSTAGES; ++k) {
        if (stage_ms) stage_ms[k] = plan->stage_ms[k];
        if (stage_launches) stage_launches[k] = plan->stage_launches[k];
    }
    if (total_launches) *total_launches = plan->launches;
    return EXPM_OK;
}

}  // extern "C"
