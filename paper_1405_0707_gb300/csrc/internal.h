// internal.h -- plan layout and kernel launchers shared by the library's CUDA sources.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <complex>
#include <vector>

#include "../../include/expm_block.h"

namespace expm {

constexpr int kMaxP = 32;          // block width limit
constexpr int kMaxMP = 512;        // m * p limit
constexpr int kProjThreads = 256;

// One axis of the convection-diffusion operator (t = 1): tridiag(l, c, u).
struct Axis {
    int N = 1;
    double l = 0, c = 0, u = 0;
};

// Strided, two-level batched real GEMM  C = A * B  (B row-major, shared by the batch).
struct GemmArgs {
    const double* A;
    const double* B;
    double* C;
    int M, N, K;
    int64_t a_rs, a_cs, a_b1, a_b2;
    int64_t c_rs, c_cs, c_b1, c_b2;
    int ldb;
    int nb1, nb2;
};

// Mixed-precision variant: A and C may be FP64 or FP32 (a_f64 / c_f64), B is FP32,
// arithmetic FP32; accumulate != 0 adds into C.
struct GemmArgsMixed {
    const void* A;
    const float* B;
    void* C;
    int M, N, K;
    int64_t a_rs, a_cs, a_b1, a_b2;
    int64_t c_rs, c_cs, c_b1, c_b2;
    int ldb;
    int nb1, nb2;
    int a_f64, c_f64, accumulate;
    // ms > 0: the row index m is a pair (m % ms, m / ms) with strides (a_rs, a_ms2) in A and
    // (c_rs, c_ms2) in C, so two grid axes form one long M dimension (no padding per line)
    int ms = 0;
    int64_t a_ms2 = 0, c_ms2 = 0;
};

// Four-step FFT geometry: N = N1 N2 (powers of two), C adjacent columns per block in the
// column pass, Rr rows per block in the row pass.
struct FftPlan {
    int64_t N = 0;
    int N1 = 0, N2 = 0, C = 1, Rr = 1;
};

enum FftMode {
    FFT_COL_FWD_REAL = 0,     // real column pairs of V (zero beyond nreal) -> forward column pass
    FFT_COL_FWD_CPLX = 1,     // complex in -> forward column pass
    FFT_COL_INV_REAL = 2,     // inverse column pass -> real/imag parts to column pairs of W (rows < nreal)
    FFT_COL_INV_CPLX = 3,     // inverse column pass -> complex out (times scale)
    FFT_COL_INV_TRUNC_FWD = 4,// inverse column pass, zero rows >= nreal, forward column pass
    FFT_ROW_FWD = 10,         // forward row pass
    FFT_ROW_MATVEC = 11,      // forward row, times scale * lam (real), inverse row
    FFT_ROW_GSF_A = 12,       // forward row; out = inv(conj(mu1) y) scale, out2 = inv(conj(mu2) y) scale
    FFT_ROW_GSF_B = 13        // forward rows of in, in2; out = inv(mu1 f1 - mu2 f2) scale
};

// Arguments of one FFT pass (complex buffers hold nseq sequences of N interleaved complex).
struct FftArgs {
    FftPlan f;
    const double* V = nullptr;  // real input columns (FFT_COL_FWD_REAL), ld ldv
    int64_t ldv = 0;
    double* W = nullptr;        // real output columns (FFT_COL_INV_REAL), ld ldw
    int64_t ldw = 0;
    int p = 0;                  // real columns (2 per sequence)
    int64_t nreal = 0;          // rows of the real columns (n)
    const double* in = nullptr;
    const double* in2 = nullptr;
    double* out = nullptr;
    double* out2 = nullptr;
    const double* lam = nullptr;   // real spectrum (transposed order)
    const double* mu1 = nullptr;   // complex spectra (transposed order)
    const double* mu2 = nullptr;
    double scale = 1.0;
    const double* tw1 = nullptr;   // W_{N1}^k
    const double* tw2 = nullptr;   // W_{N2}^k
    const double* thi = nullptr;   // W_N^{64 h}
    const double* tlo = nullptr;   // W_N^l, l < 64
    // the same tables as float pairs (re_hi, re_lo, im_hi, im_lo); with df set the passes
    // compute in double-float arithmetic (data stays FP64 in memory)
    const float* tw1f = nullptr;
    const float* tw2f = nullptr;
    const float* thif = nullptr;
    const float* tlof = nullptr;
    int df = 0;
};

// Symmetric Toeplitz operator state (device buffers owned by the plan).
struct ToeplitzOp {
    int64_t n = 0, bw = 0;
    FftPlan f{};
    double* col = nullptr;      // a_0 .. a_bw
    double* tw1 = nullptr;      // complex tables
    double* tw2 = nullptr;
    double* thi = nullptr;
    double* tlo = nullptr;
    float* tw1f = nullptr;      // float-pair copies of the tables (mixed precision)
    float* tw2f = nullptr;
    float* thif = nullptr;
    float* tlof = nullptr;
    bool use_df = false;        // products and inverses in double-float (set after setup)
    double* lam = nullptr;      // N real: spectrum of the circulant embedding (transposed order)
    double* Ua = nullptr;       // nseq_max = max(2, ceil(p_max/2)) sequences of N complex
    double* Ub = nullptr;       // (Gohberg-Semencul) 2 nseq_max sequences
    double* mu1 = nullptr;      // (Gohberg-Semencul) spectra of [x; 0] and [xh; 0], N complex each
    double* mu2 = nullptr;
    double x0 = 0.0;            // first entry of the generator x = T^{-1} e_1
    int cg_iters = 0;
    double cg_resid = 0.0;      // backward error ||e_1 - T x|| / (||T||_1 ||x|| + 1)
    bool pcg = false;           // generator solved with the circulant preconditioner
    double abs_rowsum = 0.0;    // |a_0| + 2 sum_k |a_k|  (bound of ||T||)
    bool gsf = false;           // inverse available
};

// A general sparse operator (EXPM_OP_CSR): the matrix on the device, its inverted diagonal
// (the inner solve's Jacobi preconditioner) and the inner solver's workspace.
struct CsrOp {
    int64_t n = 0, nnz = 0, ld = 0;
    int pmax = 0;
    int64_t* rowptr = nullptr;
    int* colind = nullptr;
    double* val = nullptr;
    double* dinv = nullptr;
    double abs_rowsum = 0.0;    // max_i sum_j |a_ij| (bound of ||A||_inf)
    double* work = nullptr;     // 9 x ld x pmax: the inner solver's vectors
    double* part = nullptr;     // csr_blocks(n) x 2 x pmax partial sums
    double* scal = nullptr;     // pmax x 8: the columns' solver scalars
    double* norms = nullptr;    // 2 pmax: squared residual and right-hand-side norms
    double* hnorms = nullptr;   // pinned host mirror of norms
};

}  // namespace expm

struct GraphEntry {
    int alg = 0, p = 0;
    double t = 0.0;
    int kk = 0, prologue = 0;   // deflated restart: kept Ritz vectors, kind of restart prologue
    cudaGraphExec_t exec = nullptr;
    int64_t launches = 0;
    int64_t stage_launches[EXPM_NSTAGES] = {};
};

struct expm_plan_s {
    expm_op_desc op{};
    expm_opts opts{};
    int ndim = 1;
    expm::Axis ax[3];
    bool toeplitz = false;     // EXPM_OP_TOEPLITZ_SYM
    expm::ToeplitzOp tz;
    bool csr = false;          // EXPM_OP_CSR
    expm::CsrOp cs;
    int64_t inner_iters = 0;   // CSR: inner solver iterations of the current call
    int64_t n = 0, ld = 0;
    int p_max = 0;
    cudaStream_t stream = nullptr;
    // CF table (poles with Im > 0)
    int npoles = 0;
    double tau_re[EXPM_MAX_POLES], tau_im[EXPM_MAX_POLES];
    double om_re[EXPM_MAX_POLES], om_im[EXPM_MAX_POLES];
    double omega0 = 0;
    // preconditioner tables (device)
    double* Qf[3] = {nullptr, nullptr, nullptr};   // diag(rho^j) Q      (N x N, row-major)
    double* Qi[3] = {nullptr, nullptr, nullptr};   // Q diag(rho^-j)     (N x N, row-major)
    double* lam[3] = {nullptr, nullptr, nullptr};  // axis eigenvalues (t = 1)
    double* th_m = nullptr;                          // Thomas 1/pivot, [x * nmodes + mode]
    double* th_c = nullptr;                          // Thomas c',      [x * nmodes + mode]
    int64_t nmodes = 1;
    // mixed precision: FP32 copies of the tables and FP32 transform buffers
    float* Qf32[3] = {nullptr, nullptr, nullptr};
    float* Qi32[3] = {nullptr, nullptr, nullptr};
    float* th_m32 = nullptr;
    float* th_c32 = nullptr;
    float* T1f = nullptr;      // ld x p_max
    float* T2f = nullptr;      // ld x p_max
    double* R64 = nullptr;     // ld x p_max   residual of the refined inverse
    int refine = 2;            // FP64 refinement steps of the FP32 inverse
    // workspace (device)
    double* V = nullptr;       // ld x (m+1) p_max       Krylov basis
    double* W = nullptr;       // ld x p_max
    double* T1 = nullptr;      // ld x p_max             transform temporaries
    double* T2 = nullptr;
    double* Zacc = nullptr;    // ld x p_max
    double* Bst = nullptr;     // ld x p_max             staging for the host entry point
    double* H = nullptr;       // ldH x m p_max, ldH = (m+1) p_max
    int ldH = 0;
    double* part = nullptr;    // nblk x (m+1) p_max x p_max partial sums
    int nblk = 0;
    int nblk_cgs = 0;          // CTAs of the first CGS pass (projection, update)
    double* small = nullptr;   // small scratch (see api.cu for the map)
    double* poles = nullptr;   // per-pole elimination workspace (global fallback)
    double* S = nullptr;       // per-pole restart factors, npoles x p x p complex
    double* Wc_slots = nullptr;// per-pole (m+1)p x p update coefficients
    double* stat = nullptr;    // device status block: res[16], normsq, flags (ints)
    unsigned* ctr = nullptr;   // last-CTA ticket counter of the fused reductions
    double* hpin = nullptr;    // pinned host mirror of stat
    cudaEvent_t cycle_ev = nullptr;   // recorded after every restart cycle
    double* dotpart = nullptr; // dot_blocks() x p_max partial sums (adjoint's <G, A Z>)
    double* hdot = nullptr;    // pinned host mirror of dotpart
    expm_plan_s* adj = nullptr;// plan of A^T for the adjoint (created on first use)
    double* Zst = nullptr;     // ld x p_max staging for the host entry point
    // certify mode: per-pole solutions (real/imag columns), Z_i, coefficient matrix, partials
    double* Xcert = nullptr;   // ld x 2 npoles p_max
    double* Acert = nullptr;   // ld x 2 npoles p_max   tA Xcert (Toeplitz operator)
    double* Zcert = nullptr;   // npoles x m p_max x p_max complex
    double* Ccert = nullptr;   // ((m+1) p_max) x 2 npoles p_max
    double* rcert = nullptr;   // npoles x true_resid_blocks(n)
    double* hcert = nullptr;   // host copy of rcert
    // profiling: launch counts always, event timing when enabled
    bool prof = false;
    int64_t launches = 0;
    int64_t stage_launches[EXPM_NSTAGES] = {};
    double stage_ms[EXPM_NSTAGES] = {};
    std::vector<cudaEvent_t> ev;
    std::vector<int> pend_stage;          // stage of pending event pair k (events 2k, 2k+1)
    int ev_used = 0;
    // CUDA graphs of one restart cycle, keyed by (algorithm, p, t)
    bool use_graphs = false;
    bool qr_single = true;     // mixed path: try the single accurate Cholesky-QR pass
    int cgs_tc = 0;            // mixed path, first CGS update on the tensor cores: 0 never, 1 always, 2 by shape
    int proj_tc = 0;           // mixed path, first CGS projection on the tensor cores: 0 never, 1 always, 2 by shape
    int stencil_df = 0;        // mixed path: the stencil in double-float (k_cd_apply_df)
    long tc_spin = 1L << 24;   // bound of the tensor-core kernel's mbarrier waits (iterations)
    // deflated restart (opts.k_defl > 0)
    int kdefl_max = 0;         // columns of Vk and Pkd
    double* Vk = nullptr;      // ld x kdefl_max: V_m P_k
    double* Pkd = nullptr;     // m p_max x kdefl_max: P_k in chunks of 16 columns, each row-major
    double* hH = nullptr;      // pinned: H~ after each cycle (ldH x m p_max)
    double* hPk = nullptr;     // pinned: staging of Pkd
    double* hHnew = nullptr;   // pinned: the leading (kk + p) x kk block of H~ after the restart
    std::vector<GraphEntry> graphs;
};

// ---------------------------------------------------------------- launchers
namespace expm {
// general sparse operators (k_csr.cu)
int csr_blocks(int64_t n);
cudaError_t launch_csr_spmm(const CsrOp& a, double alpha, const double* X, int64_t ldx, int p, double* Y,
                            int64_t ldy, cudaStream_t s);
cudaError_t launch_csr_dinv(CsrOp& a, cudaStream_t s);
cudaError_t csr_inverse(const CsrOp& a, double t, const double* V, int64_t ldv, int p, double* W, int64_t ldw,
                        double eta, int maxit, cudaStream_t s, int* iters, int* converged);
cudaError_t launch_gemm(const GemmArgs& g, cudaStream_t s);
cudaError_t launch_tridiag_lines(const double* in, int64_t ld_in, double* out, int64_t ld_out,
                                 int p, int L, int64_t nmodes, double l_sub, const double* th_m,
                                 const double* th_c, double inv_t, cudaStream_t s);
cudaError_t launch_thomas_setup(double* th_m, double* th_c, int L, int64_t nmodes,
                                double l, double c, double u, const double* lam_y, int Ny,
                                const double* lam_z, int Nz, cudaStream_t s);
cudaError_t launch_axis_setup(double* Qf, double* Qi, double* lam, int N, double l, double c,
                              double u, cudaStream_t s);
cudaError_t launch_cd_apply(const double* V, int64_t ldv, double* W, int64_t ldw, int p,
                            int ndim, int nx, int ny, int nz, const Axis* ax, double t,
                            cudaStream_t s, const double* Y = nullptr, int64_t ldy = 0,
                            double beta = 0.0, float* W32 = nullptr, int df = 0);
cudaError_t launch_gemm32(const GemmArgsMixed& g, cudaStream_t s);
cudaError_t launch_tridiag_lines32(float* y, int64_t ld, int p, int L, int64_t nmodes, float l_sub,
                                   const float* th_m, const float* th_c, float inv_t,
                                   cudaStream_t s);
cudaError_t launch_d2f(const double* in, float* out, int64_t n, cudaStream_t s);

// block Gram-Schmidt / Cholesky-QR pieces
cudaError_t launch_proj_partial(const double* V, int64_t ldv, int cols, const double* W,
                                int64_t ldw, int p, int64_t n, double* part, int nblk,
                                cudaStream_t s, int f32 = 0);
bool cgs_rows_fit(int cols, int p);
cudaError_t launch_cgs_rows(int upd, const double* V, int64_t ldv, int cols, double* W, int64_t ldw, int p,
                            int64_t n, const double* h, double* part, int nblk, int gram, cudaStream_t s);
// hcols < 0: every output row a < cols goes to H; else only a < hcols (the rest to h only)
cudaError_t launch_reduce_h(const double* part, int nblk, int cols, int p, double* h,
                            double* H, int ldH, int row0, int col0, int accumulate,
                            cudaStream_t s, int hcols = -1);
cudaError_t launch_update_proj(const double* V, int64_t ldv, int cols, double* W, int64_t ldw,
                               int p, int64_t n, const double* h, double* part, int nblk,
                               int gram, cudaStream_t s, int f32 = 0, int upd32 = 0, double* G = nullptr,
                               unsigned* ctr = nullptr);
// Mixed path, p <= 8: Cholesky-QR pass with an FP32 factorisation (mode 0: of G; modes 1
// and 2: of the deviation G - I), corrections in FP32, W and the R product in FP64.
cudaError_t launch_qr_mixed_rows(double* W, int64_t ldw, int p, int64_t n, int nblk, double* G, double* part,
                                 unsigned* ctr, int mode, double* R, double* Rinv, const double* Rtot_in,
                                 double* Rtot_out, double* H, int ldH, int hrow, int hcol, double* normsq_out,
                                 int* flags, double* out, int64_t ldo, cudaStream_t s,
                                 const double* Vc = nullptr, int64_t ldvc = 0, int ccols = 0,
                                 const double* h2 = nullptr, double* fin = nullptr, int64_t ldfin = 0);
constexpr int kRowsMaxP = 16;  // widths handled by the row-per-thread kernels
// The first CGS pass's update W <- W - V h on the tensor cores (k_cgs_tc.cu): p <= 16,
// cols <= 160.  The second projection and the Gram matrix follow from launch_cgs_rows(0, ...,
// gram = 1).
bool cgs_tc_fit(int cols, int p);
cudaError_t launch_cgs_tc(const double* V, int64_t ldv, int cols, double* W, int64_t ldw, int p, int64_t n,
                          const double* h, int* flags, long spin_limit, cudaStream_t s);
// The first CGS pass's projection h = V^T W on the tensor cores (k_cgs_tc.cu, kind::tf32 with
// a hi/lo split): partial[blk][a][c] for blk < nb as the FP32 projection kernel writes them;
// p <= 16, cols <= 160; nb = proj_tc_blocks(n, cols, max) CTAs looping over 256-row tiles.  A bounded wait that runs
// out sets bit 4 of flags[0].
bool proj_tc_fit(int cols, int p);
int proj_tc_blocks(int64_t n, int cols, int max_blocks);
cudaError_t launch_proj_tc(const double* V, int64_t ldv, int cols, const double* W, int64_t ldw, int p, int64_t n,
                           double* part, int nb, int* flags, long spin_limit, cudaStream_t s);
cudaError_t cgs_tc_set_smem_limits();
// Cholesky-QR passes: mode 0 (unshifted, shifted on ill-conditioning, sets flags[2] when a
// third pass is needed), mode 1, mode 2 (no-op unless flags[2]); see k_krylov.cu.
cudaError_t launch_chol(const double* part, int nblk, int p, double shift_rel, double* R,
                        double* Rinv, double* Rtot, int mode, double* H, int ldH, int hrow,
                        int hcol, double* normsq_out, int* flags, cudaStream_t s);
cudaError_t launch_trsm(double* W, int64_t ldw, int p, int64_t n, const double* Rinv,
                        double* out, int64_t ldo, double* part, int nblk, int gram,
                        const int* extra, int tmode, cudaStream_t s);
// projected solves / update
cudaError_t launch_poles(const double* H, int ldH, int mp, int p, int npoles,
                         const double* tau_re, const double* tau_im, const double* om_re,
                         const double* om_im, double* S, double* work, double* Wc_slots,
                         double* res, int* flags, int alg, cudaStream_t s, double* Zout = nullptr,
                         int kk = 0);
cudaError_t launch_certify_coeffs(const double* H, int ldH, int mp, int p, int npoles, const double* Zs,
                                  double* C, int alg, cudaStream_t s, int kk = 0);
int true_resid_blocks(int64_t n);
// AX != nullptr: tA X is given (same column layout, leading dimension ldax) instead of the stencil
cudaError_t launch_true_resid(const double* X, int64_t ldx, const double* B, int64_t ldb, int p, int npoles,
                              int ndim, int nx, int ny, int nz, const Axis* ax, double t, const double* tau_re,
                              const double* tau_im, double* part, cudaStream_t s, const double* AX = nullptr,
                              int64_t ldax = 0);
cudaError_t launch_combine(const double* Wc_slots, int npoles, int rows, int p, double* Wc,
                           cudaStream_t s);
cudaError_t launch_combine2(const double* H, int ldH, int mp, int p, int npoles,
                            const double* Y_slots, double* Wc, int alg, cudaStream_t s, int kk = 0);
cudaError_t launch_update_z(double* V, int64_t ldv, int cols, int p, int64_t n,
                            const double* Wc, double* Z, int64_t ldz, int restart_copy,
                            cudaStream_t s, int nblk, int df = 0);
int consistent_blocks(int64_t n, int requested);
// FFT and Toeplitz pieces (k_fft.cu)
FftPlan fft_geometry(int64_t nmin);
bool fft_geometry_ok(const FftPlan& f);
cudaError_t fft_set_smem_limits();
cudaError_t launch_fft_tables(const FftPlan& f, double* tw1, double* tw2, double* thi, double* tlo,
                              cudaStream_t s);
cudaError_t launch_fft_tables_df(const double* src, float* dst, int64_t count, cudaStream_t s);
cudaError_t launch_fft_cols(const FftArgs& a, int mode, int nseq, cudaStream_t s);
cudaError_t launch_fft_rows(const FftArgs& a, int mode, int nseq, cudaStream_t s);
cudaError_t launch_embed_toeplitz(const double* a, int64_t bw, int64_t N, double* U, cudaStream_t s);
cudaError_t launch_embed_gsf(const double* x, int64_t n, int64_t N, double* U, cudaStream_t s);
cudaError_t launch_real_part(const double* U, double* lam, int64_t N, cudaStream_t s);
int dot_blocks();
cudaError_t launch_dot_partial(const double* a, const double* b, int64_t n, double* part, cudaStream_t s);
cudaError_t launch_cg_step(double* x, double* r, const double* p, const double* w, double alpha, int64_t n,
                           cudaStream_t s);
cudaError_t launch_cg_dir(double* p, const double* r, double beta, int64_t n, cudaStream_t s);
cudaError_t launch_unit(double* v, int64_t n, cudaStream_t s);
cudaError_t operator_set_smem_limits();
cudaError_t krylov_set_smem_limits();
cudaError_t poles_set_smem_limits();
size_t poles_smem_bytes(int mp, int p);
cudaError_t launch_init_S(const double* R, int p, int npoles, double* S, cudaStream_t s,
                          const double* R_alt = nullptr, const int* use_alt = nullptr);
cudaError_t launch_axpby(double a, const double* X, int64_t ldx, double b, const double* Y,
                         int64_t ldy, double* out, int64_t ldo, int64_t n, int p,
                         cudaStream_t s);
cudaError_t launch_copy(const double* X, int64_t ldx, double* Y, int64_t ldy, int64_t n, int p,
                        cudaStream_t s);
cudaError_t launch_zero(double* X, int64_t ldx, int64_t n, int p, cudaStream_t s);
}  // namespace expm

bool expm_internal_cf_table(int nu, std::vector<std::complex<double>>& tau,
                            std::vector<std::complex<double>>& omega, double& omega0,
                            double& sigma);
