// rows_api.h -- the row-per-thread kernels, compiled once per row width RP in its own
// translation unit (k_rows4.cu .. k_rows16.cu, built in parallel): the launchers each width
// exports.  A block of p columns uses the smallest width RP >= p (4, 8, 12 or 16), so the
// per-row arithmetic carries at most three padded columns.  Widths above 8 run 128-thread
// CTAs (twice the registers per thread).
#pragma once
#include "internal.h"

namespace expm {

#define EXPM_ROWS_API(NS, RPV, NTRV)                                                                          \
    namespace NS {                                                                                            \
    constexpr int RP = RPV;                                                                                   \
    constexpr int NTR = NTRV;                                                                                 \
    bool cgs_fit(int cols, int p);                                                                            \
    cudaError_t cgs(int upd, const double* V, int64_t ldv, int cols, double* W, int64_t ldw, int p, int64_t n, \
                    const double* h, double* part, int nblk, int gram, cudaStream_t s);                       \
    cudaError_t qr(double* W, int64_t ldw, int p, int64_t n, int nblk, double* G, double* part, unsigned* ctr,  \
                   int mode, double* R, double* Rinv, const double* Rtot_in, double* Rtot_out, double* H,     \
                   int ldH, int hrow, int hcol, double* normsq_out, int* flags, double* out, int64_t ldo,      \
                   cudaStream_t s, const double* Vc, int64_t ldvc, int ccols, const double* h2, double* fin,   \
                   int64_t ldfin);                                                                            \
    cudaError_t upd_gram(const double* V, int64_t ldv, int cols, double* W, int64_t ldw, int p, int64_t n,     \
                         const double* h, double* part, int nblk, double* G, unsigned* ctr, int upd32,          \
                         cudaStream_t s);                                                                     \
    cudaError_t trsm(double* W, int64_t ldw, int p, int64_t n, const double* Rinv, double* out, int64_t ldo,   \
                     double* part, int nblk, int gram, const int* extra, int tmode, cudaStream_t s);           \
    cudaError_t updz(double* V, int64_t ldv, int cols, int p, int64_t n, const double* Wc, double* Z,          \
                     int64_t ldz, int restart_copy, cudaStream_t s, int nblk, int df);                        \
    cudaError_t set_smem(int optin);                                                                          \
    }

EXPM_ROWS_API(rows4, 4, 256)
EXPM_ROWS_API(rows8, 8, 256)
EXPM_ROWS_API(rows12, 12, 128)
EXPM_ROWS_API(rows16, 16, 128)
#undef EXPM_ROWS_API

// the launcher of width >= p (p <= 16): rows_call(p, f(args)) calls NS::f(args)
#define EXPM_ROWS_CALL(p, CALL) \
    ((p) <= 4 ? rows4::CALL : (p) <= 8 ? rows8::CALL : (p) <= 12 ? rows12::CALL : rows16::CALL)

}  // namespace expm
