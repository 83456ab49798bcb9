// rows_launch.cuh -- launchers of the row-per-thread kernels of one width (included after
// rows_impl.cuh inside the width's namespace; see rows_api.h).

// The first CGS pass of the mixed path by the row-chunk kernels (k_cgs_rows): used when the
// projection blocks per thread and the staged chunk fit.
constexpr int kCgsRowsKMax = 5;
constexpr size_t kCgsRowsSmemMax = 112 * 1024;

bool cgs_fit(int cols, int p) {
    if (p < 1 || p > RP || cols < 1) return false;
    return (cgs_nblk(cols, p) + NTR - 1) / NTR <= kCgsRowsKMax && cgs_rows_smem(cols, true, p) <= kCgsRowsSmemMax;
}

cudaError_t cgs(int upd, const double* V, int64_t ldv, int cols, double* W, int64_t ldw, int p, int64_t n,
                const double* h, double* part, int nblk, int gram, cudaStream_t s) {
    if (!cgs_fit(cols, p) || (upd && !h)) return cudaErrorInvalidValue;
    const int64_t rpb = rows_per_block(n, nblk);
    const int g = blocks_for(n, nblk);
    const int ng = gram ? p : 0;
    const size_t shm = cgs_rows_smem(cols, upd != 0, ng);
#define EXPM_CGS_K(KK)                                                                               \
    {                                                                                               \
        if (upd) k_cgs_rows<true, true, KK><<<g, NTR, shm, s>>>(V, ldv, cols, W, ldw, p, n, rpb, h, part, ng); \
        else if (ng) k_cgs_rows<false, true, KK><<<g, NTR, shm, s>>>(V, ldv, cols, W, ldw, p, n, rpb, h, part, ng); \
        else k_cgs_rows<false, false, KK><<<g, NTR, shm, s>>>(V, ldv, cols, W, ldw, p, n, rpb, h, part, 0);    \
    }
    const int k = (cgs_nblk(cols, p) + NTR - 1) / NTR;
    if (k <= 1) EXPM_CGS_K(1)
    else if (k <= 2) EXPM_CGS_K(2)
    else if (k <= 3) EXPM_CGS_K(3)
    else EXPM_CGS_K(5)
#undef EXPM_CGS_K
    return cudaGetLastError();
}

cudaError_t qr(double* W, int64_t ldw, int p, int64_t n, int nblk, double* G, double* part, unsigned* ctr, int mode,
               double* R, double* Rinv, const double* Rtot_in, double* Rtot_out, double* H, int ldH, int hrow,
               int hcol, double* normsq_out, int* flags, double* out, int64_t ldo, cudaStream_t s, const double* Vc,
               int64_t ldvc, int ccols, const double* h2, double* fin, int64_t ldfin) {
    if (p > RP) return cudaErrorInvalidValue;
    if (Vc && (mode != 0 || !h2 || ccols < 1 || ccols > kMaxMP)) return cudaErrorInvalidValue;
    const int64_t rpb = rows_per_block(n, nblk);
    const int gr = blocks_for(n, nblk);
    // an extra lead CTA (no rows) when the row CTAs are short; else CTA 0 leads
    const bool extra_lead = rpb <= 2 * NTR;
    const int g = gr + (extra_lead ? 1 : 0), lead_blk = extra_lead ? gr : 0;
    if (mode == 0 && Vc)
        k_qr_mixed_rows<3><<<g, NTR, 2 * sizeof(float) * (size_t)ccols * RP, s>>>(
            W, ldw, p, n, rpb, G, part, ctr, mode, R, Rinv, Rtot_in, Rtot_out, H, ldH, hrow, hcol, normsq_out,
            flags, out, ldo, Vc, ldvc, ccols, h2, lead_blk, fin, ldfin);
    else if (mode == 0)
        k_qr_mixed_rows<1><<<g, NTR, 0, s>>>(W, ldw, p, n, rpb, G, part, ctr, mode, R, Rinv, Rtot_in, Rtot_out, H,
                                             ldH, hrow, hcol, normsq_out, flags, out, ldo, nullptr, 0, 0, nullptr,
                                             lead_blk, nullptr, 0);
    else
        k_qr_mixed_rows<2><<<g, NTR, 0, s>>>(W, ldw, p, n, rpb, G, part, ctr, mode, R, Rinv, Rtot_in, Rtot_out, H,
                                             ldH, hrow, hcol, normsq_out, flags, out, ldo, nullptr, 0, 0, nullptr,
                                             lead_blk, nullptr, 0);
    return cudaGetLastError();
}

cudaError_t upd_gram(const double* V, int64_t ldv, int cols, double* W, int64_t ldw, int p, int64_t n,
                     const double* h, double* part, int nblk, double* G, unsigned* ctr, int upd32, cudaStream_t s) {
    const int64_t rpb = rows_per_block(n, nblk);
    const int g = blocks_for(n, nblk);
    const size_t shr = sizeof(double) * (size_t)cols * RP;
    if (upd32) k_update_gram_rows<true><<<g, NTR, shr, s>>>(V, ldv, cols, W, ldw, p, n, rpb, h, part, G, ctr);
    else k_update_gram_rows<false><<<g, NTR, shr, s>>>(V, ldv, cols, W, ldw, p, n, rpb, h, part, G, ctr);
    return cudaGetLastError();
}

cudaError_t trsm(double* W, int64_t ldw, int p, int64_t n, const double* Rinv, double* out, int64_t ldo,
                 double* part, int nblk, int gram, const int* extra, int tmode, cudaStream_t s) {
    const int64_t rpb = rows_per_block(n, nblk);
    const int g = blocks_for(n, nblk);
    k_trsm_rows<<<g, NTR, 0, s>>>(W, ldw, p, n, rpb, Rinv, out, ldo, part, gram, extra, tmode);
    return cudaGetLastError();
}

cudaError_t updz(double* V, int64_t ldv, int cols, int p, int64_t n, const double* Wc, double* Z, int64_t ldz,
                 int restart_copy, cudaStream_t s, int nblk, int df) {
    const int64_t rpb = rows_per_block(n, nblk);
    const int g = blocks_for(n, nblk);
    const size_t shr = sizeof(double) * (size_t)cols * RP;
    if (df) k_update_z_rows<true><<<g, NTR, shr, s>>>(V, ldv, cols, p, n, rpb, Wc, Z, ldz, restart_copy);
    else k_update_z_rows<false><<<g, NTR, shr, s>>>(V, ldv, cols, p, n, rpb, Wc, Z, ldz, restart_copy);
    return cudaGetLastError();
}

// Shared-memory opt-in of this width's kernels whose dynamic size can pass 48 KB: the
// device's per-block maximum minus the kernel's own static shared memory.
template <class KF>
static cudaError_t set_max_dynamic_rows(KF kernel, int optin) {
    cudaFuncAttributes fa;
    cudaError_t e = cudaFuncGetAttributes(&fa, kernel);
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, optin - (int)fa.sharedSizeBytes);
}

cudaError_t set_smem(int optin) {
    cudaError_t e = cudaSuccess;
#define EXPM_SET(K) \
    if (e == cudaSuccess) e = set_max_dynamic_rows(K, optin)
    EXPM_SET(k_update_gram_rows<false>);
    EXPM_SET(k_update_gram_rows<true>);
    EXPM_SET(k_update_z_rows<false>);
    EXPM_SET(k_update_z_rows<true>);
    EXPM_SET((k_cgs_rows<true, true, 1>)); EXPM_SET((k_cgs_rows<true, true, 2>));
    EXPM_SET((k_cgs_rows<true, true, 3>)); EXPM_SET((k_cgs_rows<true, true, 5>));
    EXPM_SET((k_cgs_rows<false, true, 1>)); EXPM_SET((k_cgs_rows<false, true, 2>));
    EXPM_SET((k_cgs_rows<false, true, 3>)); EXPM_SET((k_cgs_rows<false, true, 5>));
    EXPM_SET((k_cgs_rows<false, false, 1>)); EXPM_SET((k_cgs_rows<false, false, 2>));
    EXPM_SET((k_cgs_rows<false, false, 3>)); EXPM_SET((k_cgs_rows<false, false, 5>));
    EXPM_SET(k_qr_mixed_rows<3>);
#undef EXPM_SET
    return e;
}
