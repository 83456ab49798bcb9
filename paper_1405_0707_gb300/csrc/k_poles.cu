// k_poles.cu -- the projected shifted systems, one CTA per pole.
//
// For each pole tau_i (Im > 0) in one launch, Algorithm 2:
//   (I - tau_i H_m) Z_i = E_1 S_i                              eq. (3236)
//   S_i <- tau_i H_{m+1,m} E_m^T Z_i,  ||R_i||_F = ||S_i||_F     eq. (49) and the residual
//                                                             formula above it (collinear
//                                                             with V_{m+1}: restart factor)
//   Wc = sum_i 2 Re(omega_i H~_m Z_i) = H~_m sum_i 2 Re(omega_i Z_i)  (H~ real)
//                                          eq. (4.5): X_i - X_i^0 = (tA)^{-1} V_m Z_i = V_{m+1} H~_m Z_i
// Algorithm 1 (alg = 1): (H_m - tau_i I) Z_i = E_1 S_i (eq. (3.3)), S_i <- -H_{m+1,m} E_m^T Z_i
// (eq. (35)), Wc = [sum_i 2 Re(omega_i Z_i); 0] (X_i - X_i^0 = V_m Z_i).
// H_m is band upper Hessenberg with p sub-diagonals, so Gaussian elimination with partial
// pivoting only looks at rows j..j+p of column j (blocked by p x p blocks, see k_poles).
// After a deflated restart that keeps kk Ritz vectors (a multiple of p), the leading kk
// columns are dense down to row kk+p-1 (the projection of H~ onto the kept vectors) and the
// right-hand side E S_i sits at rows kk..kk+p-1; the elimination of those columns then looks
// at rows j..kk+p-1.  The
// matrix lives in shared memory when (mp)^2 + mp p complex numbers fit, else in a global
// workspace (L2-resident).
#include "internal.h"

namespace expm {
namespace {

struct cplx {
    double re, im;
};
__device__ inline cplx cmul(cplx a, cplx b) { return {a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re}; }
__device__ inline double cabs2(cplx a) { return a.re * a.re + a.im * a.im; }
// x -= a * b with four fused multiply-adds
__device__ inline void cmsub(cplx& x, cplx a, cplx b) {
    x.re = fma(-a.re, b.re, fma(a.im, b.im, x.re));
    x.im = fma(-a.re, b.im, fma(-a.im, b.re, x.im));
}

constexpr size_t kSmemLimit = 200 * 1024;
constexpr int kPoleThreads = 512;   // sixteen warps per pole: four per scheduler to cover FP64 latency

// One CTA (sixteen warps) per pole.  Shared memory holds M (mp x mp complex, row-major), the
// right-hand sides / solution X (mp x p complex), the inverses of U's diagonal blocks
// (mp x p complex) and, when it fits, the real H~ ((mp+p) x mp), staged once with coalesced
// loads.  Outputs: the restart factor S_i, ||S_i||_F and Y_i = 2 Re(omega_i Z_i) (mp x p
// real).  Since H~ is real, sum_i 2 Re(omega_i H~ Z_i) = H~ sum_i Y_i, so the product with H~
// is done once for all poles by k_combine2.
//
// M is block upper Hessenberg with p x p blocks (H_m is band Hessenberg with p sub-diagonals),
// so Gaussian elimination with partial pivoting is blocked by block columns J:
//   panel   (2p x p block [M_JJ; M_J+1,J], column by column, all threads): pivot searched
//           among the panel rows only (the band) on FP32 magnitudes, full rows swapped, one
//           reciprocal per pivot, multipliers stored in place, the panel's own columns updated;
//   update  U_J,c = L_JJ^{-1} M_J,c (one column per thread), then M_J+1,c -= L_J+1,J U_J,c
//           (one (row, column) pair per thread) for every later column c of M and of X;
// then the inverses of the diagonal blocks U_JJ (one block column per thread, all blocks at
// once) and the blocked back substitution X_J = U_JJ^{-1} X_J, X_0..J-1 -= U_0..J-1,J X_J as
// parallel products.  FP64 throughout; the FP64 pipe of one SM is the bound, so the layout
// keeps every lane of every warp busy wherever the work allows.
__global__ void __launch_bounds__(kPoleThreads) k_poles(const double* __restrict__ H, int ldH, int mp, int p,
                                                        const double* __restrict__ tau_re,
                                                        const double* __restrict__ tau_im,
                                                        const double* __restrict__ om_re,
                                                        const double* __restrict__ om_im,
                                                        double* __restrict__ S, double* __restrict__ work,
                                                        double* __restrict__ Y_slots, double* res,
                                                        int* flags, int use_smem, int h_in_smem, int alg,
                                                        double* __restrict__ Zout, int kk) {
    extern __shared__ double sm[];
    __shared__ cplx rdiag[kMaxMP];
    __shared__ double red[kPoleThreads];
    __shared__ int piv_s;
    const int i = blockIdx.x, tid = threadIdx.x, nt = blockDim.x;
    const int lane = tid & 31, warp = tid >> 5;
    const cplx tau{tau_re[i], tau_im[i]};
    const cplx om{om_re[i], om_im[i]};
    const size_t per = (size_t)mp * mp + 2 * (size_t)mp * p;
    cplx* M = use_smem ? reinterpret_cast<cplx*>(sm) : reinterpret_cast<cplx*>(work) + (size_t)i * per;
    cplx* X = M + (size_t)mp * mp;
    cplx* Ui = X + (size_t)mp * p;          // Ui[J p + a][b] = (U_JJ^{-1})[a][b]
    cplx* Si = reinterpret_cast<cplx*>(S) + (size_t)i * p * p;
    const int rows = mp + p;
    // H~ (rows x mp, column-major, ld = rows) in shared memory after M, X and Ui when it fits
    double* Hs = reinterpret_cast<double*>(sm) + (use_smem ? 2 * per : 0);
    const double* Hr = h_in_smem ? Hs : H;
    const int ldr = h_in_smem ? rows : ldH;
    if (h_in_smem)
        for (int c = 0; c < mp; ++c)
            for (int r = tid; r < rows; r += nt) Hs[(int64_t)c * rows + r] = H[(int64_t)c * ldH + r];
    __syncthreads();
    // Algorithm 2: M = I - tau H_m (eq. (3236)); Algorithm 1: M = H_m - tau I (eq. (3.3)).
    // X = E_1 S_i.
    for (int r = 0; r < mp; ++r)
        for (int c = tid; c < mp; c += nt) {
            const double h = Hr[(int64_t)c * ldr + r];
            const double d = (r == c ? 1.0 : 0.0);
            M[(size_t)r * mp + c] = (alg == 2) ? cplx{d - tau.re * h, -tau.im * h} : cplx{h - d * tau.re, -d * tau.im};
        }
    // after a deflated restart the residual coordinates sit at rows kk .. kk+p-1
    for (int e = tid; e < mp * p; e += nt) {
        const int r = e / p, c = e % p;
        X[e] = (r >= kk && r < kk + p) ? Si[(r - kk) * p + c] : cplx{0.0, 0.0};
    }
    __syncthreads();
    const int nbc = mp / p;
    for (int J = 0; J < nbc; ++J) {
        const int r0 = J * p;
        // panel rows r0 .. rend-1: the band (one block below the diagonal block); the kk
        // deflated columns of a deflated restart reach down to the block row of the old
        // V_{m+1} (rows kk .. kk+p-1: H_{m+1,m} E_m^T P_k)
        const int rend = min(mp, max(r0 + 2 * p, r0 < kk ? kk + p : 0));
        for (int jj = 0; jj < p; ++jj) {
            const int c = r0 + jj;
            if (warp == 0) {
                // pivot: arg-max of |M[r][c]|^2 in FP32 over the panel rows r >= c
                float best = -1.f;
                int piv = c;
                for (int r = c + lane; r < rend; r += 32) {
                    const cplx v = M[(size_t)r * mp + c];
                    const float fr = (float)v.re, fi = (float)v.im;
                    const float m = fmaf(fr, fr, fi * fi);
                    if (m > best) { best = m; piv = r; }
                }
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) {
                    const float ob = __shfl_xor_sync(0xffffffffu, best, o);
                    const int op = __shfl_xor_sync(0xffffffffu, piv, o);
                    if (ob > best || (ob == best && op < piv)) { best = ob; piv = op; }
                }
                if (lane == 0) piv_s = piv;
            }
            __syncthreads();
            const int piv = piv_s;
            if (piv != c) {   // swap the full rows (M from column r0 on, and X)
                for (int k = r0 + tid; k < mp; k += nt) {
                    const cplx a = M[(size_t)c * mp + k];
                    M[(size_t)c * mp + k] = M[(size_t)piv * mp + k];
                    M[(size_t)piv * mp + k] = a;
                }
                for (int k = tid; k < p; k += nt) {
                    const cplx a = X[(size_t)c * p + k];
                    X[(size_t)c * p + k] = X[(size_t)piv * p + k];
                    X[(size_t)piv * p + k] = a;
                }
                __syncthreads();
            }
            if (tid == 0) {
                const cplx d = M[(size_t)c * mp + c];
                const double n2 = d.re * d.re + d.im * d.im;
                if (!(n2 > 0.0)) atomicOr(&flags[0], 2);
                const double x = 1.0 / n2;
                rdiag[c] = cplx{d.re * x, -d.im * x};
            }
            __syncthreads();
            const cplx inv = rdiag[c];
            const int nr = rend - c - 1, wc = r0 + p - c - 1;
            for (int r = c + 1 + tid; r < rend; r += nt) M[(size_t)r * mp + c] = cmul(M[(size_t)r * mp + c], inv);
            __syncthreads();
            for (int e = tid; e < nr * wc; e += nt) {
                const int r = c + 1 + e / wc, k = c + 1 + e % wc;
                cmsub(M[(size_t)r * mp + k], M[(size_t)r * mp + c], M[(size_t)c * mp + k]);
            }
            __syncthreads();
        }
        // trailing update: columns of M right of the panel, then the columns of X
        const int ncm = mp - r0 - p, ncol = ncm + p;
        for (int q = tid; q < ncol; q += nt) {      // U_J,c = L_JJ^{-1} M_J,c (unit lower)
            cplx* col;
            size_t ld;
            if (q < ncm) { col = M + r0 + p + q; ld = mp; }
            else { col = X + (q - ncm); ld = p; }
            for (int a = 1; a < p; ++a) {
                cplx s = col[(size_t)(r0 + a) * ld];
                for (int k = 0; k < a; ++k) cmsub(s, M[(size_t)(r0 + a) * mp + r0 + k], col[(size_t)(r0 + k) * ld]);
                col[(size_t)(r0 + a) * ld] = s;
            }
        }
        __syncthreads();
        const int nbelow = rend - r0 - p;              // rows below the diagonal block
        if (nbelow > 0)
            for (int e = tid; e < nbelow * ncol; e += nt) {   // M_below,c -= L_below,J U_J,c
                const int a = e / ncol, q = e % ncol;
                cplx* col;
                size_t ld;
                if (q < ncm) { col = M + r0 + p + q; ld = mp; }
                else { col = X + (q - ncm); ld = p; }
                const int r = r0 + p + a;
                cplx s = col[(size_t)r * ld];
                for (int k = 0; k < p; ++k) cmsub(s, M[(size_t)r * mp + r0 + k], col[(size_t)(r0 + k) * ld]);
                col[(size_t)r * ld] = s;
            }
        __syncthreads();
    }
    // inverses of the diagonal blocks U_JJ (upper triangular), one block column per thread
    for (int e = tid; e < nbc * p; e += nt) {
        const int J = e / p, b = e % p, r0 = J * p;
        for (int a = p - 1; a >= 0; --a) {
            cplx s{a == b ? 1.0 : 0.0, 0.0};
            for (int k = a + 1; k <= b; ++k) cmsub(s, M[(size_t)(r0 + a) * mp + r0 + k], Ui[(size_t)(r0 + k) * p + b]);
            Ui[(size_t)(r0 + a) * p + b] = (a > b) ? cplx{0.0, 0.0} : cmul(s, rdiag[r0 + a]);
        }
    }
    __syncthreads();
    // blocked back substitution
    for (int J = nbc - 1; J >= 0; --J) {
        const int r0 = J * p;
        // X_J = U_JJ^{-1} X_J: outputs (a, c); the old X_J is read before any is written
        constexpr int kXo = (kMaxP * kMaxP + kPoleThreads - 1) / kPoleThreads;
        cplx xo[kXo];
        int cnt = 0;
        for (int e = tid; e < p * p; e += nt, ++cnt) {
            const int a = e / p, c = e % p;
            cplx s{0.0, 0.0};
            for (int k = a; k < p; ++k) {
                const cplx u = Ui[(size_t)(r0 + a) * p + k], x = X[(size_t)(r0 + k) * p + c];
                s.re = fma(u.re, x.re, fma(-u.im, x.im, s.re));
                s.im = fma(u.re, x.im, fma(u.im, x.re, s.im));
            }
            xo[cnt] = s;
        }
        __syncthreads();
        cnt = 0;
        for (int e = tid; e < p * p; e += nt, ++cnt) X[(size_t)(r0 + e / p) * p + e % p] = xo[cnt];
        __syncthreads();
        for (int e = tid; e < r0 * p; e += nt) {   // X_0..J-1 -= U_0..J-1,J X_J
            const int r = e / p, c = e % p;
            cplx s = X[(size_t)r * p + c];
            for (int k = 0; k < p; ++k) cmsub(s, M[(size_t)r * mp + r0 + k], X[(size_t)(r0 + k) * p + c]);
            X[(size_t)r * p + c] = s;
        }
        __syncthreads();
    }
    // S_i and its Frobenius norm.  Algorithm 2: tau H_{m+1,m} E_m^T Z_i (eq. (49));
    // Algorithm 1: -H_{m+1,m} E_m^T Z_i (eq. (35)).
    double ss = 0.0;
    for (int e = tid; e < p * p; e += nt) {
        const int a = e / p, c = e % p;
        cplx s{0.0, 0.0};
        for (int b = 0; b < p; ++b) {
            const double h = Hr[(int64_t)(mp - p + b) * ldr + mp + a];
            const cplx x = X[(size_t)(mp - p + b) * p + c];
            s.re += h * x.re;
            s.im += h * x.im;
        }
        const cplx snew = (alg == 2) ? cmul(tau, s) : cplx{-s.re, -s.im};
        Si[e] = snew;
        ss += cabs2(snew);
    }
    red[tid] = ss;
    __syncthreads();
    for (int st = nt / 2; st > 0; st >>= 1) {
        if (tid < st) red[tid] += red[tid + st];
        __syncthreads();
    }
    if (tid == 0) {
        res[i] = sqrt(red[0]);
        if (!isfinite(red[0])) atomicOr(&flags[0], 4);
    }
    if (Zout) {   // certify mode: Z_i itself (complex, row-major [r][c])
        cplx* Zi = reinterpret_cast<cplx*>(Zout) + (size_t)i * mp * p;
        for (int e = tid; e < mp * p; e += nt) Zi[e] = X[e];
    }
    // Y_i = 2 Re(omega_i Z_i), stored r fastest (Y[c * mp + r])
    double* Yi = Y_slots + (size_t)i * mp * p;
    for (int e = tid; e < mp * p; e += nt) {
        const int r = e % mp, c = e / mp;
        const cplx x = X[(size_t)r * p + c];
        Yi[e] = 2.0 * (om.re * x.re - om.im * x.im);
    }
}

// Wc = H~ sum_i Y_i (Algorithm 2) or [sum_i Y_i; 0] (Algorithm 1), (mp+p) x p, row-major
// [r][c] as k_update_z reads it.  One thread per output, r fastest (coalesced H~ columns).
__global__ void k_combine2(const double* __restrict__ H, int ldH, int mp, int p, int npoles,
                           const double* __restrict__ Y_slots, double* __restrict__ Wc, int alg, int kk) {
    extern __shared__ double Ys[];          // mp x p, summed over poles (fixed order)
    const int rows = mp + p;
    for (int e = threadIdx.x; e < mp * p; e += blockDim.x) {
        double s = 0.0;
        for (int i = 0; i < npoles; ++i) s += Y_slots[(size_t)i * mp * p + e];
        Ys[e] = s;
    }
    __syncthreads();
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < rows * p; e += gridDim.x * blockDim.x) {
        const int r = e % rows, c = e / rows;
        double s = 0.0;
        if (alg == 2) {
            // band rows start p columns left of the diagonal; the rows of a deflated restart's
            // leading block (r < kk + p) are dense from column 0
            for (int k = r < kk + p ? 0 : r - p; k < mp; ++k) s = fma(H[(int64_t)k * ldH + r], Ys[c * mp + k], s);
        } else if (r < mp) {
            s = Ys[c * mp + r];
        }
        Wc[r * p + c] = s;
    }
}

// Certify mode: C[a][i 2p + c] = Re(F_i)[a][c], C[a][i 2p + p + c] = Im(F_i)[a][c] with
// F_i = H~_m Z_i (Algorithm 2: X_i - X_i^0 = V_{m+1} H~_m Z_i) or F_i = [Z_i; 0] (Algorithm 1),
// so X += V_{m+1} C updates every pole's real and imaginary parts in one tall-skinny product.
__global__ void k_certify_coeffs(const double* __restrict__ H, int ldH, int mp, int p, int npoles,
                                 const double* __restrict__ Zs, double* __restrict__ C, int alg, int kk) {
    const int rows = mp + p, w = 2 * npoles * p;
    const cplx* Z = reinterpret_cast<const cplx*>(Zs);
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < rows * npoles * p; e += gridDim.x * blockDim.x) {
        const int a = e % rows, ic = e / rows, i = ic / p, c = ic % p;
        const cplx* Zi = Z + (size_t)i * mp * p;
        cplx s{0.0, 0.0};
        if (alg == 2) {
            for (int k = a < kk + p ? 0 : a - p; k < mp; ++k) {   // as in k_combine2
                const double h = H[(int64_t)k * ldH + a];
                s.re = fma(h, Zi[(size_t)k * p + c].re, s.re);
                s.im = fma(h, Zi[(size_t)k * p + c].im, s.im);
            }
        } else if (a < mp) {
            s = Zi[(size_t)a * p + c];
        }
        C[(size_t)a * w + 2 * i * p + c] = s.re;
        C[(size_t)a * w + 2 * i * p + p + c] = s.im;
    }
}

}  // namespace

cudaError_t launch_certify_coeffs(const double* H, int ldH, int mp, int p, int npoles, const double* Zs,
                                  double* C, int alg, cudaStream_t s, int kk) {
    const int tot = (mp + p) * npoles * p;
    k_certify_coeffs<<<(tot + 255) / 256, 256, 0, s>>>(H, ldH, mp, p, npoles, Zs, C, alg, kk);
    return cudaGetLastError();
}

size_t poles_smem_bytes(int mp, int p) {
    const size_t b = ((size_t)mp * mp + 2 * (size_t)mp * p) * sizeof(cplx);
    return b <= kSmemLimit ? b : 0;
}

static size_t poles_h_bytes(int mp, int p) { return (size_t)(mp + p) * mp * sizeof(double); }

cudaError_t launch_poles(const double* H, int ldH, int mp, int p, int npoles,
                         const double* tau_re, const double* tau_im, const double* om_re,
                         const double* om_im, double* S, double* work, double* Y_slots,
                         double* res, int* flags, int alg, cudaStream_t s, double* Zout, int kk) {
    size_t shm = poles_smem_bytes(mp, p);
    int h_in = 0;
    if (shm > 0 && shm + poles_h_bytes(mp, p) <= kSmemLimit) {
        shm += poles_h_bytes(mp, p);
        h_in = 1;
    }
    k_poles<<<npoles, kPoleThreads, shm, s>>>(H, ldH, mp, p, tau_re, tau_im, om_re, om_im, S, work,
                                              Y_slots, res, flags, poles_smem_bytes(mp, p) > 0 ? 1 : 0,
                                              h_in, alg, Zout, kk);
    return cudaGetLastError();
}

cudaError_t launch_combine2(const double* H, int ldH, int mp, int p, int npoles,
                            const double* Y_slots, double* Wc, int alg, cudaStream_t s, int kk) {
    const int nout = (mp + p) * p;
    const int blocks = (nout + 255) / 256;
    k_combine2<<<blocks, 256, sizeof(double) * (size_t)mp * p, s>>>(H, ldH, mp, p, npoles, Y_slots, Wc, alg, kk);
    return cudaGetLastError();
}

cudaError_t poles_set_smem_limits() {
    // kSmemLimit (200 KB) of dynamic memory plus the kernel's few KB of static memory stays
    // below the 227 KB per-block opt-in maximum
    cudaError_t e = cudaFuncSetAttribute(k_poles, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemLimit);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_combine2, cudaFuncAttributeMaxDynamicSharedMemorySize, 140 * 1024);
    return e;
}

}  // namespace expm
