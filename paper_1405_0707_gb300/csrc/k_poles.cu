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
// pivoting only looks at rows j..j+p of column j.  The matrix lives in shared memory when
// (mp)^2 + mp p complex numbers fit, else in a global workspace (L2-resident).
#include "internal.h"

namespace expm {
namespace {

struct cplx {
    double re, im;
};
__device__ inline cplx cmul(cplx a, cplx b) { return {a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re}; }
__device__ inline cplx csub(cplx a, cplx b) { return {a.re - b.re, a.im - b.im}; }
__device__ inline cplx cdiv(cplx a, cplx b) {
    const double s = fabs(b.re) + fabs(b.im);
    const double br = b.re / s, bi = b.im / s, ar = a.re / s, ai = a.im / s;
    const double d = br * br + bi * bi;
    return {(ar * br + ai * bi) / d, (ai * br - ar * bi) / d};
}
__device__ inline double cabs2(cplx a) { return a.re * a.re + a.im * a.im; }
// x -= a * b with four fused multiply-adds
__device__ inline void cmsub(cplx& x, cplx a, cplx b) {
    x.re = fma(-a.re, b.re, fma(a.im, b.im, x.re));
    x.im = fma(-a.re, b.im, fma(-a.im, b.re, x.im));
}

constexpr size_t kSmemLimit = 200 * 1024;
constexpr int kPoleThreads = 32;    // one warp per pole: warp-synchronous, no block barriers

// One CTA (one warp) per pole.  Shared memory holds M (mp x mp complex), the right-hand
// sides / solution X (mp x p complex) and, when it fits, the real H~ ((mp+p) x mp), staged
// once with coalesced loads.  Outputs: the restart factor S_i, ||S_i||_F, and
// Y_i = 2 Re(omega_i Z_i) (mp x p real).  Since H~ is real,
// sum_i 2 Re(omega_i H~ Z_i) = H~ sum_i Y_i, so the product with H~ is done once for all
// poles by k_combine.
__global__ void __launch_bounds__(kPoleThreads) k_poles(const double* __restrict__ H, int ldH, int mp, int p,
                                                        const double* __restrict__ tau_re,
                                                        const double* __restrict__ tau_im,
                                                        const double* __restrict__ om_re,
                                                        const double* __restrict__ om_im,
                                                        double* __restrict__ S, double* __restrict__ work,
                                                        double* __restrict__ Y_slots, double* res,
                                                        int* flags, int use_smem, int h_in_smem, int alg,
                                                        double* __restrict__ Zout) {
    extern __shared__ double sm[];
    __shared__ cplx f[kMaxP + 1];
    __shared__ int piv_s;
    __shared__ double red[kPoleThreads];
    const int i = blockIdx.x, tid = threadIdx.x, nt = blockDim.x;
    const cplx tau{tau_re[i], tau_im[i]};
    const cplx om{om_re[i], om_im[i]};
    const size_t per = (size_t)mp * mp + (size_t)mp * p;
    cplx* M = use_smem ? reinterpret_cast<cplx*>(sm) : reinterpret_cast<cplx*>(work) + (size_t)i * per;
    cplx* X = M + (size_t)mp * mp;
    cplx* Si = reinterpret_cast<cplx*>(S) + (size_t)i * p * p;
    const int rows = mp + p;
    // H~ (rows x mp, column-major, ld = rows) in shared memory after M and X when it fits
    double* Hs = reinterpret_cast<double*>(sm) + (use_smem ? 2 * per : 0);
    const double* Hr = h_in_smem ? Hs : H;
    const int ldr = h_in_smem ? rows : ldH;
    if (h_in_smem)
        for (int e = tid; e < rows * mp; e += nt) Hs[e] = H[(int64_t)(e / rows) * ldH + (e % rows)];
    __syncwarp();
    // Algorithm 2: M = I - tau H_m (eq. (3236)); Algorithm 1: M = H_m - tau I (eq. (3.3));
    // row-major.  X = E_1 S_i.
    for (int e = tid; e < mp * mp; e += nt) {
        const int r = e / mp, c = e % mp;
        const double h = Hr[(int64_t)c * ldr + r];
        const double d = (r == c ? 1.0 : 0.0);
        M[e] = (alg == 2) ? cplx{d - tau.re * h, -tau.im * h} : cplx{h - d * tau.re, -d * tau.im};
    }
    for (int e = tid; e < mp * p; e += nt) {
        const int r = e / p, c = e % p;
        X[e] = (r < p) ? Si[r * p + c] : cplx{0.0, 0.0};
    }
    __syncwarp();
    // elimination with partial pivoting inside the band (rows j..j+p of column j)
    for (int j = 0; j < mp; ++j) {
        const int jmax = min(j + p, mp - 1);
        // pivot: warp arg-max of |M[r][j]|^2 over r = j..jmax (ties -> smallest r)
        {
            double best = -1.0;
            int piv = j;
            for (int r = j + tid; r <= jmax; r += 32) {
                const double v = cabs2(M[(size_t)r * mp + j]);
                if (v > best) { best = v; piv = r; }
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                const double ob = __shfl_xor_sync(0xffffffffu, best, o);
                const int op = __shfl_xor_sync(0xffffffffu, piv, o);
                if (ob > best || (ob == best && op < piv)) { best = ob; piv = op; }
            }
            if (tid == 0) {
                if (!(best > 0.0)) atomicOr(&flags[0], 2);
                piv_s = piv;
            }
        }
        __syncwarp();
        const int piv = piv_s;
        if (piv != j) {
            for (int k = j + tid; k < mp; k += nt) {
                const cplx a = M[(size_t)j * mp + k];
                M[(size_t)j * mp + k] = M[(size_t)piv * mp + k];
                M[(size_t)piv * mp + k] = a;
            }
            for (int c = tid; c < p; c += nt) {
                const cplx a = X[(size_t)j * p + c];
                X[(size_t)j * p + c] = X[(size_t)piv * p + c];
                X[(size_t)piv * p + c] = a;
            }
            __syncwarp();
        }
        const int nr = jmax - j;
        if (tid < nr) f[tid] = cdiv(M[(size_t)(j + 1 + tid) * mp + j], M[(size_t)j * mp + j]);
        __syncwarp();
        const int ncM = mp - j - 1, w = ncM + p;
        for (int rr = 0; rr < nr; ++rr) {
            const int r = j + 1 + rr;
            const cplx fr = f[rr];
            for (int k = tid; k < w; k += nt) {
                if (k < ncM) {
                    const int col = j + 1 + k;
                    cmsub(M[(size_t)r * mp + col], fr, M[(size_t)j * mp + col]);
                } else {
                    const int c = k - ncM;
                    cmsub(X[(size_t)r * p + c], fr, X[(size_t)j * p + c]);
                }
            }
        }
        __syncwarp();
    }
    // back substitution on the upper triangle; thread -> (row offset, column) fixed
    const int bc = tid % p, br0 = tid / p, brs = nt / p;
    for (int j = mp - 1; j >= 0; --j) {
        if (tid < p) X[(size_t)j * p + tid] = cdiv(X[(size_t)j * p + tid], M[(size_t)j * mp + j]);
        __syncwarp();
        if (br0 < brs) {
            const cplx xj = X[(size_t)j * p + bc];
            for (int r = br0; r < j; r += brs) cmsub(X[(size_t)r * p + bc], M[(size_t)r * mp + j], xj);
        }
        __syncwarp();
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
    __syncwarp();
    for (int st = nt / 2; st > 0; st >>= 1) {
        if (tid < st) red[tid] += red[tid + st];
        __syncwarp();
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
                           const double* __restrict__ Y_slots, double* __restrict__ Wc, int alg) {
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
            for (int k = max(0, r - p); k < mp; ++k) s = fma(H[(int64_t)k * ldH + r], Ys[c * mp + k], s);
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
                                 const double* __restrict__ Zs, double* __restrict__ C, int alg) {
    const int rows = mp + p, w = 2 * npoles * p;
    const cplx* Z = reinterpret_cast<const cplx*>(Zs);
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < rows * npoles * p; e += gridDim.x * blockDim.x) {
        const int a = e % rows, ic = e / rows, i = ic / p, c = ic % p;
        const cplx* Zi = Z + (size_t)i * mp * p;
        cplx s{0.0, 0.0};
        if (alg == 2) {
            for (int k = max(0, a - p); k < mp; ++k) {
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
                                  double* C, int alg, cudaStream_t s) {
    const int tot = (mp + p) * npoles * p;
    k_certify_coeffs<<<(tot + 255) / 256, 256, 0, s>>>(H, ldH, mp, p, npoles, Zs, C, alg);
    return cudaGetLastError();
}

size_t poles_smem_bytes(int mp, int p) {
    const size_t b = ((size_t)mp * mp + (size_t)mp * p) * sizeof(cplx);
    return b <= kSmemLimit ? b : 0;
}

static size_t poles_h_bytes(int mp, int p) { return (size_t)(mp + p) * mp * sizeof(double); }

cudaError_t launch_poles(const double* H, int ldH, int mp, int p, int npoles,
                         const double* tau_re, const double* tau_im, const double* om_re,
                         const double* om_im, double* S, double* work, double* Y_slots,
                         double* res, int* flags, int alg, cudaStream_t s, double* Zout) {
    size_t shm = poles_smem_bytes(mp, p);
    int h_in = 0;
    if (shm > 0 && shm + poles_h_bytes(mp, p) <= kSmemLimit) {
        shm += poles_h_bytes(mp, p);
        h_in = 1;
    }
    k_poles<<<npoles, kPoleThreads, shm, s>>>(H, ldH, mp, p, tau_re, tau_im, om_re, om_im, S, work,
                                              Y_slots, res, flags, poles_smem_bytes(mp, p) > 0 ? 1 : 0,
                                              h_in, alg, Zout);
    return cudaGetLastError();
}

cudaError_t launch_combine2(const double* H, int ldH, int mp, int p, int npoles,
                            const double* Y_slots, double* Wc, int alg, cudaStream_t s) {
    const int nout = (mp + p) * p;
    const int blocks = (nout + 255) / 256;
    k_combine2<<<blocks, 256, sizeof(double) * (size_t)mp * p, s>>>(H, ldH, mp, p, npoles, Y_slots, Wc, alg);
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
