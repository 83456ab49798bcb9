// k_poles.cu -- the projected shifted systems, one CTA per pole.
//
// For each pole tau_i (Im > 0) in one launch, Algorithm 2:
//   (I - tau_i H_m) Z_i = E_1 S_i                              eq. (3236)
//   S_i <- tau_i H_{m+1,m} E_m^T Z_i,  ||R_i||_F = ||S_i||_F     eq. (49) and the residual
//                                                             formula above it (collinear
//                                                             with V_{m+1}: restart factor)
//   Wc_i = 2 Re(omega_i H~_m Z_i)   ((m+1)p x p, real)          eq. (4.5): X_i - X_i^0 =
//                                                             (tA)^{-1} V_m Z_i = V_{m+1} H~_m Z_i
// Algorithm 1 (alg = 1): (H_m - tau_i I) Z_i = E_1 S_i (eq. (3.3)), S_i <- -H_{m+1,m} E_m^T Z_i
// (eq. (35)), Wc_i = 2 Re(omega_i Z_i) (X_i - X_i^0 = V_m Z_i).
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

constexpr size_t kSmemLimit = 200 * 1024;

__global__ void __launch_bounds__(256) k_poles(const double* __restrict__ H, int ldH, int mp, int p,
                                               const double* __restrict__ tau_re,
                                               const double* __restrict__ tau_im,
                                               const double* __restrict__ om_re,
                                               const double* __restrict__ om_im,
                                               double* __restrict__ S, double* __restrict__ work,
                                               double* __restrict__ Wc_slots, double* res,
                                               int* flags, int use_smem, int alg) {
    extern __shared__ double sm[];
    __shared__ cplx f[kMaxP + 1];
    __shared__ int piv_s;
    __shared__ double red[256];
    const int i = blockIdx.x, tid = threadIdx.x, nt = blockDim.x;
    const cplx tau{tau_re[i], tau_im[i]};
    const cplx om{om_re[i], om_im[i]};
    const size_t per = (size_t)mp * mp + (size_t)mp * p;
    cplx* M = use_smem ? reinterpret_cast<cplx*>(sm) : reinterpret_cast<cplx*>(work) + (size_t)i * per;
    cplx* X = M + (size_t)mp * mp;
    cplx* Si = reinterpret_cast<cplx*>(S) + (size_t)i * p * p;
    // Algorithm 2: M = I - tau H_m (eq. (3236)); Algorithm 1: M = H_m - tau I (eq. (3.3));
    // row-major.  X = E_1 S_i.
    for (int e = tid; e < mp * mp; e += nt) {
        const int r = e / mp, c = e % mp;
        const double h = H[(int64_t)c * ldH + r];
        const double d = (r == c ? 1.0 : 0.0);
        M[e] = (alg == 2) ? cplx{d - tau.re * h, -tau.im * h} : cplx{h - d * tau.re, -d * tau.im};
    }
    for (int e = tid; e < mp * p; e += nt) {
        const int r = e / p, c = e % p;
        X[e] = (r < p) ? Si[r * p + c] : cplx{0.0, 0.0};
    }
    __syncthreads();
    // elimination with partial pivoting inside the band
    for (int j = 0; j < mp; ++j) {
        const int jmax = min(j + p, mp - 1);
        if (tid == 0) {
            int piv = j;
            double best = cabs2(M[(size_t)j * mp + j]);
            for (int r = j + 1; r <= jmax; ++r) {
                const double v = cabs2(M[(size_t)r * mp + j]);
                if (v > best) { best = v; piv = r; }
            }
            if (!(best > 0.0)) atomicOr(&flags[0], 2);
            piv_s = piv;
        }
        __syncthreads();
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
            __syncthreads();
        }
        const int nr = jmax - j;
        if (tid < nr) f[tid] = cdiv(M[(size_t)(j + 1 + tid) * mp + j], M[(size_t)j * mp + j]);
        __syncthreads();
        const int ncM = mp - j - 1, w = ncM + p;
        for (int e = tid; e < nr * w; e += nt) {
            const int rr = e / w, k = e % w;
            const int r = j + 1 + rr;
            if (k < ncM) {
                const int col = j + 1 + k;
                M[(size_t)r * mp + col] = csub(M[(size_t)r * mp + col], cmul(f[rr], M[(size_t)j * mp + col]));
            } else {
                const int c = k - ncM;
                X[(size_t)r * p + c] = csub(X[(size_t)r * p + c], cmul(f[rr], X[(size_t)j * p + c]));
            }
        }
        __syncthreads();
    }
    // back substitution on the upper triangle
    for (int j = mp - 1; j >= 0; --j) {
        if (tid < p) X[(size_t)j * p + tid] = cdiv(X[(size_t)j * p + tid], M[(size_t)j * mp + j]);
        __syncthreads();
        for (int e = tid; e < j * p; e += nt) {
            const int r = e / p, c = e % p;
            X[(size_t)r * p + c] = csub(X[(size_t)r * p + c], cmul(M[(size_t)r * mp + j], X[(size_t)j * p + c]));
        }
        __syncthreads();
    }
    // S_i <- tau H_{m+1,m} E_m^T Z_i and its Frobenius norm
    double ss = 0.0;
    for (int e = tid; e < p * p; e += nt) {
        const int a = e / p, c = e % p;
        cplx s{0.0, 0.0};
        for (int b = 0; b < p; ++b) {
            const double h = H[(int64_t)(mp - p + b) * ldH + mp + a];
            const cplx x = X[(size_t)(mp - p + b) * p + c];
            s.re += h * x.re;
            s.im += h * x.im;
        }
        // Algorithm 2: tau H_{m+1,m} E_m^T Z_i (eq. (49)); Algorithm 1: -H_{m+1,m} E_m^T Z_i (eq. (35))
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
    // Algorithm 2: Wc_i = 2 Re(omega_i H~_m Z_i) (H~ row r has non-zeros in columns >= r - p);
    // Algorithm 1: Wc_i = 2 Re(omega_i Z_i) on the first mp rows, 0 on the last p.
    const int rows = mp + p;
    double* Wi = Wc_slots + (size_t)i * rows * p;
    for (int e = tid; e < rows * p; e += nt) {
        const int r = e / p, c = e % p;
        cplx s{0.0, 0.0};
        if (alg == 2) {
            for (int k = max(0, r - p); k < mp; ++k) {
                const double h = H[(int64_t)k * ldH + r];
                const cplx x = X[(size_t)k * p + c];
                s.re += h * x.re;
                s.im += h * x.im;
            }
        } else if (r < mp) {
            s = X[(size_t)r * p + c];
        }
        Wi[e] = 2.0 * (om.re * s.re - om.im * s.im);
    }
}

}  // namespace

size_t poles_smem_bytes(int mp, int p) {
    const size_t b = ((size_t)mp * mp + (size_t)mp * p) * sizeof(cplx);
    return b <= kSmemLimit ? b : 0;
}

cudaError_t launch_poles(const double* H, int ldH, int mp, int p, int npoles,
                         const double* tau_re, const double* tau_im, const double* om_re,
                         const double* om_im, double* S, double* work, double* Wc_slots,
                         double* res, int* flags, int alg, cudaStream_t s) {
    const size_t shm = poles_smem_bytes(mp, p);
    k_poles<<<npoles, 256, shm, s>>>(H, ldH, mp, p, tau_re, tau_im, om_re, om_im, S, work,
                                     Wc_slots, res, flags, shm > 0 ? 1 : 0, alg);
    return cudaGetLastError();
}

cudaError_t poles_set_smem_limits() {
    return cudaFuncSetAttribute(k_poles, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemLimit);
}

}  // namespace expm
