// k_csr.cu -- general sparse operators (CSR): the product t A X for Algorithm 1's Krylov
// operator, and the inexact inverse for Algorithm 2 (Section 4.1: when a direct solver is out
// of reach, (tA)^{-1} may be applied by an inner iterative solve; Theorem 4.3 bounds the
// error that the inexactness costs).
//
// The inner solve is BiCGStab with the Jacobi preconditioner (right preconditioning, M =
// diag(A)) on every column of the block at once, each column with its own scalars.  The
// vector steps are kernels with a thread per row over all p columns, so the sparse products
// read each matrix row once for the whole block; each reduction writes one partial per CTA,
// column and dot, and a one-CTA scalar step adds them in a fixed order (deterministic) and
// updates the columns' alpha, omega, rho, beta.  A column whose relative residual has reached
// the tolerance (or whose recurrence broke down: a zero denominator) is frozen: its iterate
// and residual no longer change.
#include "internal.h"

namespace expm {
namespace {

constexpr int CT = 256;     // threads per CTA
constexpr int PMAX = 16;    // columns per block (p_max limit of the row kernels)
constexpr int NSC = 8;      // scalars per column: rho, rho_old, alpha, omega, rr, bb, beta, frozen
constexpr int SPG = 4;      // columns per thread in the sparse products

enum { S_RHO = 0, S_RHO0, S_ALPHA, S_OMEGA, S_RR, S_BB, S_BETA, S_FRZ };

// Y[:, c] = alpha A X[:, c] for every column: a thread per row reads the row's entries once and
// applies them to all p columns (the matrix is read once, not once per column)
template <int NC>
__device__ __forceinline__ void row_apply(const int64_t* __restrict__ rp, const int* __restrict__ ci,
                                          const double* __restrict__ va, const double* __restrict__ X, int64_t ldx,
                                          int p, int64_t r, double* acc) {
#pragma unroll
    for (int c = 0; c < NC; ++c) acc[c] = 0.0;
    const int64_t k1 = rp[r + 1];
    for (int64_t k = rp[r]; k < k1; ++k) {
        const double a = va[k];
        const double* xc = X + ci[k];
#pragma unroll
        for (int c = 0; c < NC; ++c)
            if (c < p) acc[c] = fma(a, xc[c * ldx], acc[c]);
    }
}

// thread per row and group of SPG columns (blockIdx.y): each row's entries are read once per
// group, from L2 after the first group (measured: one group of all 16 columns ran
// load-throttled at 0.24 ms on 96^3, p = 16; one column per CTA column re-read the matrix
// from DRAM 2.85 times)
__global__ void __launch_bounds__(CT) k_csr_spmm(const int64_t* __restrict__ rp, const int* __restrict__ ci,
                                                 const double* __restrict__ va, int64_t n, double alpha,
                                                 const double* __restrict__ X, int64_t ldx, double* __restrict__ Y,
                                                 int64_t ldy, int p) {
    const int c0 = blockIdx.y * SPG;
    const int pc = min(SPG, p - c0);
    X += c0 * ldx;
    Y += c0 * ldy;
    double acc[SPG];
    for (int64_t r = (int64_t)blockIdx.x * CT + threadIdx.x; r < n; r += (int64_t)gridDim.x * CT) {
        row_apply<SPG>(rp, ci, va, X, ldx, pc, r, acc);
#pragma unroll
        for (int c = 0; c < SPG; ++c)
            if (c < pc) Y[c * ldy + r] = alpha * acc[c];
    }
}

// The inner solver's vectors, column c at offset c * ld of each: x, r, rh (the shadow
// residual r^_0), q (search direction), qh = M^-1 q, v = A qh, s, sh = M^-1 s, u = A sh.
struct Bicg {
    const int64_t* rp;
    const int* ci;
    const double* va;
    const double* dinv;      // 1 / a_ii
    int64_t n, ld;
    int p, nb;
    double *x, *r, *rh, *q, *qh, *v, *s, *sh, *u;
    double* part;            // [nb][2][p]: the CTAs' partials of the phase's one or two dots
    double* sc;              // [p][NSC]: the columns' scalars
    double* norms;           // [2p]: rr and bb per column, for the host's stop test
    double eta2;             // squared relative tolerance
};

// The CTA's partials of up to two dot products for its SPG columns c0 .. c0 + SPG - 1: per-warp
// sums through shared memory, then thread (k, c) adds the warps' sums in a fixed order
// (deterministic).
__device__ __forceinline__ void cta_partials(const Bicg& g, int c0, const double* d1, const double* d2, int nd) {
    __shared__ double sh[CT / 32][2][SPG];
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    for (int k = 0; k < nd; ++k) {
        const double* d = k ? d2 : d1;
#pragma unroll
        for (int c = 0; c < SPG; ++c) {
            double v = d[c];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
            if (l == 0) sh[w][k][c] = v;
        }
    }
    __syncthreads();
    if (threadIdx.x < SPG * nd) {
        const int k = threadIdx.x / SPG, c = threadIdx.x - k * SPG;
        if (c0 + c < g.p) {
            double s = 0.0;
            for (int ww = 0; ww < CT / 32; ++ww) s += sh[ww][k][c];
            g.part[((size_t)blockIdx.x * 2 + k) * g.p + c0 + c] = s;
        }
    }
}

// the elementwise steps loop over columns (one column's rows at a time, coalesced) and leave
// each warp's sums in shared memory, indexed by column; cta_partials_sh then writes the
// CTA's partials in a fixed order
__device__ __forceinline__ void warp_put(double (*sh)[2][PMAX], int k, int c, double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5][k][c] = v;
}

__device__ __forceinline__ void cta_partials_sh(const Bicg& g, double (*sh)[2][PMAX], int nd) {
    __syncthreads();
    if (threadIdx.x < g.p * nd) {
        const int k = threadIdx.x / g.p, c = threadIdx.x - k * g.p;
        double s = 0.0;
        for (int ww = 0; ww < CT / 32; ++ww) s += sh[ww][k][c];
        g.part[((size_t)blockIdx.x * 2 + k) * g.p + c] = s;
    }
}

__device__ __forceinline__ double sum_part(const Bicg& g, int k, int c) {
    double s = 0.0;
    for (int b = 0; b < g.nb; ++b) s += g.part[((size_t)b * 2 + k) * g.p + c];
    return s;
}

// start: x = 0, r = rh = b, q = v = 0; partials (b, b)
__global__ void __launch_bounds__(CT) k_bicg_start(Bicg g, const double* __restrict__ B, int64_t ldb) {
    __shared__ double sh[CT / 32][2][PMAX];
    for (int c = 0; c < g.p; ++c) {
        double bb = 0.0;
        for (int64_t i = (int64_t)blockIdx.x * CT + threadIdx.x; i < g.n; i += (int64_t)gridDim.x * CT) {
            const double b = B[c * ldb + i];
            const int64_t o = c * g.ld + i;
            g.x[o] = 0.0;
            g.r[o] = b;
            g.rh[o] = b;
            g.q[o] = 0.0;
            g.v[o] = 0.0;
            bb = fma(b, b, bb);
        }
        warp_put(sh, 0, c, bb);
    }
    cta_partials_sh(g, sh, 1);
}

// The scalar steps (one CTA, a thread per column), after each reduction:
//   phase 0 (start): bb = rho = rr = (b, b); frozen iff b = 0
//   phase 1 (after v = A qh): alpha = rho / (rh, v)
//   phase 2 (after u = A sh): omega = (u, s) / (u, u)
//   phase 3 (after the update): rho_old = rho, rho = (rh, r), rr = (r, r),
//           beta = (rho / rho_old) (alpha / omega); frozen once rr <= eta^2 bb or a
//           denominator vanished (then the column's iterate stays as it is)
__global__ void k_bicg_scal(Bicg g, int phase) {
    const int c = threadIdx.x;
    if (c >= g.p) return;
    double* z = g.sc + c * NSC;
    if (phase == 0) {
        const double bb = sum_part(g, 0, c);
        z[S_BB] = bb;
        z[S_RHO] = bb;
        z[S_RR] = bb;
        z[S_FRZ] = bb > 0.0 ? 0.0 : 1.0;
    } else if (phase == 1) {
        const double d = sum_part(g, 0, c);
        if (d != 0.0) z[S_ALPHA] = z[S_RHO] / d;
        else z[S_FRZ] = 1.0;
    } else if (phase == 2) {
        const double us = sum_part(g, 0, c), uu = sum_part(g, 1, c);
        if (uu != 0.0 && us != 0.0) z[S_OMEGA] = us / uu;
        else z[S_FRZ] = 1.0;
    } else {
        const double rho = sum_part(g, 0, c), rr = sum_part(g, 1, c);
        if (z[S_FRZ] == 0.0) {
            z[S_RHO0] = z[S_RHO];
            z[S_RHO] = rho;
            z[S_RR] = rr;
            z[S_BETA] = (rho / z[S_RHO0]) * (z[S_ALPHA] / z[S_OMEGA]);
            if (!(rr > g.eta2 * z[S_BB]) || rho == 0.0) z[S_FRZ] = 1.0;
        }
    }
    g.norms[c] = z[S_RR];
    g.norms[g.p + c] = z[S_BB];
}

// q = r + beta (q - omega v) (iteration 0: q = r), qh = M^-1 q
__global__ void __launch_bounds__(CT) k_bicg_dir(Bicg g, int it) {
    for (int c = 0; c < g.p; ++c) {
        const double* z = g.sc + c * NSC;
        if (z[S_FRZ] != 0.0) continue;
        const double beta = z[S_BETA], omega = z[S_OMEGA];
        for (int64_t i = (int64_t)blockIdx.x * CT + threadIdx.x; i < g.n; i += (int64_t)gridDim.x * CT) {
            const int64_t o = c * g.ld + i;
            const double q = it > 0 ? fma(beta, fma(-omega, g.v[o], g.q[o]), g.r[o]) : g.r[o];
            g.q[o] = q;
            g.qh[o] = q * g.dinv[i];
        }
    }
}

// v = A qh, partials (rh, v); blockIdx.y: the group of SPG columns
__global__ void __launch_bounds__(CT) k_bicg_av(Bicg g) {
    const int c0 = blockIdx.y * SPG, pc = min(SPG, g.p - c0);
    double acc[SPG], d1[SPG];
#pragma unroll
    for (int c = 0; c < SPG; ++c) d1[c] = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * CT + threadIdx.x; i < g.n; i += (int64_t)gridDim.x * CT) {
        row_apply<SPG>(g.rp, g.ci, g.va, g.qh + c0 * g.ld, g.ld, pc, i, acc);
#pragma unroll
        for (int c = 0; c < SPG; ++c)
            if (c < pc) {
                const int64_t o = (c0 + c) * g.ld + i;
                g.v[o] = acc[c];
                d1[c] = fma(g.rh[o], acc[c], d1[c]);
            }
    }
    cta_partials(g, c0, d1, nullptr, 1);
}

// s = r - alpha v, sh = M^-1 s
__global__ void __launch_bounds__(CT) k_bicg_s(Bicg g) {
    for (int c = 0; c < g.p; ++c) {
        const double* z = g.sc + c * NSC;
        if (z[S_FRZ] != 0.0) continue;
        const double alpha = z[S_ALPHA];
        for (int64_t i = (int64_t)blockIdx.x * CT + threadIdx.x; i < g.n; i += (int64_t)gridDim.x * CT) {
            const int64_t o = c * g.ld + i;
            const double s = fma(-alpha, g.v[o], g.r[o]);
            g.s[o] = s;
            g.sh[o] = s * g.dinv[i];
        }
    }
}

// u = A sh, partials (u, s) and (u, u); blockIdx.y: the group of SPG columns
__global__ void __launch_bounds__(CT) k_bicg_au(Bicg g) {
    const int c0 = blockIdx.y * SPG, pc = min(SPG, g.p - c0);
    double acc[SPG], d2[SPG], d3[SPG];
#pragma unroll
    for (int c = 0; c < SPG; ++c) {
        d2[c] = 0.0;
        d3[c] = 0.0;
    }
    for (int64_t i = (int64_t)blockIdx.x * CT + threadIdx.x; i < g.n; i += (int64_t)gridDim.x * CT) {
        row_apply<SPG>(g.rp, g.ci, g.va, g.sh + c0 * g.ld, g.ld, pc, i, acc);
#pragma unroll
        for (int c = 0; c < SPG; ++c)
            if (c < pc) {
                const int64_t o = (c0 + c) * g.ld + i;
                g.u[o] = acc[c];
                d2[c] = fma(acc[c], g.s[o], d2[c]);
                d3[c] = fma(acc[c], acc[c], d3[c]);
            }
    }
    cta_partials(g, c0, d2, d3, 2);
}

// x += alpha qh + omega sh, r = s - omega u; partials (rh, r) and (r, r)
__global__ void __launch_bounds__(CT) k_bicg_x(Bicg g) {
    __shared__ double sh[CT / 32][2][PMAX];
    for (int c = 0; c < g.p; ++c) {
        const double* z = g.sc + c * NSC;
        const bool frz = z[S_FRZ] != 0.0;
        const double alpha = z[S_ALPHA], omega = z[S_OMEGA];
        double d4 = 0.0, d5 = 0.0;
        for (int64_t i = (int64_t)blockIdx.x * CT + threadIdx.x; i < g.n; i += (int64_t)gridDim.x * CT) {
            const int64_t o = c * g.ld + i;
            double r = g.r[o];
            if (!frz) {
                g.x[o] = fma(omega, g.sh[o], fma(alpha, g.qh[o], g.x[o]));
                r = fma(-omega, g.u[o], g.s[o]);
                g.r[o] = r;
            }
            d4 = fma(g.rh[o], r, d4);
            d5 = fma(r, r, d5);
        }
        warp_put(sh, 0, c, d4);
        warp_put(sh, 1, c, d5);
    }
    cta_partials_sh(g, sh, 2);
}

__global__ void __launch_bounds__(CT) k_csr_scale_out(const double* __restrict__ x, int64_t ldx, int64_t n,
                                                      double scale, double* __restrict__ W, int64_t ldw) {
    const int c = blockIdx.y;
    for (int64_t i = (int64_t)blockIdx.x * CT + threadIdx.x; i < n; i += (int64_t)gridDim.x * CT)
        W[c * ldw + i] = scale * x[c * ldx + i];
}

__global__ void k_csr_dinv(const int64_t* __restrict__ rp, const int* __restrict__ ci, const double* __restrict__ va,
                           int64_t n, double* __restrict__ dinv) {
    const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= n) return;
    double d = 0.0;
    for (int64_t k = rp[r]; k < rp[r + 1]; ++k)
        if (ci[k] == r) d += va[k];
    dinv[r] = 1.0 / d;
}

}  // namespace

int csr_blocks(int64_t n) {
    static int sms = 0;
    if (!sms) {
        int dev = 0;
        if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
            sms = 1;
    }
    return (int)std::max<int64_t>(1, std::min<int64_t>((n + CT - 1) / CT, 4 * (int64_t)sms));
}

cudaError_t launch_csr_spmm(const CsrOp& a, double alpha, const double* X, int64_t ldx, int p, double* Y, int64_t ldy,
                            cudaStream_t s) {
    if (p < 1 || p > PMAX) return cudaErrorInvalidValue;
    const dim3 grid((unsigned)csr_blocks(a.n), (unsigned)((p + SPG - 1) / SPG));
    k_csr_spmm<<<grid, CT, 0, s>>>(a.rowptr, a.colind, a.val, a.n, alpha, X, ldx, Y, ldy, p);
    return cudaGetLastError();
}

cudaError_t launch_csr_dinv(CsrOp& a, cudaStream_t s) {
    k_csr_dinv<<<(unsigned)((a.n + 255) / 256), 256, 0, s>>>(a.rowptr, a.colind, a.val, a.n, a.dinv);
    return cudaGetLastError();
}

// W = (tA)^{-1} V approximately: A y = V by BiCGStab to ||r|| <= eta ||v|| per column, then
// W = y / t.  The host reads the residual norms every `check` iterations (a stream
// synchronisation).  *iters: iterations run; *converged = 0 when maxit ran out first.
cudaError_t csr_inverse(const CsrOp& a, double t, const double* V, int64_t ldv, int p, double* W, int64_t ldw,
                        double eta, int maxit, cudaStream_t s, int* iters, int* converged) {
    *iters = 0;
    *converged = 0;
    if (p < 1 || p > PMAX) return cudaErrorInvalidValue;
    Bicg g;
    g.rp = a.rowptr;
    g.ci = a.colind;
    g.va = a.val;
    g.dinv = a.dinv;
    g.n = a.n;
    g.ld = a.ld;
    g.p = p;
    g.nb = csr_blocks(a.n);
    double* w = a.work;
    double** vecs[9] = {&g.x, &g.r, &g.rh, &g.q, &g.qh, &g.v, &g.s, &g.sh, &g.u};
    for (int k = 0; k < 9; ++k) *vecs[k] = w + (size_t)k * a.ld * a.pmax;
    g.part = a.part;
    g.sc = a.scal;
    g.norms = a.norms;
    g.eta2 = eta * eta;
    const unsigned nb = (unsigned)g.nb;
    const dim3 gsp(nb, (unsigned)((p + SPG - 1) / SPG));
    k_bicg_start<<<nb, CT, 0, s>>>(g, V, ldv);
    k_bicg_scal<<<1, PMAX, 0, s>>>(g, 0);
    cudaError_t e = cudaGetLastError();
    const int check = 8;
    for (int it = 0; it < maxit && e == cudaSuccess; ++it) {
        k_bicg_dir<<<nb, CT, 0, s>>>(g, it);
        k_bicg_av<<<gsp, CT, 0, s>>>(g);
        k_bicg_scal<<<1, PMAX, 0, s>>>(g, 1);
        k_bicg_s<<<nb, CT, 0, s>>>(g);
        k_bicg_au<<<gsp, CT, 0, s>>>(g);
        k_bicg_scal<<<1, PMAX, 0, s>>>(g, 2);
        k_bicg_x<<<nb, CT, 0, s>>>(g);
        k_bicg_scal<<<1, PMAX, 0, s>>>(g, 3);
        e = cudaGetLastError();
        *iters = it + 1;
        if (e == cudaSuccess && ((it + 1) % check == 0 || it + 1 == maxit)) {
            e = cudaMemcpyAsync(a.hnorms, a.norms, sizeof(double) * 2 * p, cudaMemcpyDeviceToHost, s);
            if (e == cudaSuccess) e = cudaStreamSynchronize(s);
            if (e != cudaSuccess) break;
            bool all = true;
            for (int c = 0; c < p; ++c) all = all && !(a.hnorms[c] > g.eta2 * a.hnorms[p + c]);
            if (all) {
                *converged = 1;
                break;
            }
        }
    }
    if (e == cudaSuccess) {
        const dim3 grid(nb, (unsigned)p);
        k_csr_scale_out<<<grid, CT, 0, s>>>(g.x, a.ld, a.n, 1.0 / t, W, ldw);
        e = cudaGetLastError();
    }
    return e;
}

}  // namespace expm
