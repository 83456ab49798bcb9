// k_csr.cu -- general sparse operators (CSR): the product t A X for Algorithm 1's Krylov
// operator, and the inexact inverse for Algorithm 2 (Section 4.1: when a direct solver is out
// of reach, (tA)^{-1} may be applied by an inner iterative solve; Theorem 4.3 bounds the
// error that the inexactness costs).
//
// The inner solve is BiCGStab with the Jacobi preconditioner (right preconditioning, M =
// diag(A)) on every column of the block at once, each column with its own scalars.  Every
// step is a kernel over (row blocks) x (columns); the reductions are deterministic: each CTA
// writes one partial per column and dot, and the CTAs of the next kernel each re-add all the
// partials of their column in the same fixed order, so every CTA derives the same alpha,
// beta, omega without a separate reduction launch.  A column whose relative residual has
// reached the tolerance (or whose recurrence broke down: a zero denominator) is frozen: its
// iterate and residual no longer change.
#include "internal.h"

namespace expm {
namespace {

constexpr int CT = 256;     // threads per CTA

__device__ __forceinline__ double block_sum(double v, double* sh) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    __syncthreads();
    if (l == 0) sh[w] = v;
    __syncthreads();
    double s = 0.0;
    if (threadIdx.x == 0)
        for (int k = 0; k < CT / 32; ++k) s += sh[k];
    return s;   // valid in thread 0
}

// y = alpha A x for one row (thread per row and column)
__device__ __forceinline__ double row_dot(const int64_t* __restrict__ rp, const int* __restrict__ ci,
                                          const double* __restrict__ va, const double* __restrict__ x, int64_t r) {
    double s = 0.0;
    for (int64_t k = rp[r]; k < rp[r + 1]; ++k) s = fma(va[k], x[ci[k]], s);
    return s;
}

__global__ void __launch_bounds__(CT) k_csr_spmm(const int64_t* __restrict__ rp, const int* __restrict__ ci,
                                                 const double* __restrict__ va, int64_t n, double alpha,
                                                 const double* __restrict__ X, int64_t ldx, double* __restrict__ Y,
                                                 int64_t ldy) {
    const int c = blockIdx.y;
    const double* x = X + c * ldx;
    for (int64_t r = (int64_t)blockIdx.x * CT + threadIdx.x; r < n; r += (int64_t)gridDim.x * CT)
        Y[c * ldy + r] = alpha * row_dot(rp, ci, va, x, r);
}

// The inner solver's vectors, column c at offset c * ld of each: x, r, rh (the shadow
// residual r^_0), q (search direction p), qh = M^-1 q, v = A qh, s, sh = M^-1 s, u = A sh.
struct Bicg {
    const int64_t* rp;
    const int* ci;
    const double* va;
    const double* dinv;      // 1 / a_ii
    int64_t n, ld;
    double *x, *r, *rh, *q, *qh, *v, *s, *sh, *u;
    // partials [nb][p] each: d1 = (rh, v), d2 = (u, s), d3 = (u, u), d4 = (rh, r) (two
    // buffers by iteration parity), d5 = (r, r), b2 = (b, b)
    double *d1, *d2, *d3, *d4a, *d4b, *d5, *b2;
    int* frz;                // per column: frozen this iteration (written by k_bicg_dir)
    double eta2;             // squared relative tolerance
};

__device__ __forceinline__ double sum_part(const double* part, int nb, int p, int c) {
    double s = 0.0;
    for (int b = 0; b < nb; ++b) s += __ldcg(part + (int64_t)b * p + c);
    return s;
}

// the scalars of column c at the start of iteration it (it >= 1), from the partials of the
// previous iteration: rho_new = (rh, r), rho_old, alpha, omega, and whether the column is
// frozen (converged at the previous check of (r, r), or a denominator vanished)
struct Scal {
    double rho, alpha, omega, beta;
    bool frozen;
};

__device__ Scal scalars(const Bicg& g, int it, int nb, int p, int c) {
    const double* d4cur = (it & 1) ? g.d4b : g.d4a;   // written by iteration it - 1
    const double* d4old = (it & 1) ? g.d4a : g.d4b;   // written by iteration it - 2 (or the start)
    Scal z;
    const double rho = sum_part(d4cur, nb, p, c), rho_old = sum_part(d4old, nb, p, c);
    const double dd1 = sum_part(g.d1, nb, p, c), dd2 = sum_part(g.d2, nb, p, c), dd3 = sum_part(g.d3, nb, p, c);
    const double rr = sum_part(g.d5, nb, p, c), bb = sum_part(g.b2, nb, p, c);
    const double alpha = dd1 != 0.0 ? rho_old / dd1 : 0.0;
    const double omega = dd3 != 0.0 ? dd2 / dd3 : 0.0;
    z.rho = rho;
    z.alpha = alpha;
    z.omega = omega;
    z.frozen = !(rr > g.eta2 * bb) || dd1 == 0.0 || dd3 == 0.0 || omega == 0.0 || rho_old == 0.0;
    z.beta = z.frozen ? 0.0 : (rho / rho_old) * (alpha / omega);
    return z;
}

// start: x = 0, r = rh = b, q = 0 (the first direction is r), partials (b, b) and (rh, r)
__global__ void __launch_bounds__(CT) k_bicg_start(Bicg g, const double* __restrict__ B, int64_t ldb, int p) {
    __shared__ double sh[CT / 32];
    const int c = blockIdx.y, nb = gridDim.x;
    double acc = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * CT + threadIdx.x; i < g.n; i += (int64_t)nb * CT) {
        const double b = B[c * ldb + i];
        const int64_t o = c * g.ld + i;
        g.x[o] = 0.0;
        g.r[o] = b;
        g.rh[o] = b;
        g.q[o] = 0.0;
        g.v[o] = 0.0;
        acc = fma(b, b, acc);
    }
    const double s = block_sum(acc, sh);
    if (threadIdx.x == 0) {
        const int64_t o = (int64_t)blockIdx.x * p + c;
        g.b2[o] = s;
        g.d4a[o] = s;      // rho_0 = (rh, r_0)
        g.d4b[o] = 1.0;    // (rho of iteration 1 is written by iteration 0 before any read)
        g.d5[o] = s;
    }
}

// q = r + beta (q - omega v), qh = M^-1 q  (iteration 0: q = r).  Every CTA derives the
// column's scalars and frozen state from the same partials; CTA 0 records the state for the
// iteration's other kernels (which overwrite some of those partials).
__global__ void __launch_bounds__(CT) k_bicg_dir(Bicg g, int it, int p) {
    const int c = blockIdx.y, nb = gridDim.x;
    Scal z;
    if (it > 0) z = scalars(g, it, nb, p, c);
    else z = Scal{0.0, 0.0, 0.0, 0.0, !(sum_part(g.b2, nb, p, c) > 0.0)};
    if (blockIdx.x == 0 && threadIdx.x == 0) g.frz[c] = z.frozen ? 1 : 0;
    if (z.frozen) return;
    for (int64_t i = (int64_t)blockIdx.x * CT + threadIdx.x; i < g.n; i += (int64_t)nb * CT) {
        const int64_t o = c * g.ld + i;
        const double q = it > 0 ? fma(z.beta, fma(-z.omega, g.v[o], g.q[o]), g.r[o]) : g.r[o];
        g.q[o] = q;
        g.qh[o] = q * g.dinv[i];
    }
}

// v = A qh, partial (rh, v)
__global__ void __launch_bounds__(CT) k_bicg_av(Bicg g, int it, int p) {
    __shared__ double sh[CT / 32];
    const int c = blockIdx.y, nb = gridDim.x;
    const bool frozen = g.frz[c] != 0;
    double acc = 0.0;
    if (!frozen)
        for (int64_t i = (int64_t)blockIdx.x * CT + threadIdx.x; i < g.n; i += (int64_t)nb * CT) {
            const int64_t o = c * g.ld + i;
            const double v = row_dot(g.rp, g.ci, g.va, g.qh + c * g.ld, i);
            g.v[o] = v;
            acc = fma(g.rh[o], v, acc);
        }
    const double s = block_sum(acc, sh);
    if (threadIdx.x == 0 && !frozen) g.d1[(int64_t)blockIdx.x * p + c] = s;
}

// alpha = rho / (rh, v); s = r - alpha v, sh = M^-1 s
__global__ void __launch_bounds__(CT) k_bicg_s(Bicg g, int it, int p) {
    const int c = blockIdx.y, nb = gridDim.x;
    if (g.frz[c]) return;
    const double* d4cur = (it & 1) ? g.d4b : g.d4a;
    const double dd1 = sum_part(g.d1, nb, p, c);
    const double alpha = dd1 != 0.0 ? sum_part(d4cur, nb, p, c) / dd1 : 0.0;
    for (int64_t i = (int64_t)blockIdx.x * CT + threadIdx.x; i < g.n; i += (int64_t)nb * CT) {
        const int64_t o = c * g.ld + i;
        const double s = fma(-alpha, g.v[o], g.r[o]);
        g.s[o] = s;
        g.sh[o] = s * g.dinv[i];
    }
}

// u = A sh, partials (u, s) and (u, u)
__global__ void __launch_bounds__(CT) k_bicg_au(Bicg g, int it, int p) {
    __shared__ double sh[CT / 32];
    const int c = blockIdx.y, nb = gridDim.x;
    const bool frozen = g.frz[c] != 0;
    double a2 = 0.0, a3 = 0.0;
    if (!frozen)
        for (int64_t i = (int64_t)blockIdx.x * CT + threadIdx.x; i < g.n; i += (int64_t)nb * CT) {
            const int64_t o = c * g.ld + i;
            const double u = row_dot(g.rp, g.ci, g.va, g.sh + c * g.ld, i);
            g.u[o] = u;
            a2 = fma(u, g.s[o], a2);
            a3 = fma(u, u, a3);
        }
    const double s2 = block_sum(a2, sh);
    const double s3 = block_sum(a3, sh);
    if (threadIdx.x == 0 && !frozen) {
        g.d2[(int64_t)blockIdx.x * p + c] = s2;
        g.d3[(int64_t)blockIdx.x * p + c] = s3;
    }
}

// omega = (u, s) / (u, u); x += alpha qh + omega sh; r = s - omega u; partials (rh, r), (r, r)
__global__ void __launch_bounds__(CT) k_bicg_x(Bicg g, int it, int p) {
    __shared__ double sh[CT / 32];
    const int c = blockIdx.y, nb = gridDim.x;
    const bool frozen = g.frz[c] != 0;
    const double* d4cur = (it & 1) ? g.d4b : g.d4a;
    double* d4next = (it & 1) ? g.d4a : g.d4b;
    const double dd1 = sum_part(g.d1, nb, p, c), dd2 = sum_part(g.d2, nb, p, c), dd3 = sum_part(g.d3, nb, p, c);
    const double alpha = dd1 != 0.0 ? sum_part(d4cur, nb, p, c) / dd1 : 0.0;
    const double omega = dd3 != 0.0 ? dd2 / dd3 : 0.0;
    double a4 = 0.0, a5 = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * CT + threadIdx.x; i < g.n; i += (int64_t)nb * CT) {
        const int64_t o = c * g.ld + i;
        double r = g.r[o];
        if (!frozen) {
            g.x[o] = fma(omega, g.sh[o], fma(alpha, g.qh[o], g.x[o]));
            r = fma(-omega, g.u[o], g.s[o]);
            g.r[o] = r;
        }
        a4 = fma(g.rh[o], r, a4);
        a5 = fma(r, r, a5);
    }
    const double s4 = block_sum(a4, sh);
    const double s5 = block_sum(a5, sh);
    if (threadIdx.x == 0) {
        const int64_t o = (int64_t)blockIdx.x * p + c;
        // a frozen column keeps its partials, so its scalars and its frozen state stay put
        d4next[o] = frozen ? d4cur[o] : s4;
        g.d5[o] = s5;
    }
}

// squared residual norms and (b, b) per column, for the host's stop test
__global__ void k_bicg_norms(Bicg g, int nb, int p, double* out) {
    const int c = threadIdx.x;
    if (c < p) {
        out[c] = sum_part(g.d5, nb, p, c);
        out[p + c] = sum_part(g.b2, nb, p, c);
    }
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
    return (int)std::max<int64_t>(1, std::min<int64_t>((n + CT - 1) / CT, 2 * (int64_t)sms));
}

cudaError_t launch_csr_spmm(const CsrOp& a, double alpha, const double* X, int64_t ldx, int p, double* Y, int64_t ldy,
                            cudaStream_t s) {
    const dim3 grid((unsigned)csr_blocks(a.n), (unsigned)p);
    k_csr_spmm<<<grid, CT, 0, s>>>(a.rowptr, a.colind, a.val, a.n, alpha, X, ldx, Y, ldy);
    return cudaGetLastError();
}

cudaError_t launch_csr_dinv(CsrOp& a, cudaStream_t s) {
    k_csr_dinv<<<(unsigned)((a.n + 255) / 256), 256, 0, s>>>(a.rowptr, a.colind, a.val, a.n, a.dinv);
    return cudaGetLastError();
}

// W = (tA)^{-1} V approximately: A y = V by BiCGStab to ||r|| <= eta ||v|| per column, then
// W = y / t.  The host reads the residual norms every `check` iterations (a stream
// synchronisation).  Returns cudaSuccess and *iters (iterations run); *converged = 0 when
// maxit ran out first.
cudaError_t csr_inverse(const CsrOp& a, double t, const double* V, int64_t ldv, int p, double* W, int64_t ldw,
                        double eta, int maxit, cudaStream_t s, int* iters, int* converged) {
    const int nb = csr_blocks(a.n);
    Bicg g;
    g.rp = a.rowptr;
    g.ci = a.colind;
    g.va = a.val;
    g.dinv = a.dinv;
    g.n = a.n;
    g.ld = a.ld;
    double* w = a.work;
    double** vecs[9] = {&g.x, &g.r, &g.rh, &g.q, &g.qh, &g.v, &g.s, &g.sh, &g.u};
    for (int k = 0; k < 9; ++k) *vecs[k] = w + (size_t)k * a.ld * a.pmax;
    double* pp = a.part;
    const size_t ps = (size_t)nb * p;
    g.d1 = pp; g.d2 = pp + ps; g.d3 = pp + 2 * ps; g.d4a = pp + 3 * ps; g.d4b = pp + 4 * ps;
    g.d5 = pp + 5 * ps; g.b2 = pp + 6 * ps;
    g.frz = a.frz;
    g.eta2 = eta * eta;
    // the partials of the dots before their first write: zero (a frozen check in iteration
    // 0 is skipped, and iteration 1 reads only what iteration 0 wrote)
    cudaError_t e = cudaMemsetAsync(pp, 0, sizeof(double) * 7 * ps, s);
    const dim3 grid((unsigned)nb, (unsigned)p);
    if (e == cudaSuccess) {
        k_bicg_start<<<grid, CT, 0, s>>>(g, V, ldv, p);
        e = cudaGetLastError();
    }
    *iters = 0;
    *converged = 0;
    const int check = 8;
    for (int it = 0; it < maxit && e == cudaSuccess; ++it) {
        k_bicg_dir<<<grid, CT, 0, s>>>(g, it, p);
        k_bicg_av<<<grid, CT, 0, s>>>(g, it, p);
        k_bicg_s<<<grid, CT, 0, s>>>(g, it, p);
        k_bicg_au<<<grid, CT, 0, s>>>(g, it, p);
        k_bicg_x<<<grid, CT, 0, s>>>(g, it, p);
        e = cudaGetLastError();
        *iters = it + 1;
        if (e == cudaSuccess && ((it + 1) % check == 0 || it + 1 == maxit)) {
            k_bicg_norms<<<1, 32, 0, s>>>(g, nb, p, a.norms);
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
        k_csr_scale_out<<<grid, CT, 0, s>>>(g.x, a.ld, a.n, 1.0 / t, W, ldw);
        e = cudaGetLastError();
    }
    return e;
}

}  // namespace expm
