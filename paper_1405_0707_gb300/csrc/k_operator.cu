// k_operator.cu -- operator and exact-inverse kernels for the convection-diffusion family.
//
// W = (tA)^{-1} V replaces the paper's "LU once, then U \ (L \ w)" (Section 4.1,
// Section 5) by an exact structured solve: tA = t (T_x (+) T_y (+) T_z) (Kronecker sum)
// with T_d = D_d^{-1} Q Lambda_d Q D_d (diagonal similarity D_d = diag(rho^j),
// rho = sqrt(u/l); Q the orthonormal DST-I, symmetric, Q Q = I).  Transform every axis
// except x with (D_d, Q), solve one tridiagonal system along x per transformed mode with
// the shift lambda_y + lambda_z, transform back.  The transforms are small dense GEMMs
// (DST-I for N + 1 prime or odd has no cheap power-of-two FFT), the line solves use a
// Thomas factorisation built once per mode at plan creation.
#include "df.cuh"
#include "internal.h"

namespace expm {
namespace {

constexpr int BM = 64, BN = 64, BK = 16;

// C = A * B, FP64.  256 threads, 4x4 outputs per thread.  CM selects the thread layout
// so that the fastest-varying thread index walks C's contiguous dimension.
template <bool CM>
__global__ void __launch_bounds__(256) k_gemm(GemmArgs g) {
    __shared__ double As[BK][BM + 1];
    __shared__ double Bs[BK][BN];
    const int b1 = blockIdx.z % g.nb1, b2 = blockIdx.z / g.nb1;
    const double* A = g.A + b1 * g.a_b1 + b2 * g.a_b2;
    double* C = g.C + b1 * g.c_b1 + b2 * g.c_b2;
    const int m0 = blockIdx.x * BM, n0 = blockIdx.y * BN;
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    const bool a_mfast = (g.a_rs == 1);
    double acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = 0.0;
    for (int k0 = 0; k0 < g.K; k0 += BK) {
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int e = tid + q * 256;
            int mm, kk;
            if (a_mfast) { mm = e % BM; kk = e / BM; }
            else { kk = e % BK; mm = e / BK; }
            const int gm = m0 + mm, gk = k0 + kk;
            As[kk][mm] = (gm < g.M && gk < g.K) ? A[(int64_t)gm * g.a_rs + (int64_t)gk * g.a_cs] : 0.0;
        }
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int e = tid + q * 256;
            const int nn = e % BN, kk = e / BN;
            const int gn = n0 + nn, gk = k0 + kk;
            Bs[kk][nn] = (gn < g.N && gk < g.K) ? g.B[(int64_t)gk * g.ldb + gn] : 0.0;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < BK; ++kk) {
            double a[4], b[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) a[i] = As[kk][(CM ? tx : ty) + 16 * i];
#pragma unroll
            for (int j = 0; j < 4; ++j) b[j] = Bs[kk][(CM ? ty : tx) + 16 * j];
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int m = m0 + (CM ? tx : ty) + 16 * i, nn = n0 + (CM ? ty : tx) + 16 * j;
            if (m < g.M && nn < g.N) C[(int64_t)m * g.c_rs + (int64_t)nn * g.c_cs] = acc[i][j];
        }
}

// Line solves along x with the precomputed Thomas factors of tridiag(l, c + lambda_mode, u):
// forward  y_x = (f_x / t - l y_{x-1}) m_x,  backward  z_x = y_x - c'_x z_{x+1} (z_L = 0).
// Both are first-order linear recurrences, i.e. compositions of affine maps v -> a v + b, so
// each line is split into TSEG segments handled by TSEG lanes of one warp: every lane composes
// its segment's map, the segments' entry values are passed lane to lane with shuffles, and
// every lane then reruns its segment from the right entry value.  Lanes of a warp hold
// 32 / TSEG consecutive modes of the same segment position, so each warp-wide load touches
// TSEG fully used 32-byte sectors (the layout is mode-fastest).  in may equal out: every
// element is read and written by the one lane that owns its segment.
constexpr int TSEG = 8;
constexpr int TUNR = 8;    // loads issued ahead inside a segment

template <typename T>
__device__ inline void tridiag_seg(const T* f, T* y, int L, int64_t nm, int64_t k, T l_sub,
                                   const T* __restrict__ thm, const T* __restrict__ thc, T inv_t, int seg,
                                   bool active) {
    const int seglen = (L + TSEG - 1) / TSEG;
    const int x0 = min(L, seg * seglen), x1 = min(L, x0 + seglen);
    const unsigned full = 0xffffffffu;
    // forward: compose y_out = A y_in + B over the segment
    T A = 1, B = 0;
    if (active)
        for (int xb = x0; xb < x1; xb += TUNR) {
            T fv[TUNR], mv[TUNR];
#pragma unroll
            for (int q = 0; q < TUNR; ++q)
                if (xb + q < x1) {
                    fv[q] = f[(int64_t)(xb + q) * nm];
                    mv[q] = thm[(int64_t)(xb + q) * nm + k];
                }
#pragma unroll
            for (int q = 0; q < TUNR; ++q)
                if (xb + q < x1) {
                    const T a = -l_sub * mv[q];
                    B = a * B + fv[q] * inv_t * mv[q];
                    A = a * A;
                }
        }
    T yin = 0;
    for (int sgi = 1; sgi < TSEG; ++sgi) {
        const T v = __shfl_up_sync(full, A * yin + B, 1);
        if (seg == sgi) yin = v;
    }
    if (active) {
        T prev = yin;
        for (int xb = x0; xb < x1; xb += TUNR) {
            T fv[TUNR], mv[TUNR];
#pragma unroll
            for (int q = 0; q < TUNR; ++q)
                if (xb + q < x1) {
                    fv[q] = f[(int64_t)(xb + q) * nm];
                    mv[q] = thm[(int64_t)(xb + q) * nm + k];
                }
#pragma unroll
            for (int q = 0; q < TUNR; ++q)
                if (xb + q < x1) {
                    prev = (fv[q] * inv_t - l_sub * prev) * mv[q];
                    y[(int64_t)(xb + q) * nm] = prev;
                }
        }
    }
    // backward: z_out(x0) = A z_in(x1) + B over the segment, from x1 - 1 down to x0
    A = 1;
    B = 0;
    if (active)
        for (int xb = x1 - 1; xb >= x0; xb -= TUNR) {
            T yv[TUNR], cv[TUNR];
#pragma unroll
            for (int q = 0; q < TUNR; ++q)
                if (xb - q >= x0) {
                    yv[q] = y[(int64_t)(xb - q) * nm];
                    cv[q] = (xb - q < L - 1) ? thc[(int64_t)(xb - q) * nm + k] : T(0);
                }
#pragma unroll
            for (int q = 0; q < TUNR; ++q)
                if (xb - q >= x0) {
                    B = yv[q] - cv[q] * B;
                    A = -cv[q] * A;
                }
        }
    T zin = 0;
    for (int sgi = TSEG - 2; sgi >= 0; --sgi) {
        const T v = __shfl_down_sync(full, A * zin + B, 1);
        if (seg == sgi) zin = v;
    }
    if (active) {
        T next = zin;
        for (int xb = x1 - 1; xb >= x0; xb -= TUNR) {
            T yv[TUNR], cv[TUNR];
#pragma unroll
            for (int q = 0; q < TUNR; ++q)
                if (xb - q >= x0) {
                    yv[q] = y[(int64_t)(xb - q) * nm];
                    cv[q] = (xb - q < L - 1) ? thc[(int64_t)(xb - q) * nm + k] : T(0);
                }
#pragma unroll
            for (int q = 0; q < TUNR; ++q)
                if (xb - q >= x0) {
                    next = yv[q] - cv[q] * next;
                    y[(int64_t)(xb - q) * nm] = next;
                }
        }
    }
}

// line index of a lane: warp-major groups of 32 / TSEG lines, TSEG segment lanes per line
__device__ inline int64_t seg_line(int& seg) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    seg = lane % TSEG;
    return ((int64_t)blockIdx.x * (blockDim.x >> 5) + warp) * (32 / TSEG) + lane / TSEG;
}

__global__ void k_tridiag_lines(const double* in, int64_t ld_in, double* out, int64_t ld_out,
                                int p, int L, int64_t nmodes, double l_sub,
                                const double* __restrict__ thm, const double* __restrict__ thc,
                                double inv_t) {
    int seg;
    const int64_t line = seg_line(seg);
    const bool active = line < nmodes * p;
    const int64_t k = active ? line % nmodes : 0;
    const int c = active ? (int)(line / nmodes) : 0;
    tridiag_seg<double>(in + c * ld_in + k, out + c * ld_out + k, L, nmodes, k, l_sub, thm, thc, inv_t, seg,
                        active);
}

// Thomas factors for every mode (one thread per mode): pivots b - l c'_{x-1}, stored as
// reciprocals, and c'_x = u / pivot_x.
__global__ void k_thomas_setup(double* thm, double* thc, int L, int64_t nmodes, double l,
                               double c, double u, const double* lam_y, int Ny,
                               const double* lam_z, int Nz) {
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= nmodes) return;
    double shift = 0.0;
    if (lam_y) shift += lam_y[k % Ny];
    if (lam_z) shift += lam_z[k / Ny];
    const double b = c + shift;
    double cp = 0.0;
    for (int x = 0; x < L; ++x) {
        const double piv = b - (x > 0 ? l * cp : 0.0);
        const double mi = 1.0 / piv;
        cp = u * mi;
        thm[(int64_t)x * nmodes + k] = mi;
        thc[(int64_t)x * nmodes + k] = cp;
    }
}

// Axis eigen-data: Q[j][k] = sqrt(2/(N+1)) sin(pi (j+1)(k+1)/(N+1)) (DST-I, exact
// integer argument reduction), Qf = diag(rho^j) Q, Qi = Q diag(rho^-j),
// lambda_k = c + 2 s cos(pi (k+1)/(N+1)), s = sign(l) sqrt(l u).
__global__ void k_axis_setup(double* Qf, double* Qi, double* lam, int N, double l, double c,
                             double u) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (int64_t)N * N) return;
    const int j = (int)(e / N), k = (int)(e % N);
    const int64_t arg = ((int64_t)(j + 1) * (k + 1)) % (2 * (int64_t)(N + 1));
    const double q = sqrt(2.0 / (N + 1)) * sinpi((double)arg / (double)(N + 1));
    const double rho = sqrt(u / l);
    Qf[e] = pow(rho, (double)j) * q;              // row j (grid index), column k (mode)
    Qi[e] = q * pow(rho, -(double)k);             // row j (mode), column k (grid index)
    if (j == 0) {
        const double s = (l > 0 ? 1.0 : -1.0) * sqrt(l * u);
        lam[k] = c + 2.0 * s * cospi((double)(k + 1) / (double)(N + 1));
    }
}

// W = t (A V) + beta Y, 3/5/7-point stencil with Dirichlet zeros outside the grid.
// (beta = 0, Y = null: the operator apply; t -> -t, beta = 1: the residual Y - tA V.)
// Stencil coefficients with t folded in (computed on the host): tc = t (c_x + c_y + c_z),
// tl[d] = t l_d, tu[d] = t u_d; 5 (2-D) or 7 (3-D) FP64 multiply-adds per point.
struct StencilT {
    double tc, tl[3], tu[3];
};

// W = tA V (+ beta Y): one thread per grid point and column; grid index arithmetic in 32 bits
// (n < 2^31 is checked by the launcher).  With W32 set, the FP64 result is stored rounded to
// FP32 there (same leading dimension) instead of in W: the refinement residual, which only
// the FP32 transforms read.
__global__ void k_cd_apply(const double* __restrict__ V, int64_t ldv, double* __restrict__ W,
                           int64_t ldw, int ndim, int nx, int ny, int nz, StencilT k,
                           const double* __restrict__ Y, int64_t ldy, double beta, float* __restrict__ W32) {
    const unsigned n = (unsigned)nx * (unsigned)ny * (unsigned)nz;
    const unsigned i = blockIdx.x * blockDim.x + threadIdx.x;
    const int c = blockIdx.y;
    if (i >= n) return;
    const double* v = V + c * ldv;
    const unsigned q = i / (unsigned)nx;
    const unsigned ix = i - q * (unsigned)nx;
    double acc = k.tc * v[i];
    if (ix > 0) acc = fma(k.tl[0], v[i - 1], acc);
    if (ix < (unsigned)nx - 1) acc = fma(k.tu[0], v[i + 1], acc);
    if (ndim > 1) {
        const unsigned iz = q / (unsigned)ny, iy = q - iz * (unsigned)ny;
        if (iy > 0) acc = fma(k.tl[1], v[i - nx], acc);
        if (iy < (unsigned)ny - 1) acc = fma(k.tu[1], v[i + nx], acc);
        if (ndim > 2) {
            const unsigned st = (unsigned)nx * (unsigned)ny;
            if (iz > 0) acc = fma(k.tl[2], v[i - st], acc);
            if (iz < (unsigned)nz - 1) acc = fma(k.tu[2], v[i + st], acc);
        }
    }
    const double r = Y ? fma(beta, Y[c * ldy + i], acc) : acc;
    if (W32) W32[c * ldw + i] = f32_rn_i(r);   // integer rounding: no FP64-pipe conversion
    else W[c * ldw + i] = r;
}

// The same stencil in double-float arithmetic on the FP32 pipe, for mixed-precision plans:
// coefficients as float pairs (host-split), every value split from its bit pattern
// (split_df_i), products and sums as in the double-float row kernels.  GB300 retires about two
// FP64 FMAs per SM per clock, so the FP64 stencil (5 or 7 per point) is bound by the FP64
// pipe, not by memory; the pair arithmetic is ~2^-48 accurate, the level of the mixed path's
// other double-float kernels.  Y (the refinement's right-hand side) enters with beta = 1.
struct StencilDF {
    float ch, cl, lh[3], ll[3], uh[3], ul[3];
};

__device__ __forceinline__ void df_term(float& sh, float& sl, double v, float ch, float cl) {
    float vh, vl;
    split_df_i(v, vh, vl);
    df_fma(sh, sl, vh, vl, ch, cl);
}

__global__ void k_cd_apply_df(const double* __restrict__ V, int64_t ldv, double* __restrict__ W,
                              int64_t ldw, int ndim, int nx, int ny, int nz, StencilDF k,
                              const double* __restrict__ Y, int64_t ldy, float* __restrict__ W32) {
    const unsigned n = (unsigned)nx * (unsigned)ny * (unsigned)nz;
    const unsigned i = blockIdx.x * blockDim.x + threadIdx.x;
    const int c = blockIdx.y;
    if (i >= n) return;
    const double* v = V + c * ldv;
    const unsigned q = i / (unsigned)nx;
    const unsigned ix = i - q * (unsigned)nx;
    float sh = 0.f, sl = 0.f;
    df_term(sh, sl, v[i], k.ch, k.cl);
    if (ix > 0) df_term(sh, sl, v[i - 1], k.lh[0], k.ll[0]);
    if (ix < (unsigned)nx - 1) df_term(sh, sl, v[i + 1], k.uh[0], k.ul[0]);
    if (ndim > 1) {
        const unsigned iz = q / (unsigned)ny, iy = q - iz * (unsigned)ny;
        if (iy > 0) df_term(sh, sl, v[i - nx], k.lh[1], k.ll[1]);
        if (iy < (unsigned)ny - 1) df_term(sh, sl, v[i + nx], k.uh[1], k.ul[1]);
        if (ndim > 2) {
            const unsigned st = (unsigned)nx * (unsigned)ny;
            if (iz > 0) df_term(sh, sl, v[i - st], k.lh[2], k.ll[2]);
            if (iz < (unsigned)nz - 1) df_term(sh, sl, v[i + st], k.uh[2], k.ul[2]);
        }
    }
    if (Y) {
        float yh, yl;
        split_df_i(Y[c * ldy + i], yh, yl);
        df_add(sh, sl, yh);
        sl += yl;
    }
    if (W32) W32[c * ldw + i] = sh + sl;
    else W[c * ldw + i] = f64_of_f32_i(sh) + f64_of_f32_i(sl);
}

// ---------------------------------------------------------------- mixed precision
// FP32 arithmetic for the DST-I transforms of the exact inverse; the result is refined
// in FP64 by the caller (residual with the FP64 stencil, Theorem 4.3 bounds what an
// inexact inverse costs).  TA / TC: element types of A and C; acc: C += A B.
constexpr int BK32 = 32;   // k-depth of one FP32 tile

// FP32 tiles of 64 x 64 outputs, 4 x 4 per thread; the next k-tile's global loads are
// issued into registers before the current tile's FMAs (software pipelining), so each
// barrier round overlaps its loads with arithmetic.  FP64 operands are converted from the
// bit pattern (f32_rn_i) and FP64 results formed with an exact float -> double widening,
// keeping the transforms off GB300's FP64 pipe except for the one accumulating add.
__device__ __forceinline__ int64_t gemm_row_off(int m, int ms, int64_t rs, int64_t ms2) {
    return ms ? (int64_t)(m % ms) * rs + (int64_t)(m / ms) * ms2 : (int64_t)m * rs;
}

__device__ __forceinline__ float gemm_in(double x) { return f32_rn_i(x); }
__device__ __forceinline__ float gemm_in(float x) { return x; }

template <typename TC>
__device__ __forceinline__ void gemm_out(TC* dst, float v, int acc) {
    if constexpr (sizeof(TC) == 8) *dst = acc ? *dst + f64_of_f32_i(v) : f64_of_f32_i(v);
    else *dst = acc ? *dst + v : v;
}

template <bool CM, typename TA, typename TC>
__global__ void __launch_bounds__(256) k_gemm32(GemmArgsMixed g) {
    // rows padded to BM + 4 floats: 16-byte aligned rows for the float4 operand loads
    __shared__ __align__(16) float As[BK32][BM + 4];
    __shared__ __align__(16) float Bs[BK32][BN];
    const int b1 = blockIdx.z % g.nb1, b2 = blockIdx.z / g.nb1;
    const TA* A = reinterpret_cast<const TA*>(g.A) + b1 * g.a_b1 + b2 * g.a_b2;
    TC* C = reinterpret_cast<TC*>(g.C) + b1 * g.c_b1 + b2 * g.c_b2;
    const int m0 = blockIdx.x * BM, n0 = blockIdx.y * BN;
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    const bool a_mfast = (g.a_rs == 1);
    float acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = 0.f;
    constexpr int NQ = BK32 * BM / 256;   // elements of each tile per thread (8)
    // A-row offset of each of this thread's fetched elements (-1 past M), fixed over k
    int64_t aoff[NQ];
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
        const int e = tid + q * 256;
        const int gm = m0 + (a_mfast ? e % BM : e / BK32);
        aoff[q] = gm < g.M ? gemm_row_off(gm, g.ms, g.a_rs, g.a_ms2) : -1;
    }
    float ra[NQ], rb[NQ];
    auto fetch = [&](int k0) {
#pragma unroll
        for (int q = 0; q < NQ; ++q) {
            const int e = tid + q * 256;
            const int gk = k0 + (a_mfast ? e / BM : e % BK32);
            ra[q] = (aoff[q] >= 0 && gk < g.K) ? gemm_in(A[aoff[q] + (int64_t)gk * g.a_cs]) : 0.f;
        }
#pragma unroll
        for (int q = 0; q < NQ; ++q) {
            const int e = tid + q * 256;
            const int nn = e % BN, kk = e / BN;
            const int gn = n0 + nn, gk = k0 + kk;
            rb[q] = (gn < g.N && gk < g.K) ? g.B[(int64_t)gk * g.ldb + gn] : 0.f;
        }
    };
    fetch(0);
    for (int k0 = 0; k0 < g.K; k0 += BK32) {
#pragma unroll
        for (int q = 0; q < NQ; ++q) {
            const int e = tid + q * 256;
            int mm, kk;
            if (a_mfast) { mm = e % BM; kk = e / BM; }
            else { kk = e % BK32; mm = e / BK32; }
            As[kk][mm] = ra[q];
            Bs[e / BN][e % BN] = rb[q];
        }
        __syncthreads();
        if (k0 + BK32 < g.K) fetch(k0 + BK32);
        // each thread owns 4 consecutive rows m and 4 consecutive columns n: one float4 load
        // per operand per k (the fastest-varying thread index walks C's contiguous dimension)
        const int mi = 4 * (CM ? tx : ty), nj = 4 * (CM ? ty : tx);
#pragma unroll
        for (int kk = 0; kk < BK32; ++kk) {
            const float4 av = *reinterpret_cast<const float4*>(&As[kk][mi]);
            const float4 bv = *reinterpret_cast<const float4*>(&Bs[kk][nj]);
            const float a[4] = {av.x, av.y, av.z, av.w}, b[4] = {bv.x, bv.y, bv.z, bv.w};
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
        }
        __syncthreads();
    }
    const int mi = 4 * (CM ? tx : ty), nj = 4 * (CM ? ty : tx);
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int m = m0 + mi + i;
        if (m >= g.M) continue;
        TC* crow = C + gemm_row_off(m, g.ms, g.c_rs, g.c_ms2);
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int nn = n0 + nj + j;
            if (nn < g.N) gemm_out(crow + (int64_t)nn * g.c_cs, acc[i][j], g.accumulate);
        }
    }
}

// Transforms along a short axis (K, N <= 96: every axis of the 3-D grids): the whole K x N
// DST matrix and a slab of SBM rows of A (all K) sit in shared memory, so one barrier
// separates staging from arithmetic and no k-tile padding is read.  A thread owns 8 rows
// (two runs of 4 consecutive rows, 64 apart) and NJ columns (16 apart): per k two float4 of
// A and NJ floats of B feed 8 NJ FMAs.  The row runs (CM: C's contiguous dimension is m) or
// the columns (otherwise) walk consecutive threads, so the stores coalesce.
constexpr int SBM = 128, SMAX = 96;
constexpr int SAS = SBM + 4;   // row stride of the staged A (float4-aligned)

// one 4-byte asynchronous global -> shared copy (zero-filled when !ok: no bytes are read,
// and src is then any valid address)
__device__ __forceinline__ void cp_async4(float* dst, const float* src, bool ok) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;" ::"r"((uint32_t)__cvta_generic_to_shared(dst)),
                 "l"(src), "r"(ok ? 4 : 0)
                 : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }
__host__ __device__ constexpr size_t gemm_small_smem(int K, int NJ) {
    return sizeof(float) * ((size_t)K * 16 * NJ + (size_t)K * SAS);
}

template <bool CM, typename TA, typename TC, int NJ>
__global__ void __launch_bounds__(256) k_gemm_small(GemmArgsMixed g) {
    extern __shared__ __align__(16) float sgm[];
    constexpr int NP = 16 * NJ;
    const int K = g.K;
    float* Bs = sgm;                  // K x NP, columns past N zero
    float* As = Bs + K * NP;          // K x SAS: As[k * SAS + mm]
    const int b1 = blockIdx.y % g.nb1, b2 = blockIdx.y / g.nb1;
    const TA* A = reinterpret_cast<const TA*>(g.A) + b1 * g.a_b1 + b2 * g.a_b2;
    TC* C = reinterpret_cast<TC*>(g.C) + b1 * g.c_b1 + b2 * g.c_b2;
    const int m0 = blockIdx.x * SBM, tid = threadIdx.x;
    // staging: every float operand is copied with cp.async, so all of a thread's copies are in
    // flight at once and the CTA waits for one round trip; an FP64 A is converted on the way
    // and goes through registers, in batches of loads issued before any is stored
    for (int e = tid; e < K * NP; e += 256) {
        const int k = e / NP, n = e - k * NP;
        const bool ok = n < g.N;
        cp_async4(Bs + e, ok ? g.B + (int64_t)k * g.ldb + n : g.B, ok);
    }
    if constexpr (sizeof(TA) == 4) {
        if (g.a_rs == 1) {
            const int mm = tid & (SBM - 1), m = m0 + mm;
            const bool ok = m < g.M;
            const int64_t ro = ok ? gemm_row_off(m, g.ms, g.a_rs, g.a_ms2) : 0;
            for (int k = tid >> 7; k < K; k += 2)
                cp_async4(As + k * SAS + mm, ok ? (const float*)A + ro + (int64_t)k * g.a_cs : (const float*)A, ok);
        } else {
            const int warp = tid >> 5, lane = tid & 31;
            for (int mm0 = warp; mm0 < SBM; mm0 += 32)
#pragma unroll
                for (int r = 0; r < 4; ++r) {
                    const int m = m0 + mm0 + 8 * r;
                    const bool ok = m < g.M;
                    const int64_t ro = ok ? gemm_row_off(m, g.ms, g.a_rs, g.a_ms2) : 0;
#pragma unroll
                    for (int j = 0; j < 3; ++j) {
                        const int k = lane + 32 * j;
                        if (k < K)
                            cp_async4(As + k * SAS + mm0 + 8 * r,
                                      ok ? (const float*)A + ro + (int64_t)k * g.a_cs : (const float*)A, ok);
                    }
                }
        }
    } else if (g.a_rs == 1) {
        // m fastest in memory: thread t keeps row mm = t % SBM (one row offset) and walks k
        const int mm = tid & (SBM - 1), m = m0 + mm;
        const bool ok = m < g.M;
        const int64_t ro = ok ? gemm_row_off(m, g.ms, g.a_rs, g.a_ms2) : 0;
        for (int k0 = tid >> 7; k0 < K; k0 += 16) {
            float v[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const int k = k0 + 2 * u;
                v[u] = (ok && k < K) ? gemm_in(A[ro + (int64_t)k * g.a_cs]) : 0.f;
            }
#pragma unroll
            for (int u = 0; u < 8; ++u)
                if (k0 + 2 * u < K) As[(k0 + 2 * u) * SAS + mm] = v[u];
        }
    } else {
        // k fastest in memory: a warp takes 4 rows at a time, lane l the entries k = l + 32 j
        const int warp = tid >> 5, lane = tid & 31;
        for (int mm0 = warp; mm0 < SBM; mm0 += 32) {
            float v[4][3];
#pragma unroll
            for (int r = 0; r < 4; ++r) {
                const int m = m0 + mm0 + 8 * r;
                const bool ok = m < g.M;
                const int64_t ro = ok ? gemm_row_off(m, g.ms, g.a_rs, g.a_ms2) : 0;
#pragma unroll
                for (int j = 0; j < 3; ++j) {
                    const int k = lane + 32 * j;
                    v[r][j] = (ok && k < K) ? gemm_in(A[ro + (int64_t)k * g.a_cs]) : 0.f;
                }
            }
#pragma unroll
            for (int r = 0; r < 4; ++r)
#pragma unroll
                for (int j = 0; j < 3; ++j)
                    if (lane + 32 * j < K) As[(lane + 32 * j) * SAS + mm0 + 8 * r] = v[r][j];
        }
    }
    cp_async_wait_all();
    __syncthreads();
    const int tm = CM ? (tid & 15) : (tid >> 4), tn = CM ? (tid >> 4) : (tid & 15);
    float acc[8][NJ];
#pragma unroll
    for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < NJ; ++j) acc[i][j] = 0.f;
    const float* ap = As + 4 * tm;
    const float* bp = Bs + tn;
#pragma unroll 4
    for (int k = 0; k < K; ++k) {
        const float4 a0 = *reinterpret_cast<const float4*>(ap + k * SAS);
        const float4 a1 = *reinterpret_cast<const float4*>(ap + k * SAS + 64);
        const float a[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
        float b[NJ];
#pragma unroll
        for (int j = 0; j < NJ; ++j) b[j] = bp[k * NP + 16 * j];
#pragma unroll
        for (int i = 0; i < 8; ++i)
#pragma unroll
            for (int j = 0; j < NJ; ++j) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
    }
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        const int m = m0 + 4 * tm + (i & 3) + 64 * (i >> 2);
        if (m >= g.M) continue;
        TC* crow = C + gemm_row_off(m, g.ms, g.c_rs, g.c_ms2);
#pragma unroll
        for (int j = 0; j < NJ; ++j) {
            const int n = tn + 16 * j;
            if (n < g.N) gemm_out(crow + (int64_t)n * g.c_cs, acc[i][j], g.accumulate);
        }
    }
}

// The FP32 line solves with the lines staged in shared memory: a CTA takes TK consecutive
// modes of one column (16 x L values of f, thm and thc, loaded once with coalesced reads),
// runs the same segmented affine scans as tridiag_seg from shared memory and writes y back.
// Each mode's line is stored contiguously with one pad element per segment, so the TSG lanes
// of a line read distinct banks (segment stride seglen + 1, odd for L = 256).
constexpr int TK = 16;
constexpr int TSG = 32;    // segments per line in the tile kernel (one line per warp)
constexpr size_t kTridiagTileSmemMax = 110 * 1024;
__host__ __device__ constexpr size_t tridiag_tile_smem(int L) { return sizeof(float) * 3 * (size_t)TK * (L + TSG); }

__global__ void __launch_bounds__(TK * TSG) k_tridiag_tile32(float* y_io, int64_t ld, int L, int64_t nmodes,
                                                             float l_sub, const float* __restrict__ thm,
                                                             const float* __restrict__ thc, float inv_t) {
    extern __shared__ float smt[];
    const int Lp = L + TSG;
    const int seglen = (L + TSG - 1) / TSG;
    float* F = smt;                  // TK x Lp: f, then y in place
    float* Mt = F + TK * Lp;
    float* Ct = Mt + TK * Lp;
    const int c = blockIdx.y;
    const int64_t k0 = (int64_t)blockIdx.x * TK;
    float* y = y_io + (int64_t)c * ld;
    constexpr int NT = TK * TSG, UB = 8;   // UB elements (3 UB loads) in flight per thread
    const int tot = L * TK;
    for (int e0 = threadIdx.x; e0 < tot; e0 += UB * NT) {
        float fv[UB], mv[UB], cv[UB];
#pragma unroll
        for (int u = 0; u < UB; ++u) {
            const int e = e0 + u * NT, x = e / TK, kk = e - x * TK;
            const int64_t k = k0 + kk;
            const bool ok = e < tot && k < nmodes;
            fv[u] = ok ? y[(int64_t)x * nmodes + k] : 0.f;
            mv[u] = ok ? thm[(int64_t)x * nmodes + k] : 0.f;
            cv[u] = ok ? thc[(int64_t)x * nmodes + k] : 0.f;
        }
#pragma unroll
        for (int u = 0; u < UB; ++u) {
            const int e = e0 + u * NT, x = e / TK, kk = e - x * TK;
            if (e < tot) {
                const int si = kk * Lp + x + x / seglen;
                F[si] = fv[u];
                Mt[si] = mv[u];
                Ct[si] = cv[u];
            }
        }
    }
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int seg = lane % TSG, kk = warp * (32 / TSG) + lane / TSG;
    const int x0 = min(L, seg * seglen), x1 = min(L, x0 + seglen);
    float* f = F + kk * Lp + seg;          // element x of the line at f[x] (x in this segment)
    const float* m = Mt + kk * Lp + seg;
    const float* cc = Ct + kk * Lp + seg;
    const unsigned full = 0xffffffffu;
    float A = 1.f, B = 0.f;
    for (int x = x0; x < x1; ++x) {
        const float a = -l_sub * m[x];
        B = a * B + f[x] * inv_t * m[x];
        A = a * A;
    }
    // inclusive scan of the segment maps y -> A y + B over the line's TSG lanes (log2 TSG
    // steps; the composition is associative), then the value entering each segment is the
    // previous segment's prefix applied to 0
#pragma unroll
    for (int d = 1; d < TSG; d <<= 1) {
        const float Ap = __shfl_up_sync(full, A, d, TSG), Bp = __shfl_up_sync(full, B, d, TSG);
        if (seg >= d) {
            B = fmaf(A, Bp, B);
            A = A * Ap;
        }
    }
    float yin = __shfl_up_sync(full, B, 1, TSG);
    if (seg == 0) yin = 0.f;
    float prev = yin;
    for (int x = x0; x < x1; ++x) {
        prev = (f[x] * inv_t - l_sub * prev) * m[x];
        f[x] = prev;
    }
    A = 1.f;
    B = 0.f;
    for (int x = x1 - 1; x >= x0; --x) {
        const float cv = (x < L - 1) ? cc[x] : 0.f;
        B = f[x] - cv * B;
        A = -cv * A;
    }
#pragma unroll
    for (int d = 1; d < TSG; d <<= 1) {
        const float An = __shfl_down_sync(full, A, d, TSG), Bn = __shfl_down_sync(full, B, d, TSG);
        if (seg + d < TSG) {
            B = fmaf(A, Bn, B);
            A = A * An;
        }
    }
    float zin = __shfl_down_sync(full, B, 1, TSG);
    if (seg == TSG - 1) zin = 0.f;
    float next = zin;
    for (int x = x1 - 1; x >= x0; --x) {
        const float cv = (x < L - 1) ? cc[x] : 0.f;
        next = f[x] - cv * next;
        f[x] = next;
    }
    __syncthreads();
    for (int e = threadIdx.x; e < L * TK; e += blockDim.x) {
        const int x = e / TK, kk2 = e - x * TK;
        const int64_t k = k0 + kk2;
        if (k < nmodes) y[(int64_t)x * nmodes + k] = F[kk2 * Lp + x + x / seglen];
    }
}

// Short lines with many modes (the x lines of a 3-D grid, L <= 128, ny nz modes): one thread
// per (mode, column) runs both sweeps of the factored solve over its line, consecutive
// threads on consecutive modes (coalesced: the layout is mode-fastest).  The sweeps' loads do
// not depend on the recurrence, but they may alias the stores as far as the compiler knows,
// so each sweep reads its line in explicit batches of TB elements into registers and issues
// the next batch's loads before it stores the current one.
constexpr int TB = 8;
__global__ void __launch_bounds__(256) k_tridiag_thread32(float* y_io, int64_t ld, int L, int64_t nmodes,
                                                          float l_sub, const float* __restrict__ thm,
                                                          const float* __restrict__ thc, float inv_t) {
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= nmodes) return;
    float* y = y_io + (int64_t)blockIdx.y * ld + k;
    const float* m = thm + k;
    const float* cc = thc + k;
    float yv[TB], mv[TB], out[TB];
    // forward sweep, x ascending
#pragma unroll
    for (int u = 0; u < TB; ++u) {
        yv[u] = u < L ? y[(int64_t)u * nmodes] : 0.f;
        mv[u] = u < L ? m[(int64_t)u * nmodes] : 0.f;
    }
    float prev = 0.f;
    for (int x0 = 0; x0 < L; x0 += TB) {
#pragma unroll
        for (int u = 0; u < TB; ++u) {
            if (x0 + u < L) prev = (yv[u] * inv_t - l_sub * prev) * mv[u];
            out[u] = prev;
        }
        if (x0 + TB < L) {
#pragma unroll
            for (int u = 0; u < TB; ++u) {
                const int x = x0 + TB + u;
                yv[u] = x < L ? y[(int64_t)x * nmodes] : 0.f;
                mv[u] = x < L ? m[(int64_t)x * nmodes] : 0.f;
            }
        }
#pragma unroll
        for (int u = 0; u < TB; ++u)
            if (x0 + u < L) y[(int64_t)(x0 + u) * nmodes] = out[u];
    }
    // backward sweep, x descending from L - 1 (whose value the forward sweep left final)
    int xb = L - 2;
#pragma unroll
    for (int u = 0; u < TB; ++u) {
        yv[u] = xb - u >= 0 ? y[(int64_t)(xb - u) * nmodes] : 0.f;
        mv[u] = xb - u >= 0 ? cc[(int64_t)(xb - u) * nmodes] : 0.f;
    }
    float next = prev;
    for (; xb >= 0; xb -= TB) {
#pragma unroll
        for (int u = 0; u < TB; ++u) {
            next = yv[u] - mv[u] * next;
            out[u] = next;
        }
        if (xb - TB >= 0) {
#pragma unroll
            for (int u = 0; u < TB; ++u) {
                const int x = xb - TB - u;
                yv[u] = x >= 0 ? y[(int64_t)x * nmodes] : 0.f;
                mv[u] = x >= 0 ? cc[(int64_t)x * nmodes] : 0.f;
            }
        }
#pragma unroll
        for (int u = 0; u < TB; ++u)
            if (xb - u >= 0) y[(int64_t)(xb - u) * nmodes] = out[u];
    }
}

__global__ void k_tridiag_lines32(float* y_io, int64_t ld, int p, int L, int64_t nmodes,
                                  float l_sub, const float* __restrict__ thm,
                                  const float* __restrict__ thc, float inv_t) {
    int seg;
    const int64_t line = seg_line(seg);
    const bool active = line < nmodes * p;
    const int64_t k = active ? line % nmodes : 0;
    const int c = active ? (int)(line / nmodes) : 0;
    float* y = y_io + c * ld + k;
    tridiag_seg<float>(y, y, L, nmodes, k, l_sub, thm, thc, inv_t, seg, active);
}

// Certify mode: partial sums of ||B - (tA - tau_i I) X_i||_F^2 per pole, X_i = Xr + i Xi stored
// as columns [i 2p + c] (real) and [i 2p + p + c] (imaginary) of X.  One partial per CTA and
// pole; the host adds them.
__global__ void k_true_resid(const double* __restrict__ X, int64_t ldx, const double* __restrict__ B,
                             int64_t ldb, int p, int npoles, int ndim, int nx, int ny, int nz, Axis ax0,
                             Axis ax1, Axis ax2, double t, const double* __restrict__ tau_re,
                             const double* __restrict__ tau_im, double* __restrict__ part,
                             const double* __restrict__ AX, int64_t ldax) {
    __shared__ double red[256];
    const int64_t n = (int64_t)nx * ny * nz;
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int pole = blockIdx.y;
    double acc = 0.0;
    if (i < n) {
        const int ix = (int)(i % nx);
        const int iy = (int)((i / nx) % ny);
        const int iz = (int)(i / ((int64_t)nx * ny));
        const double dc = ax0.c + (ndim > 1 ? ax1.c : 0.0) + (ndim > 2 ? ax2.c : 0.0);
        const double tr = tau_re[pole], ti = tau_im[pole];
        for (int c = 0; c < p; ++c) {
            double ax[2];
            for (int part_ = 0; part_ < 2; ++part_) {
                if (AX) {
                    ax[part_] = AX[(int64_t)(2 * pole * p + part_ * p + c) * ldax + i];
                    continue;
                }
                const double* v = X + (int64_t)(2 * pole * p + part_ * p + c) * ldx;
                double s = dc * v[i];
                if (ix > 0) s += ax0.l * v[i - 1];
                if (ix < nx - 1) s += ax0.u * v[i + 1];
                if (ndim > 1) {
                    if (iy > 0) s += ax1.l * v[i - nx];
                    if (iy < ny - 1) s += ax1.u * v[i + nx];
                }
                if (ndim > 2) {
                    const int64_t st = (int64_t)nx * ny;
                    if (iz > 0) s += ax2.l * v[i - st];
                    if (iz < nz - 1) s += ax2.u * v[i + st];
                }
                ax[part_] = t * s;
            }
            const double xr = X[(int64_t)(2 * pole * p + c) * ldx + i];
            const double xi = X[(int64_t)(2 * pole * p + p + c) * ldx + i];
            // (tA - tau)(xr + i xi) = (A xr - tr xr + ti xi) + i (A xi - tr xi - ti xr)
            const double rre = B[(int64_t)c * ldb + i] - (ax[0] - tr * xr + ti * xi);
            const double rim = -(ax[1] - tr * xi - ti * xr);
            acc += rre * rre + rim * rim;
        }
    }
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int st = 128; st > 0; st >>= 1) {
        if (threadIdx.x < st) red[threadIdx.x] += red[threadIdx.x + st];
        __syncthreads();
    }
    if (threadIdx.x == 0) part[(int64_t)pole * gridDim.x + blockIdx.x] = red[0];
}

__global__ void k_d2f(const double* __restrict__ in, float* __restrict__ out, int64_t n) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = (float)in[i];
}

}  // namespace

cudaError_t launch_gemm(const GemmArgs& g, cudaStream_t s) {
    dim3 grid((g.M + BM - 1) / BM, (g.N + BN - 1) / BN, g.nb1 * g.nb2);
    if (g.c_rs == 1) k_gemm<true><<<grid, 256, 0, s>>>(g);
    else k_gemm<false><<<grid, 256, 0, s>>>(g);
    return cudaGetLastError();
}

cudaError_t launch_tridiag_lines(const double* in, int64_t ld_in, double* out, int64_t ld_out,
                                 int p, int L, int64_t nmodes, double l_sub, const double* th_m,
                                 const double* th_c, double inv_t, cudaStream_t s) {
    const int64_t lines = nmodes * p, per_block = 128 / TSEG;
    k_tridiag_lines<<<(unsigned)((lines + per_block - 1) / per_block), 128, 0, s>>>(in, ld_in, out, ld_out, p, L,
                                                                                 nmodes, l_sub, th_m, th_c, inv_t);
    return cudaGetLastError();
}

cudaError_t launch_thomas_setup(double* th_m, double* th_c, int L, int64_t nmodes, double l,
                                double c, double u, const double* lam_y, int Ny,
                                const double* lam_z, int Nz, cudaStream_t s) {
    const int thr = 128;
    k_thomas_setup<<<(unsigned)((nmodes + thr - 1) / thr), thr, 0, s>>>(th_m, th_c, L, nmodes, l, c, u,
                                                                        lam_y, Ny, lam_z, Nz);
    return cudaGetLastError();
}

cudaError_t launch_axis_setup(double* Qf, double* Qi, double* lam, int N, double l, double c,
                              double u, cudaStream_t s) {
    const int64_t tot = (int64_t)N * N;
    k_axis_setup<<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(Qf, Qi, lam, N, l, c, u);
    return cudaGetLastError();
}

static void split_host(double x, float& h, float& l) {
    h = (float)x;
    l = (float)(x - (double)h);
}

cudaError_t launch_cd_apply(const double* V, int64_t ldv, double* W, int64_t ldw, int p,
                            int ndim, int nx, int ny, int nz, const Axis* ax, double t,
                            cudaStream_t s, const double* Y, int64_t ldy, double beta, float* W32, int df) {
    const int64_t n = (int64_t)nx * ny * nz;
    if (n >= ((int64_t)1 << 31)) return cudaErrorInvalidValue;
    if (df) {
        if (Y && beta != 1.0) return cudaErrorInvalidValue;
        StencilDF k;
        split_host(t * (ax[0].c + (ndim > 1 ? ax[1].c : 0.0) + (ndim > 2 ? ax[2].c : 0.0)), k.ch, k.cl);
        for (int d = 0; d < 3; ++d) {
            split_host(t * ax[d].l, k.lh[d], k.ll[d]);
            split_host(t * ax[d].u, k.uh[d], k.ul[d]);
        }
        dim3 grid((unsigned)((n + 255) / 256), p);
        k_cd_apply_df<<<grid, 256, 0, s>>>(V, ldv, W, ldw, ndim, nx, ny, nz, k, Y, ldy, W32);
        return cudaGetLastError();
    }
    StencilT k;
    k.tc = t * (ax[0].c + (ndim > 1 ? ax[1].c : 0.0) + (ndim > 2 ? ax[2].c : 0.0));
    for (int d = 0; d < 3; ++d) {
        k.tl[d] = t * ax[d].l;
        k.tu[d] = t * ax[d].u;
    }
    dim3 grid((unsigned)((n + 255) / 256), p);
    k_cd_apply<<<grid, 256, 0, s>>>(V, ldv, W, ldw, ndim, nx, ny, nz, k, Y, ldy, beta, W32);
    return cudaGetLastError();
}

template <typename TA, typename TC, int NJ>
static void launch_gemm_small_nj(const GemmArgsMixed& g, bool cm, cudaStream_t s) {
    const dim3 grid((unsigned)((g.M + SBM - 1) / SBM), (unsigned)(g.nb1 * g.nb2));
    const size_t shm = gemm_small_smem(g.K, NJ);
    if (cm) k_gemm_small<true, TA, TC, NJ><<<grid, 256, shm, s>>>(g);
    else k_gemm_small<false, TA, TC, NJ><<<grid, 256, shm, s>>>(g);
}

template <typename TA, typename TC>
static void launch_gemm_small_t(const GemmArgsMixed& g, bool cm, cudaStream_t s) {
    const int nj = (g.N + 15) / 16;
    if (nj <= 2) launch_gemm_small_nj<TA, TC, 2>(g, cm, s);
    else if (nj == 3) launch_gemm_small_nj<TA, TC, 3>(g, cm, s);
    else if (nj == 4) launch_gemm_small_nj<TA, TC, 4>(g, cm, s);
    else if (nj == 5) launch_gemm_small_nj<TA, TC, 5>(g, cm, s);
    else launch_gemm_small_nj<TA, TC, 6>(g, cm, s);
}

cudaError_t launch_gemm32(const GemmArgsMixed& g, cudaStream_t s) {
    const bool small = g.K <= SMAX && g.N <= SMAX;
    if (small) {
        const bool cm = (g.c_rs == 1);
        if (g.a_f64 && !g.c_f64) launch_gemm_small_t<double, float>(g, cm, s);
        else if (!g.a_f64 && !g.c_f64) launch_gemm_small_t<float, float>(g, cm, s);
        else if (!g.a_f64 && g.c_f64) launch_gemm_small_t<float, double>(g, cm, s);
        else return cudaErrorInvalidValue;
        return cudaGetLastError();
    }
    dim3 grid((g.M + BM - 1) / BM, (g.N + BN - 1) / BN, g.nb1 * g.nb2);
    const bool cm = (g.c_rs == 1);
    if (g.a_f64 && !g.c_f64) {
        if (cm) k_gemm32<true, double, float><<<grid, 256, 0, s>>>(g);
        else k_gemm32<false, double, float><<<grid, 256, 0, s>>>(g);
    } else if (!g.a_f64 && !g.c_f64) {
        if (cm) k_gemm32<true, float, float><<<grid, 256, 0, s>>>(g);
        else k_gemm32<false, float, float><<<grid, 256, 0, s>>>(g);
    } else if (!g.a_f64 && g.c_f64) {
        if (cm) k_gemm32<true, float, double><<<grid, 256, 0, s>>>(g);
        else k_gemm32<false, float, double><<<grid, 256, 0, s>>>(g);
    } else {
        return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t launch_tridiag_lines32(float* y, int64_t ld, int p, int L, int64_t nmodes, float l_sub,
                                   const float* th_m, const float* th_c, float inv_t,
                                   cudaStream_t s) {
    if (L <= 128 && nmodes >= 1024) {
        const dim3 grid((unsigned)((nmodes + 255) / 256), (unsigned)p);
        k_tridiag_thread32<<<grid, 256, 0, s>>>(y, ld, L, nmodes, l_sub, th_m, th_c, inv_t);
        return cudaGetLastError();
    }
    const size_t shm = tridiag_tile_smem(L);
    if (shm <= kTridiagTileSmemMax) {
        const dim3 grid((unsigned)((nmodes + TK - 1) / TK), (unsigned)p);
        k_tridiag_tile32<<<grid, TK * TSG, shm, s>>>(y, ld, L, nmodes, l_sub, th_m, th_c, inv_t);
        return cudaGetLastError();
    }
    const int64_t lines = nmodes * p, per_block = 128 / TSEG;
    k_tridiag_lines32<<<(unsigned)((lines + per_block - 1) / per_block), 128, 0, s>>>(y, ld, p, L, nmodes, l_sub,
                                                                                   th_m, th_c, inv_t);
    return cudaGetLastError();
}

template <typename TA, typename TC, int NJ>
static cudaError_t set_gemm_small_smem() {
    const int mx = (int)gemm_small_smem(SMAX, NJ);
    cudaError_t e = cudaFuncSetAttribute(k_gemm_small<true, TA, TC, NJ>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_gemm_small<false, TA, TC, NJ>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
    return e;
}

template <typename TA, typename TC>
static cudaError_t set_gemm_small_smem_t() {
    cudaError_t e = set_gemm_small_smem<TA, TC, 2>();
    if (e == cudaSuccess) e = set_gemm_small_smem<TA, TC, 3>();
    if (e == cudaSuccess) e = set_gemm_small_smem<TA, TC, 4>();
    if (e == cudaSuccess) e = set_gemm_small_smem<TA, TC, 5>();
    if (e == cudaSuccess) e = set_gemm_small_smem<TA, TC, 6>();
    return e;
}

cudaError_t operator_set_smem_limits() {
    cudaError_t e = cudaFuncSetAttribute(k_tridiag_tile32, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)kTridiagTileSmemMax);
    if (e == cudaSuccess) e = set_gemm_small_smem_t<double, float>();
    if (e == cudaSuccess) e = set_gemm_small_smem_t<float, float>();
    if (e == cudaSuccess) e = set_gemm_small_smem_t<float, double>();
    return e;
}

int true_resid_blocks(int64_t n) { return (int)((n + 255) / 256); }

cudaError_t launch_true_resid(const double* X, int64_t ldx, const double* B, int64_t ldb, int p, int npoles,
                              int ndim, int nx, int ny, int nz, const Axis* ax, double t, const double* tau_re,
                              const double* tau_im, double* part, cudaStream_t s, const double* AX,
                              int64_t ldax) {
    const int64_t n = (int64_t)nx * ny * nz;
    dim3 grid((unsigned)true_resid_blocks(n), npoles);
    k_true_resid<<<grid, 256, 0, s>>>(X, ldx, B, ldb, p, npoles, ndim, nx, ny, nz, ax[0], ax[1], ax[2], t,
                                      tau_re, tau_im, part, AX, ldax);
    return cudaGetLastError();
}

cudaError_t launch_d2f(const double* in, float* out, int64_t n, cudaStream_t s) {
    k_d2f<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(in, out, n);
    return cudaGetLastError();
}

}  // namespace expm
