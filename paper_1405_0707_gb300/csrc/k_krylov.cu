// k_krylov.cu -- block Arnoldi pieces (Section 3, eq. (2.1); Section 4.1, eq. (4.5)).
//
// One block step turns W = (tA)^{-1} V_j into V_{j+1}:
//   block classical Gram-Schmidt, twice (CGS2):  h = V^T W,  W -= V h   (x2, h summed
//   into H), then a Cholesky QR of W with a shifted first pass (three passes in all:
//   G = W^T W (+ shift on pass 1), G = R^T R, W <- W R^{-1}); the product of the three
//   R factors is H_{j+1,j}, upper triangular with a positive diagonal, so the basis is
//   the one Ruhe's vector-wise variant builds in exact arithmetic.
//
// The tall-skinny passes split the n rows over `nblk` CTAs; each CTA stages 16-row tiles
// of V and W in shared memory, and writes one partial (cols x p) product per CTA.  A
// second tiny launch sums the partials in a fixed order (deterministic), so the
// projections need no atomics.  The update of pass 1 is fused with the projection of
// pass 2, and the update of pass 2 with the Gram matrix of the QR, so V_j is read three
// times per block step instead of four.
#include "df.cuh"
#include "internal.h"
#include "rows_api.h"
#include "rows_common.cuh"

namespace expm {
namespace {

constexpr int NT = 256;     // threads per CTA for the row passes

// Load a TR x cols tile of column-major X (rows r0.., ld) into S[rr * cs + a], zero-filled,
// converted to the tile's element type.
template <typename T>
__device__ inline void load_tile(const double* __restrict__ X, int64_t ld, int cols, int64_t r0,
                                 int tr, T* S, int cs) {
    const int total = TR * cols;
    for (int e0 = threadIdx.x; e0 < total; e0 += LB * blockDim.x) {
        double v[LB];
#pragma unroll
        for (int k = 0; k < LB; ++k) {
            const int e = e0 + k * blockDim.x;
            const int rr = e % TR, a = e / TR;
            v[k] = (e < total && rr < tr) ? X[(int64_t)a * ld + r0 + rr] : 0.0;
        }
#pragma unroll
        for (int k = 0; k < LB; ++k) {
            const int e = e0 + k * blockDim.x;
            if (e < total) S[(e % TR) * cs + e / TR] = (T)v[k];
        }
    }
}

// Gram partial of a TR x p tile X (row-major X[rr * p + c]), upper triangle only (the
// Cholesky factorisation reads nothing else).  With p^2 <= NT every output gets NT / p^2
// threads that take every (NT / p^2)-th row, so the dependent chains are short; gram_write
// adds the stripes in a fixed order.  With p^2 > NT each thread owns whole outputs.
template <int OPT>
__device__ inline void gram_accumulate(const double* X, int p, int nout, double* acc) {
    if (nout <= NT) {
        const int stripes = NT / nout, o = threadIdx.x % nout, st = threadIdx.x / nout;
        const int c1 = o / p, c2 = o % p;
        if (st < stripes && c1 <= c2) {
            double s = 0.0;
            for (int rr = st; rr < TR; rr += stripes) s = fma(X[rr * p + c1], X[rr * p + c2], s);
            acc[0] += s;
        }
        return;
    }
#pragma unroll
    for (int q = 0; q < OPT; ++q) {
        const int o = threadIdx.x + q * NT;
        if (o < nout) {
            const int c1 = o / p, c2 = o % p;
            if (c1 <= c2) {
                double s = 0.0;
#pragma unroll
                for (int rr = 0; rr < TR; ++rr) s = fma(X[rr * p + c1], X[rr * p + c2], s);
                acc[q] += s;
            }
        }
    }
}

template <int OPT>
__device__ inline void gram_write(const double* acc, int p, int nout, double* __restrict__ part) {
    if (nout <= NT) {
        __shared__ double red[NT];
        const int stripes = NT / nout;
        red[threadIdx.x] = acc[0];
        __syncthreads();
        if (threadIdx.x < nout) {
            double s = 0.0;
            for (int k = 0; k < stripes; ++k) s += red[k * nout + threadIdx.x];
            part[(int64_t)blockIdx.x * nout + threadIdx.x] = s;
        }
        return;
    }
#pragma unroll
    for (int q = 0; q < OPT; ++q) {
        const int o = threadIdx.x + q * NT;
        if (o < nout) part[(int64_t)blockIdx.x * nout + o] = acc[q];
    }
}

// partial[blk][a][c] = sum_{rows of blk} V[r, a] W[r, c]      (a < cols, c < p)
// T = float: FP32 products over each 16-row tile (the mixed path's projections; only the
// FP64 updates must be exact for the Arnoldi relation), FP64 accumulation across tiles.
// Tiles of trp rows (64 when the tiles fit in 100 KB of shared memory, else 32 or 16): more
// loads in flight per barrier round than the 16-row tiles of the update kernels (the
// projection's own arithmetic is small).
template <typename T>
__device__ inline void load_tile_p(const double* __restrict__ X, int64_t ld, int cols, int64_t r0,
                                   int tr, T* S, int cs, int trp) {
    const int total = trp * cols;
    for (int e0 = threadIdx.x; e0 < total; e0 += LB * blockDim.x) {
        double v[LB];
#pragma unroll
        for (int k = 0; k < LB; ++k) {
            const int e = e0 + k * blockDim.x;
            const int rr = e % trp, a = e / trp;
            v[k] = (e < total && rr < tr) ? X[(int64_t)a * ld + r0 + rr] : 0.0;
        }
#pragma unroll
        for (int k = 0; k < LB; ++k) {
            const int e = e0 + k * blockDim.x;
            if (e < total) S[(e % trp) * cs + e / trp] = (T)v[k];
        }
    }
}

template <int OPT, typename T>
__global__ void __launch_bounds__(NT) k_proj(const double* __restrict__ V, int64_t ldv, int cols,
                                             const double* __restrict__ W, int64_t ldw, int p,
                                             int64_t n, int64_t rpb, double* __restrict__ part, int TRP) {
    extern __shared__ double sm[];
    const int cs = cols | 1;
    T* Vs = reinterpret_cast<T*>(sm);
    T* Ws = Vs + TRP * cs;
    const int nout = cols * p;
    double acc[OPT];
#pragma unroll
    for (int q = 0; q < OPT; ++q) acc[q] = 0.0;
    const int64_t rb = rows_begin(rpb), re = min(n, rb + rpb);
    for (int64_t r0 = rb; r0 < re; r0 += TRP) {
        const int tr = (int)min((int64_t)TRP, re - r0);
        load_tile_p(V, ldv, cols, r0, tr, Vs, cs, TRP);
        load_tile_p(W, ldw, p, r0, tr, Ws, p, TRP);
        __syncthreads();
#pragma unroll
        for (int q = 0; q < OPT; ++q) {
            const int o = threadIdx.x + q * NT;
            if (o < nout) {
                const int a = o / p, c = o % p;
                T s0 = 0, s1 = 0;
#pragma unroll 8
                for (int rr = 0; rr < TRP; rr += 2) {
                    s0 = fma(Vs[rr * cs + a], Ws[rr * p + c], s0);
                    s1 = fma(Vs[(rr + 1) * cs + a], Ws[(rr + 1) * p + c], s1);
                }
                acc[q] += (double)s0 + (double)s1;
            }
        }
        __syncthreads();
    }
#pragma unroll
    for (int q = 0; q < OPT; ++q) {
        const int o = threadIdx.x + q * NT;
        if (o < nout) part[(int64_t)blockIdx.x * nout + o] = acc[q];
    }
}

// Sum of the nblk partials of output o, split over `stripes` threads (stripe s takes
// b = s, s + stripes, ...) with eight independent accumulators, so eight loads are in flight
// per thread; the caller adds the stripes in a fixed order, so the result does not depend on
// scheduling.
__device__ inline double stripe_sum(const double* __restrict__ part, int nblk, int nout, int o,
                                    int s, int stripes) {
    double a[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) a[k] = 0.0;
    int b = s;
    for (; b + 7 * stripes < nblk; b += 8 * stripes) {
#pragma unroll
        for (int k = 0; k < 8; ++k) a[k] += part[(int64_t)(b + k * stripes) * nout + o];
    }
    for (; b < nblk; b += stripes) a[0] += part[(int64_t)b * nout + o];
    return ((a[0] + a[1]) + (a[2] + a[3])) + ((a[4] + a[5]) + (a[6] + a[7]));
}

constexpr int RED_OUT = 4;        // outputs per reduction CTA
constexpr int RED_STRIPES = 64;   // threads per output

// h[o] = sum_b part[b][o]; H[row0 + a, col0 + c] (+)= h[a][c].  CTA = 4 outputs x 64 stripes;
// the stripes are added in two fixed-order levels (8 groups of 8, then the 8 groups).
__global__ void __launch_bounds__(RED_OUT * RED_STRIPES)
k_reduce_h(const double* __restrict__ part, int nblk, int cols, int p, double* __restrict__ h,
           double* H, int ldH, int row0, int col0, int accumulate, int hcols) {
    __shared__ double red[RED_STRIPES][RED_OUT];
    __shared__ double red2[8][RED_OUT];
    const int nout = cols * p;
    const int ol = threadIdx.x % RED_OUT, st = threadIdx.x / RED_OUT;
    const int o = blockIdx.x * RED_OUT + ol;
    red[st][ol] = (o < nout) ? stripe_sum(part, nblk, nout, o, st, RED_STRIPES) : 0.0;
    __syncthreads();
    if (st < 8) {
        double g = 0.0;
#pragma unroll
        for (int k = 0; k < 8; ++k) g += red[st * 8 + k][ol];
        red2[st][ol] = g;
    }
    __syncthreads();
    if (st != 0 || o >= nout) return;
    const double s = ((red2[0][ol] + red2[1][ol]) + (red2[2][ol] + red2[3][ol])) +
                     ((red2[4][ol] + red2[5][ol]) + (red2[6][ol] + red2[7][ol]));
    h[o] = s;
    if (H && o < hcols * p) {
        const int a = o / p, c = o % p;
        double* dst = H + (int64_t)(col0 + c) * ldH + row0 + a;
        *dst = accumulate ? *dst + s : s;
    }
}

// W <- W - V h (FP64: keeps the Arnoldi relation exact); then partial of V^T W (gram = 0)
// or W^T W (gram = 1).  F32: the projection's products in FP32 on FP32 copies of the tiles.
// UPD32 (mixed path, second CGS pass, gram = 1): the correction V h in FP32 on FP32 copies,
// subtracted from the FP64 W (see k_update_gram_rows).
template <int OPT, bool F32, bool UPD32 = false>
__global__ void __launch_bounds__(NT) k_update(const double* __restrict__ V, int64_t ldv, int cols,
                                               double* __restrict__ W, int64_t ldw, int p,
                                               int64_t n, int64_t rpb,
                                               const double* __restrict__ h,
                                               double* __restrict__ part, int gram) {
    extern __shared__ double sm[];
    const int cs = cols | 1;
    double* hs = sm;                      // cols x p
    double* Vs = hs + cols * p;           // TR x cs
    double* Ws = Vs + TR * cs;            // TR x p
    float* Vf = reinterpret_cast<float*>(Ws + TR * p);   // F32 copies (TR x cs, TR x p)
    float* Wf = Vf + TR * cs;
    float* hf = Wf + TR * p;              // UPD32: FP32 copy of h (cols x p)
    for (int e = threadIdx.x; e < cols * p; e += blockDim.x) {
        hs[e] = h[e];
        if (UPD32) hf[e] = (float)h[e];
    }
    const int nout = gram ? p * p : cols * p;
    double acc[OPT];
#pragma unroll
    for (int q = 0; q < OPT; ++q) acc[q] = 0.0;
    const int64_t rb = rows_begin(rpb), re = min(n, rb + rpb);
    for (int64_t r0 = rb; r0 < re; r0 += TR) {
        const int tr = (int)min((int64_t)TR, re - r0);
        if (UPD32) load_tile(V, ldv, cols, r0, tr, Vf, cs);
        else load_tile(V, ldv, cols, r0, tr, Vs, cs);
        load_tile(W, ldw, p, r0, tr, Ws, p);
        __syncthreads();
        for (int e = threadIdx.x; e < TR * p; e += blockDim.x) {
            const int rr = e % TR, c = e / TR;
            double w = Ws[rr * p + c];
            if (UPD32) {
                float corr = 0.f;
                for (int a = 0; a < cols; ++a) corr = fmaf(Vf[rr * cs + a], hf[a * p + c], corr);
                w -= (double)corr;
            } else {
                for (int a = 0; a < cols; ++a) w = fma(-Vs[rr * cs + a], hs[a * p + c], w);
            }
            Ws[rr * p + c] = w;
            if (F32) Wf[rr * p + c] = (float)w;
            if (rr < tr) W[(int64_t)c * ldw + r0 + rr] = w;
        }
        if (F32 && !gram)
            for (int e = threadIdx.x; e < TR * cols; e += blockDim.x) {
                const int rr = e % TR, a = e / TR;
                Vf[rr * cs + a] = (float)Vs[rr * cs + a];
            }
        __syncthreads();
        if (gram) gram_accumulate<OPT>(Ws, p, nout, acc);
        else
#pragma unroll
        for (int q = 0; q < OPT; ++q) {
            const int o = threadIdx.x + q * NT;
            if (o < nout) {
                double s = 0.0;
                if (gram) {
                    // handled below by gram_accumulate
                } else if (F32) {
                    const int a = o / p, c = o % p;
                    float sf = 0.f;
#pragma unroll
                    for (int rr = 0; rr < TR; ++rr) sf = fmaf(Vf[rr * cs + a], Wf[rr * p + c], sf);
                    s = (double)sf;
                } else {
                    const int a = o / p, c = o % p;
#pragma unroll
                    for (int rr = 0; rr < TR; ++rr) s = fma(Vs[rr * cs + a], Ws[rr * p + c], s);
                }
                acc[q] += s;
            }
        }
        __syncthreads();
    }
    if (gram) {
        gram_write<OPT>(acc, p, nout, part);
        return;
    }
#pragma unroll
    for (int q = 0; q < OPT; ++q) {
        const int o = threadIdx.x + q * NT;
        if (o < nout) part[(int64_t)blockIdx.x * nout + o] = acc[q];
    }
}

// W <- W - V h with V h formed in double-float arithmetic on the FP32 pipe (mixed path, first
// CGS pass), then the FP32 partials of V^T W for the second pass.  Each product
// v h = vh hh + (err(vh hh) + vh hl + vl hh) with the FP32 product error recovered by an FMA;
// the large parts are accumulated with TwoSum, the small ones in FP32, and W is updated in
// FP64 by the pair's value.  Relative error ~ cols 2^-48 of |V h|, which keeps the Arnoldi
// relation exact far below the accuracy the mixed path delivers.  The work items (row, column)
// of a tile are split over S = NT / (TR p) threads each when that is more than one; their
// partial pairs are combined in a fixed order.
template <int OPT>
__global__ void __launch_bounds__(NT) k_update_df(const double* __restrict__ V, int64_t ldv, int cols,
                                                  double* __restrict__ W, int64_t ldw, int p, int64_t n,
                                                  int64_t rpb, const double* __restrict__ h,
                                                  double* __restrict__ part) {
    extern __shared__ double sm[];
    const int cs = cols | 1;
    float* hh = reinterpret_cast<float*>(sm);       // cols x p
    float* hl = hh + cols * p;
    float* Vh = hl + cols * p;                      // TR x cs
    float* Vl = Vh + TR * cs;
    float* Wf = Vl + TR * cs;                       // TR x p
    float* cmb = Wf + TR * p;                       // 2 NT
    for (int e = threadIdx.x; e < cols * p; e += blockDim.x) split_df(h[e], hh[e], hl[e]);
    const int nitems = TR * p;
    const int S = nitems >= NT ? 1 : NT / nitems;
    const int nout = cols * p;
    double acc[OPT];
#pragma unroll
    for (int q = 0; q < OPT; ++q) acc[q] = 0.0;
    const int64_t rb = rows_begin(rpb), re = min(n, rb + rpb);
    for (int64_t r0 = rb; r0 < re; r0 += TR) {
        const int tr = (int)min((int64_t)TR, re - r0);
        for (int e0 = threadIdx.x; e0 < TR * cols; e0 += LB * blockDim.x) {
            double v[LB];
#pragma unroll
            for (int k = 0; k < LB; ++k) {
                const int e = e0 + k * blockDim.x;
                const int rr = e % TR, a = e / TR;
                v[k] = (e < TR * cols && rr < tr) ? V[(int64_t)a * ldv + r0 + rr] : 0.0;
            }
#pragma unroll
            for (int k = 0; k < LB; ++k) {
                const int e = e0 + k * blockDim.x;
                if (e < TR * cols) {
                    float vh, vl;
                    split_df(v[k], vh, vl);
                    Vh[(e % TR) * cs + e / TR] = vh;
                    Vl[(e % TR) * cs + e / TR] = vl;
                }
            }
        }
        __syncthreads();
        for (int it = threadIdx.x; it < S * nitems; it += blockDim.x) {
            const int item = it % nitems, seg = it / nitems;
            const int rr = item % TR, c = item / TR;
            float sh = 0.f, sc = 0.f;
            for (int a = seg; a < cols; a += S) {
                const float vh = Vh[rr * cs + a], vl = Vl[rr * cs + a];
                const float h1 = hh[a * p + c], h2 = hl[a * p + c];
                const float pr = vh * h1;
                float t = fmaf(vh, h1, -pr);
                t = fmaf(vl, h1, t);
                t = fmaf(vh, h2, t);
                df_add(sh, sc, pr);
                sc += t;
            }
            if (S > 1) {
                cmb[2 * it] = sh;
                cmb[2 * it + 1] = sc;
            } else {
                double w = 0.0;
                if (rr < tr) {
                    w = W[(int64_t)c * ldw + r0 + rr] - ((double)sh + (double)sc);
                    W[(int64_t)c * ldw + r0 + rr] = w;
                }
                Wf[rr * p + c] = (float)w;
            }
        }
        if (S > 1) {
            __syncthreads();
            for (int item = threadIdx.x; item < nitems; item += blockDim.x) {
                const int rr = item % TR, c = item / TR;
                float sh = cmb[2 * item], sc = cmb[2 * item + 1];
                for (int sg = 1; sg < S; ++sg) {
                    df_add(sh, sc, cmb[2 * (sg * nitems + item)]);
                    sc += cmb[2 * (sg * nitems + item) + 1];
                }
                double w = 0.0;
                if (rr < tr) {
                    w = W[(int64_t)c * ldw + r0 + rr] - ((double)sh + (double)sc);
                    W[(int64_t)c * ldw + r0 + rr] = w;
                }
                Wf[rr * p + c] = (float)w;
            }
        }
        __syncthreads();
#pragma unroll
        for (int q = 0; q < OPT; ++q) {
            const int o = threadIdx.x + q * NT;
            if (o < nout) {
                const int a = o / p, c = o % p;
                float sf = 0.f;
#pragma unroll
                for (int rr = 0; rr < TR; ++rr) sf = fmaf(Vh[rr * cs + a], Wf[rr * p + c], sf);
                acc[q] += (double)sf;
            }
        }
        __syncthreads();
    }
#pragma unroll
    for (int q = 0; q < OPT; ++q) {
        const int o = threadIdx.x + q * NT;
        if (o < nout) part[(int64_t)blockIdx.x * nout + o] = acc[q];
    }
}

// Cholesky-QR factor step, one CTA.  G = sum of the p x p partials (all CHOL_T threads),
// then one warp factorises.  Pass modes (the QR of a block runs 3 passes, the third only
// when needed; the decision is made on the device so a captured graph stays valid):
//   mode 0: unshifted Cholesky of G; if a pivot is not positive or the smallest pivot is
//           below 1e-10 of the largest diagonal entry (kappa(W) above ~1e5) it is redone
//           with the shift shift_rel * trace(G) and extra[0] = 1 requests a third pass,
//           else extra[0] = 0.  Rtot = R.
//   mode 1: Rtot = R Rtot; the last pass when extra[0] == 0.
//   mode 2: returns at once when extra[0] == 0; else Rtot = R Rtot, the last pass.
// The last pass writes Rtot into H (rows hrow.., cols hcol..) when H is given and checks
// for breakdown against the column norms of W before orthogonalisation.  Breakdown (the
// block Krylov space is invariant up to rounding) only sets flags[1] for the caller's
// information: the new block is then orthonormalised rounding noise coupled to the basis
// through an entry of H below 1e-14 relative, which leaves the projected solutions
// unchanged to that order (the paper is silent on breakdown).  Columns that are exactly zero
// on entry (a zero right-hand side column, or the image of one) get zero rows in R and stay
// zero, so such blocks pass through without a division by zero.
constexpr int CHOL_T = 1024;
__global__ void __launch_bounds__(CHOL_T) k_chol(const double* __restrict__ part, int nblk, int p,
                                                 double shift_rel, double* R, double* Rinv,
                                                 double* Rtot, int mode, double* H, int ldH,
                                                 int hrow, int hcol, double* normsq_out, int* flags) {
    int* extra = flags + 2;
    if (mode == 2 && *extra == 0) return;
    __shared__ double G[kMaxP * kMaxP], G0[kMaxP * kMaxP], Rs[kMaxP * kMaxP], Ri[kMaxP * kMaxP],
        Rt[kMaxP * kMaxP];
    __shared__ double red[CHOL_T];
    __shared__ double rdiag[kMaxP];
    __shared__ int bad, ill;
    const int pp = p * p;
    {
        const int stripes = pp >= CHOL_T ? 1 : CHOL_T / pp;
        for (int base = 0; base < pp; base += CHOL_T / stripes) {
            const int ol = threadIdx.x % (CHOL_T / stripes), st = threadIdx.x / (CHOL_T / stripes);
            const int o = base + ol;
            red[threadIdx.x] = (o < pp && st < stripes) ? stripe_sum(part, nblk, pp, o, st, stripes) : 0.0;
            __syncthreads();
            if (st == 0 && o < pp) {
                double s = 0.0;
                for (int k = 0; k < stripes; ++k) s += red[k * (CHOL_T / stripes) + ol];
                G0[o] = s;
            }
            __syncthreads();
        }
    }
    const bool last = (mode == 1 && *extra == 0) || mode == 2;
    __shared__ double hn2[kMaxP];
    if (H && last) {
        const int stripes = CHOL_T / p;
        const int c = threadIdx.x % p, st = threadIdx.x / p;
        double v2 = 0.0;
        if (st < stripes)
            for (int a = st; a < hrow; a += stripes) {
                const double v = H[(int64_t)(hcol + c) * ldH + a];
                v2 += v * v;
            }
        red[threadIdx.x] = v2;
        __syncthreads();
        if (threadIdx.x < p) {
            double s2 = 0.0;
            for (int k = 0; k < stripes; ++k) s2 += red[k * p + threadIdx.x];
            hn2[threadIdx.x] = s2;
        }
        __syncthreads();
    }
    if (threadIdx.x >= 32) return;
    const int lane = threadIdx.x;
    if (lane == 0) { bad = 0; ill = 0; }
    double tr = 0.0, dmax = 0.0;
    for (int c = 0; c < p; ++c) {
        tr += G0[c * p + c];
        dmax = fmax(dmax, G0[c * p + c]);
    }
    if (normsq_out && lane == 0 && mode == 0) *normsq_out = tr;
    for (int attempt = 0; attempt < 2; ++attempt) {
        const double shift = (attempt == 1) ? shift_rel * tr : 0.0;
        for (int o = lane; o < pp; o += 32) {
            G[o] = G0[o] + ((o / p == o % p) ? shift : 0.0);
            Rs[o] = 0.0;
            Ri[o] = 0.0;
        }
        __syncwarp();
        // right-looking upper Cholesky G = R^T R (upper part), one reciprocal per pivot
        for (int j = 0; j < p; ++j) {
            if (lane == 0) {
                double d = G[j * p + j];
                if (G0[j * p + j] == 0.0) {
                    // an exactly zero column (an invariant subspace reached earlier): R row j
                    // and R^{-1} row and column j stay zero, so the column stays zero
                    Rs[j * p + j] = 0.0;
                    rdiag[j] = 0.0;
                } else {
                    if (!(d > 0.0) || !isfinite(d) || (mode == 0 && attempt == 0 && d < 1e-10 * dmax)) ill = 1;
                    if (!(d > 0.0) || !isfinite(d)) d = 1.0;
                    const double rj = sqrt(d);
                    Rs[j * p + j] = rj;
                    rdiag[j] = 1.0 / rj;
                }
            }
            __syncwarp();
            const double inv = rdiag[j];
            if (lane > j && lane < p) Rs[j * p + lane] = G[j * p + lane] * inv;
            __syncwarp();
            if (lane > j && lane < p) {
                const double rb = Rs[j * p + lane];
                for (int a = j + 1; a <= lane; ++a) G[a * p + lane] -= Rs[j * p + a] * rb;
            }
            __syncwarp();
        }
        if (mode != 0 || attempt == 1 || !ill) break;   // mode 0 retries with the shift
        __syncwarp();
    }
    if (mode == 0 && lane == 0) *extra = ill;
    if (mode != 0 && lane == 0 && ill) bad = 1;       // a later pass must factor cleanly
    __syncwarp();
    // inverse of the upper triangular R, column `lane` (reciprocal pivots, no division)
    if (lane < p) {
        const int c = lane;
        Ri[c * p + c] = rdiag[c];
        for (int r = c - 1; r >= 0; --r) {
            double s = 0.0;
            for (int k = r + 1; k <= c; ++k) s = fma(Rs[r * p + k], Ri[k * p + c], s);
            Ri[r * p + c] = -s * rdiag[r];
        }
    }
    __syncwarp();
    // Rtot = R * Rtot_old (upper triangular product), column `lane`
    if (lane < p) {
        const int c = lane;
        for (int r = 0; r < p; ++r) {
            double s;
            if (mode == 0) s = Rs[r * p + c];
            else {
                s = 0.0;
                for (int k = r; k <= c; ++k) s = fma(Rs[r * p + k], Rtot[k * p + c], s);
            }
            Rt[r * p + c] = (r <= c) ? s : 0.0;
        }
    }
    __syncwarp();
    for (int o = lane; o < pp; o += 32) {
        R[o] = Rs[o];
        Rinv[o] = Ri[o];
        Rtot[o] = Rt[o];
        if (!isfinite(Rt[o])) bad = 1;
    }
    __syncwarp();
    if (H && last) {
        for (int o = lane; o < pp; o += 32) {
            const int a = o / p, c = o % p;
            H[(int64_t)(hcol + c) * ldH + hrow + a] = Rt[o];
        }
        if (lane < p) {
            const int c = lane;
            double n0 = hn2[c];
            for (int a = 0; a <= c; ++a) n0 += Rt[a * p + c] * Rt[a * p + c];
            if (Rt[c * p + c] <= 1e-14 * sqrt(n0)) atomicOr(&flags[1], 1);
        }
    }
    __syncwarp();
    if (lane == 0 && bad) atomicOr(&flags[0], 1);
}

// W_out = W R^{-1} (row by row); gram: also partial of W_out^T W_out.
template <int OPT>
__global__ void __launch_bounds__(NT) k_trsm(double* W, int64_t ldw, int p, int64_t n,
                                             int64_t rpb, const double* __restrict__ Rinv,
                                             double* out_, int64_t ldo_,
                                             double* __restrict__ part, int gram_,
                                             const int* extra, int tmode) {
    const TrsmPass ps = trsm_pass(W, ldw, out_, ldo_, gram_, extra, tmode);
    if (ps.skip) return;
    double* out = ps.dest;
    const int64_t ldo = ps.ldd;
    const int gram = ps.gram;
    __shared__ double Ri[kMaxP * kMaxP];
    __shared__ double Ws[TR * kMaxP], Wn[TR * kMaxP];
    for (int e = threadIdx.x; e < p * p; e += blockDim.x) Ri[e] = Rinv[e];
    const int nout = p * p;
    double acc[OPT];
#pragma unroll
    for (int q = 0; q < OPT; ++q) acc[q] = 0.0;
    const int64_t rb = rows_begin(rpb), re = min(n, rb + rpb);
    for (int64_t r0 = rb; r0 < re; r0 += TR) {
        const int tr = (int)min((int64_t)TR, re - r0);
        load_tile(W, ldw, p, r0, tr, Ws, p);
        __syncthreads();
        for (int e = threadIdx.x; e < TR * p; e += blockDim.x) {
            const int rr = e % TR, c = e / TR;
            double s = 0.0;
            for (int a = 0; a <= c; ++a) s = fma(Ws[rr * p + a], Ri[a * p + c], s);
            Wn[rr * p + c] = s;
            if (rr < tr) out[(int64_t)c * ldo + r0 + rr] = s;
        }
        __syncthreads();
        if (gram) gram_accumulate<OPT>(Wn, p, nout, acc);
        __syncthreads();
    }
    if (gram) gram_write<OPT>(acc, p, nout, part);
}


// Z[r, c] += sum_{a < cols} V[r, a] Wc[a][c]; restart: V[:, 0:p] <- V[:, cols-p:cols].
__global__ void __launch_bounds__(NT) k_update_z(double* __restrict__ V, int64_t ldv, int cols,
                                                 int p, int64_t n, int64_t rpb,
                                                 const double* __restrict__ Wc,
                                                 double* __restrict__ Z, int64_t ldz,
                                                 int restart_copy) {
    extern __shared__ double sm[];
    const int cs = cols | 1;
    double* ws = sm;                 // cols x p
    double* Vs = ws + cols * p;      // TR x cs
    for (int e = threadIdx.x; e < cols * p; e += blockDim.x) ws[e] = Wc[e];
    const int64_t rb = rows_begin(rpb), re = min(n, rb + rpb);
    for (int64_t r0 = rb; r0 < re; r0 += TR) {
        const int tr = (int)min((int64_t)TR, re - r0);
        load_tile(V, ldv, cols, r0, tr, Vs, cs);
        __syncthreads();
        for (int e = threadIdx.x; e < TR * p; e += blockDim.x) {
            const int rr = e % TR, c = e / TR;
            if (rr < tr) {
                double s = 0.0;
                for (int a = 0; a < cols; ++a) s = fma(Vs[rr * cs + a], ws[a * p + c], s);
                Z[(int64_t)c * ldz + r0 + rr] += s;
                if (restart_copy) V[(int64_t)c * ldv + r0 + rr] = Vs[rr * cs + cols - p + c];
            }
        }
        __syncthreads();
    }
}

__global__ void k_combine(const double* __restrict__ slots, int npoles, int nout,
                          double* __restrict__ Wc) {
    const int o = blockIdx.x * blockDim.x + threadIdx.x;
    if (o >= nout) return;
    double s = 0.0;
    for (int i = 0; i < npoles; ++i) s += slots[(int64_t)i * nout + o];
    Wc[o] = s;
}

// S_i = R for every pole (R_alt instead when *use_alt != 0: the QR's third pass ran)
__global__ void k_init_S(const double* __restrict__ R, int p, int npoles, double* __restrict__ S,
                         const double* __restrict__ R_alt, const int* use_alt) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= npoles * p * p) return;
    const double* src = (R_alt && *use_alt) ? R_alt : R;
    S[2 * e] = src[e % (p * p)];
    S[2 * e + 1] = 0.0;
}

__global__ void k_axpby(double a, const double* __restrict__ X, int64_t ldx, double b,
                        const double* __restrict__ Y, int64_t ldy, double* __restrict__ out,
                        int64_t ldo, int64_t n) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int c = blockIdx.y;
    if (i >= n) return;
    const double y = Y ? Y[c * ldy + i] : 0.0;
    out[c * ldo + i] = a * X[c * ldx + i] + b * y;
}

__global__ void k_zero(double* __restrict__ X, int64_t ldx, int64_t n) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) X[blockIdx.y * ldx + i] = 0.0;
}


}  // namespace

// A CTA count that the row-pass launchers reproduce exactly (rows per CTA are rounded up
// to whole tiles, which can lower the count); every partial-sum reduction uses it.
int consistent_blocks(int64_t n, int requested) {
    int nb = requested < 1 ? 1 : requested;
    for (int it = 0; it < 64; ++it) {
        const int g = blocks_for(n, nb);
        if (g == nb) break;
        nb = g;
    }
    return nb;
}

#define EXPM_OPT_DISPATCH(NOUT, CALL)                  \
    do {                                               \
        const int need_ = ((NOUT) + NT - 1) / NT;      \
        if (need_ <= 1) { constexpr int O = 1; CALL; } \
        else if (need_ <= 4) { constexpr int O = 4; CALL; } \
        else if (need_ <= 16) { constexpr int O = 16; CALL; } \
        else if (need_ <= 64) { constexpr int O = 64; CALL; } \
        else return cudaErrorInvalidValue;             \
    } while (0)

cudaError_t launch_proj_partial(const double* V, int64_t ldv, int cols, const double* W,
                                int64_t ldw, int p, int64_t n, double* part, int nblk,
                                cudaStream_t s, int f32) {
    const int64_t rpb = rows_per_block(n, nblk);
    const int g = blocks_for(n, nblk);
    const size_t esz = f32 ? sizeof(float) : sizeof(double);
    int trp = 64;
    while (trp > TR && esz * trp * ((cols | 1) + p) > 100 * 1024) trp /= 2;
    const size_t shm = esz * trp * ((cols | 1) + p);
    if (f32)
        EXPM_OPT_DISPATCH(cols * p, (k_proj<O, float><<<g, NT, shm, s>>>(V, ldv, cols, W, ldw, p, n, rpb, part, trp)));
    else
        EXPM_OPT_DISPATCH(cols * p, (k_proj<O, double><<<g, NT, shm, s>>>(V, ldv, cols, W, ldw, p, n, rpb, part,
                                                                         trp)));
    return cudaGetLastError();
}

cudaError_t launch_reduce_h(const double* part, int nblk_req, int cols, int p, double* h,
                            double* H, int ldH, int row0, int col0, int accumulate,
                            cudaStream_t s, int hcols) {
    const int nout = cols * p;
    k_reduce_h<<<(nout + RED_OUT - 1) / RED_OUT, RED_OUT * RED_STRIPES, 0, s>>>(
        part, nblk_req, cols, p, h, H, ldH, row0, col0, accumulate, hcols < 0 ? cols : hcols);
    return cudaGetLastError();
}

// The first CGS pass of the mixed path by the row-chunk kernels (k_cgs_rows, p <= 16, in the
// width-specific translation units): used when the projection outputs per thread and the
// staged chunk fit.
bool cgs_rows_fit(int cols, int p) {
    if (p < 1 || p > kRowsMaxP) return false;
    return EXPM_ROWS_CALL(p, cgs_fit(cols, p));
}

cudaError_t launch_cgs_rows(int upd, const double* V, int64_t ldv, int cols, double* W, int64_t ldw, int p,
                            int64_t n, const double* h, double* part, int nblk, int gram, cudaStream_t s) {
    if (p < 1 || p > kRowsMaxP) return cudaErrorInvalidValue;
    return EXPM_ROWS_CALL(p, cgs(upd, V, ldv, cols, W, ldw, p, n, h, part, nblk, gram, s));
}

cudaError_t launch_qr_mixed_rows(double* W, int64_t ldw, int p, int64_t n, int nblk, double* G, double* part,
                                 unsigned* ctr, int mode, double* R, double* Rinv, const double* Rtot_in,
                                 double* Rtot_out, double* H, int ldH, int hrow, int hcol, double* normsq_out,
                                 int* flags, double* out, int64_t ldo, cudaStream_t s, const double* Vc,
                                 int64_t ldvc, int ccols, const double* h2, double* fin, int64_t ldfin) {
    if (p < 1 || p > kRowsMaxP) return cudaErrorInvalidValue;
    return EXPM_ROWS_CALL(p, qr(W, ldw, p, n, nblk, G, part, ctr, mode, R, Rinv, Rtot_in, Rtot_out, H, ldH, hrow,
                                hcol, normsq_out, flags, out, ldo, s, Vc, ldvc, ccols, h2, fin, ldfin));
}

cudaError_t launch_update_proj(const double* V, int64_t ldv, int cols, double* W, int64_t ldw,
                               int p, int64_t n, const double* h, double* part, int nblk,
                               int gram, cudaStream_t s, int f32, int upd32, double* G, unsigned* ctr) {
    const int64_t rpb = rows_per_block(n, nblk);
    const int g = blocks_for(n, nblk);
    size_t shm = sizeof(double) * ((size_t)cols * p + TR * (cols | 1) + TR * p);
    if (f32 || upd32) shm += sizeof(float) * (TR * (cols | 1) + TR * p);
    if (upd32) shm += sizeof(float) * (size_t)cols * p;
    const int nout = gram ? p * p : cols * p;
    if (gram && p <= kRowsMaxP)
        return EXPM_ROWS_CALL(p, upd_gram(V, ldv, cols, W, ldw, p, n, h, part, nblk, G, ctr, upd32, s));
    if (upd32 && gram)
        EXPM_OPT_DISPATCH(nout, (k_update<O, false, true><<<g, NT, shm, s>>>(V, ldv, cols, W, ldw, p, n, rpb, h, part,
                                                                             gram)));
    else if (f32 && !gram && f32 == 2) {
        const size_t shm_df = sizeof(float) * (2 * (size_t)cols * p + 2 * TR * (cols | 1) + TR * p + 2 * NT);
        EXPM_OPT_DISPATCH(nout, (k_update_df<O><<<g, NT, shm_df, s>>>(V, ldv, cols, W, ldw, p, n, rpb, h, part)));
    } else if (f32)
        EXPM_OPT_DISPATCH(nout, (k_update<O, true><<<g, NT, shm, s>>>(V, ldv, cols, W, ldw, p, n, rpb, h, part, gram)));
    else
        EXPM_OPT_DISPATCH(nout, (k_update<O, false><<<g, NT, shm, s>>>(V, ldv, cols, W, ldw, p, n, rpb, h, part, gram)));
    return cudaGetLastError();
}

cudaError_t launch_chol(const double* part, int nblk, int p, double shift_rel, double* R,
                        double* Rinv, double* Rtot, int mode, double* H, int ldH, int hrow,
                        int hcol, double* normsq_out, int* flags, cudaStream_t s) {
    k_chol<<<1, CHOL_T, 0, s>>>(part, nblk, p, shift_rel, R, Rinv, Rtot, mode, H, ldH, hrow, hcol,
                                normsq_out, flags);
    return cudaGetLastError();
}

cudaError_t launch_trsm(double* W, int64_t ldw, int p, int64_t n, const double* Rinv,
                        double* out, int64_t ldo, double* part, int nblk, int gram,
                        const int* extra, int tmode, cudaStream_t s) {
    const int64_t rpb = rows_per_block(n, nblk);
    const int g = blocks_for(n, nblk);
    if (p <= kRowsMaxP) return EXPM_ROWS_CALL(p, trsm(W, ldw, p, n, Rinv, out, ldo, part, nblk, gram, extra, tmode, s));
    EXPM_OPT_DISPATCH(p * p, (k_trsm<O><<<g, NT, 0, s>>>(W, ldw, p, n, rpb, Rinv, out, ldo, part, gram,
                                                       extra, tmode)));
    return cudaGetLastError();
}

cudaError_t launch_update_z(double* V, int64_t ldv, int cols, int p, int64_t n,
                            const double* Wc, double* Z, int64_t ldz, int restart_copy,
                            cudaStream_t s, int nblk, int df) {
    const int64_t rpb = rows_per_block(n, nblk);
    const int g = blocks_for(n, nblk);
    if (p <= kRowsMaxP) return EXPM_ROWS_CALL(p, updz(V, ldv, cols, p, n, Wc, Z, ldz, restart_copy, s, nblk, df));
    const size_t shm = sizeof(double) * ((size_t)cols * p + TR * (cols | 1));
    k_update_z<<<g, NT, shm, s>>>(V, ldv, cols, p, n, rpb, Wc, Z, ldz, restart_copy);
    return cudaGetLastError();
}

cudaError_t launch_combine(const double* Wc_slots, int npoles, int rows, int p, double* Wc,
                           cudaStream_t s) {
    const int nout = rows * p;
    k_combine<<<(nout + 127) / 128, 128, 0, s>>>(Wc_slots, npoles, nout, Wc);
    return cudaGetLastError();
}

cudaError_t launch_init_S(const double* R, int p, int npoles, double* S, cudaStream_t s, const double* R_alt,
                          const int* use_alt) {
    const int tot = npoles * p * p;
    k_init_S<<<(tot + 127) / 128, 128, 0, s>>>(R, p, npoles, S, R_alt, use_alt);
    return cudaGetLastError();
}

cudaError_t launch_axpby(double a, const double* X, int64_t ldx, double b, const double* Y,
                         int64_t ldy, double* out, int64_t ldo, int64_t n, int p,
                         cudaStream_t s) {
    dim3 grid((unsigned)((n + 255) / 256), p);
    k_axpby<<<grid, 256, 0, s>>>(a, X, ldx, b, Y, ldy, out, ldo, n);
    return cudaGetLastError();
}

cudaError_t launch_copy(const double* X, int64_t ldx, double* Y, int64_t ldy, int64_t n, int p,
                        cudaStream_t s) {
    return launch_axpby(1.0, X, ldx, 0.0, nullptr, 0, Y, ldy, n, p, s);
}

cudaError_t launch_zero(double* X, int64_t ldx, int64_t n, int p, cudaStream_t s) {
    dim3 grid((unsigned)((n + 255) / 256), p);
    k_zero<<<grid, 256, 0, s>>>(X, ldx, n);
    return cudaGetLastError();
}

// Shared-memory opt-in for the launches whose dynamic size can pass 48 KB: the device's
// per-block opt-in maximum minus the kernel's own static shared memory.
template <class K>
static cudaError_t set_max_dynamic(K kernel, int optin) {
    cudaFuncAttributes fa;
    cudaError_t e = cudaFuncGetAttributes(&fa, kernel);
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                optin - (int)fa.sharedSizeBytes);
}

cudaError_t krylov_set_smem_limits() {
    int dev = 0, optin = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
#define EXPM_SET(K) \
    if (e == cudaSuccess) e = set_max_dynamic(K, optin)
    EXPM_SET((k_proj<1, double>)); EXPM_SET((k_proj<4, double>)); EXPM_SET((k_proj<16, double>));
    EXPM_SET((k_proj<64, double>)); EXPM_SET((k_proj<1, float>)); EXPM_SET((k_proj<4, float>));
    EXPM_SET((k_proj<16, float>)); EXPM_SET((k_proj<64, float>));
    EXPM_SET((k_update<1, false>)); EXPM_SET((k_update<4, false>)); EXPM_SET((k_update<16, false>));
    EXPM_SET((k_update<64, false>)); EXPM_SET((k_update<1, true>)); EXPM_SET((k_update<4, true>));
    EXPM_SET((k_update<16, true>)); EXPM_SET((k_update<64, true>));
    EXPM_SET((k_update<1, false, true>)); EXPM_SET((k_update<4, false, true>));
    EXPM_SET((k_update<16, false, true>)); EXPM_SET((k_update<64, false, true>));
    EXPM_SET(k_update_df<1>); EXPM_SET(k_update_df<4>); EXPM_SET(k_update_df<16>); EXPM_SET(k_update_df<64>);
    EXPM_SET(k_update_z);
    if (e == cudaSuccess) e = rows4::set_smem(optin);
    if (e == cudaSuccess) e = rows8::set_smem(optin);
    if (e == cudaSuccess) e = rows12::set_smem(optin);
    if (e == cudaSuccess) e = rows16::set_smem(optin);
#undef EXPM_SET
    return e;
}

}  // namespace expm
