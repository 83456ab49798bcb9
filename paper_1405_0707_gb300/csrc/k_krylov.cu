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
#include "internal.h"

namespace expm {
namespace {

constexpr int TR = 16;      // rows per shared-memory tile
constexpr int NT = 256;     // threads per CTA for the row passes

__device__ inline int64_t rows_begin(int64_t rpb) { return (int64_t)blockIdx.x * rpb; }

// Loads are issued in batches of LB per thread into registers before any is converted or
// stored, so LB independent global loads are in flight per thread.
constexpr int LB = 8;

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

// Destination, Gram and skip of a triangular-solve pass (see k_chol's pass modes):
// tmode 0: write `out` (gram as asked); tmode 1: a third pass follows iff extra -> in place
// with Gram, else the final block `out`; tmode 2: only if extra, into `out`.
struct TrsmPass {
    double* dest;
    int64_t ldd;
    int gram;
    bool skip;
};
__device__ inline TrsmPass trsm_pass(double* W, int64_t ldw, double* out, int64_t ldo, int gram,
                                     const int* extra, int tmode) {
    if (tmode == 0) return {out, ldo, gram, false};
    const int ex = *extra;
    if (tmode == 1) return ex ? TrsmPass{W, ldw, 1, false} : TrsmPass{out, ldo, 0, false};
    return {out, ldo, 0, ex == 0};
}

// ---- double-float (FP32 pair) arithmetic for the mixed path's first CGS update
// v = hi + lo with hi = v truncated to 24 significant bits (exact as a float) and lo the
// remainder rounded to a float (relative error 2^-48 of v), built from the bit pattern with
// integer and FP32 operations only.  Values below 2^-74 in magnitude keep hi = (float)v.
__device__ __forceinline__ void split_df(double v, float& hi, float& lo) {
    const long long b = __double_as_longlong(v);
    const int e = (int)((b >> 52) & 0x7ff);
    if (e < 949 || e > 1150) {          // outside the range where the split is exact
        hi = (float)v;
        lo = 0.f;
        return;
    }
    hi = (float)__longlong_as_double(b & ~((1LL << 29) - 1));
    const float mag = (float)(int)(b & ((1LL << 29) - 1)) * __int_as_float((e - 1075 + 127) << 23);
    lo = (b < 0) ? -mag : mag;
}

// s + x into the pair (s, c): TwoSum for the large parts, the rounding error into c
__device__ __forceinline__ void df_add(float& s, float& c, float x) {
    const float t = s + x;
    const float bp = t - s;
    const float err = (s - (t - bp)) + (x - bp);
    s = t;
    c += err;
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
// b = s, s + stripes, ...) with four independent accumulators; the caller adds the stripes
// in a fixed order, so the result does not depend on scheduling.
__device__ inline double stripe_sum(const double* __restrict__ part, int nblk, int nout, int o,
                                    int s, int stripes) {
    double a0 = 0.0, a1 = 0.0, a2 = 0.0, a3 = 0.0;
    int b = s;
    for (; b + 3 * stripes < nblk; b += 4 * stripes) {
        a0 += part[(int64_t)b * nout + o];
        a1 += part[(int64_t)(b + stripes) * nout + o];
        a2 += part[(int64_t)(b + 2 * stripes) * nout + o];
        a3 += part[(int64_t)(b + 3 * stripes) * nout + o];
    }
    for (; b < nblk; b += stripes) a0 += part[(int64_t)b * nout + o];
    return (a0 + a1) + (a2 + a3);
}

constexpr int RED_OUT = 8;        // outputs per reduction CTA
constexpr int RED_STRIPES = 32;   // threads per output

// h[o] = sum_b part[b][o]; H[row0 + a, col0 + c] (+)= h[a][c].  CTA = 8 outputs x 32 stripes;
// the stripes are added in two fixed-order levels (4 groups of 8, then the 4 groups).
__global__ void __launch_bounds__(RED_OUT * RED_STRIPES)
k_reduce_h(const double* __restrict__ part, int nblk, int cols, int p, double* __restrict__ h,
           double* H, int ldH, int row0, int col0, int accumulate) {
    __shared__ double red[RED_STRIPES][RED_OUT];
    __shared__ double red2[4][RED_OUT];
    const int nout = cols * p;
    const int ol = threadIdx.x % RED_OUT, st = threadIdx.x / RED_OUT;
    const int o = blockIdx.x * RED_OUT + ol;
    red[st][ol] = (o < nout) ? stripe_sum(part, nblk, nout, o, st, RED_STRIPES) : 0.0;
    __syncthreads();
    if (st < 4) {
        double g = 0.0;
#pragma unroll
        for (int k = 0; k < 8; ++k) g += red[st * 8 + k][ol];
        red2[st][ol] = g;
    }
    __syncthreads();
    if (st != 0 || o >= nout) return;
    const double s = (red2[0][ol] + red2[1][ol]) + (red2[2][ol] + red2[3][ol]);
    h[o] = s;
    if (H) {
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

// Row-per-thread variant for p <= 8 (the common block sizes): a row of W lives in
// registers, W R^{-1} and the upper-triangular outer product w^T w are formed there, and
// the Gram partial of the CTA is one warp-shuffle reduction at the end.  Loads and stores
// are coalesced per column (consecutive threads, consecutive rows); no tile barriers.
constexpr int RP = 8;
constexpr int RG = RP * (RP + 1) / 2;

__device__ inline double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Gram partial of rows held one per lane: each warp stages its 32 rows in shared memory
// (buf, 32 x RP), then lane l sums upper-triangle entries l and l + 32 over those rows.
// FP64 work equals the useful products; no reduction tree.  Every lane of the warp must
// call it (rows past the end are zero).
__device__ inline void warp_gram_rows(const double* y, double* buf, double& acc0, double& acc1) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int c = 0; c < RP; ++c) buf[lane * RP + c] = y[c];
    __syncwarp();
    // upper-triangle entry k -> (c1, c2)
    for (int q = 0; q < 2; ++q) {
        const int kk = lane + 32 * q;
        if (kk < RG) {
            int c1 = 0, rem = kk;
            while (rem >= RP - c1) { rem -= RP - c1; ++c1; }
            const int c2 = c1 + rem;
            double s = 0.0;
#pragma unroll 8
            for (int rr = 0; rr < 32; ++rr) s = fma(buf[rr * RP + c1], buf[rr * RP + c2], s);
            if (q == 0) acc0 += s;
            else acc1 += s;
        }
    }
    __syncwarp();
}

// FP32 variant (the mixed path's Gram for the first Cholesky-QR pass, whose factorisation
// is FP32 anyway): rows staged as floats, products and per-lane sums in FP32.
__device__ inline void warp_gram_rows32(const double* y, float* buf, float& acc0, float& acc1) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int c = 0; c < RP; ++c) buf[lane * RP + c] = (float)y[c];
    __syncwarp();
    for (int q = 0; q < 2; ++q) {
        const int kk = lane + 32 * q;
        if (kk < RG) {
            int c1 = 0, rem = kk;
            while (rem >= RP - c1) { rem -= RP - c1; ++c1; }
            const int c2 = c1 + rem;
            float s = 0.f;
#pragma unroll 8
            for (int rr = 0; rr < 32; ++rr) s = fmaf(buf[rr * RP + c1], buf[rr * RP + c2], s);
            if (q == 0) acc0 += s;
            else acc1 += s;
        }
    }
    __syncwarp();
}

// Double-float variant (the mixed path's Gram matrix after the first Cholesky-QR pass, which
// the deviation pass needs to ~1e-14): rows staged as (hi, lo) float pairs; each product
// hi1 hi2 + (err(hi1 hi2) + hi1 lo2 + lo1 hi2) accumulated with TwoSum into a per-lane pair.
__device__ inline void warp_gram_rows_df(const float* yh, const float* yl, float* buf, float* ah, float* al) {
    const int lane = threadIdx.x & 31;
    float* bh = buf;                 // 32 x RP
    float* bl = buf + 32 * RP;       // 32 x RP
#pragma unroll
    for (int c = 0; c < RP; ++c) {
        bh[lane * RP + c] = yh[c];
        bl[lane * RP + c] = yl[c];
    }
    __syncwarp();
    for (int q = 0; q < 2; ++q) {
        const int kk = lane + 32 * q;
        if (kk < RG) {
            int c1 = 0, rem = kk;
            while (rem >= RP - c1) { rem -= RP - c1; ++c1; }
            const int c2 = c1 + rem;
            float sh = ah[q], sl = al[q];
#pragma unroll 4
            for (int rr = 0; rr < 32; ++rr) {
                const float h1 = bh[rr * RP + c1], h2 = bh[rr * RP + c2];
                const float pr = h1 * h2;
                float t = fmaf(h1, h2, -pr);
                t = fmaf(h1, bl[rr * RP + c2], t);
                t = fmaf(bl[rr * RP + c1], h2, t);
                df_add(sh, sl, pr);
                sl += t;
            }
            ah[q] = sh;
            al[q] = sl;
        }
    }
    __syncwarp();
}

// The CTA's Gram partial (p x p layout, upper triangle; lower = 0) from the per-lane
// accumulators of warp_gram_rows.
__device__ inline void cta_gram_write(double acc0, double acc1, int p, double (*red)[RG],
                                      double* __restrict__ part) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    red[wid][lane] = acc0;
    if (lane + 32 < RG) red[wid][lane + 32] = acc1;
    __syncthreads();
    for (int o = threadIdx.x; o < p * p; o += blockDim.x) {
        const int c1 = o / p, c2 = o % p;
        double s = 0.0;
        if (c1 <= c2) {
            const int k = c1 * RP - c1 * (c1 - 1) / 2 + (c2 - c1);
            for (int w_ = 0; w_ < NT / 32; ++w_) s += red[w_][k];
        }
        part[(int64_t)blockIdx.x * p * p + o] = s;
    }
}

// Last-CTA reduction: every CTA has written its partial; the CTA that takes the last ticket
// (atomic counter) sums the nblk partials of each output in a fixed order (independent of
// which CTA is last) and resets the counter for the next kernel.  No CTA waits on another.
__device__ inline bool take_last_ticket(unsigned* ctr) {
    __shared__ unsigned ticket;
    __threadfence();                       // this CTA's partial is visible device-wide
    __syncthreads();
    if (threadIdx.x == 0) ticket = atomicAdd(ctr, 1u);
    __syncthreads();
    return ticket == gridDim.x - 1;
}

// out[o] = sum_b part[b][o] in double-float arithmetic (each partial split into a float pair,
// TwoSum accumulation): the FP32 pipe instead of the FP64 one for the last CTA's tail.
__device__ inline void last_cta_sum_df(const double* part, int nblk, int nout, double* __restrict__ out,
                                       unsigned* ctr) {
    __shared__ float redh[NT], redl[NT];
    __threadfence();
    const int stripes = NT / nout;
    const int o = threadIdx.x % nout, st = threadIdx.x / nout;
    float sh = 0.f, sl = 0.f;
    if (st < stripes)
        for (int b = st; b < nblk; b += stripes) {
            float h, l;
            split_df(__ldcg(part + (int64_t)b * nout + o), h, l);
            df_add(sh, sl, h);
            sl += l;
        }
    redh[threadIdx.x] = sh;
    redl[threadIdx.x] = sl;
    __syncthreads();
    if (threadIdx.x < nout) {
        float th = 0.f, tl = 0.f;
        for (int k = 0; k < stripes; ++k) {
            df_add(th, tl, redh[k * nout + threadIdx.x]);
            tl += redl[k * nout + threadIdx.x];
        }
        out[threadIdx.x] = (double)th + (double)tl;
    }
    if (threadIdx.x == 0) *ctr = 0u;
}

// out[o] = sum_b part[b][o] for o < nout (nout <= RP * RP), by the last CTA: NT / nout stripes
// per output, each stripe's loads issued back to back, stripes added in a fixed order.
// ACC = float: FP32 sums (for a Gram matrix that only feeds an FP32 factorisation).
template <typename ACC = double>
__device__ inline void last_cta_sum(const double* part, int nblk, int nout, double* __restrict__ out,
                                    unsigned* ctr) {
    __shared__ double red[NT];
    __threadfence();
    const int stripes = NT / nout;         // nout <= 64 -> at least 4 stripes
    const int o = threadIdx.x % nout, st = threadIdx.x / nout;
    double acc = 0.0;
    if (st < stripes) {
        ACC a0 = 0, a1 = 0, a2 = 0, a3 = 0;
        int b = st;
        for (; b + 3 * stripes < nblk; b += 4 * stripes) {
            a0 += (ACC)__ldcg(part + (int64_t)b * nout + o);
            a1 += (ACC)__ldcg(part + (int64_t)(b + stripes) * nout + o);
            a2 += (ACC)__ldcg(part + (int64_t)(b + 2 * stripes) * nout + o);
            a3 += (ACC)__ldcg(part + (int64_t)(b + 3 * stripes) * nout + o);
        }
        for (; b < nblk; b += stripes) a0 += (ACC)__ldcg(part + (int64_t)b * nout + o);
        acc = (double)((a0 + a1) + (a2 + a3));
    }
    red[threadIdx.x] = acc;
    __syncthreads();
    if (threadIdx.x < nout) {
        double s = 0.0;
        for (int k = 0; k < stripes; ++k) s += red[k * nout + threadIdx.x];
        out[threadIdx.x] = s;
    }
    if (threadIdx.x == 0) *ctr = 0u;
}

// ---- Mixed-path Cholesky QR for p <= 8 (every CTA factors the reduced Gram matrix G
// itself, in FP32; CTA 0 alone writes R, Rtot, H and the flags).
//   KIND 1 (pass 1, mode 0): G (summed in FP64) is scaled by a power of two near its largest
//     diagonal entry (exact) and factored in FP32; pivots below 1e-6 of the largest (kappa(W)
//     above ~1e3) redo it with the shift 11 p (p+1) 2^-24 trace and request a third pass
//     (flags[2]).  R is that factor scaled back (exact), and W <- W R^{-1} is a forward
//     substitution with R in FP64, so W = W_new R holds to FP64 rounding whatever the FP32
//     factor's own accuracy.  Gram partials in FP64, reduced by the last CTA into G.
//   KIND 2 (passes 2 and 3, modes 1 and 2): now G = I + E with E small, so R = I + U is
//     found from the deviation alone, in FP32: U_jl = (E_jl - sum_{k<j} U_kj U_kl)/(1 + U_jj),
//     U_jj = x / (1 + sqrt(1 + x)) with x = E_jj - sum_{k<j} U_kj^2; R^{-1} = I + Y with
//     (I + U) Y = -U.  Each entry has FP32 relative accuracy on a quantity of size |E|, so
//     absolute errors are ~eps_32 |E|.  Rtot <- Rtot + U Rtot (FP32 correction of the FP64
//     product) and W <- W + W Y (FP32 correction of the FP64 W).
// Columns that are exactly zero stay zero (zero rows in R), as in k_chol.
struct CholF {
    float G[RP * RP], U[RP * RP], Y[RP * RP];
    float rd[RP];
    float umax;       // KIND 2: max |U|
    int ill, bad;
};

// pass 1: FP32 Cholesky of G 2^-k (upper triangle) -> U; warp 0
__device__ inline void chol32_full(CholF& cf, const double* G0, int p, int k, double tr_s) {
    const int lane = threadIdx.x;
    const int pp = p * p;
    if (lane == 0) { cf.ill = 0; cf.bad = 0; }
    __syncwarp();
    for (int attempt = 0; attempt < 2; ++attempt) {
        const double shift = attempt ? 11.0 * p * (p + 1) * 0x1p-24 * tr_s : 0.0;
        for (int o = lane; o < pp; o += 32) {
            cf.G[o] = (float)(ldexp(G0[o], -k) + ((o / p == o % p) ? shift : 0.0));
            cf.U[o] = 0.f;
        }
        __syncwarp();
        float dmax = 0.f;
        for (int c = 0; c < p; ++c) dmax = fmaxf(dmax, cf.G[c * p + c]);
        for (int j = 0; j < p; ++j) {
            if (lane == 0) {
                float d = cf.G[j * p + j];
                if (G0[j * p + j] == 0.0) {
                    cf.U[j * p + j] = 0.f;
                    cf.rd[j] = 0.f;
                } else {
                    if (!(d > 0.f) || !isfinite(d) || (attempt == 0 && d < 1e-6f * dmax)) cf.ill = 1;
                    if (!(d > 0.f) || !isfinite(d)) d = 1.f;
                    const float rj = sqrtf(d);
                    cf.U[j * p + j] = rj;
                    cf.rd[j] = 1.f / rj;
                }
            }
            __syncwarp();
            const float inv = cf.rd[j];
            if (lane > j && lane < p) cf.U[j * p + lane] = cf.G[j * p + lane] * inv;
            __syncwarp();
            if (lane > j && lane < p) {
                const float rb = cf.U[j * p + lane];
                for (int a = j + 1; a <= lane; ++a) cf.G[a * p + lane] -= cf.U[j * p + a] * rb;
            }
            __syncwarp();
        }
        if (attempt == 1 || !cf.ill) break;
        __syncwarp();
    }
}

// passes 2/3: deviation Cholesky of G = I + E -> U (R = I + U), Y (R^{-1} = I + Y); warp 0
__device__ inline void chol32_dev(CholF& cf, const double* G0, int p) {
    const int lane = threadIdx.x;
    const int pp = p * p;
    if (lane == 0) { cf.ill = 0; cf.bad = 0; }
    for (int o = lane; o < pp; o += 32) {
        const bool dg = o / p == o % p;
        cf.G[o] = (float)(G0[o] - (dg ? 1.0 : 0.0));   // E (upper triangle)
        cf.U[o] = 0.f;
        cf.Y[o] = 0.f;
    }
    __syncwarp();
    for (int j = 0; j < p; ++j) {
        if (lane == 0) {
            if (G0[j * p + j] == 0.0) {
                cf.U[j * p + j] = -1.f;                  // R_jj = 0: a zero column stays zero
                cf.rd[j] = 0.f;
            } else {
                float x = cf.G[j * p + j];
                for (int k = 0; k < j; ++k) x -= cf.U[k * p + j] * cf.U[k * p + j];
                if (!(x > -0.75f) || !isfinite(x)) cf.bad = 1;   // not close to orthonormal
                if (!(x > -0.75f) || !isfinite(x)) x = 0.f;
                const float ujj = x / (1.f + sqrtf(1.f + x));
                cf.U[j * p + j] = ujj;
                cf.rd[j] = 1.f / (1.f + ujj);
            }
        }
        __syncwarp();
        if (lane > j && lane < p) {
            float s = cf.G[j * p + lane];
            for (int k = 0; k < j; ++k) s -= cf.U[k * p + j] * cf.U[k * p + lane];
            cf.U[j * p + lane] = s * cf.rd[j];
        }
        __syncwarp();
    }
    if (lane == 0) {
        float um = 0.f;
        for (int o = 0; o < pp; ++o) um = fmaxf(um, fabsf(cf.U[o]));
        cf.umax = um;
    }
    // (I + U) Y = -U, column `lane` by back substitution
    if (lane < p) {
        const int c = lane;
        for (int r = c; r >= 0; --r) {
            float s = -cf.U[r * p + c];
            for (int k = r + 1; k <= c; ++k) s -= cf.U[r * p + k] * cf.Y[k * p + c];
            cf.Y[r * p + c] = (r == c && cf.rd[r] == 0.f) ? -1.f : s * cf.rd[r];
        }
    }
    __syncwarp();
}

template <int KIND>
__global__ void __launch_bounds__(NT) k_qr_mixed_rows(double* W, int64_t ldw, int p, int64_t n, int64_t rpb,
                                                      double* G, double* __restrict__ part, unsigned* ctr,
                                                      int mode, double* R, double* Rinv, const double* Rtot_in,
                                                      double* Rtot_out, double* H, int ldH, int hrow, int hcol,
                                                      double* normsq_out, int* flags, double* out_, int64_t ldo_) {
    int* extra = flags + 2;
    if (mode == 2 && *extra == 0) return;
    __shared__ CholF cf;
    __shared__ double G0[RP * RP];
    __shared__ double hn2[RP];
    __shared__ double Rd[RP * RP];          // KIND 1: R (padded to RP x RP); KIND 2 unused
    __shared__ double rcp[RP];              // KIND 1: 1 / R_cc (0 for a zero column)
    __shared__ float Rh[RP * RP], Rl[RP * RP];   // KIND 1: R as float pairs
    __shared__ float rch[RP], rcl[RP];           // KIND 1: 1 / R_cc as float pairs
    __shared__ float Yf[RP * RP];           // KIND 2: Y padded to RP x RP
    __shared__ double red[NT / 32][RG];
    __shared__ double buf[NT / 32][32 * RP];
    const int pp = p * p;
    for (int o = threadIdx.x; o < pp; o += blockDim.x) G0[o] = G[o];
    const bool last = (mode == 1 && *extra == 0) || mode == 2;
    const bool lead = blockIdx.x == 0;
    if (H && last && lead) {
        const int stripes = NT / p;
        const int c = threadIdx.x % p, st = threadIdx.x / p;
        double v2 = 0.0;
        if (st < stripes)
            for (int a = st; a < hrow; a += stripes) {
                const double v = H[(int64_t)(hcol + c) * ldH + a];
                v2 += v * v;
            }
        buf[0][threadIdx.x] = v2;
    }
    __syncthreads();
    if (H && last && lead && threadIdx.x < p) {
        const int stripes = NT / p;
        double s2 = 0.0;
        for (int k = 0; k < stripes; ++k) s2 += buf[0][k * p + threadIdx.x];
        hn2[threadIdx.x] = s2;
    }
    __syncthreads();
    int kexp = 0;                           // KIND 1: G is factored as G 2^-kexp (kexp even)
    if (threadIdx.x < 32) {
        const int lane = threadIdx.x;
        double tr = 0.0, dmax = 0.0;
        if (KIND == 1) {
            for (int c = 0; c < p; ++c) {
                tr += G0[c * p + c];
                dmax = fmax(dmax, G0[c * p + c]);
            }
            if (dmax > 0.0 && isfinite(dmax)) {
                frexp(dmax, &kexp);
                kexp &= ~1;
            }
            chol32_full(cf, G0, p, kexp, ldexp(tr, -kexp));
        } else {
            chol32_dev(cf, G0, p);
        }
        if (lead) {
            if (KIND == 1 && normsq_out && lane == 0) *normsq_out = tr;
            if (KIND == 1 && lane == 0) *extra = cf.ill;
            if (lane < p) {
                const int c = lane;
                for (int r = 0; r < p; ++r) {
                    const int o = r * p + c;
                    double rt;
                    if (KIND == 1) {
                        rt = (r <= c) ? ldexp((double)cf.U[o], kexp / 2) : 0.0;
                        R[o] = rt;
                    } else {
                        // Rtot_out = Rtot_in + U Rtot_in (FP32 correction of the FP64 product)
                        float corr = 0.f;
                        for (int k = r; k <= c; ++k) corr = fmaf(cf.U[r * p + k], (float)Rtot_in[k * p + c], corr);
                        rt = (r <= c) ? Rtot_in[o] + (double)corr : 0.0;
                        R[o] = (r <= c) ? (double)cf.U[o] + (r == c ? 1.0 : 0.0) : 0.0;
                        Rinv[o] = (r <= c) ? (double)cf.Y[o] + (r == c ? 1.0 : 0.0) : 0.0;
                    }
                    Rtot_out[o] = rt;
                    if (!isfinite(rt)) cf.bad = 1;
                    if (H && last) H[(int64_t)(hcol + c) * ldH + hrow + r] = rt;
                }
            }
            __syncwarp();
            if (H && last && lane < p) {
                const int c = lane;
                double n0 = hn2[c], dg = 0.0;
                for (int a = 0; a <= c; ++a) {
                    const double v = Rtot_out[a * p + c];
                    n0 += v * v;
                    if (a == c) dg = v;
                }
                if (dg <= 1e-14 * sqrt(n0)) atomicOr(&flags[1], 1);
            }
            __syncwarp();
            if (lane == 0 && cf.bad) atomicOr(&flags[0], 1);
        }
    }
    __syncthreads();
    if (KIND == 1) {
        // kexp as computed by warp 0 (every thread recomputes it from the same G0)
        double dmax = 0.0;
        for (int c = 0; c < p; ++c) dmax = fmax(dmax, G0[c * p + c]);
        kexp = 0;
        if (dmax > 0.0 && isfinite(dmax)) {
            frexp(dmax, &kexp);
            kexp &= ~1;
        }
    }
    // KIND 2 with max|U| above 1e-4 (a pass after the shifted one): the FP32 inverse I + Y
    // would leave an eps_32 |U| mismatch with the recorded R, so the solve is a forward
    // substitution with R = I + U in FP64, as in pass 1
    const bool subst = KIND == 1 || cf.umax > 1e-4f;
    for (int e = threadIdx.x; e < RP * RP; e += blockDim.x) {
        const int a = e / RP, c = e % RP;
        const bool in = a < p && c < p && a <= c;
        if (KIND == 1) Rd[e] = in ? ldexp((double)cf.U[a * p + c], kexp / 2) : 0.0;
        else {
            Yf[e] = in ? cf.Y[a * p + c] : 0.f;
            Rd[e] = in ? (double)cf.U[a * p + c] + (a == c ? 1.0 : 0.0) : 0.0;
        }
    }
    __syncthreads();
    if (subst && threadIdx.x < RP) {
        const double d = Rd[threadIdx.x * RP + threadIdx.x];
        rcp[threadIdx.x] = (d != 0.0) ? 1.0 / d : 0.0;
        if (KIND == 1) split_df(rcp[threadIdx.x], rch[threadIdx.x], rcl[threadIdx.x]);
    }
    if (KIND == 1)
        for (int e = threadIdx.x; e < RP * RP; e += blockDim.x) split_df(Rd[e], Rh[e], Rl[e]);
    __syncthreads();
    double* out;
    int64_t ldo;
    int gram;
    if (mode == 0) { out = W; ldo = ldw; gram = 1; }
    else if (mode == 1 && *extra) { out = W; ldo = ldw; gram = 1; }
    else { out = out_; ldo = ldo_; gram = 0; }
    double acc0 = 0.0, acc1 = 0.0;
    float gah[2] = {0.f, 0.f}, gal[2] = {0.f, 0.f};
    const int64_t rb = rows_begin(rpb), re = min(n, rb + rpb);
    for (int64_t r0 = rb + (threadIdx.x & ~31); r0 < re; r0 += blockDim.x) {
        const int64_t r = r0 + (threadIdx.x & 31);
        const bool ok = r < re;
        double w[RP], y[RP];
#pragma unroll
        for (int c = 0; c < RP; ++c) w[c] = (ok && c < p) ? W[(int64_t)c * ldw + r] : 0.0;
        float yh[RP], yl[RP];
        if (KIND == 1) {
            // forward substitution y R = w in double-float: R's entries are exact floats
            // (pairs Rh + Rl for safety), 1 / R_cc as a pair, y kept as pairs
#pragma unroll
            for (int c = 0; c < RP; ++c) {
                float sh, sl;
                split_df(w[c], sh, sl);
#pragma unroll
                for (int a = 0; a < c; ++a) {
                    const float r1 = Rh[a * RP + c], r2 = Rl[a * RP + c];
                    const float pr = yh[a] * r1;
                    float t = fmaf(yh[a], r1, -pr);
                    t = fmaf(yh[a], r2, t);
                    t = fmaf(yl[a], r1, t);
                    df_add(sh, sl, -pr);
                    sl -= t;
                }
                const float q1 = rch[c], q2 = rcl[c];
                const float pr = sh * q1;
                float t = fmaf(sh, q1, -pr);
                t = fmaf(sh, q2, t);
                t = fmaf(sl, q1, t);
                const float s2 = pr + t;
                yl[c] = t - (s2 - pr);
                yh[c] = s2;
                y[c] = (double)yh[c] + (double)yl[c];
            }
        } else if (subst) {
            // forward substitution y R = w (R upper triangular)
#pragma unroll
            for (int c = 0; c < RP; ++c) {
                double s = w[c];
#pragma unroll
                for (int a = 0; a < c; ++a) s = fma(-y[a], Rd[a * RP + c], s);
                y[c] = s * rcp[c];
            }
        } else {
            float wf[RP];
#pragma unroll
            for (int c = 0; c < RP; ++c) wf[c] = (float)w[c];
#pragma unroll
            for (int c = 0; c < RP; ++c) {
                float s = 0.f;
#pragma unroll
                for (int a = 0; a <= c; ++a) s = fmaf(wf[a], Yf[a * RP + c], s);
                y[c] = w[c] + (double)s;
            }
        }
#pragma unroll
        for (int c = 0; c < RP; ++c)
            if (ok && c < p) out[(int64_t)c * ldo + r] = y[c];
        if (gram) {
            if (KIND == 1) {
#pragma unroll
                for (int c = 0; c < RP; ++c)
                    if (!ok || c >= p) { yh[c] = 0.f; yl[c] = 0.f; }
                warp_gram_rows_df(yh, yl, reinterpret_cast<float*>(buf[threadIdx.x >> 5]), gah, gal);
            } else {
                warp_gram_rows(y, buf[threadIdx.x >> 5], acc0, acc1);
            }
        }
    }
    if (gram) {
        if (KIND == 1) {
            acc0 = (double)gah[0] + (double)gal[0];
            acc1 = (double)gah[1] + (double)gal[1];
        }
        cta_gram_write(acc0, acc1, p, red, part);
        if (take_last_ticket(ctr)) last_cta_sum_df(part, gridDim.x, pp, G, ctr);
    }
}

__global__ void __launch_bounds__(NT) k_trsm_rows(double* W, int64_t ldw, int p,
                                                  int64_t n, int64_t rpb, const double* __restrict__ Rinv,
                                                  double* out_, int64_t ldo_,
                                                  double* __restrict__ part, int gram_,
                                                  const int* extra, int tmode) {
    const TrsmPass ps = trsm_pass(W, ldw, out_, ldo_, gram_, extra, tmode);
    if (ps.skip) return;
    double* out = ps.dest;
    const int64_t ldo = ps.ldd;
    const int gram = ps.gram;
    __shared__ double Ri[RP * RP];
    __shared__ double red[NT / 32][RG];
    __shared__ double buf[NT / 32][32 * RP];
    for (int e = threadIdx.x; e < RP * RP; e += blockDim.x) {
        const int a = e / RP, c = e % RP;
        Ri[e] = (a < p && c < p) ? Rinv[a * p + c] : 0.0;
    }
    __syncthreads();
    double acc0 = 0.0, acc1 = 0.0;
    const int64_t rb = rows_begin(rpb), re = min(n, rb + rpb);
    // whole warps step through the rows together (rows past the end contribute zeros)
    for (int64_t r0 = rb + (threadIdx.x & ~31); r0 < re; r0 += blockDim.x) {
        const int64_t r = r0 + (threadIdx.x & 31);
        const bool ok = r < re;
        double w[RP], y[RP];
#pragma unroll
        for (int c = 0; c < RP; ++c) w[c] = (ok && c < p) ? W[(int64_t)c * ldw + r] : 0.0;
#pragma unroll
        for (int c = 0; c < RP; ++c) {
            double s = 0.0;
#pragma unroll
            for (int a = 0; a <= c; ++a) s = fma(w[a], Ri[a * RP + c], s);
            y[c] = s;
            if (ok && c < p) out[(int64_t)c * ldo + r] = s;
        }
        if (gram) warp_gram_rows(y, buf[threadIdx.x >> 5], acc0, acc1);
    }
    if (gram) cta_gram_write(acc0, acc1, p, red, part);
}

// Row-per-thread, p <= 8: W <- W - V h and the upper-triangular Gram partial of the result.
// h (cols x p) is broadcast from shared memory.  UPD32 = false: the update in FP64 (the
// Arnoldi relation stays exact to FP64 rounding).  UPD32 = true (mixed path, second CGS
// pass only): h is then the O(eps_32) remainder left by the FP32 projection of the first
// pass, so the correction V h is formed in FP32 and subtracted from the FP64 W; its error,
// eps_32 |V h| ~ eps_32^2 |W|, stays far below the accuracy the mixed path delivers.
template <bool UPD32>
__global__ void __launch_bounds__(NT) k_update_gram_rows(const double* __restrict__ V, int64_t ldv, int cols,
                                                         double* __restrict__ W, int64_t ldw, int p,
                                                         int64_t n, int64_t rpb,
                                                         const double* __restrict__ h,
                                                         double* __restrict__ part, double* G,
                                                         unsigned* ctr) {
    extern __shared__ double hs[];           // cols x RP (zero-padded columns), FP64 or FP32
    float* hsf = reinterpret_cast<float*>(hs);
    __shared__ double red[NT / 32][RG];
    for (int e = threadIdx.x; e < cols * RP; e += blockDim.x) {
        const int a = e / RP, c = e % RP;
        const double v = (c < p) ? h[a * p + c] : 0.0;
        if (UPD32) hsf[e] = (float)v;
        else hs[e] = v;
    }
    __syncthreads();
    __shared__ double buf[NT / 32][32 * RP];
    double acc0 = 0.0, acc1 = 0.0;
    float facc0 = 0.f, facc1 = 0.f;
    const int64_t rb = rows_begin(rpb), re = min(n, rb + rpb);
    for (int64_t r0 = rb + (threadIdx.x & ~31); r0 < re; r0 += blockDim.x) {
        const int64_t r = r0 + (threadIdx.x & 31);
        const bool ok = r < re;
        double w[RP];
#pragma unroll
        for (int c = 0; c < RP; ++c) w[c] = (ok && c < p) ? W[(int64_t)c * ldw + r] : 0.0;
        if (ok && UPD32) {
            float corr[RP];
#pragma unroll
            for (int c = 0; c < RP; ++c) corr[c] = 0.f;
#pragma unroll 8
            for (int a = 0; a < cols; ++a) {
                const float v = (float)V[(int64_t)a * ldv + r];
#pragma unroll
                for (int c = 0; c < RP; ++c) corr[c] = fmaf(v, hsf[a * RP + c], corr[c]);
            }
#pragma unroll
            for (int c = 0; c < RP; ++c) w[c] -= (double)corr[c];
        } else if (ok) {
#pragma unroll 8
            for (int a = 0; a < cols; ++a) {
                const double v = V[(int64_t)a * ldv + r];
#pragma unroll
                for (int c = 0; c < RP; ++c) w[c] = fma(-v, hs[a * RP + c], w[c]);
            }
        }
#pragma unroll
        for (int c = 0; c < RP; ++c)
            if (ok && c < p) W[(int64_t)c * ldw + r] = w[c];
        if (UPD32) warp_gram_rows32(w, reinterpret_cast<float*>(buf[threadIdx.x >> 5]), facc0, facc1);
        else warp_gram_rows(w, buf[threadIdx.x >> 5], acc0, acc1);
    }
    if (UPD32) {
        acc0 = facc0;
        acc1 = facc1;
    }
    cta_gram_write(acc0, acc1, p, red, part);
    if (G && take_last_ticket(ctr)) {
        if (UPD32) last_cta_sum<float>(part, gridDim.x, p * p, G, ctr);
        else last_cta_sum<double>(part, gridDim.x, p * p, G, ctr);
    }
}

// Row-per-thread, p <= 8: Z[r, :] += V[r, 0:cols] Wc; restart copy V[r, 0:p] <- V[r, cols-p:cols].
__global__ void __launch_bounds__(NT) k_update_z_rows(double* __restrict__ V, int64_t ldv, int cols, int p,
                                                      int64_t n, int64_t rpb,
                                                      const double* __restrict__ Wc,
                                                      double* __restrict__ Z, int64_t ldz,
                                                      int restart_copy) {
    extern __shared__ double ws[];           // cols x RP
    for (int e = threadIdx.x; e < cols * RP; e += blockDim.x) {
        const int a = e / RP, c = e % RP;
        ws[e] = (c < p) ? Wc[a * p + c] : 0.0;
    }
    __syncthreads();
    const int64_t rb = rows_begin(rpb), re = min(n, rb + rpb);
    for (int64_t r = rb + threadIdx.x; r < re; r += blockDim.x) {
        double z[RP];
#pragma unroll
        for (int c = 0; c < RP; ++c) z[c] = 0.0;
        for (int a = 0; a < cols; ++a) {
            const double v = V[(int64_t)a * ldv + r];
#pragma unroll
            for (int c = 0; c < RP; ++c) z[c] = fma(v, ws[a * RP + c], z[c]);
        }
#pragma unroll
        for (int c = 0; c < RP; ++c)
            if (c < p) {
                Z[(int64_t)c * ldz + r] += z[c];
                // restart copy: this thread's row only, after all its reads of the row
                if (restart_copy) V[(int64_t)c * ldv + r] = V[(int64_t)(cols - p + c) * ldv + r];
            }
    }
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

int64_t rows_per_block(int64_t n, int nblk) {
    int64_t r = (n + nblk - 1) / nblk;
    return (r + TR - 1) / TR * TR;
}
int blocks_for(int64_t n, int nblk) {
    const int64_t rpb = rows_per_block(n, nblk);
    return (int)((n + rpb - 1) / rpb);
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
                            cudaStream_t s) {
    const int nout = cols * p;
    k_reduce_h<<<(nout + RED_OUT - 1) / RED_OUT, RED_OUT * RED_STRIPES, 0, s>>>(
        part, nblk_req, cols, p, h, H, ldH, row0, col0, accumulate);
    return cudaGetLastError();
}

cudaError_t launch_qr_mixed_rows(double* W, int64_t ldw, int p, int64_t n, int nblk, double* G, double* part,
                                 unsigned* ctr, int mode, double* R, double* Rinv, const double* Rtot_in,
                                 double* Rtot_out, double* H, int ldH, int hrow, int hcol, double* normsq_out,
                                 int* flags, double* out, int64_t ldo, cudaStream_t s) {
    if (p > RP) return cudaErrorInvalidValue;
    const int64_t rpb = rows_per_block(n, nblk);
    const int g = blocks_for(n, nblk);
    if (mode == 0)
        k_qr_mixed_rows<1><<<g, NT, 0, s>>>(W, ldw, p, n, rpb, G, part, ctr, mode, R, Rinv, Rtot_in, Rtot_out, H,
                                            ldH, hrow, hcol, normsq_out, flags, out, ldo);
    else
        k_qr_mixed_rows<2><<<g, NT, 0, s>>>(W, ldw, p, n, rpb, G, part, ctr, mode, R, Rinv, Rtot_in, Rtot_out, H,
                                            ldH, hrow, hcol, normsq_out, flags, out, ldo);
    return cudaGetLastError();
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
    if (gram && p <= RP) {
        if (upd32)
            k_update_gram_rows<true><<<g, NT, sizeof(double) * (size_t)cols * RP, s>>>(V, ldv, cols, W, ldw, p, n,
                                                                                       rpb, h, part, G, ctr);
        else
            k_update_gram_rows<false><<<g, NT, sizeof(double) * (size_t)cols * RP, s>>>(V, ldv, cols, W, ldw, p, n,
                                                                                        rpb, h, part, G, ctr);
        return cudaGetLastError();
    }
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
    if (p <= RP) {
        k_trsm_rows<<<g, NT, 0, s>>>(W, ldw, p, n, rpb, Rinv, out, ldo, part, gram, extra, tmode);
        return cudaGetLastError();
    }
    EXPM_OPT_DISPATCH(p * p, (k_trsm<O><<<g, NT, 0, s>>>(W, ldw, p, n, rpb, Rinv, out, ldo, part, gram,
                                                       extra, tmode)));
    return cudaGetLastError();
}

cudaError_t launch_update_z(double* V, int64_t ldv, int cols, int p, int64_t n,
                            const double* Wc, double* Z, int64_t ldz, int restart_copy,
                            cudaStream_t s, int nblk) {
    const int64_t rpb = rows_per_block(n, nblk);
    const int g = blocks_for(n, nblk);
    if (p <= RP) {
        k_update_z_rows<<<g, NT, sizeof(double) * (size_t)cols * RP, s>>>(V, ldv, cols, p, n, rpb, Wc, Z, ldz,
                                                                         restart_copy);
        return cudaGetLastError();
    }
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
    EXPM_SET(k_update_gram_rows<false>);
    EXPM_SET(k_update_gram_rows<true>);
    EXPM_SET(k_update_z_rows);
#undef EXPM_SET
    return e;
}

}  // namespace expm
