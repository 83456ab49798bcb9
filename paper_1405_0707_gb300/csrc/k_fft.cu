// k_fft.cu -- FP64 complex FFT (four-step, Stockham radix 8/4/2) and the symmetric Toeplitz
// operator built on it: the product tT V by circulant embedding, and the exact inverse
// (tT)^{-1} V by the Gohberg-Semencul formula.
//
// Products (the fast Toeplitz product of Example 5.4; the 2n circulant of the commented
// remark in Section 2).  T (first column a_0..a_bw, zero beyond, symmetric) is the leading
// n x n block of the N x N circulant C with first column [a_0..a_bw, 0.., a_bw..a_1],
// N >= n + bw a power of two.  C = F^{-1} diag(lambda) F with lambda = F c real, so
//     T v = first n entries of F^{-1}(lambda . F [v; 0]),
// and because lambda is real, two real columns share one complex transform (v1 + i v2).
//
// Inverse (Section 4.1: the Gohberg-Semencul formula for A^{-1} when A is Toeplitz;
// Example 5.4).  With x = T^{-1} e_1 and xh = (0, x_{n-1}, .., x_1),
//     T^{-1} = ( L(x) L(x)^T - L(xh) L(xh)^T ) / x_0,
// L(y) the lower-triangular Toeplitz matrix with first column y.  L(y) is the leading block
// of the circulant of [y; 0] (spectrum mu = F[y; 0]) and L(y)^T that of its transpose
// (spectrum conj(mu)), so one apply is six transforms per column pair:
//     u_k = trunc_n F^{-1}(conj(mu_k) . F v),
//     T^{-1} v = trunc_n F^{-1}(mu_1 . F u_1 - mu_2 . F u_2) / x_0.
//
// Four-step transform, N = N1 N2, x index n = N2 n1 + n2, spectrum index k = k1 + N1 k2:
//   column pass (per n2): length-N1 DFT over n1, times W_N^{n2 k1}  -> U[k1][n2]
//   row pass    (per k1): length-N2 DFT over n2                     -> U[k1][k2] = X[k1 + N1 k2]
// The spectrum stays in this transposed order: pointwise products do not care, the plan's
// spectra are computed by the same passes, and the inverse runs the steps backwards (row
// pass, times W_N^{-n2 k1}, then column pass), so every pass reads and writes either
// contiguous rows or groups of C adjacent columns.  The pointwise spectral products are
// fused into the row pass (forward DFT, product, inverse DFT in one kernel), so a product
// costs three passes over the data and a Gohberg-Semencul apply five.  Every pass reads
// all of its lines into shared memory before it writes, and no two blocks share a line,
// so the passes may run in place.
//
// Line FFT: one line of length L (8 <= L <= 2048, so N <= 2^22) sits in shared memory
// (padded by one element per eight: conflict-free strides); L/8 threads hold 8 values each in
// registers per stage (one radix-8 butterfly, two radix-4 or four radix-2), Stockham
// ordering (natural order in and out, no bit reversal).  Twiddles come from tables built
// once with sincospi (exact argument reduction): W_L^k, k < L, and for the four-step factor
// W_N^e = T_hi[e >> 6] T_lo[e & 63].
#include <algorithm>

#include "df.cuh"
#include "internal.h"

namespace expm {
namespace {

struct c2 {
    double x, y;
};
__device__ __forceinline__ c2 cmul(c2 a, c2 b) { return {a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x}; }
// a * conj(b)
__device__ __forceinline__ c2 cmulc(c2 a, c2 b) { return {a.x * b.x + a.y * b.y, a.y * b.x - a.x * b.y}; }
__device__ __forceinline__ c2 cadd(c2 a, c2 b) { return {a.x + b.x, a.y + b.y}; }
__device__ __forceinline__ c2 csub(c2 a, c2 b) { return {a.x - b.x, a.y - b.y}; }
__device__ __forceinline__ c2 cscale(c2 a, double s) { return {a.x * s, a.y * s}; }
// multiply by -i (forward) or +i (inverse)
template <bool INV>
__device__ __forceinline__ c2 mul_mi(c2 a) { return INV ? c2{-a.y, a.x} : c2{a.y, -a.x}; }

__device__ __forceinline__ int pad(int i) { return i + (i >> 3); }

constexpr double kRsqrt2 = 0.70710678118654752440;

// ---- double-float complex numbers (each component a float pair h + l, ~2^-48 relative):
// the mixed path runs the butterflies on the FP32 pipe, 72x the FP64 rate on this GPU.
struct df {
    float h, l;
};
struct cdf {
    df x, y;
};
__device__ __forceinline__ df df_of(double v) {
    df r;
    split_df(v, r.h, r.l);
    return r;
}
__device__ __forceinline__ double df_val(df a) { return (double)a.h + (double)a.l; }
__device__ __forceinline__ df dadd(df a, df b) {
    const float s = a.h + b.h, bp = s - a.h;
    float e = (a.h - (s - bp)) + (b.h - bp);
    e += a.l + b.l;
    const float h = s + e;
    return {h, e - (h - s)};
}
__device__ __forceinline__ df dneg(df a) { return {-a.h, -a.l}; }
__device__ __forceinline__ df dsub(df a, df b) { return dadd(a, dneg(b)); }
__device__ __forceinline__ df dmul(df a, df b) {
    const float p = a.h * b.h;
    float e = fmaf(a.h, b.h, -p);
    e = fmaf(a.h, b.l, e);
    e = fmaf(a.l, b.h, e);
    const float h = p + e;
    return {h, e - (h - p)};
}
__device__ __forceinline__ cdf cadd(cdf a, cdf b) { return {dadd(a.x, b.x), dadd(a.y, b.y)}; }
__device__ __forceinline__ cdf csub(cdf a, cdf b) { return {dsub(a.x, b.x), dsub(a.y, b.y)}; }
__device__ __forceinline__ cdf cmul(cdf a, cdf b) {
    return {dsub(dmul(a.x, b.x), dmul(a.y, b.y)), dadd(dmul(a.x, b.y), dmul(a.y, b.x))};
}
__device__ __forceinline__ cdf cmulc(cdf a, cdf b) {
    return {dadd(dmul(a.x, b.x), dmul(a.y, b.y)), dsub(dmul(a.y, b.x), dmul(a.x, b.y))};
}
__device__ __forceinline__ cdf cscale(cdf a, double s) {
    const df d = df_of(s);
    return {dmul(a.x, d), dmul(a.y, d)};
}
template <bool INV>
__device__ __forceinline__ cdf mul_mi(cdf a) { return INV ? cdf{dneg(a.y), a.x} : cdf{a.y, dneg(a.x)}; }

// element access for both complex types
template <class T> __device__ __forceinline__ T czero();
template <> __device__ __forceinline__ c2 czero<c2>() { return {0.0, 0.0}; }
template <> __device__ __forceinline__ cdf czero<cdf>() { return {{0.f, 0.f}, {0.f, 0.f}}; }
template <class T> __device__ __forceinline__ T cmake(double re, double im);
template <> __device__ __forceinline__ c2 cmake<c2>(double re, double im) { return {re, im}; }
template <> __device__ __forceinline__ cdf cmake<cdf>(double re, double im) { return {df_of(re), df_of(im)}; }
__device__ __forceinline__ double cre(c2 a) { return a.x; }
__device__ __forceinline__ double cim(c2 a) { return a.y; }
__device__ __forceinline__ double cre(cdf a) { return df_val(a.x); }
__device__ __forceinline__ double cim(cdf a) { return df_val(a.y); }

// W8^1 o, W8^3 o (W8 = e^{-2 pi i / 8}, conjugated for the inverse)
template <bool INV>
__device__ __forceinline__ c2 w8_1(c2 o) {
    return INV ? c2{(o.x - o.y) * kRsqrt2, (o.x + o.y) * kRsqrt2} : c2{(o.x + o.y) * kRsqrt2, (o.y - o.x) * kRsqrt2};
}
template <bool INV>
__device__ __forceinline__ c2 w8_3(c2 o) {
    return INV ? c2{-(o.x + o.y) * kRsqrt2, (o.x - o.y) * kRsqrt2} : c2{(o.y - o.x) * kRsqrt2, -(o.x + o.y) * kRsqrt2};
}
__device__ __forceinline__ df r2df() { return {0.70710676908493042f, 1.2101617485882343e-08f}; }
template <bool INV>
__device__ __forceinline__ cdf w8_1(cdf o) {
    const df r = r2df();
    return INV ? cdf{dmul(dsub(o.x, o.y), r), dmul(dadd(o.x, o.y), r)}
               : cdf{dmul(dadd(o.x, o.y), r), dmul(dsub(o.y, o.x), r)};
}
template <bool INV>
__device__ __forceinline__ cdf w8_3(cdf o) {
    const df r = r2df();
    return INV ? cdf{dneg(dmul(dadd(o.x, o.y), r)), dmul(dsub(o.x, o.y), r)}
               : cdf{dmul(dsub(o.y, o.x), r), dneg(dmul(dadd(o.x, o.y), r))};
}

template <class T>
__device__ __forceinline__ void dft2(T& a, T& b) {
    const T t = a;
    a = cadd(t, b);
    b = csub(t, b);
}

template <bool INV, class T>
__device__ __forceinline__ void dft4(T& x0, T& x1, T& x2, T& x3) {
    const T s02 = cadd(x0, x2), d02 = csub(x0, x2), s13 = cadd(x1, x3), d13 = mul_mi<INV>(csub(x1, x3));
    x0 = cadd(s02, s13);
    x2 = csub(s02, s13);
    x1 = cadd(d02, d13);
    x3 = csub(d02, d13);
}

// 8-point DFT in place (natural order in and out): 4-point DFTs E, O of the even and odd
// samples, then X_k = E_k + W8^k O_k, X_{k+4} = E_k - W8^k O_k.
template <bool INV, class T>
__device__ __forceinline__ void dft8(T* v) {
    T e0 = v[0], e1 = v[2], e2 = v[4], e3 = v[6];
    T o0 = v[1], o1 = v[3], o2 = v[5], o3 = v[7];
    dft4<INV>(e0, e1, e2, e3);
    dft4<INV>(o0, o1, o2, o3);
    const T w1 = w8_1<INV>(o1);
    const T w2 = mul_mi<INV>(o2);
    const T w3 = w8_3<INV>(o3);
    v[0] = cadd(e0, o0);
    v[4] = csub(e0, o0);
    v[1] = cadd(e1, w1);
    v[5] = csub(e1, w1);
    v[2] = cadd(e2, w2);
    v[6] = csub(e2, w2);
    v[3] = cadd(e3, w3);
    v[7] = csub(e3, w3);
}

__device__ __forceinline__ c2 ld2(const double* p, int64_t i) {
    const double2 v = __ldg(reinterpret_cast<const double2*>(p) + i);
    return {v.x, v.y};
}
__device__ __forceinline__ void st2(double* p, int64_t i, c2 v) {
    reinterpret_cast<double2*>(p)[i] = make_double2(v.x, v.y);
}
// complex element i of an interleaved FP64 array, as T
template <class T> __device__ __forceinline__ T ldc(const double* p, int64_t i);
template <> __device__ __forceinline__ c2 ldc<c2>(const double* p, int64_t i) { return ld2(p, i); }
template <> __device__ __forceinline__ cdf ldc<cdf>(const double* p, int64_t i) {
    const c2 v = ld2(p, i);
    return {df_of(v.x), df_of(v.y)};
}
__device__ __forceinline__ void stc(double* p, int64_t i, c2 v) { st2(p, i, v); }
__device__ __forceinline__ void stc(double* p, int64_t i, cdf v) { st2(p, i, c2{cre(v), cim(v)}); }
// twiddle k of a table: interleaved FP64 (c2) or float4 pairs (cdf)
template <class T> __device__ __forceinline__ T ldtw(const void* tab, int64_t k);
template <> __device__ __forceinline__ c2 ldtw<c2>(const void* tab, int64_t k) {
    return ld2(static_cast<const double*>(tab), k);
}
template <> __device__ __forceinline__ cdf ldtw<cdf>(const void* tab, int64_t k) {
    const float4 v = __ldg(static_cast<const float4*>(tab) + k);
    return {{v.x, v.y}, {v.z, v.w}};
}

// Stockham FFT of the line s[pad(0..L)) by the L/8 threads q of its group.  Every thread of
// the block calls this with the same L (the barriers are block-wide); a thread whose group
// is inactive only takes part in the barriers.  Ends with a barrier.
template <bool INV, class T>
__device__ void line_fft(T* s, int L, int q, const void* tw, bool active) {
    const int G = L >> 3;
    T v[8];
    for (int Ns = 1; Ns < L;) {
        const int R = (L / Ns >= 8) ? 8 : L / Ns;
        const int LR = L / R;
        if (active) {
            if (R == 8) {
#pragma unroll
                for (int r = 0; r < 8; ++r) v[r] = s[pad(q + r * LR)];
            } else if (R == 4) {
#pragma unroll
                for (int b = 0; b < 2; ++b)
#pragma unroll
                    for (int r = 0; r < 4; ++r) v[4 * b + r] = s[pad(q + b * G + r * LR)];
            } else {
#pragma unroll
                for (int b = 0; b < 4; ++b)
#pragma unroll
                    for (int r = 0; r < 2; ++r) v[2 * b + r] = s[pad(q + b * G + r * LR)];
            }
        }
        __syncthreads();
        if (active) {
            const int tstep = L / (Ns * R);
            if (R == 8) {
                const int k = q & (Ns - 1);
                if (Ns > 1) {
#pragma unroll
                    for (int r = 1; r < 8; ++r) {
                        const T t = ldtw<T>(tw, r * k * tstep);
                        v[r] = INV ? cmulc(v[r], t) : cmul(v[r], t);
                    }
                }
                dft8<INV>(v);
                const int base = (q - k) * 8 + k;
#pragma unroll
                for (int r = 0; r < 8; ++r) s[pad(base + r * Ns)] = v[r];
            } else if (R == 4) {
#pragma unroll
                for (int b = 0; b < 2; ++b) {
                    const int j = q + b * G, k = j & (Ns - 1);
                    T* w = v + 4 * b;
                    if (Ns > 1) {
#pragma unroll
                        for (int r = 1; r < 4; ++r) {
                            const T t = ldtw<T>(tw, r * k * tstep);
                            w[r] = INV ? cmulc(w[r], t) : cmul(w[r], t);
                        }
                    }
                    dft4<INV>(w[0], w[1], w[2], w[3]);
                    const int base = (j - k) * 4 + k;
#pragma unroll
                    for (int r = 0; r < 4; ++r) s[pad(base + r * Ns)] = w[r];
                }
            } else {
#pragma unroll
                for (int b = 0; b < 4; ++b) {
                    const int j = q + b * G, k = j & (Ns - 1);
                    T* w = v + 2 * b;
                    if (Ns > 1) {
                        const T t = ldtw<T>(tw, k * tstep);
                        w[1] = INV ? cmulc(w[1], t) : cmul(w[1], t);
                    }
                    dft2(w[0], w[1]);
                    const int base = (j - k) * 2 + k;
                    s[pad(base)] = w[0];
                    s[pad(base + Ns)] = w[1];
                }
            }
        }
        __syncthreads();
        Ns *= R;
    }
}

// the twiddle tables of one arithmetic: FP64 (c2) or float pairs (cdf)
template <class T> __device__ __forceinline__ const void* tab_tw1(const FftArgs& a);
template <> __device__ __forceinline__ const void* tab_tw1<c2>(const FftArgs& a) { return a.tw1; }
template <> __device__ __forceinline__ const void* tab_tw1<cdf>(const FftArgs& a) { return a.tw1f; }
template <class T> __device__ __forceinline__ const void* tab_tw2(const FftArgs& a);
template <> __device__ __forceinline__ const void* tab_tw2<c2>(const FftArgs& a) { return a.tw2; }
template <> __device__ __forceinline__ const void* tab_tw2<cdf>(const FftArgs& a) { return a.tw2f; }

// W_N^e from the split tables
template <class T>
__device__ __forceinline__ T twN(const FftArgs& a, int64_t e);
template <>
__device__ __forceinline__ c2 twN<c2>(const FftArgs& a, int64_t e) {
    return cmul(ld2(a.thi, e >> 6), ld2(a.tlo, e & 63));
}
template <>
__device__ __forceinline__ cdf twN<cdf>(const FftArgs& a, int64_t e) {
    return cmul(ldtw<cdf>(a.thif, e >> 6), ldtw<cdf>(a.tlof, e & 63));
}

// ------------------------------------------------------------------ column pass
template <int MODE, class T>
__global__ void __launch_bounds__(512) k_fft_cols(const FftArgs a) {
    extern __shared__ __align__(16) unsigned char sm_raw[];
    T* sm = reinterpret_cast<T*>(sm_raw);
    const int L = a.f.N1, G = L >> 3, C = a.f.C;
    const int N2 = a.f.N2, PL = pad(L);
    const int64_t N = a.f.N;
    const int b = blockIdx.y, c0 = blockIdx.x * C;
    const int tid = threadIdx.x, nthr = blockDim.x;
    const int line = tid / G, q = tid - line * G;
    T* s = sm + line * PL;
    const int64_t seq = (int64_t)b * N;
    for (int e = tid; e < C * L; e += nthr) {
        const int c = e % C, r = e / C;
        const int64_t g = (int64_t)r * N2 + c0 + c;
        T v = czero<T>();
        if (MODE == FFT_COL_FWD_REAL) {
            if (g < a.nreal) {
                const double re = a.V[(int64_t)(2 * b) * a.ldv + g];
                const double im = (2 * b + 1 < a.p) ? a.V[(int64_t)(2 * b + 1) * a.ldv + g] : 0.0;
                v = cmake<T>(re, im);
            }
        } else {
            v = ldc<T>(a.in, seq + g);
        }
        sm[c * PL + pad(r)] = v;
    }
    __syncthreads();
    constexpr bool kInv = (MODE == FFT_COL_INV_REAL || MODE == FFT_COL_INV_CPLX || MODE == FFT_COL_INV_TRUNC_FWD);
    line_fft<kInv, T>(s, L, q, tab_tw1<T>(a), true);
    if (MODE == FFT_COL_INV_TRUNC_FWD) {
        // keep the first n entries only, then transform forward again
        for (int e = tid; e < C * L; e += nthr) {
            const int c = e % C, r = e / C;
            if ((int64_t)r * N2 + c0 + c >= a.nreal) sm[c * PL + pad(r)] = czero<T>();
        }
        __syncthreads();
        line_fft<false, T>(s, L, q, tab_tw1<T>(a), true);
    }
    for (int e = tid; e < C * L; e += nthr) {
        const int c = e % C, r = e / C;
        const int64_t g = (int64_t)r * N2 + c0 + c;
        const T v = sm[c * PL + pad(r)];
        if (MODE == FFT_COL_INV_REAL) {
            if (g < a.nreal) {
                a.W[(int64_t)(2 * b) * a.ldw + g] = cre(v) * a.scale;
                if (2 * b + 1 < a.p) a.W[(int64_t)(2 * b + 1) * a.ldw + g] = cim(v) * a.scale;
            }
        } else if (MODE == FFT_COL_INV_CPLX) {
            stc(a.out, seq + g, cscale(v, a.scale));
        } else {
            stc(a.out, seq + g, cmul(v, twN<T>(a, (int64_t)(c0 + c) * r)));
        }
    }
}

// ------------------------------------------------------------------ row pass
template <int MODE, int LPR, class T>
__device__ __forceinline__ void row_spectral_inverse(const FftArgs& a, T* sm, T* s, int L, int Rr, int PL,
                                                     int k1_0, int64_t seq, int q, int sub);

template <int MODE, class T>
__global__ void __launch_bounds__(512) k_fft_rows(const FftArgs a) {
    extern __shared__ __align__(16) unsigned char sm_raw[];
    T* sm = reinterpret_cast<T*>(sm_raw);
    constexpr int LPR = (MODE == FFT_ROW_GSF_A || MODE == FFT_ROW_GSF_B) ? 2 : 1;   // lines per row
    const int L = a.f.N2, G = L >> 3, Rr = a.f.Rr;
    const int PL = pad(L);
    const int64_t N = a.f.N;
    const int b = blockIdx.y, k1_0 = blockIdx.x * Rr;
    const int tid = threadIdx.x, nthr = blockDim.x;
    const int line = tid / G, q = tid - line * G, sub = line % LPR;
    T* s = sm + line * PL;
    const int64_t seq = (int64_t)b * N;
    for (int e = tid; e < Rr * LPR * L; e += nthr) {
        const int ln = e / L, i = e - ln * L, row = ln / LPR, sb = ln % LPR;
        if (MODE == FFT_ROW_GSF_A && sb == 1) continue;
        const double* src = sb == 0 ? a.in : a.in2;
        sm[ln * PL + pad(i)] = ldc<T>(src, seq + (int64_t)(k1_0 + row) * L + i);
    }
    __syncthreads();
    line_fft<false, T>(s, L, q, tab_tw2<T>(a), !(MODE == FFT_ROW_GSF_A && sub == 1));
    if constexpr (MODE == FFT_ROW_FWD) {
        for (int e = tid; e < Rr * L; e += nthr) {
            const int row = e / L, i = e - row * L;
            stc(a.out, seq + (int64_t)(k1_0 + row) * L + i, sm[row * PL + pad(i)]);
        }
        return;
    } else {
        row_spectral_inverse<MODE, LPR, T>(a, sm, s, L, Rr, PL, k1_0, seq, q, sub);
    }
}

// The rest of a row pass: pointwise spectral step, inverse row DFT, W_N^{-n2 k1}, store.
template <int MODE, int LPR, class T>
__device__ __forceinline__ void row_spectral_inverse(const FftArgs& a, T* sm, T* s, int L, int Rr, int PL,
                                                     int k1_0, int64_t seq, int q, int sub) {
    const int tid = threadIdx.x, nthr = blockDim.x;
    // pointwise spectral step (the plan's spectra are stored in the same transposed order)
    for (int e = tid; e < Rr * L; e += nthr) {
        const int row = e / L, i = e - row * L;
        const int64_t idx = (int64_t)(k1_0 + row) * L + i;
        T* s0 = sm + (row * LPR) * PL + pad(i);
        if (MODE == FFT_ROW_MATVEC) {
            *s0 = cscale(*s0, a.lam[idx] * a.scale);
        } else if (MODE == FFT_ROW_GSF_A) {
            const T y = *s0;
            s0[PL] = cscale(cmulc(y, ldc<T>(a.mu2, idx)), a.scale);
            *s0 = cscale(cmulc(y, ldc<T>(a.mu1, idx)), a.scale);
        } else {   // FFT_ROW_GSF_B
            *s0 = cscale(csub(cmul(*s0, ldc<T>(a.mu1, idx)), cmul(s0[PL], ldc<T>(a.mu2, idx))), a.scale);
        }
    }
    __syncthreads();
    line_fft<true, T>(s, L, q, tab_tw2<T>(a), MODE == FFT_ROW_GSF_A || sub == 0);
    for (int e = tid; e < Rr * LPR * L; e += nthr) {
        const int ln = e / L, i = e - ln * L, row = ln / LPR, sb = ln % LPR;
        if (MODE != FFT_ROW_GSF_A && sb == 1) continue;
        const int k1 = k1_0 + row;
        double* dst = sb == 0 ? a.out : a.out2;
        stc(dst, seq + (int64_t)k1 * L + i, cmulc(sm[ln * PL + pad(i)], twN<T>(a, (int64_t)i * k1)));
    }
}

// ------------------------------------------------------------------ tables and helpers
__global__ void k_fft_tables(double* tw1, int N1, double* tw2, int N2, double* thi, double* tlo, int64_t N) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    double s, c;
    if (e < N1) { sincospi(-2.0 * (double)e / N1, &s, &c); st2(tw1, e, c2{c, s}); }
    if (e < N2) { sincospi(-2.0 * (double)e / N2, &s, &c); st2(tw2, e, c2{c, s}); }
    if (e < N / 64) { sincospi(-2.0 * (double)(64 * e) / (double)N, &s, &c); st2(thi, e, c2{c, s}); }
    if (e < 64) { sincospi(-2.0 * (double)e / (double)N, &s, &c); st2(tlo, e, c2{c, s}); }
}

// a complex FP64 table as float pairs (re_hi, re_lo, im_hi, im_lo) for the double-float passes
__global__ void k_tab_df(const double* __restrict__ src, float* __restrict__ dst, int64_t count) {
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= count) return;
    float4 v;
    split_df(src[2 * k], v.x, v.y);
    split_df(src[2 * k + 1], v.z, v.w);
    reinterpret_cast<float4*>(dst)[k] = v;
}

// sequence 0: the circulant's first column (Toeplitz embedding), imaginary parts zero
__global__ void k_embed_toeplitz(const double* __restrict__ a, int64_t bw, int64_t N, double* __restrict__ U) {
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= N) return;
    double v = 0.0;
    if (k <= bw) v = a[k];
    else if (N - k <= bw) v = a[N - k];
    st2(U, k, c2{v, 0.0});
}

// sequences 0 and 1: [x; 0] and [xh; 0], xh = (0, x_{n-1}, .., x_1)
__global__ void k_embed_gsf(const double* __restrict__ x, int64_t n, int64_t N, double* __restrict__ U) {
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= N) return;
    st2(U, k, c2{k < n ? x[k] : 0.0, 0.0});
    st2(U, N + k, c2{(k >= 1 && k < n) ? x[n - k] : 0.0, 0.0});
}

__global__ void k_real_part(const double* __restrict__ U, double* __restrict__ lam, int64_t N) {
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k < N) lam[k] = U[2 * k];
}

// ---- conjugate gradients for the generator x = T^{-1} e_1 (plan setup only)
constexpr int kDotBlocks = 256;
__global__ void __launch_bounds__(256) k_dot_partial(const double* __restrict__ a, const double* __restrict__ b,
                                                     int64_t n, double* __restrict__ part) {
    __shared__ double red[256];
    double s = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        s = fma(a[i], b[i], s);
    red[threadIdx.x] = s;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) part[blockIdx.x] = red[0];
}

// x += alpha p, r -= alpha w
__global__ void k_cg_step(double* __restrict__ x, double* __restrict__ r, const double* __restrict__ p,
                          const double* __restrict__ w, double alpha, int64_t n) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    x[i] = fma(alpha, p[i], x[i]);
    r[i] = fma(-alpha, w[i], r[i]);
}

// p = r + beta p
__global__ void k_cg_dir(double* __restrict__ p, const double* __restrict__ r, double beta, int64_t n) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) p[i] = fma(beta, p[i], r[i]);
}

__global__ void k_unit(double* __restrict__ v, int64_t n) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) v[i] = i == 0 ? 1.0 : 0.0;
}

inline unsigned blocks_for(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

constexpr int kFftSmemMax = 200 * 1024;

template <class K>
cudaError_t set_smem(K kernel) {
    return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kFftSmemMax);
}

}  // namespace

// ------------------------------------------------------------------ host side
FftPlan fft_geometry(int64_t nmin) {
    FftPlan f;
    int k = 6;
    while ((int64_t(1) << k) < nmin) ++k;
    f.N = int64_t(1) << k;
    f.N1 = 1 << (k / 2);
    f.N2 = 1 << (k - k / 2);
    const int G1 = f.N1 / 8, G2 = f.N2 / 8;
    const int line1 = (f.N1 + f.N1 / 8) * 16, line2 = (f.N2 + f.N2 / 8) * 16;
    // columns per block: at least 4 adjacent columns (64-byte segments), ~256 threads
    int C = std::max(4, 256 / G1);
    C = std::min(C, 512 / G1);
    C = std::min(C, kFftSmemMax / line1);
    f.C = std::max(1, std::min(C, f.N2));
    // rows per block; the Gohberg-Semencul row passes hold two lines per row
    int Rr = std::max(1, 256 / G2);
    Rr = std::min(Rr, 512 / (2 * G2));
    Rr = std::min(Rr, kFftSmemMax / (2 * line2));
    f.Rr = std::max(1, std::min(Rr, f.N1));
    return f;
}

bool fft_geometry_ok(const FftPlan& f) {
    return f.N >= 64 && f.N1 >= 8 && f.N2 >= 8 && f.N1 <= 2048 && f.N2 <= 2048 && f.C >= 1 && f.Rr >= 1 &&
           f.N2 % f.C == 0 && f.N1 % f.Rr == 0 && 2 * f.Rr * (f.N2 / 8) <= 512 && f.C * (f.N1 / 8) <= 512 &&
           (size_t)f.C * (f.N1 + f.N1 / 8) * 16 <= (size_t)kFftSmemMax &&
           (size_t)2 * f.Rr * (f.N2 + f.N2 / 8) * 16 <= (size_t)kFftSmemMax;
}

template <class T>
cudaError_t fft_set_smem_limits_t() {
    cudaError_t e = set_smem(k_fft_cols<FFT_COL_FWD_REAL, T>);
    if (e == cudaSuccess) e = set_smem(k_fft_cols<FFT_COL_FWD_CPLX, T>);
    if (e == cudaSuccess) e = set_smem(k_fft_cols<FFT_COL_INV_REAL, T>);
    if (e == cudaSuccess) e = set_smem(k_fft_cols<FFT_COL_INV_CPLX, T>);
    if (e == cudaSuccess) e = set_smem(k_fft_cols<FFT_COL_INV_TRUNC_FWD, T>);
    if (e == cudaSuccess) e = set_smem(k_fft_rows<FFT_ROW_FWD, T>);
    if (e == cudaSuccess) e = set_smem(k_fft_rows<FFT_ROW_MATVEC, T>);
    if (e == cudaSuccess) e = set_smem(k_fft_rows<FFT_ROW_GSF_A, T>);
    if (e == cudaSuccess) e = set_smem(k_fft_rows<FFT_ROW_GSF_B, T>);
    return e;
}

cudaError_t fft_set_smem_limits() {
    const cudaError_t e = fft_set_smem_limits_t<c2>();
    return e == cudaSuccess ? fft_set_smem_limits_t<cdf>() : e;
}

cudaError_t launch_fft_tables(const FftPlan& f, double* tw1, double* tw2, double* thi, double* tlo,
                              cudaStream_t s) {
    const int64_t tot = std::max<int64_t>(f.N / 64, std::max(std::max(f.N1, f.N2), 64));
    k_fft_tables<<<blocks_for(tot, 256), 256, 0, s>>>(tw1, f.N1, tw2, f.N2, thi, tlo, f.N);
    return cudaGetLastError();
}

template <class T>
cudaError_t launch_fft_cols_t(const FftArgs& a, int mode, int nseq, cudaStream_t s) {
    const dim3 grid((unsigned)(a.f.N2 / a.f.C), (unsigned)nseq);
    const int threads = a.f.C * (a.f.N1 / 8);
    const size_t smem = (size_t)a.f.C * (a.f.N1 + a.f.N1 / 8) * sizeof(T);
    switch (mode) {
        case FFT_COL_FWD_REAL: k_fft_cols<FFT_COL_FWD_REAL, T><<<grid, threads, smem, s>>>(a); break;
        case FFT_COL_FWD_CPLX: k_fft_cols<FFT_COL_FWD_CPLX, T><<<grid, threads, smem, s>>>(a); break;
        case FFT_COL_INV_REAL: k_fft_cols<FFT_COL_INV_REAL, T><<<grid, threads, smem, s>>>(a); break;
        case FFT_COL_INV_CPLX: k_fft_cols<FFT_COL_INV_CPLX, T><<<grid, threads, smem, s>>>(a); break;
        case FFT_COL_INV_TRUNC_FWD: k_fft_cols<FFT_COL_INV_TRUNC_FWD, T><<<grid, threads, smem, s>>>(a); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

template <class T>
cudaError_t launch_fft_rows_t(const FftArgs& a, int mode, int nseq, cudaStream_t s) {
    const int lpr = (mode == FFT_ROW_GSF_A || mode == FFT_ROW_GSF_B) ? 2 : 1;
    const dim3 grid((unsigned)(a.f.N1 / a.f.Rr), (unsigned)nseq);
    const int threads = a.f.Rr * lpr * (a.f.N2 / 8);
    const size_t smem = (size_t)a.f.Rr * lpr * (a.f.N2 + a.f.N2 / 8) * sizeof(T);
    switch (mode) {
        case FFT_ROW_FWD: k_fft_rows<FFT_ROW_FWD, T><<<grid, threads, smem, s>>>(a); break;
        case FFT_ROW_MATVEC: k_fft_rows<FFT_ROW_MATVEC, T><<<grid, threads, smem, s>>>(a); break;
        case FFT_ROW_GSF_A: k_fft_rows<FFT_ROW_GSF_A, T><<<grid, threads, smem, s>>>(a); break;
        case FFT_ROW_GSF_B: k_fft_rows<FFT_ROW_GSF_B, T><<<grid, threads, smem, s>>>(a); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

// The passes run in FP64, or (a.df, with the float-pair tables set) in double-float.
cudaError_t launch_fft_cols(const FftArgs& a, int mode, int nseq, cudaStream_t s) {
    if (a.df && !(a.tw1f && a.thif && a.tlof)) return cudaErrorInvalidValue;
    return a.df ? launch_fft_cols_t<cdf>(a, mode, nseq, s) : launch_fft_cols_t<c2>(a, mode, nseq, s);
}

cudaError_t launch_fft_rows(const FftArgs& a, int mode, int nseq, cudaStream_t s) {
    if (a.df && !(a.tw2f && a.thif && a.tlof)) return cudaErrorInvalidValue;
    return a.df ? launch_fft_rows_t<cdf>(a, mode, nseq, s) : launch_fft_rows_t<c2>(a, mode, nseq, s);
}

cudaError_t launch_fft_tables_df(const double* src, float* dst, int64_t count, cudaStream_t s) {
    k_tab_df<<<blocks_for(count, 256), 256, 0, s>>>(src, dst, count);
    return cudaGetLastError();
}

cudaError_t launch_embed_toeplitz(const double* a, int64_t bw, int64_t N, double* U, cudaStream_t s) {
    k_embed_toeplitz<<<blocks_for(N, 256), 256, 0, s>>>(a, bw, N, U);
    return cudaGetLastError();
}

cudaError_t launch_embed_gsf(const double* x, int64_t n, int64_t N, double* U, cudaStream_t s) {
    k_embed_gsf<<<blocks_for(N, 256), 256, 0, s>>>(x, n, N, U);
    return cudaGetLastError();
}

cudaError_t launch_real_part(const double* U, double* lam, int64_t N, cudaStream_t s) {
    k_real_part<<<blocks_for(N, 256), 256, 0, s>>>(U, lam, N);
    return cudaGetLastError();
}

int dot_blocks() { return kDotBlocks; }

cudaError_t launch_dot_partial(const double* a, const double* b, int64_t n, double* part, cudaStream_t s) {
    k_dot_partial<<<kDotBlocks, 256, 0, s>>>(a, b, n, part);
    return cudaGetLastError();
}

cudaError_t launch_cg_step(double* x, double* r, const double* p, const double* w, double alpha, int64_t n,
                           cudaStream_t s) {
    k_cg_step<<<blocks_for(n, 256), 256, 0, s>>>(x, r, p, w, alpha, n);
    return cudaGetLastError();
}

cudaError_t launch_cg_dir(double* p, const double* r, double beta, int64_t n, cudaStream_t s) {
    k_cg_dir<<<blocks_for(n, 256), 256, 0, s>>>(p, r, beta, n);
    return cudaGetLastError();
}

cudaError_t launch_unit(double* v, int64_t n, cudaStream_t s) {
    k_unit<<<blocks_for(n, 256), 256, 0, s>>>(v, n);
    return cudaGetLastError();
}

}  // namespace expm
