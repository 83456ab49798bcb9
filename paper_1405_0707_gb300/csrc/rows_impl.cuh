// rows_impl.cuh -- row-per-thread kernels of the block Gram-Schmidt / Cholesky-QR passes.
//
// Row-per-thread kernels for p <= RP (compiled for RP = 8 and RP = 16, see k_krylov.cu): a
// row of W lives in registers, W R^{-1} and the upper-triangular outer product w^T w are
// formed there, and the Gram partial of the CTA is staged through shared memory at the end.
// Loads and stores are coalesced per column (consecutive threads, consecutive rows); no tile
// barriers.  Included by k_krylov.cu inside a namespace that defines RP (columns per row),
// RG = RP (RP + 1) / 2 (Gram entries), NQ = ceil(RG / 32) (entries per lane) and NTR
// (threads per CTA).

__device__ inline double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Gram partial of rows held one per lane: each warp stages its 32 rows in shared memory
// (buf, 32 x RP), then lane l sums upper-triangle entries l and l + 32 over those rows.
// FP64 work equals the useful products; no reduction tree.  Every lane of the warp must
// call it (rows past the end are zero).
__device__ inline void warp_gram_rows(const double* y, double* buf, double* acc) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int c = 0; c < RP; ++c) buf[lane * RP + c] = y[c];
    __syncwarp();
    // upper-triangle entry k -> (c1, c2)
    for (int q = 0; q < NQ; ++q) {
        const int kk = lane + 32 * q;
        if (kk < RG) {
            int c1 = 0, rem = kk;
            while (rem >= RP - c1) { rem -= RP - c1; ++c1; }
            const int c2 = c1 + rem;
            double s = 0.0;
#pragma unroll 8
            for (int rr = 0; rr < 32; ++rr) s = fma(buf[rr * RP + c1], buf[rr * RP + c2], s);
            acc[q] += s;
        }
    }
    __syncwarp();
}

// FP32 variant (the mixed path's Gram for the first Cholesky-QR pass, whose factorisation
// is FP32 anyway): rows staged as floats, products and per-lane sums in FP32.
__device__ inline void warp_gram_rows32(const double* y, float* buf, float* acc) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int c = 0; c < RP; ++c) buf[lane * RP + c] = f32_rn_i(y[c]);
    __syncwarp();
    for (int q = 0; q < NQ; ++q) {
        const int kk = lane + 32 * q;
        if (kk < RG) {
            int c1 = 0, rem = kk;
            while (rem >= RP - c1) { rem -= RP - c1; ++c1; }
            const int c2 = c1 + rem;
            float s = 0.f;
#pragma unroll 8
            for (int rr = 0; rr < 32; ++rr) s = fmaf(buf[rr * RP + c1], buf[rr * RP + c2], s);
            acc[q] += s;
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
    for (int q = 0; q < NQ; ++q) {
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
__device__ inline void cta_gram_write(const double* acc, int p, double (*red)[RG], double* __restrict__ part) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int q = 0; q < NQ; ++q)
        if (lane + 32 * q < RG) red[wid][lane + 32 * q] = acc[q];
    __syncthreads();
    for (int o = threadIdx.x; o < p * p; o += blockDim.x) {
        const int c1 = o / p, c2 = o % p;
        double s = 0.0;
        if (c1 <= c2) {
            const int k = c1 * RP - c1 * (c1 - 1) / 2 + (c2 - c1);
            for (int w_ = 0; w_ < NTR / 32; ++w_) s += red[w_][k];
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
// TwoSum accumulation): the FP32 pipe instead of the FP64 one for the last CTA's tail.  With
// nout < NTR outputs, NTR / nout stripes per output are added in a fixed order; otherwise one
// thread per output.
__device__ inline void last_cta_sum_df(const double* part, int nblk, int nout, double* __restrict__ out,
                                       unsigned* ctr) {
    __shared__ float redh[NTR], redl[NTR];
    __threadfence();
    if (nout >= NTR) {
        for (int o = threadIdx.x; o < nout; o += blockDim.x) {
            float sh = 0.f, sl = 0.f;
            for (int b = 0; b < nblk; ++b) {
                float h, l;
                split_df(__ldcg(part + (int64_t)b * nout + o), h, l);
                df_add(sh, sl, h);
                sl += l;
            }
            out[o] = (double)sh + (double)sl;
        }
        __syncthreads();
        if (threadIdx.x == 0) *ctr = 0u;
        return;
    }
    const int stripes = NTR / nout;
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

// out[o] = sum_b part[b][o] by the last CTA (same layout as last_cta_sum_df).  ACC = float:
// FP32 sums (for a Gram matrix that only feeds an FP32 factorisation).
template <typename ACC = double>
__device__ inline void last_cta_sum(const double* part, int nblk, int nout, double* __restrict__ out,
                                    unsigned* ctr) {
    __shared__ double red[NTR];
    __threadfence();
    if (nout >= NTR) {
        for (int o = threadIdx.x; o < nout; o += blockDim.x) {
            ACC a0 = 0, a1 = 0;
            int b = 0;
            for (; b + 1 < nblk; b += 2) {
                a0 += (ACC)__ldcg(part + (int64_t)b * nout + o);
                a1 += (ACC)__ldcg(part + (int64_t)(b + 1) * nout + o);
            }
            if (b < nblk) a0 += (ACC)__ldcg(part + (int64_t)b * nout + o);
            out[o] = (double)(a0 + a1);
        }
        __syncthreads();
        if (threadIdx.x == 0) *ctr = 0u;
        return;
    }
    const int stripes = NTR / nout;
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

struct CholF {
    float G[RP * RP], U[RP * RP], Y[RP * RP];
    float rd[RP];
    float umax;       // KIND 2: max |U|
    int ill, bad;
};

// The p x p factorisations run on warp 0 with lane l holding column l of the working matrix
// and of the factor in registers; the pivot row's entries reach the other lanes by shuffles
// (no shared-memory round trips on the serial path).  Every lane of warp 0 must call them.

// pass 1: FP32 Cholesky of G 2^-k (upper triangle) -> U; warp 0
__device__ inline void chol32_full(CholF& cf, const double* G0, int p, int k, double tr_s) {
    const int lane = threadIdx.x;
    const unsigned full = 0xffffffffu;
    const bool act = lane < p;
    float u[RP];                      // u[a] = U[a][lane]
    int ill = 0;
    for (int attempt = 0; attempt < 2; ++attempt) {
        const double shift = attempt ? 11.0 * p * (p + 1) * 0x1p-24 * tr_s : 0.0;
        float g[RP];                  // g[a] = G[a][lane], updated in place
        float dg = 0.f;
#pragma unroll
        for (int a = 0; a < RP; ++a) {
            g[a] = (act && a < p) ? (float)(ldexp(G0[a * p + lane], -k) + (a == lane ? shift : 0.0)) : 0.f;
            u[a] = 0.f;
            if (a == lane) dg = g[a];
        }
        float dmax = act ? dg : 0.f;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) dmax = fmaxf(dmax, __shfl_xor_sync(full, dmax, o));
        int ill_l = 0;
#pragma unroll
        for (int j = 0; j < RP; ++j) {
            if (j >= p) break;
            float inv = 0.f;
            if (lane == j) {
                float d = g[j];
                if (G0[j * p + j] == 0.0) {
                    u[j] = 0.f;
                } else {
                    if (!(d > 0.f) || !isfinite(d) || (attempt == 0 && d < 1e-6f * dmax)) ill_l = 1;
                    if (!(d > 0.f) || !isfinite(d)) d = 1.f;
                    const float rj = sqrtf(d);
                    u[j] = rj;
                    inv = 1.f / rj;
                }
            }
            inv = __shfl_sync(full, inv, j);
            if (act && lane > j) u[j] = g[j] * inv;
            // trailing update G[a][l] -= U[j][a] U[j][l] for j < a <= l
#pragma unroll
            for (int a = j + 1; a < RP; ++a) {
                const float uja = __shfl_sync(full, u[j], a);
                if (act && a < p && a <= lane) g[a] -= uja * u[j];
            }
        }
        if (__any_sync(full, ill_l)) ill = 1;     // sticky: a shifted pass 1 asks for pass 3
        if (attempt == 1 || !ill) break;
    }
    if (act)
#pragma unroll
        for (int a = 0; a < RP; ++a)
            if (a < p) cf.U[a * p + lane] = u[a];
    if (lane == 0) {
        cf.ill = ill;
        cf.bad = 0;
    }
    __syncwarp();
}

// passes 2/3: deviation Cholesky of G = I + E -> U (R = I + U), Y (R^{-1} = I + Y); warp 0
__device__ inline void chol32_dev(CholF& cf, const double* G0, int p) {
    const int lane = threadIdx.x;
    const unsigned full = 0xffffffffu;
    const bool act = lane < p;
    float e[RP], u[RP], y[RP];        // column `lane` of E, U and Y
#pragma unroll
    for (int a = 0; a < RP; ++a) {
        e[a] = (act && a < p) ? (float)(G0[a * p + lane] - (a == lane ? 1.0 : 0.0)) : 0.f;
        u[a] = 0.f;
        y[a] = 0.f;
    }
    int bad = 0;
    float rdl = 0.f;                  // lane j: 1 / (1 + U_jj)
#pragma unroll
    for (int j = 0; j < RP; ++j) {
        if (j >= p) break;
        // U[k][j] for k < j from lane j
        float ucol[RP];
#pragma unroll
        for (int k2 = 0; k2 < RP; ++k2) ucol[k2] = (k2 < j) ? __shfl_sync(full, u[k2], j) : 0.f;
        if (lane == j) {
            if (G0[j * p + j] == 0.0) {
                u[j] = -1.f;                          // R_jj = 0: a zero column stays zero
                rdl = 0.f;
            } else {
                float x = e[j];
#pragma unroll
                for (int k2 = 0; k2 < RP; ++k2)
                    if (k2 < j) x -= u[k2] * u[k2];
                if (!(x > -0.75f) || !isfinite(x)) bad = 1;   // not close to orthonormal
                if (!(x > -0.75f) || !isfinite(x)) x = 0.f;
                const float ujj = x / (1.f + sqrtf(1.f + x));
                u[j] = ujj;
                rdl = 1.f / (1.f + ujj);
            }
        }
        const float rdj = __shfl_sync(full, rdl, j);
        if (act && lane > j) {
            float s2 = e[j];
#pragma unroll
            for (int k2 = 0; k2 < RP; ++k2)
                if (k2 < j) s2 -= ucol[k2] * u[k2];
            u[j] = s2 * rdj;
        }
    }
    float um = 0.f;
    if (act)
#pragma unroll
        for (int a = 0; a < RP; ++a)
            if (a < p) um = fmaxf(um, fabsf(u[a]));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) um = fmaxf(um, __shfl_xor_sync(full, um, o));
    // (I + U) Y = -U, column `lane` by back substitution: row r of U comes from lanes k > r
#pragma unroll
    for (int r = RP - 1; r >= 0; --r) {
        const float rdr = __shfl_sync(full, rdl, r);
        float urow[RP];
#pragma unroll
        for (int k2 = 0; k2 < RP; ++k2) urow[k2] = (k2 > r) ? __shfl_sync(full, u[r], k2) : 0.f;
        if (act && r < p && r <= lane) {
            float s2 = -u[r];
#pragma unroll
            for (int k2 = 0; k2 < RP; ++k2)
                if (k2 > r && k2 <= lane) s2 -= urow[k2] * y[k2];
            y[r] = (r == lane && rdr == 0.f) ? -1.f : s2 * rdr;
        }
    }
    if (act)
#pragma unroll
        for (int a = 0; a < RP; ++a)
            if (a < p) {
                cf.U[a * p + lane] = u[a];
                cf.Y[a * p + lane] = y[a];
            }
    bad = __any_sync(full, bad) ? 1 : 0;
    if (lane == 0) {
        cf.ill = 0;
        cf.bad = bad;
        cf.umax = um;
    }
    __syncwarp();
}

// ---- float-pair (double-float) scalars for the accurate first-pass factor
struct fp2 {
    float h, l;
};
__device__ __forceinline__ fp2 f2_make(float h, float l) {
    fp2 r;
    r.h = h;
    r.l = l;
    return r;
}
__device__ __forceinline__ fp2 f2_norm(float s, float e) {
    const float h = s + e;
    return f2_make(h, e - (h - s));
}
__device__ __forceinline__ fp2 f2_add(fp2 a, fp2 b) {
    const float s = a.h + b.h, bp = s - a.h;
    const float e = ((a.h - (s - bp)) + (b.h - bp)) + (a.l + b.l);
    return f2_norm(s, e);
}
__device__ __forceinline__ fp2 f2_mul(fp2 a, fp2 b) {
    const float pr = a.h * b.h;
    float e = fmaf(a.h, b.h, -pr);
    e = fmaf(a.h, b.l, e);
    e = fmaf(a.l, b.h, e);
    return f2_norm(pr, e);
}
// sqrt(a), a > 0: s = sqrtf(a_h), corrected by one Newton step (a - s^2) / (2 s), with s^2
// formed exactly by an FMA
__device__ __forceinline__ fp2 f2_sqrt(fp2 a) {
    const float sq = sqrtf(a.h);
    const float pr = sq * sq, pe = fmaf(sq, sq, -pr);
    return f2_norm(sq, (((a.h - pr) - pe) + a.l) / (2.f * sq));
}
// 1 / a: x0 = 1 / a_h corrected by x0 (1 - a x0)
__device__ __forceinline__ fp2 f2_rcp(fp2 a) {
    const float x0 = 1.f / a.h;
    float e = fmaf(-a.h, x0, 1.f);
    e = fmaf(-a.l, x0, e);
    return f2_norm(x0, x0 * e);
}
__device__ __forceinline__ fp2 f2_shfl(fp2 a, int src) {
    return f2_make(__shfl_sync(0xffffffffu, a.h, src), __shfl_sync(0xffffffffu, a.l, src));
}

struct CholD {
    float Uh[RP * RP], Ul[RP * RP];   // the factor of G 2^-k (upper triangle) as float pairs
    float ih[RP], il[RP];             // 1 / U_cc as float pairs
    int ok;
};

// Cholesky factor of G 2^-k in float-pair arithmetic on warp 0, lane l holding column l (as
// chol32_full).  ok = every pivot is positive and at least rel_min times the largest diagonal
// entry and no column is zero: then one pass with this factor leaves the block orthonormal to
// ~kappa^2 2^-48, and the caller skips the deviation pass.  Otherwise the caller discards it.
// dep: a pivot that is zero, or below rel_min times the largest diagonal entry, marks a
// dependent column instead of a failure: R_jj = 0 and row j of R zero, so the column's
// direction is dropped (the block Krylov space loses a direction that lies in the span of
// the others to within the pivot) and the forward substitution leaves it zero.
__device__ inline void chol_df(CholD& cd, const double* G0, int p, int k, float rel_min, bool dep = false) {
    const int lane = threadIdx.x;
    const unsigned full = 0xffffffffu;
    const bool act = lane < p;
    fp2 g[RP], u[RP];
    float dg = 0.f;
#pragma unroll
    for (int a = 0; a < RP; ++a) {
        float h = 0.f, l = 0.f;
        if (act && a < p) split_df(ldexp(G0[a * p + lane], -k), h, l);
        g[a] = f2_make(h, l);
        u[a] = f2_make(0.f, 0.f);
        if (a == lane) dg = h;
    }
    float dmax = act ? dg : 0.f;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) dmax = fmaxf(dmax, __shfl_xor_sync(full, dmax, o));
    int ok_l = 1;
    fp2 myinv = f2_make(0.f, 0.f);
#pragma unroll
    for (int j = 0; j < RP; ++j) {
        if (j >= p) break;
        fp2 inv = f2_make(0.f, 0.f);
        if (lane == j) {
            fp2 d = g[j];
            if (dep && isfinite(d.h) && (G0[j * p + j] == 0.0 || !(d.h >= rel_min * dmax))) {
                u[j] = f2_make(0.f, 0.f);           // dependent column: R_jj = 0, inverse 0
            } else {
                if (G0[j * p + j] == 0.0 || !(d.h > 0.f) || !isfinite(d.h) || d.h < rel_min * dmax) {
                    ok_l = 0;
                    d = f2_make(1.f, 0.f);
                }
                u[j] = f2_sqrt(d);
                inv = f2_rcp(u[j]);
            }
            myinv = inv;
        }
        inv = f2_shfl(inv, j);
        if (act && lane > j) u[j] = f2_mul(g[j], inv);
        // trailing update G[a][l] -= U[j][a] U[j][l] for j < a <= l
#pragma unroll
        for (int a = j + 1; a < RP; ++a) {
            const fp2 uja = f2_shfl(u[j], a);
            if (act && a < p && a <= lane) {
                const fp2 pr = f2_mul(uja, u[j]);
                g[a] = f2_add(g[a], f2_make(-pr.h, -pr.l));
            }
        }
    }
    const int ok = __all_sync(full, ok_l);
    if (act) {
#pragma unroll
        for (int a = 0; a < RP; ++a)
            if (a < p) {
                cd.Uh[a * p + lane] = u[a].h;
                cd.Ul[a * p + lane] = u[a].l;
            }
        cd.ih[lane] = myinv.h;
        cd.il[lane] = myinv.l;
    }
    if (lane == 0) cd.ok = ok;
    __syncwarp();
}

// KIND 1: the first pass (FP32 factor of G, exact double-float application).  KIND 3: the
// same, fused with the second CGS pass's correction W <- W - Vc h2 (FP32, as
// k_update_gram_rows<true>): the input Gram matrix Gin = h2 + ccols p (p x p, stored after
// h2, accumulated in double-float) is then that of W before the correction, and the factor
// is taken of Gin - h2^T h2 (formed in double-float: the Gram matrix after the correction when
// V is orthonormal).  With a final destination fin_, KIND 3 first factors it in double-float:
// when the block is well-conditioned (chol_df) that factor is applied, the pass writes the
// final block and H and sets the done flag, and the later passes return at once; else the
// FP32 factor and the passes after it run as for KIND 1.  The passes that feed another write
// the Gram matrix of their result to G (last CTA).  KIND 2: the deviation passes.
template <int KIND>
__global__ void __launch_bounds__(NTR) k_qr_mixed_rows(double* W, int64_t ldw, int p, int64_t n, int64_t rpb,
                                                      double* G, double* __restrict__ part, unsigned* ctr,
                                                      int mode, double* R, double* Rinv, const double* Rtot_in,
                                                      double* Rtot_out, double* H, int ldH, int hrow, int hcol,
                                                      double* normsq_out, int* flags, double* out_, int64_t ldo_,
                                                      const double* __restrict__ Vc, int64_t ldvc, int ccols,
                                                      const double* __restrict__ h2, int lead_blk, double* fin_,
                                                      int64_t ldfin_) {
    constexpr bool K1 = KIND == 1 || KIND == 3;
    int* extra = flags + 2;
    int* done = flags + 3;                  // KIND 3 single pass: the block is final after pass 1
    if (mode >= 1 && *done) return;
    if (mode == 2 && *extra == 0) return;
    extern __shared__ float h2f[];          // KIND 3: h2 as float pairs (hi, then lo), ccols x RP each
    float* h2l = h2f + ccols * RP;
    __shared__ CholF cf;
    __shared__ CholD cd;                    // K1: the float-pair factor (single pass, or an ill block)
    __shared__ int sgl_s;                   // K1: the single pass (the block is final after it)
    __shared__ double G0[RP * RP];
    __shared__ double hn2[RP];
    __shared__ double Rd[RP * RP];          // KIND 1: R (padded to RP x RP); KIND 2 unused
    __shared__ double rcp[RP];              // KIND 1: 1 / R_cc (0 for a zero column)
    __shared__ float Rh[RP * RP], Rl[RP * RP];   // KIND 1: R as float pairs
    __shared__ float rch[RP], rcl[RP];           // KIND 1: 1 / R_cc as float pairs
    __shared__ float Yf[RP * RP];           // KIND 2: Y padded to RP x RP
    __shared__ double red[NTR / 32][RG];
    __shared__ double buf[NTR / 32][32 * RP];
    const int pp = p * p;
    if (KIND == 3) {
        for (int e = threadIdx.x; e < ccols * RP; e += blockDim.x) {
            const int a = e / RP, c = e - a * RP;
            float hh = 0.f, hl = 0.f;
            if (c < p) split_df(h2[a * p + c], hh, hl);
            h2f[e] = hh;
            h2l[e] = hl;
        }
        __syncthreads();
        // G - h2^T h2 with the products in float-pair arithmetic (the single pass needs G to
        // ~2^-48); the Gram sums follow h2 in memory
        for (int o = threadIdx.x; o < pp; o += blockDim.x) {
            const int i = o / p, k = o - i * p;
            float sh = 0.f, sl = 0.f;
            for (int a = 0; a < ccols; ++a)
                df_fma(sh, sl, h2f[a * RP + i], h2l[a * RP + i], h2f[a * RP + k], h2l[a * RP + k]);
            G0[o] = h2[ccols * p + o] - ((double)sh + (double)sl);
        }
    } else {
        for (int o = threadIdx.x; o < pp; o += blockDim.x) G0[o] = G[o];
    }
    const bool last = (mode == 1 && *extra == 0) || mode == 2;
    // the lead CTA writes R, Rtot, the entries of H and the flags: CTA lead_blk, which the
    // launcher places beyond the rows (an extra CTA that owns none, so the lead work runs
    // concurrently with the row CTAs) when each CTA holds few rows
    const bool lead = (int)blockIdx.x == lead_blk;
    const bool need_hn2 = H && lead && (last || (KIND == 3 && fin_));
    if (need_hn2) {
        const int stripes = NTR / p;
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
    if (need_hn2 && threadIdx.x < p) {
        const int stripes = NTR / p;
        double s2 = 0.0;
        for (int k = 0; k < stripes; ++k) s2 += buf[0][k * p + threadIdx.x];
        hn2[threadIdx.x] = s2;
    }
    __syncthreads();
    int kexp = 0;                           // KIND 1: G is factored as G 2^-kexp (kexp even)
    if (threadIdx.x < 32) {
        int sgl_r = 0;                      // warp 0's copy of the single-pass decision
        const int lane = threadIdx.x;
        double tr = 0.0, dmax = 0.0;
        if (K1) {
            for (int c = 0; c < p; ++c) {
                tr += G0[c * p + c];
                dmax = fmax(dmax, G0[c * p + c]);
            }
            if (dmax > 0.0 && isfinite(dmax)) {
                frexp(dmax, &kexp);
                kexp &= ~1;
            }
            // KIND 3 with a final destination: the accurate factor first; the FP32 one (and
            // the deviation passes after it) only when the block is too ill-conditioned for
            // a single pass
            int sgl = 0;
            if (KIND == 3 && fin_) {
                chol_df(cd, G0, p, kexp, 1e-5f);
                // the Gram matrix after the correction must keep most of the one before it,
                // else its relative accuracy is lost to cancellation
                double tin = 0.0;
                for (int c = 0; c < p; ++c) tin += h2[ccols * p + c * p + c];
                sgl = cd.ok && tr >= 1e-4 * tin;
                if (lane == 0) cd.ok = sgl;
            } else if (lane == 0) {
                cd.ok = 0;
            }
            __syncwarp();
            if (sgl) {
                if (lane == 0) {
                    cf.ill = 0;
                    cf.bad = 0;
                    cf.umax = 0.f;
                }
                __syncwarp();
            } else {
                chol32_full(cf, G0, p, kexp, ldexp(tr, -kexp));
                // an ill-conditioned block (an FP32 pivot below 1e-6 of the largest diagonal
                // entry: the FP32 factor needed a shift, after which the block would be too far
                // from orthonormal for the deviation passes): factor the Gram matrix, accurate
                // to ~2^-48, unshifted in double-float instead and apply that factor exactly;
                // both deviation passes then run (cf.ill stays set).  Up to kappa(W) ~ 8e6; a
                // direction below that (a pivot under 2^-46 of the largest, where G's ~2^-48
                // accuracy no longer resolves it) counts as dependent and is dropped, as the
                // FP64 path drops zero pivots (info.breakdown).
                if (cf.ill) chol_df(cd, G0, p, kexp, 0x1p-46f, true);
            }
            sgl_r = sgl;
            if (lane == 0) sgl_s = sgl;     // for the other warps, read after the barrier
        } else {
            chol32_dev(cf, G0, p);
        }
        const bool df_w = K1 && cd.ok;      // warp 0: the float-pair factor is applied
        const bool sgl_w = df_w && sgl_r;   // warp 0's view of the single-pass decision
        const bool fin = last || sgl_w;     // this pass writes the final block and H
        if (lead) {
            if (K1 && normsq_out && lane == 0) *normsq_out = tr;
            if (K1 && lane == 0) {
                *extra = cf.ill;
                *done = sgl_w ? 1 : 0;
            }
            if (lane < p) {
                const int c = lane;
                for (int r = 0; r < p; ++r) {
                    const int o = r * p + c;
                    double rt;
                    if (df_w) {
                        float rh = 0.f, rl = 0.f;
                        if (r <= c) split_df(ldexp((double)cd.Uh[o] + (double)cd.Ul[o], kexp / 2), rh, rl);
                        rt = (double)rh + (double)rl;   // exactly the R the substitution applies
                        R[o] = rt;
                    } else if (K1) {
                        rt = (r <= c) ? ldexp((double)cf.U[o], kexp / 2) : 0.0;
                        R[o] = rt;
                    } else {
                        // Rtot_out = Rtot_in + U Rtot_in: an FP32 correction of the FP64 product
                        // when U is O(eps_32); in FP64 after an ill-conditioned first pass (U
                        // up to ~0.1), so that H records the transform the pass applies
                        double corr = 0.0;
                        if (cf.umax > 1e-4f) {
                            for (int k = r; k <= c; ++k) corr = fma((double)cf.U[r * p + k], Rtot_in[k * p + c], corr);
                        } else {
                            float cf32 = 0.f;
                            for (int k = r; k <= c; ++k) cf32 = fmaf(cf.U[r * p + k], (float)Rtot_in[k * p + c], cf32);
                            corr = (double)cf32;
                        }
                        rt = (r <= c) ? Rtot_in[o] + corr : 0.0;
                        R[o] = (r <= c) ? (double)cf.U[o] + (r == c ? 1.0 : 0.0) : 0.0;
                        Rinv[o] = (r <= c) ? (double)cf.Y[o] + (r == c ? 1.0 : 0.0) : 0.0;
                    }
                    Rtot_out[o] = rt;
                    if (!isfinite(rt)) cf.bad = 1;
                    if (H && fin) H[(int64_t)(hcol + c) * ldH + hrow + r] = rt;
                }
            }
            __syncwarp();
            if (H && fin && lane < p) {
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
    if (K1) {
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
    const bool single = K1 && cd.ok;        // the float-pair factor is applied
    const bool final1 = single && sgl_s;    // ... as the single, final pass
    const bool subst = K1 || cf.umax > 1e-4f;
    for (int e = threadIdx.x; e < RP * RP; e += blockDim.x) {
        const int a = e / RP, c = e % RP;
        const bool in = a < p && c < p && a <= c;
        if (single) {
            // the pair (Rh, Rl) is what the substitution applies and what H records
            float rh = 0.f, rl = 0.f;
            if (in) split_df(ldexp((double)cd.Uh[a * p + c] + (double)cd.Ul[a * p + c], kexp / 2), rh, rl);
            Rh[e] = rh;
            Rl[e] = rl;
            Rd[e] = (double)rh + (double)rl;
        } else if (K1) Rd[e] = in ? ldexp((double)cf.U[a * p + c], kexp / 2) : 0.0;
        else {
            Yf[e] = in ? cf.Y[a * p + c] : 0.f;
            Rd[e] = in ? (double)cf.U[a * p + c] + (a == c ? 1.0 : 0.0) : 0.0;
        }
    }
    __syncthreads();
    if (subst && threadIdx.x < RP) {
        const int c = threadIdx.x;
        if (single) {
            // 1 / R_cc from the factor's float-pair reciprocal, scaled back
            const double ic = (c < p) ? ldexp((double)cd.ih[c] + (double)cd.il[c], -(kexp / 2)) : 0.0;
            rcp[c] = ic;
            split_df(ic, rch[c], rcl[c]);
        } else {
            const double d = Rd[c * RP + c];
            rcp[c] = (d != 0.0) ? 1.0 / d : 0.0;
            if (K1) split_df(rcp[c], rch[c], rcl[c]);
        }
    }
    if (K1 && !single)
        for (int e = threadIdx.x; e < RP * RP; e += blockDim.x) split_df(Rd[e], Rh[e], Rl[e]);
    __syncthreads();
    double* out;
    int64_t ldo;
    int gram;
    if (final1) { out = fin_; ldo = ldfin_; gram = 0; }
    else if (mode == 0) { out = W; ldo = ldw; gram = 1; }
    else if (mode == 1 && *extra) { out = W; ldo = ldw; gram = 1; }
    else { out = out_; ldo = ldo_; gram = 0; }
    double acc[NQ];
    float gah[NQ], gal[NQ];
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
        acc[q] = 0.0;
        gah[q] = 0.f;
        gal[q] = 0.f;
    }
    const int64_t rb = rows_begin(rpb), re = min(n, rb + rpb);
    for (int64_t r0 = rb + (threadIdx.x & ~31); r0 < re; r0 += blockDim.x) {
        const int64_t r = r0 + (threadIdx.x & 31);
        const bool ok = r < re;
        double w[RP], y[RP];
#pragma unroll
        for (int c = 0; c < RP; ++c) w[c] = (ok && c < p) ? W[(int64_t)c * ldw + r] : 0.0;
        // KIND 3: the FP32 correction V h2, subtracted inside the double-float substitution
        // below (no FP64 add)
        float corr[RP];
#pragma unroll
        for (int c = 0; c < RP; ++c) corr[c] = 0.f;
        if (KIND == 3 && ok) {
#pragma unroll 8
            for (int a = 0; a < ccols; ++a) {
                const float v = f32_rn_i(Vc[(int64_t)a * ldvc + r]);
#pragma unroll
                for (int c = 0; c < RP; ++c) corr[c] = fmaf(v, h2f[a * RP + c], corr[c]);
            }
        }
        float yh[RP], yl[RP];
        if (K1) {
            // forward substitution y R = w in double-float: R's entries are exact floats
            // (pairs Rh + Rl for safety), 1 / R_cc as a pair, y kept as pairs
#pragma unroll
            for (int c = 0; c < RP; ++c) {
                float sh, sl;
                split_df_i(w[c], sh, sl);
                if (KIND == 3) df_add(sh, sl, -corr[c]);
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
            for (int c = 0; c < RP; ++c) wf[c] = f32_rn_i(w[c]);
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
            if (K1) {
#pragma unroll
                for (int c = 0; c < RP; ++c)
                    if (!ok || c >= p) { yh[c] = 0.f; yl[c] = 0.f; }
                warp_gram_rows_df(yh, yl, reinterpret_cast<float*>(buf[threadIdx.x >> 5]), gah, gal);
            } else {
                warp_gram_rows(y, buf[threadIdx.x >> 5], acc);
            }
        }
    }
    if (gram) {
        if (K1) {
#pragma unroll
            for (int q = 0; q < NQ; ++q) acc[q] = (double)gah[q] + (double)gal[q];
        }
        cta_gram_write(acc, p, red, part);
        if (take_last_ticket(ctr)) last_cta_sum_df(part, gridDim.x, pp, G, ctr);
    }
}

__global__ void __launch_bounds__(NTR) k_trsm_rows(double* W, int64_t ldw, int p,
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
    __shared__ double red[NTR / 32][RG];
    __shared__ double buf[NTR / 32][32 * RP];
    for (int e = threadIdx.x; e < RP * RP; e += blockDim.x) {
        const int a = e / RP, c = e % RP;
        Ri[e] = (a < p && c < p) ? Rinv[a * p + c] : 0.0;
    }
    __syncthreads();
    double acc[NQ];
#pragma unroll
    for (int q = 0; q < NQ; ++q) acc[q] = 0.0;
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
        if (gram) warp_gram_rows(y, buf[threadIdx.x >> 5], acc);
    }
    if (gram) cta_gram_write(acc, p, red, part);
}

// Row-per-thread, p <= 8: W <- W - V h and the upper-triangular Gram partial of the result.
// h (cols x p) is broadcast from shared memory.  UPD32 = false: the update in FP64 (the
// Arnoldi relation stays exact to FP64 rounding).  UPD32 = true (mixed path, second CGS
// pass only): h is then the O(eps_32) remainder left by the FP32 projection of the first
// pass, so the correction V h is formed in FP32 and subtracted from the FP64 W; its error,
// eps_32 |V h| ~ eps_32^2 |W|, stays far below the accuracy the mixed path delivers.
template <bool UPD32>
__global__ void __launch_bounds__(NTR) k_update_gram_rows(const double* __restrict__ V, int64_t ldv, int cols,
                                                         double* __restrict__ W, int64_t ldw, int p,
                                                         int64_t n, int64_t rpb,
                                                         const double* __restrict__ h,
                                                         double* __restrict__ part, double* G,
                                                         unsigned* ctr) {
    extern __shared__ double hs[];           // cols x RP (zero-padded columns), FP64 or FP32
    float* hsf = reinterpret_cast<float*>(hs);
    __shared__ double red[NTR / 32][RG];
    for (int e = threadIdx.x; e < cols * RP; e += blockDim.x) {
        const int a = e / RP, c = e % RP;
        const double v = (c < p) ? h[a * p + c] : 0.0;
        if (UPD32) hsf[e] = (float)v;
        else hs[e] = v;
    }
    __syncthreads();
    __shared__ double buf[NTR / 32][32 * RP];
    double acc[NQ];
    float facc[NQ];
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
        acc[q] = 0.0;
        facc[q] = 0.f;
    }
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
                const float v = f32_rn_i(V[(int64_t)a * ldv + r]);
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
        if (UPD32) warp_gram_rows32(w, reinterpret_cast<float*>(buf[threadIdx.x >> 5]), facc);
        else warp_gram_rows(w, buf[threadIdx.x >> 5], acc);
    }
    if (UPD32) {
#pragma unroll
        for (int q = 0; q < NQ; ++q) acc[q] = facc[q];
    }
    cta_gram_write(acc, p, red, part);
    if (G && take_last_ticket(ctr)) {
        if (UPD32) last_cta_sum<float>(part, gridDim.x, p * p, G, ctr);
        else last_cta_sum<double>(part, gridDim.x, p * p, G, ctr);
    }
}

// Row-per-thread: Z[r, :] += V[r, 0:cols] Wc; restart copy V[r, 0:p] <- V[r, cols-p:cols].
// DF = false: FP64 products.  DF = true (mixed path): the products in double-float arithmetic
// on the FP32 pipe (V and Wc split into float pairs, TwoSum accumulation as in the first CGS
// update, relative error ~ cols 2^-48 of |V Wc|), added to the FP64 Z.
template <bool DF>
__global__ void __launch_bounds__(NTR) k_update_z_rows(double* __restrict__ V, int64_t ldv, int cols, int p,
                                                      int64_t n, int64_t rpb,
                                                      const double* __restrict__ Wc,
                                                      double* __restrict__ Z, int64_t ldz,
                                                      int restart_copy) {
    extern __shared__ __align__(16) double ws[];   // cols x RP (FP64), or 2 cols x RP floats (DF)
    float* wh = reinterpret_cast<float*>(ws);
    float* wl = wh + cols * RP;
    for (int e = threadIdx.x; e < cols * RP; e += blockDim.x) {
        const int a = e / RP, c = e % RP;
        const double w = (c < p) ? Wc[a * p + c] : 0.0;
        if (DF) split_df(w, wh[e], wl[e]);
        else ws[e] = w;
    }
    __syncthreads();
    const int64_t rb = rows_begin(rpb), re = min(n, rb + rpb);
    for (int64_t r = rb + threadIdx.x; r < re; r += blockDim.x) {
        double z[RP];
        if (DF) {
            float sh[RP], sl[RP];
#pragma unroll
            for (int c = 0; c < RP; ++c) {
                sh[c] = 0.f;
                sl[c] = 0.f;
            }
            int a = 0;
            for (; a + 4 <= cols; a += 4) {
                double v[4];
#pragma unroll
                for (int u = 0; u < 4; ++u) v[u] = V[(int64_t)(a + u) * ldv + r];
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    float vh, vl;
                    split_df_i(v[u], vh, vl);
                    const float4* x4 = reinterpret_cast<const float4*>(wh + (a + u) * RP);
                    const float4* y4 = reinterpret_cast<const float4*>(wl + (a + u) * RP);
#pragma unroll
                    for (int q = 0; q < RP / 4; ++q) {
                        const float4 x = x4[q], y = y4[q];
                        df_fma(sh[4 * q], sl[4 * q], vh, vl, x.x, y.x);
                        df_fma(sh[4 * q + 1], sl[4 * q + 1], vh, vl, x.y, y.y);
                        df_fma(sh[4 * q + 2], sl[4 * q + 2], vh, vl, x.z, y.z);
                        df_fma(sh[4 * q + 3], sl[4 * q + 3], vh, vl, x.w, y.w);
                    }
                }
            }
            for (; a < cols; ++a) {
                float vh, vl;
                split_df_i(V[(int64_t)a * ldv + r], vh, vl);
#pragma unroll
                for (int c = 0; c < RP; ++c) df_fma(sh[c], sl[c], vh, vl, wh[a * RP + c], wl[a * RP + c]);
            }
#pragma unroll
            for (int c = 0; c < RP; ++c) z[c] = f64_of_f32_i(sh[c]) + f64_of_f32_i(sl[c]);
        } else {
#pragma unroll
            for (int c = 0; c < RP; ++c) z[c] = 0.0;
            for (int a = 0; a < cols; ++a) {
                const double v = V[(int64_t)a * ldv + r];
#pragma unroll
                for (int c = 0; c < RP; ++c) z[c] = fma(v, ws[a * RP + c], z[c]);
            }
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


// ---- first block CGS2 pass of the mixed path, in chunks of RB = NTR / 2 rows
//
// k_cgs_rows<false>: partial[blk][a][c] = sum over the CTA's rows of V[r, a] W[r, c] (FP32
// products; the projection of the first pass, or of the second after the tensor-core update),
// with ng = p also the double-float Gram partial as below.
// k_cgs_rows<true>:  W <- W - V h in double-float arithmetic (each product
// v h = vh hh + (err(vh hh) + vl hh + vh hl), the large parts accumulated with TwoSum), then
// the FP32 partials of V^T W for the second pass; with ng = p also the Gram partial W^T W
// in double-float (outputs cols p .. (cols + p) p, full p x p), which feeds the double-float
// factorisation of the single-pass Cholesky-QR.
// Per chunk the FP32 copy of V (cols x RB) and of W (RB x RP) are staged in shared memory.
// The projection is register-blocked: a thread owns blocks of 2 basis columns x 4 block
// columns and per pair of rows reads two float4 of W and four floats of V for 32 FMAs, so
// the shared-memory pipe is no longer the bound (one load per FMA without blocking).  Each
// chunk's FP32 sums (two chains per output, even and odd rows) are added to float-pair
// accumulators, so the CTA's partial carries FP32 products but no growth of the summation
// error with the number of chunks.  In the update two threads share a row, each owning half
// of the block's columns for every basis column a; both threads of a pair then read the same
// h entries in lockstep (one broadcast per load) and each finishes its own columns of W.
// Conversions from FP64 are built from the bit pattern (split_df_i, f32_rn_i): a hardware
// double -> float conversion issues to the FP64 pipe.
constexpr int RB = NTR / 2;
constexpr int VS = RB + 1;                  // row stride of the FP32 copy of V (per basis column)
constexpr int WS4 = RP + 4;                 // row stride of the FP32 copy of W (float4 rows)
constexpr int WG = RP + 1;                  // row stride of the float pairs of W (Gram)
constexpr int HP = RP / 2;                  // columns of W per thread in the update
constexpr int KG = (RG + NTR - 1) / NTR;    // Gram entries (upper triangle) per thread

__host__ __device__ constexpr int cgs_nblk(int cols, int p) { return ((cols + 1) / 2) * ((p + 3) / 4); }

__host__ __device__ constexpr size_t cgs_rows_smem(int cols, bool upd, int ng) {
    return sizeof(float) * ((upd ? 2 * (size_t)cols * RP : 0) + (size_t)RB * WS4 + (size_t)((cols + 1) & ~1) * VS +
                            (ng ? 2 * (size_t)RB * WG : 0));
}

// The projection blocks of one chunk: block b = ab ncb + cb covers basis columns 2ab, 2ab + 1
// and block columns 4cb .. 4cb + 3 (columns past p read zeros and are not written).
template <int KB>
__device__ __forceinline__ void chunk_project(const float* Vs, const float* Wf, int nblk, int ncb, float (*ah)[8],
                                              float (*al)[8]) {
#pragma unroll
    for (int k = 0; k < KB; ++k) {
        const int b = threadIdx.x + k * NTR;
        if (b < nblk) {
            const int ab = b / ncb, cb = b - ab * ncb;
            const float* v0 = Vs + 2 * ab * VS;
            const float* v1 = v0 + VS;
            const float* wp = Wf + 4 * cb;
            float se[8], so[8];
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                se[q] = 0.f;
                so[q] = 0.f;
            }
#pragma unroll 4
            for (int rr = 0; rr < RB; rr += 2) {
                const float4 w0 = *reinterpret_cast<const float4*>(wp + rr * WS4);
                const float4 w1 = *reinterpret_cast<const float4*>(wp + (rr + 1) * WS4);
                const float x0 = v0[rr], x1 = v1[rr], y0 = v0[rr + 1], y1 = v1[rr + 1];
                se[0] = fmaf(x0, w0.x, se[0]);
                se[1] = fmaf(x0, w0.y, se[1]);
                se[2] = fmaf(x0, w0.z, se[2]);
                se[3] = fmaf(x0, w0.w, se[3]);
                se[4] = fmaf(x1, w0.x, se[4]);
                se[5] = fmaf(x1, w0.y, se[5]);
                se[6] = fmaf(x1, w0.z, se[6]);
                se[7] = fmaf(x1, w0.w, se[7]);
                so[0] = fmaf(y0, w1.x, so[0]);
                so[1] = fmaf(y0, w1.y, so[1]);
                so[2] = fmaf(y0, w1.z, so[2]);
                so[3] = fmaf(y0, w1.w, so[3]);
                so[4] = fmaf(y1, w1.x, so[4]);
                so[5] = fmaf(y1, w1.y, so[5]);
                so[6] = fmaf(y1, w1.z, so[6]);
                so[7] = fmaf(y1, w1.w, so[7]);
            }
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                df_add(ah[k][q], al[k][q], se[q]);
                df_add(ah[k][q], al[k][q], so[q]);
            }
        }
    }
}

// The Gram entries (i <= j) of one chunk in double-float from the float pairs of W.
__device__ __forceinline__ void chunk_gram(const float* Wh, const float* Wl, const int* gi, const int* gj, int ngu,
                                           float* gh, float* gl) {
#pragma unroll
    for (int k = 0; k < KG; ++k) {
        if ((int)threadIdx.x + k * NTR < ngu) {
            const int i = gi[k], j = gj[k];
            float sh = 0.f, sl = 0.f;
#pragma unroll 4
            for (int rr = 0; rr < RB; ++rr)
                df_fma(sh, sl, Wh[rr * WG + i], Wl[rr * WG + i], Wh[rr * WG + j], Wl[rr * WG + j]);
            df_add(gh[k], gl[k], sh);
            gl[k] += sl;
        }
    }
}

// h entries of the thread's HP columns (four floats per load when HP is a multiple of 4, else
// two; the rows of hh and hl and the thread's offset keep those loads aligned)
__device__ __forceinline__ void df_row_update(float* sh, float* sl, float vh, float vl, const float* x, const float* y) {
    if constexpr (HP % 4 == 0) {
#pragma unroll
        for (int q = 0; q < HP / 4; ++q) {
            const float4 a = reinterpret_cast<const float4*>(x)[q], b = reinterpret_cast<const float4*>(y)[q];
            df_fma(sh[4 * q], sl[4 * q], vh, vl, a.x, b.x);
            df_fma(sh[4 * q + 1], sl[4 * q + 1], vh, vl, a.y, b.y);
            df_fma(sh[4 * q + 2], sl[4 * q + 2], vh, vl, a.z, b.z);
            df_fma(sh[4 * q + 3], sl[4 * q + 3], vh, vl, a.w, b.w);
        }
    } else {
#pragma unroll
        for (int q = 0; q < HP / 2; ++q) {
            const float2 a = reinterpret_cast<const float2*>(x)[q], b = reinterpret_cast<const float2*>(y)[q];
            df_fma(sh[2 * q], sl[2 * q], vh, vl, a.x, b.x);
            df_fma(sh[2 * q + 1], sl[2 * q + 1], vh, vl, a.y, b.y);
        }
    }
}

// GR: the Gram outputs are compiled in (the update always; the projection only in its Gram
// variant, so the plain projection keeps its lower register count)
template <bool UPD, bool GR, int KB>
__global__ void __launch_bounds__(NTR) k_cgs_rows(const double* __restrict__ V, int64_t ldv, int cols,
                                                 double* __restrict__ W, int64_t ldw, int p, int64_t n,
                                                 int64_t rpb, const double* __restrict__ h,
                                                 double* __restrict__ part, int ng) {
    extern __shared__ __align__(16) float smf[];
    float* hh = smf;                                   // UPD: cols x RP (zero-padded columns)
    float* hl = hh + (UPD ? cols * RP : 0);
    float* Wf = hl + (UPD ? cols * RP : 0);            // RB x WS4
    float* Vs = Wf + RB * WS4;                         // ((cols + 1) & ~1) x VS
    float* Wh = Vs + ((cols + 1) & ~1) * VS;           // ng: W as float pairs, RB x WG each
    float* Wl = Wh + RB * WG;
    if (UPD) {
        for (int e = threadIdx.x; e < cols * RP; e += NTR) {
            const int a = e / RP, c = e - a * RP;
            float x = 0.f, y = 0.f;
            if (c < p) split_df(h[a * p + c], x, y);
            hh[e] = x;
            hl[e] = y;
        }
    }
    if (cols & 1)                                      // the padding column of the last block
        for (int e = threadIdx.x; e < VS; e += NTR) Vs[cols * VS + e] = 0.f;
    const int ncb = (p + 3) >> 2, nblk = cgs_nblk(cols, p);
    const int gp = GR ? ng : 0, ngu = gp * (gp + 1) / 2;
    float ah[KB][8], al[KB][8], gh[KG], gl[KG];
    int gi[KG], gj[KG];
#pragma unroll
    for (int k = 0; k < KB; ++k)
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            ah[k][q] = 0.f;
            al[k][q] = 0.f;
        }
#pragma unroll
    for (int k = 0; k < KG; ++k) {
        gh[k] = 0.f;
        gl[k] = 0.f;
        int i = 0, rem = threadIdx.x + k * NTR;        // upper-triangle entry -> (i, j), i <= j
        if (rem < ngu)
            while (rem >= gp - i) {
                rem -= gp - i;
                ++i;
            }
        gi[k] = i;
        gj[k] = i + rem;
    }
    const int rr = threadIdx.x >> 1, hf = threadIdx.x & 1, c0 = hf * HP;
    const int64_t rb = rows_begin(rpb), re = min(n, rb + rpb);
    for (int64_t r0 = rb; r0 < re; r0 += RB) {
        const int tr = (int)min((int64_t)RB, re - r0);
        if (UPD) {
            __syncthreads();                           // hh/hl written; previous chunk consumed
            const bool ok = rr < tr;
            const int64_t r = r0 + rr;
            float sh[HP], sl[HP];
#pragma unroll
            for (int c = 0; c < HP; ++c) {
                sh[c] = 0.f;
                sl[c] = 0.f;
            }
            // groups of 8 basis columns: each thread of the pair loads and splits the 4 of its
            // parity (a = 8g + 2q + hf) and takes the other 4 from its partner by a shuffle;
            // the next group's loads are issued before this group's products
            const int ng8 = cols >> 3;
            double nx[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) nx[q] = (ok && ng8 > 0) ? V[(int64_t)(2 * q + hf) * ldv + r] : 0.0;
            for (int g = 0; g < ng8; ++g) {
                float mh[4], ml[4];
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    split_df_i(nx[q], mh[q], ml[q]);
                    Vs[(8 * g + 2 * q + hf) * VS + rr] = mh[q];
                }
                if (g + 1 < ng8) {
#pragma unroll
                    for (int q = 0; q < 4; ++q) nx[q] = ok ? V[(int64_t)(8 * (g + 1) + 2 * q + hf) * ldv + r] : 0.0;
                }
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const float oh = __shfl_xor_sync(0xffffffffu, mh[q], 1);
                    const float ol = __shfl_xor_sync(0xffffffffu, ml[q], 1);
                    const int a = 8 * g + 2 * q;
                    df_row_update(sh, sl, hf ? oh : mh[q], hf ? ol : ml[q], hh + a * RP + c0, hl + a * RP + c0);
                    df_row_update(sh, sl, hf ? mh[q] : oh, hf ? ml[q] : ol, hh + (a + 1) * RP + c0,
                                  hl + (a + 1) * RP + c0);
                }
            }
            for (int a = 8 * ng8; a < cols; ++a) {
                const double v = ok ? V[(int64_t)a * ldv + r] : 0.0;
                float vh, vl;
                split_df_i(v, vh, vl);
                if ((a & 1) == hf) Vs[a * VS + rr] = vh;
                df_row_update(sh, sl, vh, vl, hh + a * RP + c0, hl + a * RP + c0);
            }
#pragma unroll
            for (int q = 0; q < HP; ++q) {
                const int c = c0 + q;
                float wf = 0.f, wh = 0.f, wl = 0.f;
                if (ok && c < p) {
                    const double w = W[(int64_t)c * ldw + r] - (f64_of_f32_i(sh[q]) + f64_of_f32_i(sl[q]));
                    W[(int64_t)c * ldw + r] = w;
                    wf = f32_rn_i(w);
                    if (ng) split_df_i(w, wh, wl);
                }
                Wf[rr * WS4 + c] = wf;
                if (ng) {
                    Wh[rr * WG + c] = wh;
                    Wl[rr * WG + c] = wl;
                }
            }
        } else {
            __syncthreads();                           // previous chunk consumed
            // batches of LB loads per thread.  With many basis columns (KB >= 3) the next batch
            // is issued before the current one is converted and stored, so two batches are in
            // flight (measured faster at 160 columns, 96^3; slower with few columns, where the
            // extra registers cost a resident CTA)
            const int tot = cols * RB;
            if constexpr (KB >= 3) {
                double v[LB], vn[LB];
#pragma unroll
                for (int k = 0; k < LB; ++k) {
                    const int e = threadIdx.x + k * NTR, a = e / RB, r2 = e - a * RB;
                    v[k] = (e < tot && r2 < tr) ? V[(int64_t)a * ldv + r0 + r2] : 0.0;
                }
                for (int e0 = threadIdx.x; e0 < tot; e0 += LB * NTR) {
                    const int e1 = e0 + LB * NTR;
                    if (e1 < tot) {
#pragma unroll
                        for (int k = 0; k < LB; ++k) {
                            const int e = e1 + k * NTR, a = e / RB, r2 = e - a * RB;
                            vn[k] = (e < tot && r2 < tr) ? V[(int64_t)a * ldv + r0 + r2] : 0.0;
                        }
                    }
#pragma unroll
                    for (int k = 0; k < LB; ++k) {
                        const int e = e0 + k * NTR, a = e / RB, r2 = e - a * RB;
                        if (e < tot) Vs[a * VS + r2] = f32_rn_i(v[k]);
                    }
#pragma unroll
                    for (int k = 0; k < LB; ++k) v[k] = vn[k];
                }
            } else {
                for (int e0 = threadIdx.x; e0 < tot; e0 += LB * NTR) {
                    double v[LB];
#pragma unroll
                    for (int k = 0; k < LB; ++k) {
                        const int e = e0 + k * NTR, a = e / RB, r2 = e - a * RB;
                        v[k] = (e < tot && r2 < tr) ? V[(int64_t)a * ldv + r0 + r2] : 0.0;
                    }
#pragma unroll
                    for (int k = 0; k < LB; ++k) {
                        const int e = e0 + k * NTR, a = e / RB, r2 = e - a * RB;
                        if (e < tot) Vs[a * VS + r2] = f32_rn_i(v[k]);
                    }
                }
            }
            for (int e = threadIdx.x; e < RP * RB; e += NTR) {
                const int c = e / RB, r2 = e - c * RB;
                const double w = (c < p && r2 < tr) ? W[(int64_t)c * ldw + r0 + r2] : 0.0;
                Wf[r2 * WS4 + c] = f32_rn_i(w);
                if (GR && ng) split_df_i(w, Wh[r2 * WG + c], Wl[r2 * WG + c]);
            }
        }
        __syncthreads();
        chunk_project<KB>(Vs, Wf, nblk, ncb, ah, al);
        if (ngu) chunk_gram(Wh, Wl, gi, gj, ngu, gh, gl);
    }
    const int nout = (cols + gp) * p;
    double* out = part + (int64_t)blockIdx.x * nout;
#pragma unroll
    for (int k = 0; k < KB; ++k) {
        const int b = threadIdx.x + k * NTR;
        if (b < nblk) {
            const int ab = b / ncb, cb = b - ab * ncb;
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                const int a = 2 * ab + (q >> 2), c = 4 * cb + (q & 3);
                if (a < cols && c < p) out[a * p + c] = (double)ah[k][q] + (double)al[k][q];
            }
        }
    }
#pragma unroll
    for (int k = 0; k < KG; ++k) {
        if ((int)threadIdx.x + k * NTR < ngu) {
            const double g = (double)gh[k] + (double)gl[k];
            out[(cols + gi[k]) * p + gj[k]] = g;
            out[(cols + gj[k]) * p + gi[k]] = g;
        }
    }
}
