// k_cgs_tc.cu -- the first block CGS2 pass of the mixed path on the 5th-generation tensor
// cores (tcgen05, accumulators in tensor memory), for blocks of p <= 16 columns against at
// most 192 basis columns.
//
// The pass computes W <- W - V h (V: n x cols, the orthonormal Krylov basis, FP64; h: cols x p,
// the projection of the first Gram-Schmidt pass), and then, from the updated W, the FP32
// partials of V^T W (the second pass's projection) and the double-float Gram matrix W^T W
// (which feeds the single-pass Cholesky-QR), exactly as the CUDA-core kernel k_cgs_rows does.
// The update must hold to FP64 rounding (the block Arnoldi relation of eq. (4.5) is what the
// collinear-residual restart relies on), which bf16 products reach by exact slicing:
//   * |V| <= 1 (orthonormal columns), so every entry is cut into seven signed integer slices
//     (|s_i| <= 256) of fixed weights 2^-8, 2^-16, ..., 2^-56, exactly from its bit pattern:
//     v = sum_i s_i 2^-8(i+1) + O(2^-56);
//   * each column c of h gets its own exponent f_c (|h[:, c]| < 2^f_c) and six slices
//     t_j 2^(f_c - 8(j+1));
//   * every product s_i t_j of the 27 pairs with i + j <= 6 (the rest are below 2^-56 of
//     max|h|) is summed over the basis columns by tcgen05.mma kind::f16 (bf16 in, FP32 out)
//     into its own 128 x 16 accumulator in tensor memory: |s_i t_j| <= 2^16 and at most 192
//     terms keep every sum an integer below 2^24, so the FP32 accumulation is exact;
//   * the epilogue adds the accumulators of each level l = i + j as 32-bit integers, packs the
//     seven levels into two 64-bit integers and forms the correction in FP64 with one rounding.
// The error of V h is thus ~2^-56 max|h| per term, the same order as the double-float
// arithmetic it replaces, at a fraction of its FP32 instruction count.
//
// Layout: one CTA per SM (the 27 accumulators take 432 of the SM's 512 tensor-memory columns),
// 256 threads, persistent over 128-row tiles.  Per 16-column chunk of the basis each thread
// loads 8 FP64 values of one row (coalesced per column), keeps an FP32 copy for the second
// projection, cuts them into slices with integer operations and stores each slice's 8 bf16
// values as one 16-byte row
// of a core matrix (the canonical K-major layout without swizzle); thread 0 then issues the
// 27 MMAs of the chunk and commits them to the chunk's mbarrier.  Two slice buffers alternate,
// so the slicing of chunk k+1 overlaps the MMAs of chunk k.  Every mbarrier wait is bounded:
// a wait that runs out records EXPM_TIMEOUT's flag, stops issuing, drains the MMAs already
// issued (with a second, generous bound) and frees the tensor memory.
#include <cuda_bf16.h>

#include "df.cuh"
#include "internal.h"

namespace expm {
namespace {

constexpr int TCT = 256;          // threads per CTA
constexpr int TCM = 128;          // rows per tile (tensor-memory lanes)
constexpr int NVS = 7;            // slices of V
constexpr int NHS = 6;            // slices of h
constexpr int NPAIR = 27;         // pairs (i, j) with i + j <= 6
constexpr int TC_COLS_MAX = 192;
constexpr int TMEM_COLS = 512;
constexpr int VFS = TCM + 1;      // row stride of the FP32 copy of V (per basis column)
constexpr int WFS = 17;           // row stride of the FP32 copy of W
constexpr uint32_t kATile = 4096; // one 128 x 16 bf16 slice, bytes
constexpr uint32_t kBTile = 512;  // one 16 x 16 bf16 slice, bytes

__host__ __device__ constexpr size_t tc_smem_bytes(int cols) {
    return (size_t)2 * NVS * kATile + (size_t)((cols + 15) / 16) * NHS * kBTile + sizeof(float) * (size_t)cols * VFS +
           sizeof(float) * (TCM * WFS + 2 * TCM * 16);
}

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// byte offset of element (row, k) of a K-major tile with 16 K per row block: core matrices of
// 8 rows x 16 bytes, adjacent along K 128 bytes apart (LBO), along the rows 256 bytes (SBO)
__device__ __forceinline__ uint32_t kmaj(int row, int k) {
    return (uint32_t)((row >> 3) * 256 + (k >> 3) * 128 + (row & 7) * 16 + (k & 7) * 2);
}

// shared-memory matrix descriptor: start >> 4, LBO >> 4, SBO >> 4, the fixed 0b001 at bit 46,
// no swizzle
__device__ __forceinline__ uint64_t sdesc(uint32_t addr) {
    return (uint64_t)((addr & 0x3FFFF) >> 4) | ((uint64_t)(128 >> 4) << 16) | ((uint64_t)(256 >> 4) << 32) |
           ((uint64_t)1 << 46);
}

// instruction descriptor of kind::f16: D FP32, A and B bf16, both K-major, N = 16, M = 128
constexpr uint32_t kIdesc = (1u << 4) | (1u << 7) | (1u << 10) | ((16u >> 3) << 17) | ((128u >> 4) << 24);

__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, long limit) {
    uint32_t done = 0;
    for (long it = 0; it <= limit && !done; ++it)
        asm volatile("{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
                     "selp.u32 %0, 1, 0, p;\n\t}"
                     : "=r"(done)
                     : "r"(smem_u32(bar)), "r"(parity));
    return done != 0;
}

__device__ __forceinline__ void mma_issue(uint32_t dtmem, uint64_t da, uint64_t db, uint32_t acc) {
    asm volatile("{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                 "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(dtmem),
                 "l"(da), "l"(db), "r"(kIdesc), "r"(acc));
}

// 8 consecutive accumulator columns of this warp's 32 lanes
__device__ __forceinline__ void tmem_ld8(uint32_t taddr, uint32_t* v) {
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                 : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7])
                 : "r"(taddr));
}

// The seven slices of v (|v| <= 1 + 2^-8): X = round-toward-zero(|v| 2^56) as a 64-bit integer
// from the bit pattern, its base-256 digits d_0 .. d_6 (d_0 <= 256, X = sum d_i 2^(8 (6 - i))),
// each turned into an exact float (2^23 + d - 2^23) and given v's sign.  Returns false when
// |v| is too large for the slicing (d_0 > 256).
__device__ __forceinline__ bool slice7(double v, float* s) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(v);
    const int E = (int)((b >> 52) & 0x7FF);
    const unsigned sgn = (unsigned)(b >> 63) << 31;
    const unsigned long long m = (b & 0xFFFFFFFFFFFFFull) | (1ull << 52);
    const int sh = E - 1019;                  // |v| 2^56 = m 2^sh
    unsigned long long X = 0;
    if (E != 0 && sh > -53) X = sh >= 0 ? (sh < 8 ? m << sh : ~0ull) : m >> (-sh);
    const unsigned d0 = (unsigned)(X >> 48);
#pragma unroll
    for (int i = 0; i < 7; ++i) {
        const unsigned d = i == 0 ? min(d0, 256u) : (unsigned)(X >> (8 * (6 - i))) & 0xFFu;
        const float f = __int_as_float(0x4B000000 | d) - 8388608.f;
        s[i] = __int_as_float(__float_as_int(f) ^ (int)sgn);
    }
    return d0 <= 256u;
}

__device__ __forceinline__ uint32_t pack_bf16(float a, float b) {
    const __nv_bfloat162 v = __floats2bfloat162_rn(a, b);   // exact: |a|, |b| <= 256 integers
    return *reinterpret_cast<const uint32_t*>(&v);
}

template <int K>
__global__ void __launch_bounds__(TCT, 1) k_cgs_tc(const double* __restrict__ V, int64_t ldv, int cols,
                                                   double* __restrict__ W, int64_t ldw, int p, int64_t n,
                                                   const double* __restrict__ h, double* __restrict__ part,
                                                   int* flags, long spin_limit) {
    extern __shared__ __align__(1024) unsigned char smc[];
    const int nk = (cols + 15) >> 4;
    unsigned char* As = smc;                                   // [2][NVS][kATile]
    unsigned char* Bs = As + 2 * NVS * kATile;                 // [nk][NHS][kBTile]
    float* Vf = reinterpret_cast<float*>(Bs + (size_t)nk * NHS * kBTile);   // [cols][VFS]
    float* Wf = Vf + (size_t)cols * VFS;                       // [TCM][WFS]
    float* Wh = Wf + TCM * WFS;                                // [TCM][16]
    float* Wl = Wh + TCM * 16;
    __shared__ __align__(8) uint64_t mbar[2];
    __shared__ uint32_t tbase_s;
    __shared__ int fexp[16];
    __shared__ int bad_s;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int nout = (cols + p) * p;

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tbase_s)),
                     "r"(TMEM_COLS));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&mbar[0])));
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&mbar[1])));
        asm volatile("fence.mbarrier_init.release.cluster;");
        bad_s = 0;
    }
    // h: per-column exponents and six bf16 slices per 16 x 16 chunk (B operands), staged
    // through the (not yet used) FP32 copy of V
    double* hs = reinterpret_cast<double*>(Vf);
    for (int e = tid; e < cols * p; e += TCT) hs[e] = h[e];
    __syncthreads();
    if (tid < 16) {
        double mx = 0.0;
        if (tid < p)
            for (int a = 0; a < cols; ++a) mx = fmax(mx, fabs(hs[a * p + tid]));
        int e = 0;
        if (mx > 0.0 && isfinite(mx)) frexp(mx, &e);   // mx < 2^e
        fexp[tid] = e;
    }
    __syncthreads();
    for (int e = tid; e < nk * 256; e += TCT) {
        const int kc = e >> 8, rem = e & 255, c = rem >> 4, k = rem & 15, a = kc * 16 + k;
        double x = (a < cols && c < p) ? ldexp(hs[a * p + c], -fexp[c]) : 0.0;   // |x| < 1
        for (int j = 0; j < NHS; ++j) {
            x *= 256.0;
            const double s = trunc(x);
            x -= s;
            *reinterpret_cast<__nv_bfloat16*>(Bs + ((size_t)kc * NHS + j) * kBTile + kmaj(c, k)) = __float2bfloat16((float)s);
        }
    }
    asm volatile("fence.proxy.async.shared::cta;");
    __syncthreads();
    const uint32_t tbase = tbase_s;

    float ah[K], al[K];
#pragma unroll
    for (int q = 0; q < K; ++q) {
        ah[q] = 0.f;
        al[q] = 0.f;
    }
    int uses0 = 0, uses1 = 0;          // commits so far to mbar[0], mbar[1] (uniform)
    bool stop = false;                 // a bounded wait ran out: issue nothing more
    const int r = tid & (TCM - 1), g = tid >> 7;
    const int64_t ntiles = (n + TCM - 1) / TCM;
    for (int64_t tile = blockIdx.x; tile < ntiles && !stop; tile += gridDim.x) {
        const int64_t row0 = tile * TCM;
        const bool rok = row0 + r < n;
        double v[8], vn[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const int a = g * 8 + u;
            v[u] = (rok && a < cols) ? V[(int64_t)a * ldv + row0 + r] : 0.0;
        }
        for (int kc = 0; kc < nk; ++kc) {
            const int buf = kc & 1;
            const int uses = buf ? uses1 : uses0;
            if (uses > 0 && !mbar_wait(&mbar[buf], (uint32_t)((uses - 1) & 1), spin_limit)) {
                if (lane == 0) atomicOr(&bad_s, 2);
            }
            __syncthreads();
            if (bad_s & 2) {
                stop = true;
                break;
            }
            if (kc + 1 < nk) {
#pragma unroll
                for (int u = 0; u < 8; ++u) {
                    const int a = (kc + 1) * 16 + g * 8 + u;
                    vn[u] = (rok && a < cols) ? V[(int64_t)a * ldv + row0 + r] : 0.0;
                }
            }
            float sl[NVS][8];
            bool ok = true;
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const int a = kc * 16 + g * 8 + u;
                if (a < cols) Vf[a * VFS + r] = (float)v[u];
                float d[NVS];
                ok &= slice7(v[u], d);
#pragma unroll
                for (int i = 0; i < NVS; ++i) sl[i][u] = d[i];
            }
            if (!ok) atomicOr(&bad_s, 1);
            unsigned char* Ab = As + (size_t)buf * NVS * kATile;
#pragma unroll
            for (int i = 0; i < NVS; ++i) {
                uint4 q;
                q.x = pack_bf16(sl[i][0], sl[i][1]);
                q.y = pack_bf16(sl[i][2], sl[i][3]);
                q.z = pack_bf16(sl[i][4], sl[i][5]);
                q.w = pack_bf16(sl[i][6], sl[i][7]);
                *reinterpret_cast<uint4*>(Ab + (size_t)i * kATile + kmaj(r, g * 8)) = q;
            }
            asm volatile("fence.proxy.async.shared::cta;");
            asm volatile("tcgen05.fence::before_thread_sync;");
            __syncthreads();
            asm volatile("tcgen05.fence::after_thread_sync;");
            if (tid == 0) {
                const unsigned char* Bk = Bs + (size_t)kc * NHS * kBTile;
                int pr = 0;
#pragma unroll 1
                for (int j = 0; j < NHS; ++j)
#pragma unroll 1
                    for (int i = 0; i + j <= 6; ++i, ++pr)
                        mma_issue(tbase + 16u * pr, sdesc(smem_u32(Ab + (size_t)i * kATile)),
                                  sdesc(smem_u32(Bk + (size_t)j * kBTile)), kc > 0 ? 1u : 0u);
                asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                    smem_u32(&mbar[buf])));
            }
            if (buf) ++uses1;
            else ++uses0;
#pragma unroll
            for (int u = 0; u < 8; ++u) v[u] = vn[u];
        }
        if (stop) break;
        // all MMAs of the tile are tracked by the last commit
        const int lbuf = (nk - 1) & 1, luses = lbuf ? uses1 : uses0;
        if (!mbar_wait(&mbar[lbuf], (uint32_t)((luses - 1) & 1), spin_limit)) {
            if (lane == 0) atomicOr(&bad_s, 2);
        }
        asm volatile("tcgen05.fence::after_thread_sync;");
        __syncthreads();
        if (bad_s & 2) {
            stop = true;
            break;
        }
        // epilogue: warp w reads lanes 32 (w % 4) .. +31 (rows), columns 8 (w / 4) .. +7
        {
            const int q4 = warp & 3, c0 = (warp >> 2) * 8, rr = q4 * 32 + lane;
            int L[7][8];
#pragma unroll
            for (int l = 0; l < 7; ++l)
#pragma unroll
                for (int c = 0; c < 8; ++c) L[l][c] = 0;
            const uint32_t tl = tbase + ((uint32_t)(q4 * 32) << 16) + (uint32_t)c0;
            int pr = 0;
#pragma unroll
            for (int j = 0; j < NHS; ++j)
#pragma unroll
                for (int i = 0; i + j <= 6; ++i, ++pr) {
                    uint32_t x[8];
                    tmem_ld8(tl + 16u * pr, x);
                    asm volatile("tcgen05.wait::ld.sync.aligned;");
#pragma unroll
                    for (int c = 0; c < 8; ++c) L[i + j][c] += __float2int_rz(__uint_as_float(x[c]));
                }
            const int64_t row = row0 + rr;
#pragma unroll
            for (int c = 0; c < 8; ++c) {
                const int cc = c0 + c;
                float wf = 0.f, wh = 0.f, wl = 0.f;
                if (row < n && cc < p) {
                    // sum_l L_l 2^-8l = hi 2^-16 + lo 2^-48, exact in 64-bit integers
                    const long long hi = ((long long)L[0][c] << 16) + ((long long)L[1][c] << 8) + (long long)L[2][c];
                    const long long lo = ((long long)L[3][c] << 24) + ((long long)L[4][c] << 16) +
                                         ((long long)L[5][c] << 8) + (long long)L[6][c];
                    const double corr = ldexp(fma((double)hi, 0x1p-16, (double)lo * 0x1p-48), fexp[cc] - 16);
                    const double w = W[(int64_t)cc * ldw + row] - corr;
                    W[(int64_t)cc * ldw + row] = w;
                    wf = (float)w;
                    split_df(w, wh, wl);
                }
                Wf[rr * WFS + cc] = wf;
                Wh[rr * 16 + cc] = wh;
                Wl[rr * 16 + cc] = wl;
            }
        }
        asm volatile("tcgen05.fence::before_thread_sync;");
        __syncthreads();
        // the second pass's FP32 projection V^T W and the double-float Gram W^T W of this tile
#pragma unroll
        for (int q = 0; q < K; ++q) {
            const int o = tid + q * TCT;
            if (o < nout) {
                const int a = o / p, c = o - a * p;
                if (a >= cols) {
                    const int a2 = a - cols;
                    float sh = 0.f, sx = 0.f;
#pragma unroll 4
                    for (int k = 0; k < TCM; ++k) {
                        const float vh = Wh[k * 16 + a2], vl = Wl[k * 16 + a2], h1 = Wh[k * 16 + c], h2 = Wl[k * 16 + c];
                        const float pr = vh * h1;
                        float t = fmaf(vh, h1, -pr);
                        t = fmaf(vl, h1, t);
                        t = fmaf(vh, h2, t);
                        df_add(sh, sx, pr);
                        sx += t;
                    }
                    df_add(ah[q], al[q], sh);
                    al[q] += sx;
                } else {
                    const float* va = Vf + (size_t)a * VFS;
                    float s0 = 0.f, s1 = 0.f;
#pragma unroll 8
                    for (int k = 0; k < TCM; k += 2) {
                        s0 = fmaf(va[k], Wf[k * WFS + c], s0);
                        s1 = fmaf(va[k + 1], Wf[(k + 1) * WFS + c], s1);
                    }
                    df_add(ah[q], al[q], s0);
                    df_add(ah[q], al[q], s1);
                }
            }
        }
        __syncthreads();
    }
    // drain: after a wait ran out, the MMAs already issued still complete before the tensor
    // memory is released (generous bound; they do not depend on anything this CTA still does)
    if (stop) {
        const int b0 = uses0 > 0 ? mbar_wait(&mbar[0], (uint32_t)((uses0 - 1) & 1), 1L << 26) : 1;
        const int b1 = uses1 > 0 ? mbar_wait(&mbar[1], (uint32_t)((uses1 - 1) & 1), 1L << 26) : 1;
        if (!(b0 && b1) && lane == 0) atomicOr(&bad_s, 4);
    }
#pragma unroll
    for (int q = 0; q < K; ++q) {
        const int o = tid + q * TCT;
        if (o < nout) part[(int64_t)blockIdx.x * nout + o] = (double)ah[q] + (double)al[q];
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tbase), "r"(TMEM_COLS));
    if (tid == 0 && bad_s) {
        if (bad_s & 1) atomicOr(&flags[0], 1);        // |V| > 1 + 2^-8: not an orthonormal basis
        if (bad_s & 6) atomicOr(&flags[0], 16);       // a bounded wait ran out (EXPM_TIMEOUT)
    }
}

int tc_sms() {
    static int sms = 0;
    if (!sms) {
        int dev = 0;
        if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
            sms = 1;
    }
    return sms;
}

}  // namespace

bool cgs_tc_fit(int cols, int p) { return p >= 1 && p <= 16 && cols >= 1 && cols <= TC_COLS_MAX; }

// grid_out: the CTA count (one per SM at most): the partials' row count for the reduction
cudaError_t launch_cgs_tc(const double* V, int64_t ldv, int cols, double* W, int64_t ldw, int p, int64_t n,
                          const double* h, double* part, int* grid_out, int* flags, long spin_limit, cudaStream_t s) {
    if (!cgs_tc_fit(cols, p) || !h || !part || !grid_out || !flags) return cudaErrorInvalidValue;
    const int64_t tiles = (n + TCM - 1) / TCM;
    const int g = (int)std::min<int64_t>(tiles, tc_sms());
    *grid_out = g;
    const size_t shm = tc_smem_bytes(cols);
    const int k = ((cols + p) * p + TCT - 1) / TCT;
#define EXPM_TC_K(KK) k_cgs_tc<KK><<<g, TCT, shm, s>>>(V, ldv, cols, W, ldw, p, n, h, part, flags, spin_limit)
    if (k <= 4) EXPM_TC_K(4);
    else if (k <= 8) EXPM_TC_K(8);
    else EXPM_TC_K(14);
#undef EXPM_TC_K
    return cudaGetLastError();
}

cudaError_t cgs_tc_set_smem_limits() {
    int dev = 0, optin = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    auto set = [&](auto kern) {
        if (e != cudaSuccess) return;
        cudaFuncAttributes fa;
        e = cudaFuncGetAttributes(&fa, kern);
        if (e == cudaSuccess) e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, optin - (int)fa.sharedSizeBytes);
    };
    set(k_cgs_tc<4>);
    set(k_cgs_tc<8>);
    set(k_cgs_tc<14>);
    return e;
}

}  // namespace expm
