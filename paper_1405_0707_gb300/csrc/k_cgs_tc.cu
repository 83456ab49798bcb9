// k_cgs_tc.cu -- the first block CGS2 pass of the mixed path on the 5th-generation tensor
// cores (tcgen05, accumulators in tensor memory), for blocks of p <= 16 columns against at
// most 160 basis columns: the update (k_cgs_tc, below) and the projection (k_proj_tc, further
// down).
//
// The kernel computes W <- W - V h (V: n x cols, the orthonormal Krylov basis, FP64; h: cols x
// p, the projection of the first Gram-Schmidt pass).  The update must hold to FP64 rounding
// (the block Arnoldi relation of eq. (4.5) is what the collinear-residual restart relies on),
// which bf16 products reach by exact slicing into balanced base-256 digits:
//   * |V| <= 1 (orthonormal columns): X = trunc(|v| 2^55) is cut into seven digits s_i
//     (i = 0 most significant) in [-128, 128] (the top one in [0, 129]) with
//     |v| = 2^-55 sum_i s_i 256^(6 - i) + O(2^-55), each digit given v's sign;
//   * column c of h gets an exponent f_c with max_a |h[a, c]| < 2^f_c and six digits t_j in
//     [-128, 128] of X = trunc(|h| 2^(47 - f_c)) < 2^47, so h = 2^(f_c - 47) sum_j t_j
//     256^(5 - j) + O(2^(f_c - 47));
//   * the product v h is the sum over pairs of s_i t_j 2^(f_c - 14 - 8 (i + j)); the 27 pairs
//     with level l = i + j <= 6 are kept (the rest lie below 2^-56 of max|h| per term) and
//     summed over the basis columns by tcgen05.mma kind::f16 (bf16 operands, exact for
//     integers up to 256, FP32 accumulation) into one 128 x 16 accumulator per LEVEL: at most
//     6 pairs per level, |s t| <= 129 * 128 and at most 160 terms keep every partial sum an
//     integer below 2^24, so the FP32 accumulation is exact;
//   * the epilogue sums the seven level sums S = sum_l L_l 2^(-8 l) in double-float (Horner
//     from level 6; each L_l is an exact integer in FP32) and subtracts S 2^(f_c - 14) from W
//     in FP64, the power of two applied to the exponent fields (two FP64 adds per entry).
// One MMA per V digit covers all its levels at once: the six h digits of a 16-column chunk are
// stacked along N (16 rows each), so digit i multiplies [t_0; ...; t_(nj-1)] (N = 16 nj,
// nj = min(6, 7 - i)) into the accumulator columns of levels i .. i + nj - 1: 7 MMAs per chunk
// (8 in the first chunk, where level 6 is started by its own MMA so that no accumulator needs
// zeroing) into 112 of the CTA's 128 tensor-memory columns.
//
// Layout: persistent CTAs over 128-row tiles, two per SM (86 KB of shared memory, 128
// tensor-memory columns each), 256 threads.  Per 16-column chunk of the basis each thread
// loads 8 FP64 values of one row (coalesced per column), cuts them into digits with integer
// operations and stores each digit's 8 bf16 values as one 16-byte row of a core matrix (the
// canonical K-major layout without swizzle); thread 0 then issues the chunk's MMAs and commits
// them to the chunk's mbarrier.  Two digit buffers alternate, so the slicing of chunk k+1
// overlaps the MMAs of chunk k, and the other CTA on the SM overlaps this one's epilogue.
// Every mbarrier wait is bounded: a wait that runs out records EXPM_TIMEOUT's flag, stops
// issuing, drains the MMAs already issued (with a second, generous bound) and frees the tensor
// memory.  The second pass's projection and the Gram matrix of the updated block are left to
// the CUDA-core projection kernel (k_cgs_rows<false> with the Gram outputs).
#include <cuda_bf16.h>

#include "df.cuh"
#include "internal.h"

namespace expm {
namespace {

constexpr int TCT = 256;          // threads per CTA
constexpr int TCM = 128;          // rows per tile (tensor-memory lanes)
constexpr int NVS = 7;            // digits of V
constexpr int NHS = 6;            // digits of h
constexpr int NLEV = 7;           // levels i + j = 0 .. 6
constexpr int TC_COLS_MAX = 160;
constexpr int TMEM_COLS = 128;    // 7 levels x 16 columns, allocated as a power of two
constexpr uint32_t kATile = 4096; // one 128 x 16 bf16 digit slice of V, bytes
constexpr uint32_t kBTile = 512;  // one 16 x 16 bf16 digit slice of h, bytes

__host__ __device__ constexpr size_t tc_smem_bytes(int cols) {
    return (size_t)2 * NVS * kATile + (size_t)((cols + 15) / 16) * NHS * kBTile;
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

// instruction descriptor of kind::f16: D FP32, A and B bf16, both K-major, M = 128, N given
__device__ __forceinline__ uint32_t idesc(uint32_t n) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((n >> 3) << 17) | ((128u >> 4) << 24);
}

__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, long limit) {
    uint32_t done = 0;
    for (long it = 0; it <= limit && !done; ++it)
        asm volatile("{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
                     "selp.u32 %0, 1, 0, p;\n\t}"
                     : "=r"(done)
                     : "r"(smem_u32(bar)), "r"(parity));
    return done != 0;
}

__device__ __forceinline__ void mma_issue(uint32_t dtmem, uint64_t da, uint64_t db, uint32_t n, uint32_t acc) {
    asm volatile("{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                 "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(dtmem),
                 "l"(da), "l"(db), "r"(idesc(n)), "r"(acc));
}

// 8 consecutive accumulator columns of this warp's 32 lanes
__device__ __forceinline__ void tmem_ld8(uint32_t taddr, uint32_t* v) {
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                 : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7])
                 : "r"(taddr));
}

// The seven balanced digits of v (|v| <= 1 + 2^-8) from its bit pattern: X = trunc(|v| 2^55)
// in base 256 with the six low digits in [-128, 127] and the top one taking the last carry
// (X < 2^55 + 2^47 keeps it <= 129).  Adding 128 at each low byte position, Y = X + 0x80..80,
// turns those digits into the plain bytes of Y (d = byte - 128), so no carry chain is run:
// each byte is placed into the float 2^23 + byte by one byte permute and the digit, with v's
// sign, follows from one FMA.  Returns false when |v| is too large for the slicing.
__device__ __forceinline__ bool slice7(double v, float* s) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(v);
    const int E = (int)((b >> 52) & 0x7FF);
    const unsigned long long m = (b & 0xFFFFFFFFFFFFFull) | (1ull << 52);
    const int sh = E - 1020;                  // |v| 2^55 = m 2^sh
    unsigned long long X = 0;
    if (E != 0 && sh > -53) X = sh >= 0 ? (sh <= 3 ? m << sh : ~0ull) : m >> (-sh);
    const unsigned long long Y = X + 0x808080808080ull;
    const unsigned lo = (unsigned)Y, hi = (unsigned)(Y >> 32);
    const float sg = (b >> 63) ? -1.f : 1.f, off = -8388736.f * sg, off0 = -8388608.f * sg;
    // byte k of Y (k = 6 - i for digit i) as the float 2^23 + byte
    s[6] = fmaf(__uint_as_float(__byte_perm(0x4B000000u, lo, 0x3214u)), sg, off);
    s[5] = fmaf(__uint_as_float(__byte_perm(0x4B000000u, lo, 0x3215u)), sg, off);
    s[4] = fmaf(__uint_as_float(__byte_perm(0x4B000000u, lo, 0x3216u)), sg, off);
    s[3] = fmaf(__uint_as_float(__byte_perm(0x4B000000u, lo, 0x3217u)), sg, off);
    s[2] = fmaf(__uint_as_float(__byte_perm(0x4B000000u, hi, 0x3214u)), sg, off);
    s[1] = fmaf(__uint_as_float(__byte_perm(0x4B000000u, hi, 0x3215u)), sg, off);
    s[0] = fmaf(__uint_as_float(__byte_perm(0x4B000000u, hi, 0x3216u)), sg, off0);
    return (X >> 48) <= 128;
}

// x 2^k by an add to the exponent field (integer operations only); a result below the normal
// range flushes to a signed zero and one above it becomes inf
__device__ __forceinline__ double scale2_i(double x, int k) {
    const long long b = __double_as_longlong(x);
    const int e = (int)((b >> 52) & 0x7FF);
    long long r = b + ((long long)k << 52);
    if (e == 0 || e + k <= 0) r = b & (1LL << 63);
    if (e != 0 && e + k >= 0x7FF) r = (b & (1LL << 63)) | (0x7FFLL << 52);
    return __longlong_as_double(r);
}

__device__ __forceinline__ uint32_t pack_bf16(float a, float b) {
    const __nv_bfloat162 v = __floats2bfloat162_rn(a, b);   // exact: integers |a|, |b| <= 256
    return *reinterpret_cast<const uint32_t*>(&v);
}

template <int dummy>
__global__ void __launch_bounds__(TCT, 2) k_cgs_tc(const double* __restrict__ V, int64_t ldv, int cols,
                                                   double* __restrict__ W, int64_t ldw, int p, int64_t n,
                                                   const double* __restrict__ h, int* flags, long spin_limit) {
    extern __shared__ __align__(1024) unsigned char smc[];
    const int nk = (cols + 15) >> 4;
    unsigned char* As = smc;                                   // [2][NVS][kATile]
    unsigned char* Bs = As + 2 * NVS * kATile;                 // [nk][NHS][kBTile]
    __shared__ __align__(8) uint64_t mbar[2];
    __shared__ uint32_t tbase_s;
    __shared__ int fexp[16], emax_s[16];
    __shared__ int bad_s;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

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
    // per column c: the exponent f_c with max_a |h[a, c]| < 2^f_c, from the bit pattern
    if (tid < 16) {
        int emax = 0;
        if (tid < p)
            for (int a = 0; a < cols; ++a)
                emax = max(emax, (int)(((unsigned long long)__double_as_longlong(h[a * p + tid]) >> 52) & 0x7FF));
        emax_s[tid] = emax;
        fexp[tid] = emax > 0 ? emax - 1022 : -1021;            // |h| < 2^(E - 1022)
    }
    __syncthreads();
    if (tid == 0)
        for (int c = 0; c < p; ++c)
            if (emax_s[c] == 0x7FF) bad_s |= 1;                // h not finite
    // h's digits as the B operands, chunk kc: six 16 x 16 K-major blocks stacked along N
    for (int e = tid; e < nk * 256; e += TCT) {
        const int kc = e >> 8, rem = e & 255, c = rem >> 4, k = rem & 15, a = kc * 16 + k;
        unsigned long long X = 0;
        bool neg = false;
        if (a < cols && c < p) {
            const unsigned long long b = (unsigned long long)__double_as_longlong(h[a * p + c]);
            const int E = (int)((b >> 52) & 0x7FF);
            neg = (b >> 63) != 0;
            const int sh = E - 1028 - fexp[c];                 // |h| 2^(47 - f) = m 2^sh, sh <= -6
            if (E != 0 && sh > -64) X = ((b & 0xFFFFFFFFFFFFFull) | (1ull << 52)) >> (-sh);
        }
        int carry = 0;
        for (int j = NHS - 1; j >= 0; --j) {
            int d = (int)((X >> (8 * (NHS - 1 - j))) & 0xFFu) + carry;
            if (j > 0) {
                carry = d >= 128;
                d -= carry << 8;
            }
            *reinterpret_cast<__nv_bfloat16*>(Bs + ((size_t)kc * NHS + j) * kBTile + kmaj(c, k)) =
                __float2bfloat16((float)(neg ? -d : d));
        }
    }
    asm volatile("fence.proxy.async.shared::cta;");
    __syncthreads();
    const uint32_t tbase = tbase_s;

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
                const uint64_t db = sdesc(smem_u32(Bk));
#pragma unroll 1
                for (int i = 0; i < NVS; ++i) {
                    const uint64_t da = sdesc(smem_u32(Ab + (size_t)i * kATile));
                    const int nj = min(NHS, NLEV - i);
                    if (kc == 0 && i == 1) {
                        // level 6 is first written here: its own MMA starts it (pair (1, 5))
                        mma_issue(tbase + 16u * 6u, da, sdesc(smem_u32(Bk + (size_t)5 * kBTile)), 16u, 0u);
                        mma_issue(tbase + 16u, da, db, 16u * 5u, 1u);
                    } else {
                        mma_issue(tbase + 16u * (uint32_t)i, da, db, 16u * (uint32_t)nj, (kc > 0 || i > 0) ? 1u : 0u);
                    }
                }
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
            const int q4 = warp & 3, c0 = (warp >> 2) * 8;
            const uint32_t tl = tbase + ((uint32_t)(q4 * 32) << 16) + (uint32_t)c0;
            uint32_t x[NLEV][8];
#pragma unroll
            for (int l = 0; l < NLEV; ++l) tmem_ld8(tl + 16u * l, x[l]);
            asm volatile("tcgen05.wait::ld.sync.aligned;");
            const int64_t row = row0 + q4 * 32 + lane;
#pragma unroll
            for (int c = 0; c < 8; ++c) {
                const int cc = c0 + c;
                if (row < n && cc < p) {
                    // S = sum_l L_l 2^(-8 l) by Horner from level 6 in double-float (the level
                    // sums are exact integers in FP32), then corr = S 2^(f - 14), with the
                    // power of two applied to the exponent field
                    float sh = __uint_as_float(x[NLEV - 1][c]), sl = 0.f;
#pragma unroll
                    for (int l = NLEV - 2; l >= 0; --l) {
                        sh *= 0x1p-8f;
                        sl *= 0x1p-8f;
                        df_add(sh, sl, __uint_as_float(x[l][c]));
                    }
                    const int k = fexp[cc] - 14;
                    const double w = W[(int64_t)cc * ldw + row] - scale2_i(f64_of_f32_i(sh), k);
                    W[(int64_t)cc * ldw + row] = w - scale2_i(f64_of_f32_i(sl), k);
                }
            }
        }
        asm volatile("tcgen05.fence::before_thread_sync;");
        __syncthreads();
    }
    // drain: after a wait ran out, the MMAs already issued still complete before the tensor
    // memory is released (generous bound; they do not depend on anything this CTA still does)
    if (stop) {
        const int b0 = uses0 > 0 ? mbar_wait(&mbar[0], (uint32_t)((uses0 - 1) & 1), 1L << 26) : 1;
        const int b1 = uses1 > 0 ? mbar_wait(&mbar[1], (uint32_t)((uses1 - 1) & 1), 1L << 26) : 1;
        if (!(b0 && b1) && lane == 0) atomicOr(&bad_s, 4);
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tbase), "r"(TMEM_COLS));
    if (tid == 0 && bad_s) {
        if (bad_s & 1) atomicOr(&flags[0], 1);        // |V| > 1 + 2^-8: not an orthonormal basis
        if (bad_s & 6) atomicOr(&flags[0], 16);       // a bounded wait ran out (EXPM_TIMEOUT)
    }
}

// ---- the first CGS pass's projection h = V^T W on the tensor cores (tcgen05.mma kind::tf32)
//
// partial[blk][a][c] = sum over the CTA's rows r of V[r, a] W[r, c]: the output of the FP32
// projection kernel (k_cgs_rows<false>), for the same reduction.  This projection only seeds
// the second Gram-Schmidt pass, which removes whatever it leaves, so FP32-level accuracy is
// enough: each FP64 operand is rounded to FP32 (integer operations) and split x = x_hi + x_lo,
// x_hi its top 11 significant bits (a TF32 value) and x_lo = x - x_hi (exact in FP32, read
// by the MMA as TF32: its top 11 bits).  v w is taken as v_hi w_hi + v_hi w_lo + v_lo w_hi,
// about 2^-21 relative per product.  Both operands are K-major with K = the rows, contiguous
// in the column-major V and W: A = V^T (M = the basis columns, one or two 128-row M tiles),
// B = W^T (N = 16; block columns past p are zero).
// Layout: persistent CTAs of 128 threads over 256-row tiles of 16 chunks of 16 rows.  Per
// chunk each thread converts its tasks (4 consecutive rows of one column) and stores x_hi and
// x_lo as one 16-byte core-matrix row each into one of two stages; thread 0 then issues the
// chunk's MMAs (per M tile and 8-row K block: hi.lo, lo.hi, hi.hi) into the tile's
// accumulator (16 tensor-memory columns per M tile) and commits them to the stage's mbarrier.
// The next chunk's loads are in flight in registers while the current chunk is stored.  At
// the end of a tile the FP32 accumulators (sums over 256 rows) are read back and added into
// float-pair sums per thread (thread = accumulator lane = basis column), so the summation
// error does not grow with the number of tiles.  Every mbarrier wait is bounded as in
// k_cgs_tc.
constexpr int PT = 128;              // threads per M tile (its tensor-memory lanes)
constexpr int PKC = 16;              // rows per chunk
constexpr int PCH = 16;              // chunks per tile
constexpr int PTILE = PKC * PCH;     // rows per tile
constexpr int PCOLS_MAX = 160;       // basis columns (the second M tile partly used)
constexpr uint32_t kPA = 4096;       // one 128 x 8 TF32 block of A
constexpr uint32_t kPB = 512;        // one 16 x 8 TF32 block of B
constexpr int PTMEM = 32;            // two M tiles x 16 accumulator columns

__host__ __device__ constexpr size_t ptc_stage_bytes(int mt) { return (size_t)mt * 4 * kPA + 4 * kPB; }
__host__ __device__ constexpr size_t ptc_smem_bytes(int mt) { return 2 * ptc_stage_bytes(mt); }

// byte offset of element (row, k) of a K-major block with 8 TF32 per row: core matrices of
// 8 rows x 16 bytes, adjacent along K 128 bytes apart (LBO), along the rows 256 bytes (SBO)
__device__ __forceinline__ uint32_t kmaj32(int row, int k) {
    return (uint32_t)((row >> 3) * 256 + (k >> 2) * 128 + (row & 7) * 16 + (k & 3) * 4);
}

// instruction descriptor of kind::tf32: D FP32, A and B TF32, both K-major, M = 128, N = 16
__device__ __forceinline__ uint32_t idesc_tf32() {
    return (1u << 4) | (2u << 7) | (2u << 10) | ((16u >> 3) << 17) | ((128u >> 4) << 24);
}

__device__ __forceinline__ void mma_tf32(uint32_t dtmem, uint64_t da, uint64_t db, uint32_t acc) {
    asm volatile("{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                 "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(dtmem),
                 "l"(da), "l"(db), "r"(idesc_tf32()), "r"(acc));
}

// x as the pair (hi, lo): FP32 rounding by integer operations, hi = its top 11 significant
// bits, lo = the rest (exact)
__device__ __forceinline__ void split_tf32(double x, float& hi, float& lo) {
    const float f = f32_rn_i(x);
    hi = __uint_as_float(__float_as_uint(f) & 0xFFFFE000u);
    lo = f - hi;
}

template <int MT>
__global__ void __launch_bounds__(PT * MT) k_proj_tc(const double* __restrict__ V, int64_t ldv, int cols,
                                                const double* __restrict__ W, int64_t ldw, int p, int64_t n,
                                                double* __restrict__ part, int* flags, long spin_limit) {
    extern __shared__ __align__(1024) unsigned char smp[];
    __shared__ __align__(8) uint64_t mbar[2];
    __shared__ uint32_t tbase_s;
    __shared__ int bad_s;
    constexpr uint32_t SB = (uint32_t)ptc_stage_bytes(MT);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tbase_s)),
                     "r"(PTMEM));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&mbar[0])));
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&mbar[1])));
        asm volatile("fence.mbarrier_init.release.cluster;");
        bad_s = 0;
    }
    // both stages zeroed once: rows of the last M tile past cols are never written
    for (uint32_t o = (uint32_t)tid * 16u; o < 2u * SB; o += PT * MT * 16u)
        *reinterpret_cast<uint4*>(smp + o) = make_uint4(0u, 0u, 0u, 0u);
    asm volatile("fence.proxy.async.shared::cta;");
    __syncthreads();
    const uint32_t tbase = tbase_s;

    constexpr int NTH = PT * MT;                     // threads: warp w reads M tile w / 4
    constexpr int PTASK = (4 * (MT == 1 ? 128 : PCOLS_MAX) + NTH - 1) / NTH;   // V tasks per thread, at most
    const int ntask = 4 * cols;                      // V tasks per chunk: (column, 4-row group)
    const int64_t ntiles = (n + PTILE - 1) / PTILE;
    const int mt_own = warp >> 2;                    // the M tile whose sums this thread keeps
    float sh[16], sl[16];
#pragma unroll
    for (int c = 0; c < 16; ++c) {
        sh[c] = 0.f;
        sl[c] = 0.f;
    }
    double pv[PTASK][4], pw[4];
    auto load = [&](int64_t r0) {
#pragma unroll
        for (int t = 0; t < PTASK; ++t) {
            const int task = tid + t * NTH;
            const int a = task >> 2;
            const int64_t r = r0 + 4 * (task & 3);
#pragma unroll
            for (int u = 0; u < 4; ++u)
                pv[t][u] = (task < ntask && r + u < n) ? V[(int64_t)a * ldv + r + u] : 0.0;
        }
        const int c = tid >> 2;
        const int64_t r = r0 + 4 * (tid & 3);
#pragma unroll
        for (int u = 0; u < 4; ++u) pw[u] = (tid < 64 && c < p && r + u < n) ? W[(int64_t)c * ldw + r + u] : 0.0;
    };

    int uses0 = 0, uses1 = 0, gch = 0;   // commits to mbar[0], mbar[1]; chunks issued (uniform)
    bool stop = false;
    if ((int64_t)blockIdx.x < ntiles) load((int64_t)blockIdx.x * PTILE);
    for (int64_t tile = blockIdx.x; tile < ntiles && !stop; tile += gridDim.x) {
        for (int kc = 0; kc < PCH; ++kc) {
            const int buf = gch & 1;
            const int uses = buf ? uses1 : uses0;
            if (uses > 0 && !mbar_wait(&mbar[buf], (uint32_t)((uses - 1) & 1), spin_limit)) {
                if (lane == 0) atomicOr(&bad_s, 2);
            }
            __syncthreads();
            if (bad_s & 2) {
                stop = true;
                break;
            }
            unsigned char* S = smp + (size_t)buf * SB;
#pragma unroll
            for (int t = 0; t < PTASK; ++t) {
                const int task = tid + t * NTH;
                if (task < ntask) {
                    const int a = task >> 2, g = task & 3;
                    float hi[4], lo[4];
#pragma unroll
                    for (int u = 0; u < 4; ++u) split_tf32(pv[t][u], hi[u], lo[u]);
                    const uint32_t o = (uint32_t)(((a >> 7) * 2 + (g >> 1)) * 2) * kPA + kmaj32(a & 127, (g & 1) * 4);
                    *reinterpret_cast<float4*>(S + o) = make_float4(hi[0], hi[1], hi[2], hi[3]);
                    *reinterpret_cast<float4*>(S + o + kPA) = make_float4(lo[0], lo[1], lo[2], lo[3]);
                }
            }
            if (tid < 64) {
                const int c = tid >> 2, g = tid & 3;
                float hi[4], lo[4];
#pragma unroll
                for (int u = 0; u < 4; ++u) split_tf32(pw[u], hi[u], lo[u]);
                const uint32_t o = (uint32_t)MT * 4u * kPA + (uint32_t)((g >> 1) * 2) * kPB + kmaj32(c, (g & 1) * 4);
                *reinterpret_cast<float4*>(S + o) = make_float4(hi[0], hi[1], hi[2], hi[3]);
                *reinterpret_cast<float4*>(S + o + kPB) = make_float4(lo[0], lo[1], lo[2], lo[3]);
            }
            // the next chunk's loads (possibly of the CTA's next tile) while this one is used
            if (kc + 1 < PCH) load(tile * PTILE + (int64_t)(kc + 1) * PKC);
            else if (tile + gridDim.x < ntiles) load((tile + gridDim.x) * PTILE);
            asm volatile("fence.proxy.async.shared::cta;");
            asm volatile("tcgen05.fence::before_thread_sync;");
            __syncthreads();
            asm volatile("tcgen05.fence::after_thread_sync;");
            if (tid == 0) {
                const uint32_t sa = smem_u32(S), sb = sa + (uint32_t)MT * 4u * kPA;
#pragma unroll
                for (int mt = 0; mt < MT; ++mt)
#pragma unroll
                    for (int kb = 0; kb < 2; ++kb) {
                        const uint32_t ah = sa + (uint32_t)((mt * 2 + kb) * 2) * kPA, bh = sb + (uint32_t)(kb * 2) * kPB;
                        const uint32_t d = tbase + 16u * (uint32_t)mt;
                        mma_tf32(d, sdesc(ah), sdesc(bh + kPB), (kc > 0 || kb > 0) ? 1u : 0u);   // hi . lo
                        mma_tf32(d, sdesc(ah + kPA), sdesc(bh), 1u);                              // lo . hi
                        mma_tf32(d, sdesc(ah), sdesc(bh), 1u);                                    // hi . hi
                    }
                asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                    smem_u32(&mbar[buf])));
            }
            if (buf) ++uses1;
            else ++uses0;
            ++gch;
        }
        if (stop) break;
        // the tile's sums: every MMA of the tile is tracked by its last commit
        const int lbuf = (gch - 1) & 1, luses = lbuf ? uses1 : uses0;
        if (!mbar_wait(&mbar[lbuf], (uint32_t)((luses - 1) & 1), spin_limit)) {
            if (lane == 0) atomicOr(&bad_s, 2);
        }
        asm volatile("tcgen05.fence::after_thread_sync;");
        __syncthreads();
        if (bad_s & 2) {
            stop = true;
            break;
        }
        {
            // warp w reads lanes 32 (w % 4) .. + 31 of M tile w / 4 (its accumulator columns)
            uint32_t x[16];
            const uint32_t ta = tbase + ((uint32_t)((warp & 3) * 32) << 16) + 16u * (uint32_t)mt_own;
            tmem_ld8(ta, x);
            tmem_ld8(ta + 8u, x + 8);
            asm volatile("tcgen05.wait::ld.sync.aligned;");
#pragma unroll
            for (int c = 0; c < 16; ++c) df_add(sh[c], sl[c], __uint_as_float(x[c]));
        }
        asm volatile("tcgen05.fence::before_thread_sync;");
        __syncthreads();
    }
    if (stop) {
        const int b0 = uses0 > 0 ? mbar_wait(&mbar[0], (uint32_t)((uses0 - 1) & 1), 1L << 26) : 1;
        const int b1 = uses1 > 0 ? mbar_wait(&mbar[1], (uint32_t)((uses1 - 1) & 1), 1L << 26) : 1;
        if (!(b0 && b1) && lane == 0) atomicOr(&bad_s, 4);
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tbase), "r"(PTMEM));
    double* out = part + (int64_t)blockIdx.x * cols * p;
    if (tid < cols)     // thread tid holds basis column a = 128 (tid / 128) + tid % 128 = tid
#pragma unroll
        for (int c = 0; c < 16; ++c)
            if (c < p) out[tid * p + c] = (double)sh[c] + (double)sl[c];
    if (tid == 0 && (bad_s & 6)) atomicOr(&flags[0], 16);   // a bounded wait ran out (EXPM_TIMEOUT)
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

// W <- W - V h on the tensor cores; persistent CTAs, two per SM at most
cudaError_t launch_cgs_tc(const double* V, int64_t ldv, int cols, double* W, int64_t ldw, int p, int64_t n,
                          const double* h, int* flags, long spin_limit, cudaStream_t s) {
    if (!cgs_tc_fit(cols, p) || !h || !flags) return cudaErrorInvalidValue;
    const int64_t tiles = (n + TCM - 1) / TCM;
    const int g = (int)std::min<int64_t>(tiles, 2 * (int64_t)tc_sms());
    k_cgs_tc<0><<<g, TCT, tc_smem_bytes(cols), s>>>(V, ldv, cols, W, ldw, p, n, h, flags, spin_limit);
    return cudaGetLastError();
}

// The projection of the first CGS pass on the tensor cores: persistent CTAs, one partial each
// (max_blocks of them, or one per 256-row tile when there are fewer tiles: a grid capped at
// one wave by the occupancy calculator measured slower than the plan's CGS grid)
int proj_tc_blocks(int64_t n, int cols, int max_blocks) {
    (void)cols;
    const int64_t tiles = (n + PTILE - 1) / PTILE;
    return (int)std::max<int64_t>(1, std::min<int64_t>(tiles, max_blocks));
}

bool proj_tc_fit(int cols, int p) { return p >= 1 && p <= 16 && cols >= 1 && cols <= PCOLS_MAX; }

cudaError_t launch_proj_tc(const double* V, int64_t ldv, int cols, const double* W, int64_t ldw, int p, int64_t n,
                           double* part, int nb, int* flags, long spin_limit, cudaStream_t s) {
    if (!proj_tc_fit(cols, p) || nb < 1 || !part || !flags) return cudaErrorInvalidValue;
    if (cols <= 128)
        k_proj_tc<1><<<nb, PT, ptc_smem_bytes(1), s>>>(V, ldv, cols, W, ldw, p, n, part, flags, spin_limit);
    else
        k_proj_tc<2><<<nb, 2 * PT, ptc_smem_bytes(2), s>>>(V, ldv, cols, W, ldw, p, n, part, flags, spin_limit);
    return cudaGetLastError();
}

cudaError_t cgs_tc_set_smem_limits() {
    cudaError_t e = cudaFuncSetAttribute(k_cgs_tc<0>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)tc_smem_bytes(TC_COLS_MAX));
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_proj_tc<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ptc_smem_bytes(1));
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_proj_tc<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ptc_smem_bytes(2));
    return e;
}

}  // namespace expm
