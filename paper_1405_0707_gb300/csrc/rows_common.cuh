// rows_common.cuh -- the row-pass geometry shared by k_krylov.cu and the per-width row-kernel
// translation units (k_rows4/8/12/16.cu): rows per CTA, whole 16-row tiles, and the
// destination rules of a triangular-solve pass.
#pragma once
#include "df.cuh"
#include "internal.h"

namespace expm {
namespace {

constexpr int TR = 16;      // rows per shared-memory tile

__device__ inline int64_t rows_begin(int64_t rpb) { return (int64_t)blockIdx.x * rpb; }

// Loads are issued in batches of LB per thread into registers before any is converted or
// stored, so LB independent global loads are in flight per thread.
constexpr int LB = 8;

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

inline int64_t rows_per_block(int64_t n, int nblk) {
    int64_t r = (n + nblk - 1) / nblk;
    return (r + TR - 1) / TR * TR;
}
inline int blocks_for(int64_t n, int nblk) {
    const int64_t rpb = rows_per_block(n, nblk);
    return (int)((n + rpb - 1) / rpb);
}

}  // namespace
}  // namespace expm
