// k_rows8.cu -- the row-per-thread Gram-Schmidt / Cholesky-QR / Z-update kernels compiled for
// blocks of up to 8 columns (see rows_api.h; one translation unit per width, built in parallel).
#include "rows_api.h"
#include "rows_common.cuh"

namespace expm {
namespace rows8 {
constexpr int RG = RP * (RP + 1) / 2;
constexpr int NQ = (RG + 31) / 32;
#include "rows_impl.cuh"
#include "rows_launch.cuh"
}  // namespace rows8
}  // namespace expm
