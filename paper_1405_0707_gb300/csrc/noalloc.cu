// noalloc.cu -- an allocation-free variant of the exact-inverse apply (expm_prec_apply).
//
// Why it exists: some callers cannot call cudaMalloc.  A host application may hand all of
// the device's memory to its own pool allocator and forbid plug-in libraries from making
// raw allocations of their own, or a latency-critical loop may not be allowed to enter the
// CUDA allocator at all.  Such a caller still wants W = (tA)^{-1} V for one operator
// without creating a plan (plan creation allocates the Krylov workspace).
//
// How: every table the apply needs (the DST-I transform pair, the axis eigenvalues, the
// Thomas factors) and the transform temporary live in one file-scope device array of fixed
// size, kScratchDoubles doubles (8 MiB).  Every GPU that loads this library holds that array
// until the process exits.  Host code never uses the array's name as a device address (in
// host code it is only a stand-in for the symbol); the device address comes from
// cudaGetSymbolAddress, fetched once per device with that device current, cached, and
// passed to the kernels.
//
// Sharing: all calls use the same array.  Each call rebuilds every table it reads and writes
// the temporary before reading it, so nothing carries over from the previous call and
// nothing needs clearing.  Calls that overlap on the GPU (two streams, or two host threads
// on one device) race on the array: the caller must order them.
#include <cmath>
#include <mutex>

#include "internal.h"

using namespace expm;

namespace {

constexpr int64_t kScratchDoubles = int64_t(1) << 20;   // 8 MiB of FP64
constexpr int kMaxDevices = 64;

__device__ __align__(256) double g_noalloc_scratch[kScratchDoubles];

std::mutex g_mu;
double* g_addr[kMaxDevices] = {};

// Device address of the scratch array on the current device (looked up on first use).
expm_status scratch_address(double** out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return EXPM_CUDA_ERROR;
    if (dev < 0 || dev >= kMaxDevices) return EXPM_INVALID_ARG;
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_addr[dev]) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess) return EXPM_CUDA_ERROR;
        g_addr[dev] = static_cast<double*>(p);
    }
    *out = g_addr[dev];
    return EXPM_OK;
}

inline int64_t up32(int64_t a) { return (a + 31) / 32 * 32; }

}  // namespace

extern "C" expm_status expm_prec_apply_noalloc(const expm_op_desc* op, double t, const double* dV,
                                               int64_t ldv, int p, double* dW, int64_t ldw,
                                               void* stream) {
    if (!op || !dV || !dW || dV == dW) return EXPM_INVALID_ARG;
    if (op->kind != EXPM_OP_CONV_DIFF || op->ndim < 1 || op->ndim > 2) return EXPM_INVALID_ARG;
    if (!(op->diff > 0.0) || !std::isfinite(op->diff)) return EXPM_INVALID_ARG;
    if (!(t > 0.0) || !std::isfinite(t) || p < 1 || p > kMaxP) return EXPM_INVALID_ARG;
    Axis ax[2];
    int64_t n = 1;
    for (int d = 0; d < op->ndim; ++d) {
        const int N = op->side[d];
        // every side is bounded by the scratch size before any product is formed, so the
        // layout arithmetic below stays far from int64 overflow
        if (N < 1 || N > kScratchDoubles || !std::isfinite(op->vel[d])) return EXPM_INVALID_ARG;
        const double h = 1.0 / (N + 1);
        ax[d].N = N;
        ax[d].l = op->diff / (h * h) + op->vel[d] / (2.0 * h);
        ax[d].c = -2.0 * op->diff / (h * h);
        ax[d].u = op->diff / (h * h) - op->vel[d] / (2.0 * h);
        if (!(ax[d].l * ax[d].u > 0.0)) return EXPM_INVALID_ARG;   // cell Peclet >= 1
        n *= N;
    }
    if (ldv < n || ldw < n) return EXPM_INVALID_ARG;
    // scratch layout: [Qf Ny^2 | Qi Ny^2 | lambda Ny | Thomas m n | Thomas c' n | T1 n p]
    const int64_t Ny = op->ndim == 2 ? ax[1].N : 0;
    const int64_t oQf = 0, oQi = up32(Ny * Ny), oLam = oQi + up32(Ny * Ny), oThm = oLam + up32(Ny);
    const int64_t oThc = oThm + up32(n), oT1 = oThc + up32(n);
    const int64_t need = op->ndim == 2 ? oT1 + n * p : oT1;
    if (need > kScratchDoubles) return EXPM_INVALID_ARG;   // beyond the fixed 8 MiB scratch
    double* S = nullptr;
    expm_status st = scratch_address(&S);
    if (st != EXPM_OK) return st;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    const double inv_t = 1.0 / t;
    if (op->ndim == 1) {
        if (launch_thomas_setup(S + oThm, S + oThc, ax[0].N, 1, ax[0].l, ax[0].c, ax[0].u, nullptr, 1,
                                nullptr, 1, s) != cudaSuccess)
            return EXPM_CUDA_ERROR;
        if (launch_tridiag_lines(dV, ldv, dW, ldw, p, ax[0].N, 1, ax[0].l, S + oThm, S + oThc, inv_t, s) !=
            cudaSuccess)
            return EXPM_CUDA_ERROR;
        return EXPM_OK;
    }
    const int nx = ax[0].N, ny = ax[1].N;
    double* T1 = S + oT1;
    if (launch_axis_setup(S + oQf, S + oQi, S + oLam, ny, ax[1].l, ax[1].c, ax[1].u, s) != cudaSuccess ||
        launch_thomas_setup(S + oThm, S + oThc, nx, ny, ax[0].l, ax[0].c, ax[0].u, S + oLam, ny, nullptr, 1,
                            s) != cudaSuccess)
        return EXPM_CUDA_ERROR;
    GemmArgs g1{dV, S + oQf, T1, nx, ny, ny, 1, nx, ldv, 0, ny, 1, n, 0, ny, p, 1};
    GemmArgs g2{T1, S + oQi, dW, nx, ny, ny, ny, 1, n, 0, 1, nx, ldw, 0, ny, p, 1};
    if (launch_gemm(g1, s) != cudaSuccess ||
        launch_tridiag_lines(T1, n, T1, n, p, nx, ny, ax[0].l, S + oThm, S + oThc, inv_t, s) != cudaSuccess ||
        launch_gemm(g2, s) != cudaSuccess)
        return EXPM_CUDA_ERROR;
    return EXPM_OK;
}
