"""User-facing wrapper: a plan per operator, torch tensors in and out.

Matrices are column-major, as in the C ABI: an (n, p) torch tensor with stride (1, ld).
``colmajor(n, p)`` allocates one.  All work is issued on the plan's CUDA stream.
"""
from __future__ import annotations

import ctypes as C

from . import _native as N


def colmajor(n, p, device="cuda", dtype=None, ld=None):
    import torch
    dtype = dtype or torch.float64
    ld = ld or n
    return torch.empty((p, ld), dtype=dtype, device=device).T[:n]


def _check_colmajor(X, n, p, name):
    import torch
    if X.dtype != torch.float64:
        raise TypeError(f"{name} must be float64")
    if X.dim() != 2 or X.shape[0] != n or X.shape[1] != p:
        raise ValueError(f"{name} must have shape ({n}, {p}), got {tuple(X.shape)}")
    if X.stride(0) != 1 and p > 1:
        raise ValueError(f"{name} must be column-major (stride (1, ld))")
    return X.stride(1) if p > 1 else max(n, X.stride(1) if X.dim() == 2 else n)


def cf_coeffs(nu=14):
    """(tau[nu/2], omega[nu/2], omega0, sigma) of the CF table computed by the library."""
    return N.expm_cf_coeffs(nu)


class Plan:
    """A plan for tA = t (diff Laplacian_h - vel . grad_h) on a 1/2/3-D grid (x fastest), or
    (``Plan.toeplitz``) for tA = t T with T symmetric Toeplitz."""

    def __init__(self, sides, diff, vel, p_max, m=10, tol=1e-10, max_cycles=200,
                 fixed_cycles=0, stream=None, algorithm=0, precision="fp64", certify=False, nu=0,
                 k_defl=0, row_ctas=0, cgs_ctas=0, inner_tol=0.0, inner_maxit=0, grid_sms=0,
                 _op=None):
        import torch
        if _op is None:
            sides = tuple(int(s) for s in sides)
            vel = tuple(float(v) for v in vel)
            if len(sides) != len(vel) or not 1 <= len(sides) <= 3:
                raise ValueError("sides and vel must have the same length 1..3")
            op = N.expm_op_desc()
            op.kind = N.EXPM_OP_CONV_DIFF
            op.ndim = len(sides)
            for d in range(3):
                op.side[d] = sides[d] if d < len(sides) else 1
                op.vel[d] = vel[d] if d < len(vel) else 0.0
            op.diff = float(diff)
        else:
            op = _op
        opts = N.expm_opts()
        opts.m, opts.max_cycles, opts.tol = int(m), int(max_cycles), float(tol)
        opts.precision = {"fp64": N.EXPM_PREC_FP64, "mixed": N.EXPM_PREC_MIXED}[precision]
        opts.fixed_cycles = int(fixed_cycles)
        opts.algorithm = int(algorithm)        # 0 auto, 1 SBFOM (Algorithm 1), 2 PSBFOM (Algorithm 2)
        opts.certify = 1 if certify else 0
        opts.nu_cf = int(nu)                   # 0: the paper's degree 14
        opts.k_defl = int(k_defl)              # 0: plain restart
        opts.row_ctas_per_sm = int(row_ctas)   # launch shape (0: library defaults; see autotune)
        opts.cgs_ctas_per_sm = int(cgs_ctas)
        opts.inner_tol = float(inner_tol)      # CSR operators: inner solve (0: library default)
        opts.inner_maxit = int(inner_maxit)
        opts.grid_sms = int(grid_sms)          # 0: row-pass grids sized for the whole device
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        self.sides, self.diff, self.vel, self.p_max, self.m = sides, diff, vel, p_max, m
        self.tol, self.max_cycles, self.algorithm, self.precision = tol, max_cycles, algorithm, precision
        if _op is None:
            self.n = 1
            for s in sides:
                self.n *= s
        else:
            self.n = int(op.n)
        self._h = N.expm_plan_create(op, int(p_max), opts, self.stream.cuda_stream)

    @classmethod
    def toeplitz(cls, col, n, p_max, **kw):
        """Plan for t T, T the n x n symmetric Toeplitz matrix with first column
        (col[0], .., col[bw], 0, ..), bw = len(col) - 1 (Example 5.4)."""
        import numpy as np
        a = np.ascontiguousarray(np.asarray(col, dtype=np.float64))
        op = N.expm_op_desc()
        op.kind = N.EXPM_OP_TOEPLITZ_SYM
        op.ndim = 1
        for d in range(3):
            op.side[d] = 1
        op.n = int(n)
        op.toeplitz_col = a.ctypes.data_as(C.POINTER(C.c_double))
        op.toeplitz_bw = len(a) - 1
        plan = cls(None, 0.0, None, p_max, _op=op, **kw)
        plan.toeplitz_col = a
        return plan

    @classmethod
    def csr(cls, A, p_max, **kw):
        """Plan for t A, A a general sparse n x n matrix (anything scipy.sparse.csr_matrix
        accepts), whose diagonal is negative and whose rows are weakly diagonally dominant.
        Algorithm 2 applies (tA)^{-1} inexactly by an inner iterative solve (inner_tol,
        inner_maxit)."""
        import numpy as np
        import scipy.sparse as sp
        M = sp.csr_matrix(A)
        n = M.shape[0]
        if M.shape != (n, n):
            raise ValueError("A must be square")
        rowptr = np.ascontiguousarray(M.indptr, dtype=np.int64)
        colind = np.ascontiguousarray(M.indices, dtype=np.int32)
        val = np.ascontiguousarray(M.data, dtype=np.float64)
        op = N.expm_op_desc()
        op.kind = N.EXPM_OP_CSR
        op.ndim = 1
        for d in range(3):
            op.side[d] = 1
        op.n = int(n)
        op.csr_rowptr = rowptr.ctypes.data_as(C.POINTER(C.c_int64))
        op.csr_colind = colind.ctypes.data_as(C.POINTER(C.c_int32))
        op.csr_val = val.ctypes.data_as(C.POINTER(C.c_double))
        plan = cls(None, 0.0, None, p_max, _op=op, **kw)
        plan.csr_arrays = (rowptr, colind, val)
        return plan

    def close(self):
        if getattr(self, "_h", None):
            N.expm_plan_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def profile(self, enable=True):
        """Reset and enable (or disable) per-kernel-class event timing inside the library."""
        N.expm_plan_profile(self._h, enable)

    def get_profile(self):
        """({stage: (ms, launches)}, total launches) since the last profile(True)."""
        return N.expm_plan_get_profile(self._h)

    # ------------------------------------------------------------------ entry points
    def expm_block(self, t, B, Z=None):
        """Z = r(tA) B on the device (Algorithm 2).  Returns (Z, info)."""
        n, p = self.n, B.shape[1]
        ldb = _check_colmajor(B, n, p, "B")
        if Z is None:
            Z = colmajor(n, p, device=B.device)
        ldz = _check_colmajor(Z, n, p, "Z")
        code, info = N.expm_block(self._h, float(t), B.data_ptr(), ldb, p, Z.data_ptr(), ldz)
        return Z, info

    def expm_block_host(self, t, hB, hZ):
        """Host buffers (torch CPU float64, column-major, ideally pinned): copies inside."""
        n, p = self.n, hB.shape[1]
        ldb = _check_colmajor(hB, n, p, "B")
        ldz = _check_colmajor(hZ, n, p, "Z")
        code, info = N.expm_block_host(self._h, float(t), hB.data_ptr(), ldb, p, hZ.data_ptr(), ldz)
        return hZ, info

    def expm_block_adjoint(self, t, G, Z=None, want_dB=True, want_dt=True):
        """Adjoint of Z = r(tA) B for G = dL/dZ: (dL/dB = r(tA^T) G or None, dL/dt = <G, A Z> or
        None, info).  Z (the forward result) is needed for dL/dt."""
        n, p = self.n, G.shape[1]
        ldg = _check_colmajor(G, n, p, "G")
        dGB = colmajor(n, p, device=G.device) if want_dB else None
        if want_dt and Z is None:
            raise ValueError("dL/dt needs the forward result Z")
        ldz = _check_colmajor(Z, n, p, "Z") if Z is not None else n
        gt, info = N.expm_block_adjoint(self._h, float(t), G.data_ptr(), ldg, p,
                                        Z.data_ptr() if Z is not None else 0, ldz,
                                        dGB.data_ptr() if dGB is not None else 0,
                                        _check_colmajor(dGB, n, p, "dGB") if dGB is not None else n,
                                        want_dt)
        return dGB, gt, info

    def op_apply(self, t, V, W=None):
        n, p = self.n, V.shape[1]
        ldv = _check_colmajor(V, n, p, "V")
        W = colmajor(n, p, device=V.device) if W is None else W
        N.expm_op_apply(self._h, float(t), V.data_ptr(), ldv, p, W.data_ptr(), _check_colmajor(W, n, p, "W"))
        return W

    def prec_apply(self, t, V, W=None):
        n, p = self.n, V.shape[1]
        ldv = _check_colmajor(V, n, p, "V")
        W = colmajor(n, p, device=V.device) if W is None else W
        N.expm_prec_apply(self._h, float(t), V.data_ptr(), ldv, p, W.data_ptr(), _check_colmajor(W, n, p, "W"))
        return W

    def arnoldi(self, t, V1):
        """One block Arnoldi pass from the orthonormal V1: returns (V_{m+1}, H~_m)."""
        import torch
        n, p = self.n, V1.shape[1]
        ldv = _check_colmajor(V1, n, p, "V1")
        m = self.m
        V = colmajor(n, (m + 1) * p, device=V1.device)
        H = torch.zeros(((m) * p, (m + 1) * p), dtype=torch.float64, device=V1.device).T
        N.expm_arnoldi(self._h, float(t), V1.data_ptr(), ldv, p, V.data_ptr(), V.stride(1),
                       H.data_ptr(), H.stride(1))
        return V, H


def expm_block_batched(plans, ts, Bs, Zs=None):
    """Independent solves Z_i = r(t_i A_i) B_i in one library call (each plan once; plans on
    distinct streams overlap on the GPU).  B_i on the device, or all on the host (torch CPU
    tensors, ideally pinned: expm_block_batched_host, the copies inside the call).  Returns
    (list of Z, list of info)."""
    host = all(not B.is_cuda for B in Bs)
    if Zs is None:
        if host:
            import torch
            Zs = [torch.empty((B.shape[1], pl.n), dtype=torch.float64).T for pl, B in zip(plans, Bs)]
        else:
            Zs = [colmajor(pl.n, B.shape[1], device=B.device) for pl, B in zip(plans, Bs)]
    ldbs = [_check_colmajor(B, pl.n, B.shape[1], "B") for pl, B in zip(plans, Bs)]
    ldzs = [_check_colmajor(Z, pl.n, B.shape[1], "Z") for pl, B, Z in zip(plans, Bs, Zs)]
    code, infos = N.expm_block_batched([pl._h for pl in plans], [float(t) for t in ts],
                                       [B.data_ptr() for B in Bs], ldbs, [B.shape[1] for B in Bs],
                                       [Z.data_ptr() for Z in Zs], ldzs, host=host)
    return Zs, infos


class Batch:
    """Many independent solves Z_i = r(t_i A_i) B_i as one CUDA graph launch with device-side
    stop tests (expm_batch_create / expm_batch_run).  The buffers stay in place: build once,
    call run() as often as needed (each run recomputes every Z_i from the current B_i)."""

    def __init__(self, plans, ts, Bs, Zs=None, stream=None):
        import torch
        self.plans, self.Bs = list(plans), list(Bs)
        self.Zs = Zs if Zs is not None else [colmajor(pl.n, B.shape[1], device=B.device) for pl, B in zip(plans, Bs)]
        ldbs = [_check_colmajor(B, pl.n, B.shape[1], "B") for pl, B in zip(plans, Bs)]
        ldzs = [_check_colmajor(Z, pl.n, B.shape[1], "Z") for pl, B, Z in zip(plans, Bs, self.Zs)]
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        self._h = N.expm_batch_create([pl._h for pl in plans], [float(t) for t in ts], [B.data_ptr() for B in Bs],
                                      ldbs, [B.shape[1] for B in Bs], [Z.data_ptr() for Z in self.Zs], ldzs,
                                      self.stream.cuda_stream)

    def run(self):
        """Launch the graph; returns (list of Z, list of info)."""
        code, infos = N.expm_batch_run(self._h, len(self.plans))
        return self.Zs, infos

    def close(self):
        if getattr(self, "_h", None):
            N.expm_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
