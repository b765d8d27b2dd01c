"""Solver: an object wrapper over one hdd_ctx (include/hdd.h) with PyTorch device memory."""
from __future__ import annotations

import ctypes as C

from ._binding import (AssembleParams, DDParams, HDDError, KernelStat, SolveParams, SolveStats,
                       lib)

LOCAL_OPS = {"A": 0, "Z": 1, "Zt": 2, "Einv": 3, "PA": 4, "R": 5, "Ainv": 6}


def _torch():
    import torch
    return torch


class Solver:
    """One problem on one GPU: assemble → setup_dd → setup_deflation → solve."""

    def __init__(self, device: int = 0):
        torch = _torch()
        if not torch.cuda.is_available():
            raise RuntimeError("paper_2103_17081_gb300 needs a CUDA GPU (no CPU fallback)")
        self.device = int(device)
        torch.cuda.set_device(self.device)
        self._L = lib()
        h = C.c_void_p()
        self._check(self._L.hdd_create(C.byref(h), self.device), "hdd_create", ctx=False)
        self._h = h
        self.N = None
        self.k = None
        self.nsub = 0
        self.nrhs = 1

    # -- plumbing ------------------------------------------------------------------------------
    def _check(self, rc: int, where: str, ctx: bool = True):
        if rc != 0:
            msg = ""
            if ctx and getattr(self, "_h", None):
                msg = self._L.hdd_last_error(self._h).decode()
            raise HDDError(rc, where, msg)

    def _stream(self, stream=None):
        torch = _torch()
        s = stream if stream is not None else torch.cuda.current_stream(self.device)
        return C.c_void_p(s.cuda_stream)

    def _vec(self, t, n=None, name="vector"):
        torch = _torch()
        if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == torch.complex128
                and t.is_contiguous()):
            raise TypeError(f"{name} must be a contiguous complex128 CUDA tensor")
        if n is not None and t.numel() < n:
            raise ValueError(f"{name} has {t.numel()} entries, needs {n}")
        return C.c_void_p(t.data_ptr())

    def close(self):
        if getattr(self, "_h", None):
            self._L.hdd_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- set-up --------------------------------------------------------------------------------
    def assemble(self, k: float, N: int, diag: int = 0, bc: int = 0):
        """bc 0: u = 0 on the boundary, (N-1)² unknowns; bc 1: impedance (Sommerfeld) condition
        du/dn - i k u = 0 on all four sides, (N+1)² unknowns."""
        p = AssembleParams(float(k), int(N), int(diag), int(bc))
        self._check(self._L.hdd_assemble(self._h, C.byref(p)), "hdd_assemble")
        self.N, self.k, self.bc = int(N), float(k), int(bc)
        self.n = (self.N + 1) ** 2 if self.bc else (self.N - 1) ** 2
        return self

    def setup_dd(self, Sx: int, Sy: int, overlap: int, ifx=None, ify=None):
        ax = (C.c_int * (Sx + 1))(*ifx) if ifx is not None else None
        ay = (C.c_int * (Sy + 1))(*ify) if ify is not None else None
        p = DDParams(int(Sx), int(Sy), int(overlap),
                     C.cast(ax, C.POINTER(C.c_int)) if ax is not None else None,
                     C.cast(ay, C.POINTER(C.c_int)) if ay is not None else None)
        self._check(self._L.hdd_setup_dd(self._h, C.byref(p)), "hdd_setup_dd")
        self.nsub = self._L.hdd_num_subdomains(self._h)
        self.nrhs = 1
        return self

    def setup_batch(self, nrhs: int):
        """Solve `nrhs` right-hand sides per call (vectors stored RHS-major)."""
        self._check(self._L.hdd_setup_batch(self._h, int(nrhs)), "hdd_setup_batch")
        self.nrhs = self._L.hdd_num_rhs(self._h)
        return self

    def setup_deflation(self, stream=None):
        self._check(self._L.hdd_setup_deflation(self._h, self._stream(stream)), "hdd_setup_deflation")
        return self

    def setup_exact(self, stream=None):
        self._check(self._L.hdd_setup_exact(self._h, self._stream(stream)), "hdd_setup_exact")
        return self

    def setup_coarse_grid(self, c: int = 2, stream=None):
        """Grid coarse space of the two-level variant: P1 on the mesh of N/c intervals."""
        self._check(self._L.hdd_setup_coarse_grid(self._h, int(c), self._stream(stream)),
                    "hdd_setup_coarse_grid")
        return self

    @property
    def coarse_grid_size(self) -> int:
        return int(self._L.hdd_coarse_grid_size(self._h))

    def coarse_grid_op(self, stages: str, x, prec: int = 128, stream=None):
        """Apply the stages of Q = P A_H⁻¹ Pᵀ named in `stages` ("R" restrict, "S" solve,
        "P" prolong, in that order; "RSP" is Q) to nrhs complex128 vectors."""
        bits = {"R": 1, "S": 2, "P": 4}
        st = 0
        for ch in stages:
            st |= bits[ch]
        mm = self.coarse_grid_size
        nin = self.nrhs * (self.n if st & 1 else mm)
        nout = self.nrhs * (self.n if st & 4 else mm)
        out = self.empty(nout)
        self._check(self._L.hdd_coarse_grid_op(self._h, st, int(prec), self._vec(x, nin, "x"),
                                               self._vec(out), self._stream(stream)),
                    "hdd_coarse_grid_op")
        return out

    @classmethod
    def from_workload(cls, w, device: int = 0, deflation: bool = True, exact: bool = False):
        s = cls(device).assemble(w.k, w.N, bc=getattr(w, "bc", 0))
        s.setup_dd(w.Sx, w.Sy, w.overlap, w.ifx, w.ify)
        if w.nrhs > 1:
            s.setup_batch(w.nrhs)
        if deflation:
            s.setup_deflation()
        if exact:
            s.setup_exact()
        return s

    # -- queries -------------------------------------------------------------------------------
    def subdomain(self, s: int) -> dict:
        info = (C.c_int * 12)()
        self._check(self._L.hdd_get_subdomain(self._h, int(s), info), "hdd_get_subdomain")
        keys = ("ix0", "ix1", "iy0", "iy1", "ox0", "ox1", "oy0", "oy1", "nx", "ny", "mx", "my")
        return dict(zip(keys, list(info)))

    def offsets(self):
        fo = (C.c_longlong * (self.nsub + 1))()
        co = (C.c_longlong * (self.nsub + 1))()
        self._check(self._L.hdd_get_offsets(self._h, fo, co), "hdd_get_offsets")
        return list(fo), list(co)

    # -- vectors -------------------------------------------------------------------------------
    def empty(self, n=None):
        torch = _torch()
        return torch.empty(self.n if n is None else n, dtype=torch.complex128, device=f"cuda:{self.device}")

    def build_rhs(self, spec, out=None, stream=None):
        """Load vector of a workloads.RHSSpec (point sources and Gaussian bumps) on the device."""
        pts = [v for p in spec.points for v in (p.x, p.y, p.amp)]
        bps = [v for b in spec.bumps for v in (b.cx, b.cy, b.sigma, b.amp)]
        f = self.empty() if out is None else out
        P = (C.c_double * max(1, len(pts)))(*pts)
        B = (C.c_double * max(1, len(bps)))(*bps)
        self._check(self._L.hdd_build_rhs(self._h, len(spec.points), P, len(spec.bumps), B,
                                          self._vec(f, self.n, "f"), self._stream(stream)),
                    "hdd_build_rhs")
        return f

    def apply_A(self, x, out=None, stream=None):
        nrhs = x.numel() // self.n
        y = self.empty(x.numel()) if out is None else out
        self._check(self._L.hdd_apply_A(self._h, self._vec(x), self._vec(y), nrhs, self._stream(stream)),
                    "hdd_apply_A")
        return y

    # -- solves --------------------------------------------------------------------------------
    @staticmethod
    def params(outer_tol=1e-6, outer_restart=2000, outer_maxit=2000, inner_tol=1e-2,
               inner_restart=30, inner_maxit=1000, inner_prec=64, warm_start=0,
               outer_reorth32=1, two_level=0) -> SolveParams:
        return SolveParams(outer_tol, outer_restart, outer_maxit, inner_tol, inner_restart,
                           inner_maxit, inner_prec, int(bool(warm_start)), int(bool(outer_reorth32)),
                           int(bool(two_level)))

    def build_rhs_batch(self, specs):
        """Load vectors of several RHSSpecs, stacked RHS-major in one tensor."""
        f = self.empty(len(specs) * self.n)
        for r, spec in enumerate(specs):
            self.build_rhs(spec, out=f[r * self.n:(r + 1) * self.n])
        return f

    def solve(self, f, out=None, stream=None, raise_on_error=True, **kw):
        prm = self.params(**kw)
        nt = self.nrhs * self.n
        x = self.empty(nt) if out is None else out
        st = SolveStats()
        rc = self._L.hdd_solve(self._h, self._vec(f, nt, "f"), self._vec(x, nt, "x"),
                               C.byref(prm), C.byref(st), self._stream(stream))
        stats = {k: getattr(st, k) for k, _ in SolveStats._fields_ if k != "res_history"}
        stats["res_history"] = [st.res_history[i] for i in range(st.n_history)]
        stats["status_code"] = rc
        if rc != 0 and raise_on_error:
            self._check(rc, "hdd_solve")
        return x, stats

    def autotune(self, stream=None, **kw):
        """Pick the fastest tile shapes for RAS applications with these solve parameters (see
        hdd_autotune); they apply to every later call on this solver."""
        prm = self.params(**kw)
        f, c, ms = C.c_int(0), C.c_int(0), C.c_double(0.0)
        self._check(self._L.hdd_autotune(self._h, C.byref(prm), self._stream(stream), C.byref(f), C.byref(c),
                                         C.byref(ms)), "hdd_autotune")
        return {"fine_rows": f.value, "coarse_rows": c.value, "ras_ms": ms.value}

    def ras_apply(self, v, out=None, stream=None, **kw):
        prm = self.params(**kw)
        nt = self.nrhs * self.n
        z = self.empty(nt) if out is None else out
        its = (C.c_int * max(1, self.nsub * self.nrhs))()
        self._check(self._L.hdd_ras_apply(self._h, self._vec(v, nt, "v"), self._vec(z, nt, "z"),
                                          C.byref(prm), its, self._stream(stream)), "hdd_ras_apply")
        return z, list(its)[: self.nsub * self.nrhs]

    def local_op(self, op: str, x, prec: int = 128, stream=None):
        """Apply one local operator to packed vectors of every (subdomain, RHS) task."""
        fo, co = self.offsets()
        F, Cc = self.nrhs * fo[-1], self.nrhs * co[-1]
        nin = {"A": F, "Z": Cc, "Zt": F, "Einv": Cc, "PA": F, "R": self.nrhs * self.n, "Ainv": F}[op]
        nout = {"A": F, "Z": F, "Zt": Cc, "Einv": Cc, "PA": F, "R": F, "Ainv": F}[op]
        out = self.empty(nout)
        self._check(self._L.hdd_local_op(self._h, LOCAL_OPS[op], int(prec), self._vec(x, nin, "x"),
                                         self._vec(out), self._stream(stream)), "hdd_local_op")
        return out

    # -- profiling -----------------------------------------------------------------------------
    def profile(self, enable: bool = True):
        """Clear the per-family counters and switch CUDA-event timing of every launch on/off."""
        self._check(self._L.hdd_profile(self._h, 1 if enable else 0), "hdd_profile")

    def profile_stats(self) -> list:
        out = []
        for i in range(self._L.hdd_profile_count(self._h)):
            k = KernelStat()
            self._check(self._L.hdd_profile_get(self._h, i, C.byref(k)), "hdd_profile_get")
            out.append({"name": k.name.decode(), "launches": k.launches, "ms": k.ms,
                        "bytes": k.bytes, "flops": k.flops,
                        "bound": {0: "hbm", 1: "fp64", 2: "fp32"}.get(k.bound, "hbm")})
        return out

    def launch_count(self) -> int:
        return int(self._L.hdd_launch_count(self._h))

    OPTIONS = {"coarse_lookahead": 1, "fused_inner": 2, "outer_dots_df": 3, "outer_update_df": 4, "outer_dcgs2": 5,
               "coarse_df": 6, "coarse_spike": 7, "outer_dots_biased": 8}

    def set_option(self, name: str, value: int):
        """Implementation choice of this context (hdd_set_option): "coarse_lookahead" selects
        the look-ahead block solve (1) or the plain one (0); "fused_inner" the one-kernel inner
        Arnoldi step (1) or the separate kernels (0); "outer_dots_df" the outer CGS dot products
        in double-FP32 arithmetic (1) or in FP64 (0); "outer_update_df" the first-pass update in
        double-FP32 (1) or FP64 (0); "outer_dcgs2" the delayed CGS2 outer Arnoldi (1) or plain
        CGS2 (0); "coarse_df" the complex64 inner iteration's coarse solves in double-FP32 (1) or
        FP64 (0); "coarse_spike" those solves split over 2 or 4 SMs (SPIKE) when SMs are free (1)
        or not (0; takes effect at the next hdd_setup_deflation); "outer_dots_biased" the delayed
        CGS2 first-pass dot products with biased accumulators (1: half their FP32 instructions,
        a few 1e-12 of Σ|v w|; the second pass removes what they leave) or with the two-sum (0)."""
        self._check(self._L.hdd_set_option(self._h, self.OPTIONS[name], int(value)), "hdd_set_option")
        return self

    # -- learned warm start ----------------------------------------------------------------------
    def cnn_num_params(self) -> int:
        return int(self._L.hdd_cnn_num_params())

    def cnn_set_params(self, params):
        import numpy as np
        a = np.ascontiguousarray(params, dtype=np.float32)
        if a.size != self.cnn_num_params():
            raise ValueError(f"expected {self.cnn_num_params()} parameters, got {a.size}")
        self._check(self._L.hdd_cnn_set_params(self._h, a.ctypes.data_as(C.POINTER(C.c_float))),
                    "hdd_cnn_set_params")

    def cnn_get_params(self):
        import numpy as np
        a = np.zeros(self.cnn_num_params(), dtype=np.float32)
        self._check(self._L.hdd_cnn_get_params(self._h, a.ctypes.data_as(C.POINTER(C.c_float))),
                    "hdd_cnn_get_params")
        return a

    def cnn_load(self, path: str):
        """Load warm-start parameters from a file written by warmstart.save / cnn_save (C ABI)."""
        self._check(self._L.hdd_warmstart_load(self._h, str(path).encode()), "hdd_warmstart_load")

    def cnn_save(self, path: str):
        self._check(self._L.hdd_warmstart_save(self._h, str(path).encode()), "hdd_warmstart_save")

    def packed_len(self) -> int:
        fo, _ = self.offsets()
        return self.nrhs * fo[-1]

    def cnn_forward(self, f_packed, stream=None):
        x0 = self.empty(self.packed_len())
        self._check(self._L.hdd_cnn_forward(self._h, self._vec(f_packed, self.packed_len(), "f"),
                                            self._vec(x0), self._stream(stream)), "hdd_cnn_forward")
        return x0

    def cnn_infer(self, f_packed, stream=None):
        """The warm start's inference path: tensor-core layers, BF16 activations."""
        x0 = self.empty(self.packed_len())
        self._check(self._L.hdd_cnn_infer(self._h, self._vec(f_packed, self.packed_len(), "f"),
                                          self._vec(x0), self._stream(stream)), "hdd_cnn_infer")
        return x0

    def cnn_loss_grad(self, f_packed, with_grad=True):
        import numpy as np
        loss = C.c_double(0.0)
        g = np.zeros(self.cnn_num_params(), dtype=np.float32) if with_grad else None
        gp = g.ctypes.data_as(C.POINTER(C.c_float)) if with_grad else None
        self._check(self._L.hdd_cnn_loss_grad(self._h, self._vec(f_packed, self.packed_len(), "f"),
                                              C.byref(loss), gp), "hdd_cnn_loss_grad")
        return loss.value, g

    def cnn_train_step(self, f_packed, lr, stream=None) -> float:
        loss = C.c_double(0.0)
        self._check(self._L.hdd_cnn_train_step(self._h, self._vec(f_packed, self.packed_len(), "f"),
                                               float(lr), C.byref(loss), self._stream(stream)),
                    "hdd_cnn_train_step")
        return loss.value

    def outer_vector(self, j, stream=None):
        v = self.empty(self.nrhs * self.n)
        self._check(self._L.hdd_get_outer_vector(self._h, int(j), self._vec(v), self._stream(stream)),
                    "hdd_get_outer_vector")
        return v
