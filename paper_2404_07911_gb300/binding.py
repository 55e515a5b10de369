"""ctypes binding of libunfitted (argument marshalling only; every step of the operator runs in
the library).  Names follow the C ABI of include/unfitted.h.

PyTorch supplies device memory and streams: vmult takes torch CUDA tensors and passes their data
pointers and the current (or given) stream to the library.
"""
import ctypes
import os

import numpy as np

from . import build as _build

UF_OK, UF_EINVAL, UF_ENOMEM, UF_ECUDA, UF_EUNSUPPORTED, UF_EGEOMETRY, UF_ENODEVICE = range(7)
UF_FP64, UF_FP32 = 1, 2
UF_LS_SPHERE = 0
UF_LS_PLANE = 1
UF_LS_SPHERES = 2
UF_DG, UF_CG = 0, 1
UF_GP_FACE, UF_GP_VOLUME = 0, 1

_STATUS = {0: "UF_OK", 1: "UF_EINVAL", 2: "UF_ENOMEM", 3: "UF_ECUDA", 4: "UF_EUNSUPPORTED",
           5: "UF_EGEOMETRY", 6: "UF_ENODEVICE"}


class UnfittedError(RuntimeError):
    def __init__(self, status, message):
        super().__init__(f"{_STATUS.get(status, status)}: {message}")
        self.status = status


class uf_params(ctypes.Structure):
    _fields_ = [
        ("dim", ctypes.c_int),
        ("degree", ctypes.c_int),
        ("n_cells", ctypes.c_int * 3),
        ("lo", ctypes.c_double * 3),
        ("hi", ctypes.c_double * 3),
        ("ls_kind", ctypes.c_int),
        ("ls_center", ctypes.c_double * 3),
        ("ls_radius", ctypes.c_double),
        ("quad_order", ctypes.c_int),
        ("sipg_gamma", ctypes.c_double),
        ("nitsche_gamma", ctypes.c_double),
        ("gp_max_order", ctypes.c_int),
        ("gp_gamma", ctypes.c_double),
        ("precisions", ctypes.c_int),
        ("device", ctypes.c_int),
        ("kappa", ctypes.POINTER(ctypes.c_double)),
        ("discretization", ctypes.c_int),
        ("ls_normal", ctypes.c_double * 3),
        ("ls_offset", ctypes.c_double),
        ("gp_kind", ctypes.c_int),
        ("gp_tau", ctypes.c_double),
        ("ls_spheres", ctypes.POINTER(ctypes.c_double)),
        ("ls_n_spheres", ctypes.c_int),
    ]


class uf_info(ctypes.Structure):
    _fields_ = [(name, ctypes.c_int64) for name in (
        "n_active", "n_inside", "n_cut", "n_dofs", "n_faces", "n_faces_full", "n_faces_cut",
        "n_faces_empty", "n_faces_gp", "n_vol_points", "n_surf_points", "n_face_points",
        "n_vol_lines", "n_face_lines")] + [
        ("dim", ctypes.c_int32), ("degree", ctypes.c_int32), ("dofs_per_cell", ctypes.c_int32),
        ("quad_order", ctypes.c_int32), ("h", ctypes.c_double), ("bytes_fp64", ctypes.c_double),
        ("bytes_fp32", ctypes.c_double), ("flops", ctypes.c_double),
        ("kernel_bytes_fp64", ctypes.c_double * 2), ("kernel_bytes_fp32", ctypes.c_double * 2),
        ("kernel_flops", ctypes.c_double * 2), ("kernel_flops_built", ctypes.c_double * 2),
        ("kernel_flops_built_fp32", ctypes.c_double * 2), ("n_vol_groups", ctypes.c_int64),
        ("cut_lane_classes", ctypes.c_int64 * 3)]


class uf_kernel_times(ctypes.Structure):
    _fields_ = [("ms_total", ctypes.c_double * 8), ("launches", ctypes.c_int64 * 8),
                ("kernel_launches", ctypes.c_int64 * 8)]


class uf_solve_params(ctypes.Structure):
    _fields_ = [("mode", ctypes.c_int), ("tol", ctypes.c_double), ("inner_tol", ctypes.c_double),
                ("max_iter", ctypes.c_int), ("max_outer", ctypes.c_int)]


class uf_solve_stats(ctypes.Structure):
    _fields_ = [("converged", ctypes.c_int), ("outer", ctypes.c_int), ("iterations", ctypes.c_int),
                ("rel_residual", ctypes.c_double), ("seconds", ctypes.c_double)]


UF_SOLVE_FP64, UF_SOLVE_IR, UF_SOLVE_IR_SPLIT = 0, 1, 2

EXPORTED = ["uf_create_unfitted_operator", "uf_get_info", "uf_vmult", "uf_vmult_adjoint",
            "uf_vmult_host", "uf_vmult_adjoint_host", "uf_vmult_host_async",
            "uf_vmult_adjoint_host_async", "uf_host_wait", "uf_profile_begin", "uf_profile_end",
            "uf_set_kappa", "uf_export_cells", "uf_export_cut_cell_rule",
            "uf_export_cut_cell_counts", "uf_export_cut_cell_lines",
            "uf_export_cut_face_rule", "uf_assemble_csr", "uf_csr_info", "uf_csr_spmv",
            "uf_export_csr", "uf_release_csr", "uf_kappa_gradient", "uf_kappa_gradient_noalloc",
            "uf_set_kappa_device", "uf_vmult_split", "uf_set_split_fraction", "uf_export_cg", "uf_solve", "uf_manufactured_rhs", "uf_l2_error",
            "uf_destroy", "uf_debug_fail_allocation", "uf_debug_live_allocations", "uf_last_error"]

_lib = None


def load_library(path=None):
    """Load libunfitted.so (building it first if it is missing or stale).  Raises if the
    library cannot be built or loaded: there is no fallback implementation."""
    global _lib
    if _lib is not None:
        return _lib
    if path is None:
        path = _build.build()
    if not os.path.exists(path):
        raise RuntimeError(f"libunfitted not found at {path}")
    lib = ctypes.CDLL(path)
    P = ctypes.c_void_p
    lib.uf_create_unfitted_operator.argtypes = [ctypes.POINTER(uf_params), ctypes.POINTER(P)]
    lib.uf_get_info.argtypes = [P, ctypes.POINTER(uf_info)]
    lib.uf_vmult.argtypes = [P, ctypes.c_int, P, P, P]
    lib.uf_vmult_adjoint.argtypes = [P, ctypes.c_int, P, P, P]
    lib.uf_vmult_host.argtypes = [P, ctypes.c_int, P, P, P]
    lib.uf_vmult_adjoint_host.argtypes = [P, ctypes.c_int, P, P, P]
    lib.uf_vmult_host_async.argtypes = [P, ctypes.c_int, P, P, P]
    lib.uf_vmult_adjoint_host_async.argtypes = [P, ctypes.c_int, P, P, P]
    lib.uf_host_wait.argtypes = [P, P]
    lib.uf_profile_begin.argtypes = [P, ctypes.c_int]
    lib.uf_profile_end.argtypes = [P, ctypes.POINTER(uf_kernel_times)]
    lib.uf_set_kappa.argtypes = [P, ctypes.POINTER(ctypes.c_double)]
    lib.uf_export_cells.argtypes = [P, P, P]
    lib.uf_export_cut_cell_rule.argtypes = [P, ctypes.c_int64, ctypes.c_int, P, P, P,
                                            ctypes.POINTER(ctypes.c_int64)]
    lib.uf_export_cut_face_rule.argtypes = [P, ctypes.c_int64, ctypes.c_int, ctypes.c_int, P, P,
                                            ctypes.POINTER(ctypes.c_int64)]
    lib.uf_export_cut_cell_counts.argtypes = [P, P, P, P, P]
    lib.uf_export_cut_cell_lines.argtypes = [P, ctypes.c_int64, P, P, P, ctypes.POINTER(ctypes.c_int64)]
    lib.uf_assemble_csr.argtypes = [P, ctypes.c_int]
    lib.uf_csr_info.argtypes = [P, ctypes.c_int, ctypes.POINTER(ctypes.c_int64),
                                ctypes.POINTER(ctypes.c_double)]
    lib.uf_csr_spmv.argtypes = [P, ctypes.c_int, P, P, P]
    lib.uf_export_csr.argtypes = [P, ctypes.c_int, P, P, P]
    lib.uf_release_csr.argtypes = [P]
    lib.uf_kappa_gradient.argtypes = [P, P, P, P, P]
    lib.uf_kappa_gradient_noalloc.argtypes = [P, P, P, P, P]
    lib.uf_set_kappa_device.argtypes = [P, P, P]
    lib.uf_vmult_split.argtypes = [P, P, P, P]
    lib.uf_set_split_fraction.argtypes = [P, ctypes.c_double]
    lib.uf_export_cg.argtypes = [P, P, P, P]
    lib.uf_solve.argtypes = [P, ctypes.POINTER(uf_solve_params), P, P, ctypes.POINTER(uf_solve_stats), P]
    lib.uf_manufactured_rhs.argtypes = [P, ctypes.c_double, ctypes.POINTER(ctypes.c_double)]
    lib.uf_l2_error.argtypes = [P, ctypes.c_double, ctypes.POINTER(ctypes.c_double),
                                ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double)]
    lib.uf_destroy.argtypes = [P]
    lib.uf_debug_fail_allocation.argtypes = [ctypes.c_int64]
    lib.uf_debug_live_allocations.argtypes = [ctypes.POINTER(ctypes.c_int64)]
    lib.uf_last_error.restype = ctypes.c_char_p
    for name in EXPORTED:
        if name != "uf_last_error":
            getattr(lib, name).restype = ctypes.c_int
    _lib = lib
    return lib


def _check(st):
    if st != UF_OK:
        raise UnfittedError(st, _lib.uf_last_error().decode())


def debug_fail_allocation(after):
    """Fault injection: the library's next `after` allocations succeed, the one after them fails
    with UF_ENOMEM (negative: disarm)."""
    _check(load_library().uf_debug_fail_allocation(int(after)))


def debug_live_allocations():
    """The library's device, pinned-host and operator allocations not yet released."""
    live = ctypes.c_int64()
    _check(load_library().uf_debug_live_allocations(ctypes.byref(live)))
    return live.value


def _ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p) if a is not None else None


def make_params(cfg, precisions=UF_FP64 | UF_FP32, device=0, kappa=None):
    p = uf_params()
    p.dim = int(cfg["dim"])
    p.degree = int(cfg["degree"])
    for a in range(3):
        p.n_cells[a] = int(cfg["n_cells"][a]) if a < len(cfg["n_cells"]) else 1
        p.lo[a] = float(cfg["lo"][a]) if a < len(cfg["lo"]) else 0.0
        p.hi[a] = float(cfg["hi"][a]) if a < len(cfg["hi"]) else 0.0
        p.ls_center[a] = float(cfg["center"][a]) if a < len(cfg["center"]) else 0.0
    p.ls_kind = UF_LS_SPHERE
    p.ls_radius = float(cfg["radius"])
    p.gp_kind = UF_GP_VOLUME if cfg.get("gp_kind", "face") == "volume" else UF_GP_FACE
    p.gp_tau = float(cfg.get("gp_tau", 1.0))
    if cfg.get("ls_kind", "sphere") == "plane":
        p.ls_kind = UF_LS_PLANE
        for a in range(3):
            p.ls_normal[a] = float(cfg["normal"][a]) if a < len(cfg["normal"]) else 0.0
        p.ls_offset = float(cfg["offset"])
    p.quad_order = int(cfg["quad_order"])
    p.sipg_gamma = float(cfg["sipg_gamma"])
    p.nitsche_gamma = float(cfg["nitsche_gamma"])
    p.gp_max_order = int(cfg["gp_max_order"])
    p.gp_gamma = float(cfg["gp_gamma"])
    p.precisions = int(precisions)
    p.device = int(device)
    p.kappa = None
    p.discretization = UF_CG if cfg.get("discretization", "dg") == "cg" else UF_DG
    return p


class UnfittedOperator:
    """Owner of one uf_operator.  device = -1 builds the host setup only (no GPU)."""

    def __init__(self, cfg, precisions=UF_FP64 | UF_FP32, device=0, kappa=None):
        lib = load_library()
        self._keep = None
        params = make_params(cfg, precisions, device)
        if kappa is not None:
            self._keep = np.ascontiguousarray(kappa, dtype=np.float64)
            params.kappa = self._keep.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
        spheres = None
        if cfg.get("ls_kind", "sphere") == "spheres":
            spheres = np.ascontiguousarray(np.asarray(cfg["spheres"], dtype=np.float64).reshape(-1, 4))
            params.ls_kind = UF_LS_SPHERES
            params.ls_spheres = spheres.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
            params.ls_n_spheres = len(spheres)
        handle = ctypes.c_void_p()
        _check(lib.uf_create_unfitted_operator(ctypes.byref(params), ctypes.byref(handle)))
        self._h = handle
        self.device = device
        self.precisions = precisions
        self.info = self.get_info()
        if kappa is not None and len(self._keep) != self.info["n_active"]:
            self.close()
            raise ValueError("kappa must have one entry per active cell")

    # ---- lifetime
    def close(self):
        if getattr(self, "_h", None):
            _lib.uf_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ---- queries
    def get_info(self):
        inf = uf_info()
        _check(_lib.uf_get_info(self._h, ctypes.byref(inf)))
        out = {}
        for name, _ in uf_info._fields_:
            v = getattr(inf, name)
            out[name] = list(v) if isinstance(v, ctypes.Array) else v
        return out

    @property
    def n_dofs(self):
        return self.info["n_dofs"]

    # ---- operator application (device tensors)
    @staticmethod
    def _stream_ptr(stream):
        import torch

        s = stream if stream is not None else torch.cuda.current_stream()
        return ctypes.c_void_p(s.cuda_stream)

    def _apply(self, fn, x, y, stream):
        import torch

        if not (x.is_cuda and x.is_contiguous() and x.numel() == self.n_dofs):
            raise ValueError("x must be a contiguous CUDA tensor with n_dofs entries")
        prec = {torch.float64: UF_FP64, torch.float32: UF_FP32}.get(x.dtype)
        if prec is None:
            raise ValueError("x must be float64 or float32")
        if y is None:
            y = torch.empty_like(x)
        elif not (y.is_cuda and y.is_contiguous() and y.dtype == x.dtype and y.numel() == self.n_dofs):
            raise ValueError("y must match x")
        _check(fn(self._h, prec, ctypes.c_void_p(y.data_ptr()), ctypes.c_void_p(x.data_ptr()),
                  self._stream_ptr(stream)))
        return y

    def vmult(self, x, y=None, stream=None):
        """y = A x on the device (stream-ordered)."""
        return self._apply(_lib.uf_vmult, x, y, stream)

    def vmult_split(self, x, y=None, stream=None):
        """The split FP32 operator (rows of cut and ghost-penalty cells from the FP64 kernels,
        rounded once); x float32 CUDA tensor."""
        import torch

        if x.dtype != torch.float32:
            raise ValueError("x must be float32")
        return self._apply(lambda h, prec, yp, xp, sp: _lib.uf_vmult_split(h, yp, xp, sp), x, y, stream)

    def set_split_fraction(self, fraction):
        """Cut cells below this volume fraction (and their face neighbours) get FP64 rows in the
        split operator (>= 1: every cut cell)."""
        _check(_lib.uf_set_split_fraction(self._h, float(fraction)))

    def vmult_adjoint(self, g, y=None, stream=None):
        """y = A^T g on the device (stream-ordered)."""
        return self._apply(_lib.uf_vmult_adjoint, g, y, stream)

    def vmult_host(self, x, y=None, stream=None):
        """y = A x with host numpy buffers (copies inside; synchronous)."""
        x = np.ascontiguousarray(x)
        prec = {np.dtype(np.float64): UF_FP64, np.dtype(np.float32): UF_FP32}[x.dtype]
        if y is None:
            y = np.empty_like(x)
        st = ctypes.c_void_p(stream.cuda_stream) if stream is not None else None
        _check(_lib.uf_vmult_host(self._h, prec, _ptr(y), _ptr(x), st))
        return y

    def vmult_host_ptr(self, precision, y_ptr, x_ptr, stream_ptr, adjoint=False, wait=True):
        """uf_vmult_host / uf_vmult_adjoint_host on raw host pointers (pinned torch tensors);
        wait=False: the _async entry points (the result is ready once the stream completes)."""
        if wait:
            fn = _lib.uf_vmult_adjoint_host if adjoint else _lib.uf_vmult_host
        else:
            fn = _lib.uf_vmult_adjoint_host_async if adjoint else _lib.uf_vmult_host_async
        _check(fn(self._h, precision, ctypes.c_void_p(y_ptr), ctypes.c_void_p(x_ptr),
                  ctypes.c_void_p(stream_ptr)))

    def host_wait(self, stream_ptr):
        """uf_host_wait: the queued asynchronous host-buffer products are complete."""
        _check(_lib.uf_host_wait(self._h, ctypes.c_void_p(stream_ptr)))

    def profile_begin(self, capacity):
        """Bracket the next `capacity` operator applications' kernels with CUDA events."""
        _check(_lib.uf_profile_begin(self._h, int(capacity)))

    def profile_end(self):
        """{(precision, kernel, direction): (total ms, evaluations)} of the profiled kernels; the
        number of kernel launches they made is left in self.profiled_kernel_launches."""
        t = uf_kernel_times()
        _check(_lib.uf_profile_end(self._h, ctypes.byref(t)))
        self.profiled_kernel_launches = int(sum(t.kernel_launches))
        out = {}
        for pi, prec in enumerate(("fp64", "fp32")):
            for ki, kern in enumerate(("struct", "cut")):
                for di, dirn in enumerate(("vmult", "adjoint")):
                    k = pi * 4 + ki * 2 + di
                    if t.launches[k]:
                        out[(prec, kern, dirn)] = (t.ms_total[k], t.launches[k])
        return out

    def set_kappa(self, kappa):
        k = np.ascontiguousarray(kappa, dtype=np.float64)
        if k.shape != (self.info["n_active"],):
            raise ValueError("kappa must have one entry per active cell")
        _check(_lib.uf_set_kappa(self._h, k.ctypes.data_as(ctypes.POINTER(ctypes.c_double))))

    # ---- differentiation with respect to the per-cell coefficient
    def kappa_gradient(self, r, x, dk=None, stream=None):
        """dk[e] = r^T (dA/dkappa_e) x (FP64 device tensors)."""
        import torch

        for t in (r, x):
            if not (t.is_cuda and t.is_contiguous() and t.dtype == torch.float64 and t.numel() == self.n_dofs):
                raise ValueError("r and x must be contiguous float64 CUDA tensors with n_dofs entries")
        if dk is None:
            dk = torch.empty(self.info["n_active"], dtype=torch.float64, device=r.device)
        _check(_lib.uf_kappa_gradient(self._h, ctypes.c_void_p(dk.data_ptr()), ctypes.c_void_p(r.data_ptr()),
                                      ctypes.c_void_p(x.data_ptr()), self._stream_ptr(stream)))
        return dk

    def set_kappa_device(self, kappa, stream=None):
        """Replace kappa from a float64 CUDA tensor [n_active] (stream-ordered)."""
        import torch

        if not (kappa.is_cuda and kappa.dtype == torch.float64 and kappa.numel() == self.info["n_active"]):
            raise ValueError("kappa must be a float64 CUDA tensor with n_active entries")
        kappa = kappa.contiguous()
        _check(_lib.uf_set_kappa_device(self._h, ctypes.c_void_p(kappa.data_ptr()), self._stream_ptr(stream)))
        self._kappa_ref = kappa  # keep alive until the copy has run

    # ---- assembled-matrix baseline
    def assemble_csr(self, precision=UF_FP64):
        """Assemble the operator's CSR matrix on the device (synchronous)."""
        _check(_lib.uf_assemble_csr(self._h, precision))

    def csr_info(self, precision=UF_FP64):
        nnz = ctypes.c_int64()
        byts = ctypes.c_double()
        _check(_lib.uf_csr_info(self._h, precision, ctypes.byref(nnz), ctypes.byref(byts)))
        return nnz.value, byts.value

    def csr_spmv(self, x, y=None, stream=None):
        """y = A x with the assembled CSR matrix (device tensors)."""
        return self._apply(_lib.uf_csr_spmv, x, y, stream)

    def export_csr(self, precision=UF_FP64):
        """(row_ptr, col, val) host copies of the assembled matrix."""
        nnz, _ = self.csr_info(precision)
        rp = np.zeros(self.n_dofs + 1, dtype=np.int64)
        col = np.zeros(nnz, dtype=np.int32)
        val = np.zeros(nnz)
        _check(_lib.uf_export_csr(self._h, precision, _ptr(rp), _ptr(col), _ptr(val)))
        return rp, col, val

    def release_csr(self):
        _check(_lib.uf_release_csr(self._h))

    # ---- exports of the setup product
    def export_cells(self):
        na = self.info["n_active"]
        t = np.zeros(na, dtype=np.int32)
        idx = np.zeros(na * 3, dtype=np.int32)
        _check(_lib.uf_export_cells(self._h, _ptr(t), _ptr(idx)))
        return t, idx.reshape(na, 3)

    def export_cut_cell_rule(self, c, kind):
        cnt = ctypes.c_int64()
        _check(_lib.uf_export_cut_cell_rule(self._h, c, kind, None, None, None, ctypes.byref(cnt)))
        d = self.info["dim"]
        xi = np.zeros((cnt.value, d))
        w = np.zeros(cnt.value)
        nrm = np.zeros((cnt.value, d))
        _check(_lib.uf_export_cut_cell_rule(self._h, c, kind, _ptr(xi), _ptr(w), _ptr(nrm),
                                            ctypes.byref(cnt)))
        return (xi, w, nrm) if kind == 1 else (xi, w)

    def export_cut_cell_counts(self):
        """Per cut cell (active order): volume points, volume lines, cut-face lines and the lanes
        of its class in the FP64 cut-cell kernel, as int32 arrays [n_cut]."""
        nc = self.info["n_cut"]
        out = [np.zeros(nc, dtype=np.int32) for _ in range(4)]
        _check(_lib.uf_export_cut_cell_counts(self._h, *[_ptr(a) for a in out]))
        return tuple(out)

    def export_cut_cell_lines(self, c):
        """(axis, group_start, points) of cut cell c's volume lines in kernel order."""
        cnt = ctypes.c_int64()
        _check(_lib.uf_export_cut_cell_lines(self._h, c, None, None, None, ctypes.byref(cnt)))
        out = [np.zeros(cnt.value, dtype=np.int32) for _ in range(3)]
        _check(_lib.uf_export_cut_cell_lines(self._h, c, *[_ptr(a) for a in out], ctypes.byref(cnt)))
        return tuple(out)

    def solve(self, b, x=None, mode="ir", tol=1e-10, inner_tol=1e-4, max_iter=100000,
              max_outer=50, stream=None):
        """Solve A x = b with Jacobi-PCG (FP64, or FP32 inside FP64 refinement); b, x float64
        CUDA tensors.  Returns (x, stats)."""
        import torch

        if x is None:
            x = torch.zeros_like(b)
        modes = {"ir": UF_SOLVE_IR, "fp64": UF_SOLVE_FP64, "ir_split": UF_SOLVE_IR_SPLIT}
        if mode not in modes:
            raise ValueError("mode must be 'fp64', 'ir' or 'ir_split'")
        prm = uf_solve_params(modes[mode], tol, inner_tol,
                              max_iter, max_outer)
        st = uf_solve_stats()
        _check(_lib.uf_solve(self._h, ctypes.byref(prm), ctypes.c_void_p(x.data_ptr()),
                             ctypes.c_void_p(b.contiguous().data_ptr()), ctypes.byref(st),
                             self._stream_ptr(stream)))
        return x, {name: getattr(st, name) for name, _ in uf_solve_stats._fields_}

    def manufactured_rhs(self, omega):
        """Load vector of the sphere accuracy benchmark's right-hand side (host float64)."""
        b = np.zeros(self.n_dofs)
        _check(_lib.uf_manufactured_rhs(self._h, float(omega),
                                        b.ctypes.data_as(ctypes.POINTER(ctypes.c_double))))
        return b

    def l2_error(self, omega, x):
        """(||u_h - u||_L2, ||u||_L2) of the discrete function x (host float64) against the
        benchmark's exact solution."""
        x = np.ascontiguousarray(x, dtype=np.float64)
        if x.shape != (self.n_dofs,):
            raise ValueError("x must have n_dofs entries")
        err = ctypes.c_double()
        nrm = ctypes.c_double()
        _check(_lib.uf_l2_error(self._h, float(omega), x.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                ctypes.byref(err), ctypes.byref(nrm)))
        return err.value, nrm.value

    def export_cg(self):
        """(l2g[n_active, n^d], rhs[n_dofs], diag[n_dofs]) of a continuous operator."""
        na, nd = self.info["n_active"], self.info["dofs_per_cell"]
        l2g = np.zeros(na * nd, dtype=np.int32)
        rhs = np.zeros(self.n_dofs)
        diag = np.zeros(self.n_dofs)
        _check(_lib.uf_export_cg(self._h, _ptr(l2g), _ptr(rhs), _ptr(diag)))
        return l2g.reshape(na, nd), rhs, diag

    def export_cut_face_rule(self, e, axis, side):
        cnt = ctypes.c_int64()
        _check(_lib.uf_export_cut_face_rule(self._h, e, axis, side, None, None, ctypes.byref(cnt)))
        d = self.info["dim"]
        eta = np.zeros((cnt.value, d - 1))
        w = np.zeros(cnt.value)
        _check(_lib.uf_export_cut_face_rule(self._h, e, axis, side, _ptr(eta), _ptr(w),
                                            ctypes.byref(cnt)))
        return eta, w
