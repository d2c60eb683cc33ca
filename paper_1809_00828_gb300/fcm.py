"""Python binding of libfcm.so (the C ABI in include/fcm.h).

Argument marshalling only: every step of the set-up and the solve runs in the
library.  PyTorch provides device memory and the current CUDA stream.  The
binding fails loudly when the library is missing; there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libfcm.so")

FCM_OK, FCM_EINVAL, FCM_ENOMEM, FCM_ECUDA, FCM_ENOTCONV, FCM_EBREAKDOWN, FCM_ETIMEOUT, FCM_ESTATE = range(8)
STATUS_NAMES = ["FCM_OK", "FCM_EINVAL", "FCM_ENOMEM", "FCM_ECUDA", "FCM_ENOTCONV", "FCM_EBREAKDOWN",
                "FCM_ETIMEOUT", "FCM_ESTATE"]
PREC_FP64, PREC_MIXED, PREC_MIXED_FP64 = 0, 1, 2

# Every symbol include/fcm.h declares (checked by the tests).
EXPORTED = ("fcm_setup", "fcm_info", "fcm_rhs", "fcm_precond_build", "fcm_pcg_solve", "fcm_pcg_solve_host",
            "fcm_last_solve", "fcm_apply_K", "fcm_apply_S", "fcm_apply_S_noalloc", "fcm_apply_S_many",
            "fcm_set_wait_limit", "fcm_set_k_precision", "fcm_last_error", "fcm_destroy",
            "fcm_unet_create", "fcm_unet_params", "fcm_unet_get", "fcm_unet_set", "fcm_unet_forward",
            "fcm_unet_backward", "fcm_unet_zero_grad", "fcm_unet_adam", "fcm_unet_destroy", "fcm_coarse_restrict",
            "fcm_coarse_prolong", "fcm_coarse_apply", "fcm_fpcg_solve", "fcm_fpcg_solve_host",
            "fcm_fpcg_set_stall_window", "fcm_coarse_set_preconditioner", "fcm_coarse_set_storage", "fcm_coarse_levels",
            "fcm_coarse_vcycle",
            "fcm_mlhp_create", "fcm_mlhp_get_info", "fcm_mlhp_leaf", "fcm_mlhp_function",
            "fcm_mlhp_block", "fcm_mlhp_colour", "fcm_mlhp_restriction", "fcm_mlhp_assemble", "fcm_mlhp_system_size",
            "fcm_mlhp_system",
            "fcm_mlhp_factorize", "fcm_mlhp_factorize_device", "fcm_mlhp_factor_info", "fcm_mlhp_factors", "fcm_mlhp_device_setup",
            "fcm_mlhp_set_precision", "fcm_mlhp_device_info", "fcm_mlhp_apply_K", "fcm_mlhp_apply_S",
            "fcm_mlhp_pcg_solve", "fcm_mlhp_last_error", "fcm_mlhp_destroy")
NOALLOC_MAX_LATTICE = 1048576  # FCM_NOALLOC_MAX_LATTICE in include/fcm.h


class FcmError(RuntimeError):
    def __init__(self, status, message):
        super().__init__(f"{STATUS_NAMES[status] if 0 <= status < len(STATUS_NAMES) else status}: {message}")
        self.status = status


class Grid(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int * 3), ("lo", ctypes.c_double * 3), ("hi", ctypes.c_double * 3)]


class Geometry(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int), ("nsph", ctypes.c_int), ("sph", ctypes.POINTER(ctypes.c_double)),
                ("vdim", ctypes.c_int * 3), ("vox", ctypes.POINTER(ctypes.c_ubyte)), ("plane", ctypes.c_double * 4),
                ("octree_depth", ctypes.c_int)]


class BC(ctypes.Structure):
    _fields_ = [("E", ctypes.c_double), ("nu", ctypes.c_double), ("bc", ctypes.c_int), ("traction", ctypes.c_double * 3)]


class Info(ctypes.Structure):
    _fields_ = [("n_lattice", ctypes.c_int64), ("n_free", ctypes.c_int64), ("n_cells_active", ctypes.c_int64),
                ("n_cells_cut", ctypes.c_int64), ("n_patches", ctypes.c_int64), ("n_factors", ctypes.c_int64),
                ("factor_bytes", ctypes.c_int64), ("element_bytes", ctypes.c_int64), ("max_block", ctypes.c_int),
                ("p", ctypes.c_int), ("setup_seconds", ctypes.c_double), ("precond_seconds", ctypes.c_double),
                ("n_blocks", ctypes.c_int64), ("n_blocks_fp32", ctypes.c_int64), ("kapply_fmas", ctypes.c_int64),
                ("sapply_fmas", ctypes.c_int64), ("max_block_cond", ctypes.c_double),
                ("coarse_seconds", ctypes.c_double), ("n_jacobi", ctypes.c_int64),
                ("stream_rows", ctypes.c_int), ("schwarz_concurrent", ctypes.c_int),
                ("tune_seconds", ctypes.c_double * 8),
                ("device_error", ctypes.c_int), ("n_factors_ff", ctypes.c_int64), ("n_gemm_blocks", ctypes.c_int64),
                ("k_double_float", ctypes.c_int), ("s_apply_launches", ctypes.c_int),
                ("k_apply_launches", ctypes.c_int)]


class PrecondOpts(ctypes.Structure):
    _fields_ = [("eps", ctypes.c_double), ("precision", ctypes.c_int), ("cond_fp64", ctypes.c_double),
                ("block_rule", ctypes.c_int), ("eta_bar", ctypes.c_double), ("fixed_tiles", ctypes.c_int),
                ("simt_shared", ctypes.c_int)]


BLOCKS_VERTEX, BLOCKS_ELEMENT = 0, 3


class SolveInfo(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_int), ("relres", ctypes.c_double), ("true_relres", ctypes.c_double),
                ("status", ctypes.c_int), ("seconds", ctypes.c_double), ("flexible_iterations", ctypes.c_int),
                ("fallback", ctypes.c_int)]


class MLHPInfo(ctypes.Structure):
    _fields_ = [("levels", ctypes.c_int), ("n_leaves", ctypes.c_int64), ("n_functions", ctypes.c_int64),
                ("n_functions_trunk", ctypes.c_int64), ("n_max_full", ctypes.c_int), ("n_max_truncated", ctypes.c_int),
                ("max_block_full", ctypes.c_int), ("max_block_truncated", ctypes.c_int)]


_lib = None


def load(path: str = LIB_PATH):
    """Load libfcm.so; raise if it has not been built."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is missing: build it with `python -c 'import __graft_entry__ as g; g.build()'`")
    L = ctypes.CDLL(path)
    P = ctypes.c_void_p
    dp = ctypes.POINTER(ctypes.c_double)
    ip = ctypes.POINTER(ctypes.c_int)
    L.fcm_setup.argtypes = [ctypes.POINTER(Grid), ctypes.POINTER(Geometry), ctypes.c_int, ctypes.c_double,
                            ctypes.POINTER(BC), P, ctypes.POINTER(P)]
    L.fcm_info.argtypes = [P, ctypes.POINTER(Info)]
    L.fcm_rhs.argtypes = [P, ctypes.c_int, P]
    L.fcm_precond_build.argtypes = [P, ctypes.POINTER(PrecondOpts)]
    L.fcm_pcg_solve.argtypes = [P, P, ctypes.c_int, ctypes.c_double, ctypes.c_int, P, ip, dp]
    L.fcm_pcg_solve_host.argtypes = [P, P, ctypes.c_int, ctypes.c_double, ctypes.c_int, P, ip, dp]
    L.fcm_last_solve.argtypes = [P, ctypes.POINTER(SolveInfo)]
    L.fcm_apply_K.argtypes = [P, P, P]
    L.fcm_apply_S.argtypes = [P, P, P]
    L.fcm_apply_S_noalloc.argtypes = [P, P, P]
    L.fcm_apply_S_many.argtypes = [P, P, ctypes.c_int, P]
    L.fcm_set_wait_limit.argtypes = [P, ctypes.c_int]
    L.fcm_set_k_precision.argtypes = [P, ctypes.c_int]
    L.fcm_last_error.argtypes = [P]
    L.fcm_last_error.restype = ctypes.c_char_p
    L.fcm_destroy.argtypes = [P]
    i64 = ctypes.c_int64
    L.fcm_mlhp_create.argtypes = [ctypes.POINTER(Grid), ctypes.POINTER(Geometry), ctypes.c_int, ctypes.c_int,
                                  ctypes.POINTER(P)]
    L.fcm_mlhp_get_info.argtypes = [P, ctypes.POINTER(MLHPInfo)]
    L.fcm_mlhp_leaf.argtypes = [P, i64, ip, ip]
    L.fcm_mlhp_function.argtypes = [P, i64, ip, ip, ip]
    L.fcm_mlhp_block.argtypes = [P, i64, ctypes.c_int, ctypes.POINTER(i64), ctypes.c_int, ip]
    L.fcm_mlhp_colour.argtypes = [P, ctypes.c_int, ip, ip]
    L.fcm_mlhp_restriction.argtypes = [P, i64, i64, dp]
    L.fcm_mlhp_assemble.argtypes = [P, ctypes.c_double, ctypes.POINTER(BC)]
    L.fcm_mlhp_system_size.argtypes = [P, ctypes.POINTER(i64), ctypes.POINTER(i64)]
    L.fcm_mlhp_system.argtypes = [P, P, P, P, P, P, P]
    L.fcm_mlhp_factorize.argtypes = [P, ctypes.c_int, ctypes.c_double, ctypes.c_double]
    L.fcm_mlhp_factor_info.argtypes = [P, ip, ip, ctypes.POINTER(i64)]
    L.fcm_mlhp_factors.argtypes = [P, P, P, P, P, P, P]
    L.fcm_mlhp_device_setup.argtypes = [P, P]
    L.fcm_mlhp_factorize_device.argtypes = [P, ctypes.c_int, ctypes.c_double, ctypes.c_double, P]
    L.fcm_mlhp_set_precision.argtypes = [P, ctypes.c_int]
    L.fcm_mlhp_device_info.argtypes = [P, ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int64)]
    L.fcm_mlhp_apply_K.argtypes = [P, P, P]
    L.fcm_mlhp_apply_S.argtypes = [P, P, P]
    L.fcm_mlhp_pcg_solve.argtypes = [P, P, ctypes.c_double, ctypes.c_int, P, ip, dp]
    L.fcm_mlhp_destroy.argtypes = [P]
    L.fcm_mlhp_destroy.restype = None
    L.fcm_mlhp_last_error.argtypes = [P]
    for f in EXPORTED:
        if f not in ("fcm_last_error", "fcm_destroy", "fcm_unet_destroy", "fcm_mlhp_destroy", "fcm_mlhp_last_error"):
            getattr(L, f).restype = ctypes.c_int
    L.fcm_destroy.restype = None
    L.fcm_mlhp_last_error.restype = ctypes.c_char_p
    _lib = L
    return L


def _dev(t, n, dtype="float64", device=None, what="vector", multiple=False):
    """Device pointer of tensor t, after checking what the kernels will index through it.

    The C ABI receives a bare pointer and cannot see a tensor's type or extent, so a wrong
    tensor would be read or written out of bounds on the device.  Checked here: a torch
    tensor of `dtype`, contiguous, with exactly n elements (a positive multiple of n when
    `multiple`), on the CUDA device `device` (any CUDA device when None).  ValueError otherwise.
    """
    import torch
    want = getattr(torch, dtype)
    if not isinstance(t, torch.Tensor):
        raise ValueError(f"{what}: expected a torch tensor, got {type(t).__name__}")
    if t.dtype != want:
        raise ValueError(f"{what}: dtype {t.dtype}, expected {want}")
    if not t.is_contiguous():
        raise ValueError(f"{what}: tensor is not contiguous")
    k = t.numel()
    if (multiple and (k == 0 or k % n != 0)) or (not multiple and k != n):
        raise ValueError(f"{what}: {k} elements, expected {'a positive multiple of ' if multiple else ''}{n}")
    if not t.is_cuda:
        raise ValueError(f"{what}: a CUDA tensor is required, got one on {t.device}")
    if device is not None and t.device.index != device:
        raise ValueError(f"{what}: tensor on cuda:{t.device.index}, the context lives on cuda:{device}")
    return ctypes.c_void_p(t.data_ptr())


def _host_vec(a, n, what, multiple=False, writable=False):
    """The same checks for a host numpy buffer handed to a *_host entry point: float64,
    C-contiguous, n elements (or a positive multiple), writable for outputs."""
    if not isinstance(a, np.ndarray) or a.dtype != np.float64 or not a.flags["C_CONTIGUOUS"]:
        raise ValueError(f"{what}: expected a C-contiguous float64 numpy array")
    if (multiple and (a.size == 0 or a.size % n != 0)) or (not multiple and a.size != n):
        raise ValueError(f"{what}: {a.size} elements, expected {'a positive multiple of ' if multiple else ''}{n}")
    if writable and not a.flags["WRITEABLE"]:
        raise ValueError(f"{what}: array is read-only")
    return a


class Solver:
    """One finite cell problem on the current CUDA device (libfcm context)."""

    def __init__(self, workload, stream=None):
        import torch

        self._torch = torch
        L = load()
        w = workload
        g = Grid()
        g.n[:] = list(w.n)
        g.lo[:] = list(w.lo)
        g.hi[:] = list(w.hi)
        geo = Geometry()
        geo.kind = w.geometry.kind
        self._sph = w.geometry.sphere_array()
        geo.nsph = self._sph.shape[0]
        geo.sph = self._sph.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
        if w.geometry.voxels is not None:
            self._vox = np.ascontiguousarray(w.geometry.voxels, dtype=np.uint8)
            geo.vdim[:] = [self._vox.shape[2], self._vox.shape[1], self._vox.shape[0]]
            geo.vox = self._vox.ctypes.data_as(ctypes.POINTER(ctypes.c_ubyte))
        geo.plane[:] = list(w.geometry.plane)
        geo.octree_depth = w.geometry.octree_depth
        bc = BC()
        bc.E, bc.nu, bc.bc = w.E, w.nu, w.bc
        bc.traction[:] = list(w.traction)
        if stream is None:
            stream = torch.cuda.current_stream().cuda_stream
        self.ctx = ctypes.c_void_p()
        st = L.fcm_setup(ctypes.byref(g), ctypes.byref(geo), w.p, w.alpha, ctypes.byref(bc), ctypes.c_void_p(stream),
                         ctypes.byref(self.ctx))
        if st != FCM_OK:
            raise FcmError(st, L.fcm_last_error(None).decode())
        self.workload = w
        self.device = torch.cuda.current_device()
        self.info = self.get_info()
        self.n = self.info["n_lattice"]

    def _vec(self, t, what, nrhs=1, multiple=False):
        return _dev(t, self.n * nrhs, device=self.device, what=what, multiple=multiple)

    def _check(self, st):
        if st != FCM_OK:
            raise FcmError(st, load().fcm_last_error(self.ctx).decode())

    def get_info(self):
        inf = Info()
        self._check(load().fcm_info(self.ctx, ctypes.byref(inf)))
        return {k: (list(getattr(inf, k)) if k == "tune_seconds" else getattr(inf, k)) for k, _ in Info._fields_}

    def empty(self, nrhs=1):
        return self._torch.zeros(nrhs * self.n, dtype=self._torch.float64, device="cuda")

    def rhs(self, load_case=0):
        b = self.empty()
        self._check(load().fcm_rhs(self.ctx, load_case, self._vec(b, "b")))
        return b

    def precond_build(self, eps=1e-13, precision="fp64", cond_fp64=1e7, blocks="vertex", eta_bar=1.0,
                      autotune=True, launch=None, tensor_cores=True):
        """precision: "fp64", "mixed" (FP32 factors, double-float pairs above cond_fp64) or
        "mixed_fp64" (FP32 factors, FP64 above cond_fp64).  blocks: "vertex" (vertex patches)
        or "element" (element blocks of the cells with eta_T <= eta_bar, diagonal scaling for
        the DOFs in no block).  autotune: time the Schwarz apply for a few launch shapes and
        keep the fastest (results do not depend on the choice).  launch ("serial" or
        "concurrent": the shared-factor products after or beside the streamed factors) fixes
        the default shape instead.  tensor_cores: FP32 shared factors on tcgen05 (TF32 three-pass)
        or, when False, on the CUDA cores."""
        if blocks not in ("vertex", "element"):
            raise ValueError(f"unknown block rule {blocks!r}")
        o = PrecondOpts()
        o.eps = eps
        o.precision = {"fp64": PREC_FP64, "mixed": PREC_MIXED, "mixed_fp64": PREC_MIXED_FP64}[precision]
        o.cond_fp64 = cond_fp64
        o.block_rule = BLOCKS_ELEMENT if blocks == "element" else BLOCKS_VERTEX
        o.eta_bar = eta_bar
        o.fixed_tiles = {None: 0 if autotune else 1, "serial": 1, "concurrent": 2}[launch]
        o.simt_shared = 0 if tensor_cores else 1
        self._check(load().fcm_precond_build(self.ctx, ctypes.byref(o)))
        self.info = self.get_info()

    def pcg_solve(self, b, tol, maxit=100000, out=None, check=True):
        pb = self._vec(b, "b", multiple=True)
        nrhs = b.numel() // self.n
        u = out if out is not None else self.empty(nrhs)
        pu = self._vec(u, "out", nrhs)
        its = ctypes.c_int(0)
        rel = ctypes.c_double(0.0)
        st = load().fcm_pcg_solve(self.ctx, pb, nrhs, tol, maxit, pu, ctypes.byref(its), ctypes.byref(rel))
        if check:
            self._check(st)
        return u, its.value, rel.value, st

    def pcg_solve_host(self, b_host: np.ndarray, tol, maxit=100000, out: np.ndarray | None = None):
        b_host = _host_vec(b_host, self.n, "b_host", multiple=True)
        nrhs = b_host.size // self.n
        u = out if out is not None else np.empty_like(b_host)
        u = _host_vec(u, self.n * nrhs, "out", writable=True)
        its = ctypes.c_int(0)
        rel = ctypes.c_double(0.0)
        st = load().fcm_pcg_solve_host(self.ctx, ctypes.c_void_p(b_host.ctypes.data), nrhs, tol, maxit,
                                       ctypes.c_void_p(u.ctypes.data), ctypes.byref(its), ctypes.byref(rel))
        self._check(st)
        return u, its.value, rel.value

    def last_solve(self):
        s = SolveInfo()
        self._check(load().fcm_last_solve(self.ctx, ctypes.byref(s)))
        return {k: getattr(s, k) for k, _ in SolveInfo._fields_}

    def apply_K(self, x, out=None):
        y = out if out is not None else self.empty()
        self._check(load().fcm_apply_K(self.ctx, self._vec(x, "x"), self._vec(y, "out")))
        return y

    def apply_S(self, r, out=None):
        """z = S r; r may hold 1..8 vectors (n_lattice apart), applied in one call."""
        pr = self._vec(r, "r", multiple=True)
        nr = r.numel() // self.n
        z = out if out is not None else self.empty(nr)
        pz = self._vec(z, "out", nr)
        if nr == 1:
            self._check(load().fcm_apply_S(self.ctx, pr, pz))
        else:
            self._check(load().fcm_apply_S_many(self.ctx, pr, nr, pz))
        return z

    def set_k_precision(self, mode):
        """K x in "fp64" or "double_float" arithmetic (every K apply of the context, solves included)."""
        self._check(load().fcm_set_k_precision(self.ctx, {"fp64": 0, "double_float": 1}[mode]))
        self.info = self.get_info()

    def set_wait_limit(self, tries):
        """Polls of the Schwarz kernels' bounded bulk-copy wait (0: give up at once; < 0: default)."""
        self._check(load().fcm_set_wait_limit(self.ctx, int(tries)))

    def close(self):
        if getattr(self, "ctx", None) and self.ctx.value:
            load().fcm_destroy(self.ctx)
            self.ctx = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ----------------------------------------------------------------------------------------------
# Learned coarse correction (U-Net on the cell grid) and the flexible PCG that uses it.
# ----------------------------------------------------------------------------------------------
class UNetDesc(ctypes.Structure):
    _fields_ = [("in_ch", ctypes.c_int), ("out_ch", ctypes.c_int), ("base", ctypes.c_int), ("levels", ctypes.c_int),
                ("seed", ctypes.c_uint64)]


_unet_bound = False


def _bind_unet(L):
    global _unet_bound
    if _unet_bound:
        return
    P = ctypes.c_void_p
    dp = ctypes.POINTER(ctypes.c_double)
    ip = ctypes.POINTER(ctypes.c_int)
    L.fcm_unet_create.argtypes = [ctypes.POINTER(UNetDesc), P, ctypes.POINTER(P)]
    L.fcm_unet_params.argtypes = [P, ctypes.POINTER(ctypes.c_int64)]
    L.fcm_unet_get.argtypes = [P, P, P]
    L.fcm_unet_set.argtypes = [P, P]
    L.fcm_unet_forward.argtypes = [P, P, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, P]
    L.fcm_unet_backward.argtypes = [P, P, P]
    L.fcm_unet_zero_grad.argtypes = [P]
    L.fcm_unet_adam.argtypes = [P, ctypes.c_float, ctypes.c_float, ctypes.c_float, ctypes.c_float, ctypes.c_int]
    L.fcm_unet_destroy.argtypes = [P]
    L.fcm_unet_destroy.restype = None
    L.fcm_coarse_restrict.argtypes = [P, P, ctypes.c_float, ctypes.c_int, P]
    L.fcm_coarse_prolong.argtypes = [P, P, ctypes.c_double, P]
    L.fcm_coarse_apply.argtypes = [P, P, P]
    L.fcm_fpcg_solve.argtypes = [P, P, ctypes.c_double, ctypes.c_int, P, ctypes.c_double, ctypes.c_int, P, ip, dp]
    L.fcm_fpcg_solve_host.argtypes = [P, P, ctypes.c_double, ctypes.c_int, P, ctypes.c_double, ctypes.c_int, P, ip,
                                      dp]
    L.fcm_fpcg_set_stall_window.argtypes = [P, ctypes.c_int]
    L.fcm_coarse_set_preconditioner.argtypes = [P, ctypes.c_int]
    L.fcm_coarse_set_storage.argtypes = [P, ctypes.c_int]
    L.fcm_coarse_levels.argtypes = [P, ip, ip, dp, dp]
    L.fcm_coarse_vcycle.argtypes = [P, ctypes.c_int, P, P]
    for f in ("fcm_unet_create", "fcm_unet_params", "fcm_unet_get", "fcm_unet_set", "fcm_unet_forward",
              "fcm_unet_backward", "fcm_unet_zero_grad", "fcm_unet_adam", "fcm_coarse_restrict", "fcm_coarse_prolong",
              "fcm_coarse_apply", "fcm_fpcg_solve", "fcm_fpcg_solve_host", "fcm_fpcg_set_stall_window",
              "fcm_coarse_set_preconditioner", "fcm_coarse_set_storage", "fcm_coarse_levels", "fcm_coarse_vcycle"):
        getattr(L, f).restype = ctypes.c_int
    _unet_bound = True


def _unet_check(st):
    if st != FCM_OK:
        raise FcmError(st, load().fcm_last_error(None).decode())


class UNet:
    """The U-Net of the learned coarse correction (device weights, our own kernels)."""

    def __init__(self, in_ch=4, out_ch=3, base=16, levels=4, seed=0, stream=None):
        import torch

        self._torch = torch
        L = load()
        _bind_unet(L)
        d = UNetDesc(in_ch, out_ch, base, levels, seed)
        if stream is None:
            stream = torch.cuda.current_stream().cuda_stream
        self.h = ctypes.c_void_p()
        _unet_check(L.fcm_unet_create(ctypes.byref(d), ctypes.c_void_p(stream), ctypes.byref(self.h)))
        self.desc = (in_ch, out_ch, base, levels)
        n = ctypes.c_int64(0)
        _unet_check(L.fcm_unet_params(self.h, ctypes.byref(n)))
        self.nparam = n.value

    def get(self, with_grad=False):
        w = np.zeros(self.nparam, dtype=np.float32)
        g = np.zeros(self.nparam, dtype=np.float32) if with_grad else None
        _unet_check(load().fcm_unet_get(self.h, ctypes.c_void_p(w.ctypes.data),
                                        ctypes.c_void_p(g.ctypes.data) if with_grad else None))
        return (w, g) if with_grad else w

    def set(self, w):
        w = np.ascontiguousarray(w, dtype=np.float32)
        assert w.size == self.nparam
        _unet_check(load().fcm_unet_set(self.h, ctypes.c_void_p(w.ctypes.data)))

    def forward(self, x, out=None):
        if x.dim() != 5 or x.shape[1] != self.desc[0]:
            raise ValueError(f"input: expected [batch][{self.desc[0]}][z][y][x], got shape {tuple(x.shape)}")
        B, C, Z, Y, X = x.shape
        if out is None:
            out = self._torch.empty((B, self.desc[1], Z, Y, X), dtype=self._torch.float32, device=x.device)
        px = _dev(x, x.numel(), "float32", what="input")
        po = _dev(out, B * self.desc[1] * Z * Y * X, "float32", device=x.device.index, what="out")
        self._shape = (B, Z, Y, X)
        _unet_check(load().fcm_unet_forward(self.h, px, B, X, Y, Z, po))
        return out

    def backward(self, gout, want_din=False):
        B, Z, Y, X = getattr(self, "_shape", (0, 0, 0, 0))
        pg = _dev(gout, B * self.desc[1] * Z * Y * X, "float32", what="gradient of the output (after forward)")
        din = None
        if want_din:
            din = self._torch.empty((B, self.desc[0], Z, Y, X), dtype=self._torch.float32, device=gout.device)
        _unet_check(load().fcm_unet_backward(self.h, pg, _dev(din, din.numel(), "float32") if want_din else None))
        return din

    def zero_grad(self):
        _unet_check(load().fcm_unet_zero_grad(self.h))

    def adam(self, lr, step, beta1=0.9, beta2=0.999, eps=1e-8):
        _unet_check(load().fcm_unet_adam(self.h, lr, beta1, beta2, eps, step))

    def close(self):
        if getattr(self, "h", None) and self.h.value:
            load().fcm_unet_destroy(self.h)
            self.h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _solver_coarse_restrict(self, v, s=1.0, eta_channel=True, out=None):
    _bind_unet(load())
    nc = self.workload.n[0] * self.workload.n[1] * self.workload.n[2]
    if out is None:
        out = self._torch.empty((4 if eta_channel else 3) * nc, dtype=self._torch.float32, device="cuda")
    po = _dev(out, (4 if eta_channel else 3) * nc, "float32", device=self.device, what="out")
    self._check(load().fcm_coarse_restrict(self.ctx, self._vec(v, "v"), s, 1 if eta_channel else 0, po))
    return out


def _solver_coarse_prolong(self, cells, s=1.0, out=None):
    _bind_unet(load())
    y = out if out is not None else self.empty()
    nc = self.workload.n[0] * self.workload.n[1] * self.workload.n[2]
    pc = _dev(cells, 3 * nc, "float32", device=self.device, what="cells", multiple=True)
    if cells.numel() not in (3 * nc, 4 * nc):
        raise ValueError(f"cells: {cells.numel()} elements, expected {3 * nc} (or {4 * nc} with the eta channel)")
    self._check(load().fcm_coarse_prolong(self.ctx, pc, s, self._vec(y, "out")))
    return y


def _solver_coarse_apply(self, x, out=None):
    """y = K_H x on cell vectors (3 * n_cells floats, component-major)."""
    _bind_unet(load())
    y = out if out is not None else self._torch.empty_like(x)
    nc = self.workload.n[0] * self.workload.n[1] * self.workload.n[2]
    px = _dev(x, 3 * nc, "float32", device=self.device, what="x")
    self._check(load().fcm_coarse_apply(self.ctx, px, _dev(y, 3 * nc, "float32", device=self.device, what="out")))
    return y


def _solver_fpcg_solve(self, net, gamma, b, tol, maxit=100000, out=None, check=True, coarse_iters=0):
    """Flexible PCG with the coarse correction; net may be None when coarse_iters >= 1."""
    _bind_unet(load())
    u = out if out is not None else self.empty()
    its = ctypes.c_int(0)
    rel = ctypes.c_double(0.0)
    st = load().fcm_fpcg_solve(self.ctx, net.h if net is not None else None, gamma, coarse_iters,
                               self._vec(b, "b"), tol, maxit, self._vec(u, "out"), ctypes.byref(its),
                               ctypes.byref(rel))
    if check:
        self._check(st)
    return u, its.value, rel.value, st


def _solver_fpcg_solve_host(self, net, gamma, b_host, tol, maxit=100000, out=None, check=True, coarse_iters=0):
    """fpcg_solve with host numpy buffers (float64, n_lattice); copies are inside the call."""
    _bind_unet(load())
    b_host = _host_vec(np.ascontiguousarray(b_host, dtype=np.float64), self.n, "b_host")
    u = _host_vec(out if out is not None else np.empty_like(b_host), self.n, "out", writable=True)
    its = ctypes.c_int(0)
    rel = ctypes.c_double(0.0)
    st = load().fcm_fpcg_solve_host(self.ctx, net.h if net is not None else None, gamma, coarse_iters,
                                    ctypes.c_void_p(b_host.ctypes.data), tol, maxit, ctypes.c_void_p(u.ctypes.data),
                                    ctypes.byref(its), ctypes.byref(rel))
    if check:
        self._check(st)
    return u, its.value, rel.value, st


def _solver_set_stall_window(self, window):
    """Iterations without halving of the stopping residual after which fpcg_solve falls back."""
    _bind_unet(load())
    self._check(load().fcm_fpcg_set_stall_window(self.ctx, int(window)))


COARSE_PREC = {"jacobi": 0, "vcycle": 1, "hybrid": 2}  # FCM_COARSE_JACOBI, FCM_COARSE_VCYCLE, FCM_COARSE_HYBRID


def _solver_set_coarse_preconditioner(self, kind):
    """Preconditioner of the coarse CG in fpcg_solve: "jacobi" (3x3 diagonal blocks of K_H), "vcycle" (one
    V-cycle of the cell-grid multigrid hierarchy, built on the next coarse solve) or "hybrid" (the same,
    additive on the finest cell grid)."""
    _bind_unet(load())
    if kind not in COARSE_PREC:
        raise ValueError(f"coarse preconditioner {kind!r}: expected one of {sorted(COARSE_PREC)}")
    self._check(load().fcm_coarse_set_preconditioner(self.ctx, COARSE_PREC[kind]))


def _solver_set_coarse_storage(self, storage):
    """Storage of K_H: "fp32" (default), "fp16" (symmetrically scaled FP16, half the bytes per product) or
    "fp16_cycles" (FP16 only in the V-cycle's products on the finest cell grid)."""
    _bind_unet(load())
    kinds = {"fp32": 0, "fp16": 1, "fp16_cycles": 2}  # FCM_COARSE_STORE_FP32, _FP16, _FP16_CYCLES
    if storage not in kinds:
        raise ValueError(f"coarse storage {storage!r}: expected one of {sorted(kinds)}")
    self._check(load().fcm_coarse_set_storage(self.ctx, kinds[storage]))


def _solver_coarse_levels(self):
    """The multigrid hierarchy: {"levels": n, "dims": [(nx, ny, nz), ...], "lambda_max": [...], "seconds": s}."""
    _bind_unet(load())
    n = ctypes.c_int(0)
    dims = (ctypes.c_int * 36)()
    lam = (ctypes.c_double * 12)()
    sec = ctypes.c_double(0.0)
    self._check(load().fcm_coarse_levels(self.ctx, ctypes.byref(n), dims, lam, ctypes.byref(sec)))
    return {"levels": n.value, "dims": [tuple(dims[3 * i:3 * i + 3]) for i in range(n.value)],
            "lambda_max": [lam[i] for i in range(max(0, n.value - 1))], "seconds": sec.value}


def _solver_coarse_vcycle(self, f, out=None, kind="vcycle"):
    """x = one cycle ("vcycle" or "hybrid") of the cell-grid multigrid hierarchy applied to f (3 * n_cells
    floats, component-major)."""
    _bind_unet(load())
    nc = self.workload.n[0] * self.workload.n[1] * self.workload.n[2]
    x = out if out is not None else self._torch.empty_like(f)
    pf = _dev(f, 3 * nc, "float32", device=self.device, what="f")
    px = _dev(x, 3 * nc, "float32", device=self.device, what="out")
    if pf == px:
        raise ValueError("coarse_vcycle: f and out must be distinct buffers")
    if kind not in ("vcycle", "hybrid"):
        raise ValueError(f"coarse_vcycle: kind {kind!r}, expected 'vcycle' or 'hybrid'")
    self._check(load().fcm_coarse_vcycle(self.ctx, COARSE_PREC[kind], pf, px))
    return x


Solver.coarse_vcycle = _solver_coarse_vcycle
Solver.set_coarse_storage = _solver_set_coarse_storage
Solver.set_coarse_preconditioner = _solver_set_coarse_preconditioner
Solver.coarse_levels = _solver_coarse_levels
Solver.set_stall_window = _solver_set_stall_window
Solver.coarse_restrict = _solver_coarse_restrict
Solver.coarse_prolong = _solver_coarse_prolong
Solver.coarse_apply = _solver_coarse_apply
Solver.fpcg_solve = _solver_fpcg_solve
Solver.fpcg_solve_host = _solver_fpcg_solve_host


# ----------------------------------------------------------------------------------------------
# Multi-level hp overlays: the host-side plan of the hierarchy, its basis and its leaf blocks.
# ----------------------------------------------------------------------------------------------
class MLHPPlan:
    """fcm_mlhp plan: base grid n on [lo, hi] refined k times toward the surfaces of `spheres`
    (rows cx, cy, cz, r), basis order p; the spheres are also the voids of `assemble`, integrated with
    an octree of `octree_depth` levels per leaf.  Host memory only; no device is needed."""

    def __init__(self, n, lo, hi, spheres, p, k, octree_depth=3, geometry=None):
        """geometry (an inputs.Geometry: spheres, voxels or a half space) replaces `spheres` when given."""
        L = load()
        g = Grid()
        g.n[:] = list(n)
        g.lo[:] = list(lo)
        g.hi[:] = list(hi)
        geo = Geometry()
        geo.kind = 0 if geometry is None else geometry.kind
        geo.octree_depth = octree_depth
        sph = spheres if geometry is None else geometry.sphere_array()
        self._sph = np.ascontiguousarray(np.asarray(sph, dtype=np.float64).reshape(-1, 4))
        geo.nsph = self._sph.shape[0]
        geo.sph = self._sph.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
        if geometry is not None and geometry.voxels is not None:
            self._vox = np.ascontiguousarray(geometry.voxels, dtype=np.uint8)
            geo.vdim[:] = [self._vox.shape[2], self._vox.shape[1], self._vox.shape[0]]
            geo.vox = self._vox.ctypes.data_as(ctypes.POINTER(ctypes.c_ubyte))
        if geometry is not None:
            geo.plane[:] = list(geometry.plane)
        self.p = p
        self.h = ctypes.c_void_p()
        st = L.fcm_mlhp_create(ctypes.byref(g), ctypes.byref(geo), p, k, ctypes.byref(self.h))
        if st != FCM_OK:
            raise FcmError(st, "fcm_mlhp_create")
        inf = MLHPInfo()
        self._check(L.fcm_mlhp_get_info(self.h, ctypes.byref(inf)))
        self.info = {k2: getattr(inf, k2) for k2, _ in MLHPInfo._fields_}

    def _check(self, st):
        if st != FCM_OK:
            msg = load().fcm_mlhp_last_error(self.h) if getattr(self, "h", None) else b""
            raise FcmError(st, "fcm_mlhp: " + (msg.decode() if msg else "failed"))

    def leaf(self, i):
        lv = ctypes.c_int()
        c = (ctypes.c_int * 3)()
        self._check(load().fcm_mlhp_leaf(self.h, i, ctypes.byref(lv), c))
        return lv.value, tuple(c)

    def function(self, f):
        lv = ctypes.c_int()
        q = (ctypes.c_int * 3)()
        m = (ctypes.c_int * 3)()
        self._check(load().fcm_mlhp_function(self.h, f, ctypes.byref(lv), q, m))
        return lv.value, tuple(q), tuple(m)

    def block(self, leaf, kind):
        """kind "full" or "truncated": the scalar functions of the leaf's block."""
        cnt = ctypes.c_int()
        k = {"full": 0, "truncated": 1}[kind]
        load().fcm_mlhp_block(self.h, leaf, k, None, 0, ctypes.byref(cnt))
        out = np.zeros(max(cnt.value, 1), dtype=np.int64)
        self._check(load().fcm_mlhp_block(self.h, leaf, k, out.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)),
                                          cnt.value, ctypes.byref(cnt)))
        return out[:cnt.value]

    def colour(self, kind):
        """Colour of every leaf's block (kind "full" or "truncated"); blocks of one colour share no function."""
        c = np.zeros(self.info["n_leaves"], dtype=np.int32)
        nc = ctypes.c_int()
        self._check(load().fcm_mlhp_colour(self.h, {"full": 0, "truncated": 1}[kind],
                                           c.ctypes.data_as(ctypes.POINTER(ctypes.c_int)), ctypes.byref(nc)))
        return c, nc.value

    def restriction(self, leaf, f):
        """(3, p+1) coefficients of function f on the leaf in the leaf's basis (N0, N1, phi_2..phi_p)."""
        c = np.zeros(3 * (self.p + 1))
        self._check(load().fcm_mlhp_restriction(self.h, leaf, f, c.ctypes.data_as(ctypes.POINTER(ctypes.c_double))))
        return c.reshape(3, self.p + 1)

    def assemble(self, alpha, bc_kind="clamp", E=1.0, nu=0.3, traction=(0.0, 0.0, -1.0)):
        """Assemble the system on the host; returns (free_dofs, K as scipy CSR, rhs, leaf_eta)."""
        import scipy.sparse as sp
        bc = BC()
        bc.E, bc.nu = E, nu
        bc.bc = {"none": -1, "clamp": 0, "roller": 1}[bc_kind]
        bc.traction[:] = list(traction)
        L = load()
        self._check(L.fcm_mlhp_assemble(self.h, alpha, ctypes.byref(bc)))
        nf, nnz = ctypes.c_int64(), ctypes.c_int64()
        self._check(L.fcm_mlhp_system_size(self.h, ctypes.byref(nf), ctypes.byref(nnz)))
        free = np.zeros(nf.value, dtype=np.int64)
        rowptr = np.zeros(nf.value + 1, dtype=np.int64)
        cols = np.zeros(nnz.value, dtype=np.int64)
        vals = np.zeros(nnz.value)
        rhs = np.zeros(nf.value)
        eta = np.zeros(self.info["n_leaves"])
        ptr = lambda a: ctypes.c_void_p(a.ctypes.data)  # noqa: E731
        self._check(L.fcm_mlhp_system(self.h, ptr(free), ptr(rowptr), ptr(cols), ptr(vals), ptr(rhs), ptr(eta)))
        K = sp.csr_matrix((vals, cols, rowptr), shape=(nf.value, nf.value))
        return free, K, rhs, eta

    def factorize(self, kind="truncated", eps=1e-13, eta_bar=1.0, device=False):
        """Schwarz factors for the leaves with eta_T <= eta_bar; returns (blocks, factors, colour_ptr,
        jacobi): block b's free DOFs and its pseudo inverse, blocks of colour c at colour_ptr[c] ..
        colour_ptr[c+1], and 1 / K_ll on the DOFs in no block.  device: the eigensolves batched on the
        current CUDA device (torch's current stream) instead of the host."""
        L = load()
        if kind not in ("full", "truncated"):
            raise ValueError(f"kind {kind!r}: expected 'full' or 'truncated'")
        k = {"full": 0, "truncated": 1}[kind]
        if device:
            import torch
            st = torch.cuda.current_stream().cuda_stream
            self._check(L.fcm_mlhp_factorize_device(self.h, k, eps, eta_bar, ctypes.c_void_p(st)))
        else:
            self._check(L.fcm_mlhp_factorize(self.h, k, eps, eta_bar))
        nb, nc, ne = ctypes.c_int(), ctypes.c_int(), ctypes.c_int64()
        self._check(L.fcm_mlhp_factor_info(self.h, ctypes.byref(nb), ctypes.byref(nc), ctypes.byref(ne)))
        nfree = ctypes.c_int64()
        nnz = ctypes.c_int64()
        self._check(L.fcm_mlhp_system_size(self.h, ctypes.byref(nfree), ctypes.byref(nnz)))
        bptr = np.zeros(nb.value + 1, dtype=np.int64)
        fptr = np.zeros(nb.value + 1, dtype=np.int64)
        cptr = np.zeros(nc.value + 1, dtype=np.int64)
        fac = np.zeros(ne.value)
        jac = np.zeros(nfree.value)
        ptr = lambda a: ctypes.c_void_p(a.ctypes.data)  # noqa: E731
        self._check(L.fcm_mlhp_factors(self.h, ptr(bptr), None, None, None, None, None))
        dofs = np.zeros(bptr[-1], dtype=np.int64)
        self._check(L.fcm_mlhp_factors(self.h, ptr(bptr), ptr(dofs), ptr(fptr), ptr(fac), ptr(cptr), ptr(jac)))
        blocks = [dofs[bptr[b]:bptr[b + 1]] for b in range(nb.value)]
        factors = [fac[fptr[b]:fptr[b + 1]].reshape(len(blocks[b]), len(blocks[b])) for b in range(nb.value)]
        return blocks, factors, cptr, jac

    def device_setup(self, stream=None, precision="fp64"):
        """Upload the assembled system and factors to the current CUDA device (torch's current stream).
        precision "mixed": FP32 factors for the blocks with retained condition number <= 1e7."""
        import torch
        if precision not in ("fp64", "mixed"):
            raise ValueError(f"precision {precision!r}: expected 'fp64' or 'mixed'")
        if stream is None:
            stream = torch.cuda.current_stream().cuda_stream
        self._stream = stream
        self._check(load().fcm_mlhp_set_precision(self.h, PREC_FP64 if precision == "fp64" else PREC_MIXED))
        self._check(load().fcm_mlhp_device_setup(self.h, ctypes.c_void_p(stream)))
        nf, nnz = ctypes.c_int64(), ctypes.c_int64()
        self._check(load().fcm_mlhp_system_size(self.h, ctypes.byref(nf), ctypes.byref(nnz)))
        self._nfree = nf.value
        self._device = torch.cuda.current_device()

    def device_info(self):
        """(blocks stored in FP32, device factor bytes) after device_setup."""
        n32, nb = ctypes.c_int64(), ctypes.c_int64()
        self._check(load().fcm_mlhp_device_info(self.h, ctypes.byref(n32), ctypes.byref(nb)))
        return n32.value, nb.value

    def _vec(self, t, what):
        if getattr(self, "_nfree", None) is None:
            raise RuntimeError("call device_setup first")
        return _dev(t, self._nfree, device=self._device, what=what)

    def apply_K(self, x, out=None):
        import torch
        y = out if out is not None else torch.empty_like(x)
        self._check(load().fcm_mlhp_apply_K(self.h, self._vec(x, "x"), self._vec(y, "out")))
        return y

    def apply_S(self, r, out=None):
        import torch
        z = out if out is not None else torch.empty_like(r)
        self._check(load().fcm_mlhp_apply_S(self.h, self._vec(r, "r"), self._vec(z, "out")))
        return z

    def pcg_solve(self, b, tol, maxit=100000, out=None, check=True):
        import torch
        u = out if out is not None else torch.empty_like(b)
        its = ctypes.c_int(0)
        rel = ctypes.c_double(0.0)
        st = load().fcm_mlhp_pcg_solve(self.h, self._vec(b, "b"), tol, maxit, self._vec(u, "out"),
                                       ctypes.byref(its), ctypes.byref(rel))
        if check:
            self._check(st)
        return u, its.value, rel.value, st

    def close(self):
        if getattr(self, "h", None) and self.h.value:
            load().fcm_mlhp_destroy(self.h)
            self.h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
