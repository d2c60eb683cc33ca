"""ctypes binding of the plain FP64 CPU oracle (oracle/fcm_oracle.c).

TEST INFRASTRUCTURE ONLY: imported by the tests, by `__graft_entry__.smoke()`
and by the bench's CPU-baseline leg.  The product path never loads it.

Every function here only marshals arguments; the arithmetic lives in the C
file, which cites the paper's sections for each step.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import sys

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "fcm_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (plain C, -O2, no fast-math)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=c11", "-D_DEFAULT_SOURCE", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"]
        subprocess.check_call(cmd)
        os.replace(tmp, _LIB)
    return _LIB


class Desc(ctypes.Structure):
    _fields_ = [
        ("n", ctypes.c_int * 3),
        ("lo", ctypes.c_double * 3),
        ("hi", ctypes.c_double * 3),
        ("p", ctypes.c_int),
        ("depth", ctypes.c_int),
        ("alpha", ctypes.c_double),
        ("E", ctypes.c_double),
        ("nu", ctypes.c_double),
        ("bc", ctypes.c_int),
        ("traction", ctypes.c_double * 3),
        ("gkind", ctypes.c_int),
        ("nsph", ctypes.c_int),
        ("sph", ctypes.POINTER(ctypes.c_double)),
        ("vdim", ctypes.c_int * 3),
        ("vox", ctypes.POINTER(ctypes.c_ubyte)),
        ("plane", ctypes.c_double * 4),
    ]


_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(build())
        L = _lib
        P = ctypes.c_void_p
        dp = ctypes.POINTER(ctypes.c_double)
        ip = ctypes.POINTER(ctypes.c_int)
        lp = ctypes.POINTER(ctypes.c_int64)
        D = ctypes.POINTER(Desc)
        L.ora_gauss.argtypes = [ctypes.c_int, dp, dp]
        L.ora_shape1d.argtypes = [ctypes.c_int, ctypes.c_double, dp, dp]
        L.ora_solid_at.argtypes = [D, dp]
        L.ora_box_cut.argtypes = [D, dp, dp]
        L.ora_cell_matrix.argtypes = [D, ip, dp, dp]
        L.ora_cell_traction.argtypes = [D, ip, dp]
        L.ora_problem_build.argtypes = [D]
        L.ora_problem_build.restype = P
        L.ora_problem_free.argtypes = [P]
        for f in ("ora_nfree", "ora_nnz", "ora_nlat"):
            getattr(L, f).argtypes = [P]
            getattr(L, f).restype = ctypes.c_int64
        L.ora_ncells.argtypes = [P]
        L.ora_get_free_lat.argtypes = [P, lp]
        L.ora_get_rhs.argtypes = [P, dp]
        L.ora_get_load.argtypes = [P, ctypes.c_int, dp]
        L.ora_get_eta.argtypes = [P, dp]
        L.ora_get_csr.argtypes = [P, lp, lp, dp]
        L.ora_apply_K.argtypes = [P, dp, dp]
        L.ora_jacobi_eig.argtypes = [ctypes.c_int, dp, dp, dp]
        L.ora_pseudo_inverse.argtypes = [ctypes.c_int, dp, ctypes.c_double, dp, dp, ip, ip]
        L.ora_precond_build.argtypes = [P, ctypes.c_int, ctypes.c_double, ctypes.c_double]
        L.ora_nblocks.argtypes = [P]
        L.ora_block_size.argtypes = [P, ctypes.c_int]
        L.ora_block_get.argtypes = [P, ctypes.c_int, ip, dp, dp]
        L.ora_apply_S.argtypes = [P, dp, dp]
        L.ora_pcg.argtypes = [P, dp, ctypes.c_double, ctypes.c_int, dp, dp]
        L.ora_energy_error.argtypes = [P, dp, dp]
        L.ora_energy_error.restype = ctypes.c_double
        L.ora_patch_factor.argtypes = [D, ip, ctypes.c_double, lp, dp, dp]
        L.ora_sample_Kx.argtypes = [D, ctypes.c_int, lp, dp, dp]
    return _lib


def _dp(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _ip(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int))


def _lp(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int64))


def make_desc(n, p, alpha, geometry, E=1.0, nu=0.3, bc=0, traction=(0.0, 0.0, -1.0),
              lo=(0.0, 0.0, 0.0), hi=(1.0, 1.0, 1.0), depth=None):
    """Build the C descriptor.  Returns (desc, keepalive) -- keep both alive."""
    d = Desc()
    d.n[:] = list(n)
    d.lo[:] = list(lo)
    d.hi[:] = list(hi)
    d.p = p
    d.depth = geometry.octree_depth if depth is None else depth
    d.alpha, d.E, d.nu = alpha, E, nu
    d.bc = bc
    d.traction[:] = list(traction)
    d.gkind = geometry.kind
    keep = []
    sph = geometry.sphere_array()
    keep.append(sph)
    d.nsph = sph.shape[0]
    d.sph = _dp(sph)
    if geometry.voxels is not None:
        vox = np.ascontiguousarray(geometry.voxels, dtype=np.uint8)
        keep.append(vox)
        d.vdim[:] = [vox.shape[2], vox.shape[1], vox.shape[0]]
        d.vox = vox.ctypes.data_as(ctypes.POINTER(ctypes.c_ubyte))
    d.plane[:] = list(geometry.plane)
    return d, keep


def desc_for(w, **over):
    kw = dict(n=w.n, p=w.p, alpha=w.alpha, geometry=w.geometry, E=w.E, nu=w.nu, bc=w.bc,
              traction=w.traction, lo=w.lo, hi=w.hi)
    kw.update(over)
    return make_desc(**kw)


def gauss(n):
    x = np.zeros(n)
    w = np.zeros(n)
    lib().ora_gauss(n, _dp(x), _dp(w))
    return x, w


def shape1d(p, xi):
    f = np.zeros(p + 1)
    df = np.zeros(p + 1)
    lib().ora_shape1d(p, float(xi), _dp(f), _dp(df))
    return f, df


def cell_matrix(desc, c, want_K=True):
    p = desc.p
    nd = 3 * (p + 1) ** 3
    K = np.zeros((nd, nd)) if want_K else None
    eta = np.zeros(1)
    cc = np.array(c, dtype=np.int32)
    lib().ora_cell_matrix(ctypes.byref(desc), _ip(cc), _dp(K) if want_K else None, _dp(eta))
    return K, float(eta[0])


def cell_traction(desc, c):
    p = desc.p
    be = np.zeros(3 * (p + 1) ** 3)
    cc = np.array(c, dtype=np.int32)
    lib().ora_cell_traction(ctypes.byref(desc), _ip(cc), _dp(be))
    return be


def pseudo_inverse(A, eps=1e-13):
    A = np.ascontiguousarray(A, dtype=np.float64)
    n = A.shape[0]
    F = np.zeros((n, n))
    cond = np.zeros(1)
    nneg = np.zeros(1, dtype=np.int32)
    nfilt = np.zeros(1, dtype=np.int32)
    lib().ora_pseudo_inverse(n, _dp(A), eps, _dp(F), _dp(cond), _ip(nneg), _ip(nfilt))
    return F, float(cond[0]), int(nneg[0]), int(nfilt[0])


def jacobi_eig(A):
    W = np.ascontiguousarray(A, dtype=np.float64).copy()
    n = W.shape[0]
    V = np.zeros((n, n))
    lam = np.zeros(n)
    sweeps = lib().ora_jacobi_eig(n, _dp(W), _dp(V), _dp(lam))
    return lam, V, sweeps


class Problem:
    """Assembled finite cell problem on the CPU (free DOFs only)."""

    def __init__(self, desc, keep):
        self._desc = desc
        self._keep = keep
        self.h = lib().ora_problem_build(ctypes.byref(desc))
        L = lib()
        self.nfree = L.ora_nfree(self.h)
        self.nlat = L.ora_nlat(self.h)
        self.free_lat = np.zeros(self.nfree, dtype=np.int64)
        L.ora_get_free_lat(self.h, _lp(self.free_lat))
        self.ncells = L.ora_ncells(self.h)

    @classmethod
    def from_workload(cls, w, **over):
        d, keep = desc_for(w, **over)
        return cls(d, keep)

    def __del__(self):
        try:
            if getattr(self, "h", None):
                lib().ora_problem_free(self.h)
                self.h = None
        except Exception:
            pass

    def rhs(self):
        b = np.zeros(self.nfree)
        lib().ora_get_rhs(self.h, _dp(b))
        return b

    def load(self, load_case):
        """Load case 0 (traction) or 1..6 (unit Voigt strains xx, yy, zz, yz, xz, xy)."""
        b = np.zeros(self.nfree)
        if lib().ora_get_load(self.h, load_case, _dp(b)) != 0:
            raise ValueError("load case must be in 0..6")
        return b

    def eta(self):
        e = np.zeros(self.ncells)
        lib().ora_get_eta(self.h, _dp(e))
        return e

    def csr(self):
        import scipy.sparse as sp
        L = lib()
        nnz = L.ora_nnz(self.h)
        rp = np.zeros(self.nfree + 1, dtype=np.int64)
        col = np.zeros(nnz, dtype=np.int64)
        val = np.zeros(nnz)
        L.ora_get_csr(self.h, _lp(rp), _lp(col), _dp(val))
        return sp.csr_matrix((val, col, rp), shape=(self.nfree, self.nfree))

    def apply_K(self, x):
        x = np.ascontiguousarray(x, dtype=np.float64)
        y = np.zeros(self.nfree)
        lib().ora_apply_K(self.h, _dp(x), _dp(y))
        return y

    def precond_build(self, rule=0, eps=1e-13, eta_bar=1.0):
        return lib().ora_precond_build(self.h, rule, eps, eta_bar)

    def nblocks(self):
        return lib().ora_nblocks(self.h)

    def block(self, b):
        L = lib()
        n = L.ora_block_size(self.h, b)
        idx = np.zeros(n, dtype=np.int32)
        F = np.zeros((n, n))
        info = np.zeros(3)
        L.ora_block_get(self.h, b, _ip(idx), _dp(F), _dp(info))
        return idx, F, info

    def apply_S(self, r):
        r = np.ascontiguousarray(r, dtype=np.float64)
        z = np.zeros(self.nfree)
        lib().ora_apply_S(self.h, _dp(r), _dp(z))
        return z

    def pcg(self, b=None, tol=1e-10, maxit=10000):
        if b is None:
            b = self.rhs()
        b = np.ascontiguousarray(b, dtype=np.float64)
        x = np.zeros(self.nfree)
        hist = np.zeros(maxit + 1)
        its = lib().ora_pcg(self.h, _dp(b), tol, maxit, _dp(x), _dp(hist))
        n_hist = its + 1 if 0 <= its <= maxit else maxit + 1
        return x, its, hist[:n_hist].copy()

    def energy_error(self, xref, x):
        return lib().ora_energy_error(self.h, _dp(np.ascontiguousarray(xref)), _dp(np.ascontiguousarray(x)))

    def to_lattice(self, xf):
        out = np.zeros(self.nlat)
        out[self.free_lat] = xf
        return out

    def from_lattice(self, xl):
        return np.asarray(xl)[self.free_lat].copy()


def patch_factor(desc, v, eps=1e-13):
    p = desc.p
    nmax = 3 * (2 * p - 1) ** 3
    lat = np.zeros(nmax, dtype=np.int64)
    F = np.zeros(nmax * nmax)
    cond = np.zeros(1)
    vv = np.array(v, dtype=np.int32)
    nb = lib().ora_patch_factor(ctypes.byref(desc), _ip(vv), eps, _lp(lat), _dp(F), _dp(cond))
    return lat[:nb].copy(), F[: nb * nb].reshape(nb, nb).copy(), float(cond[0])


def sample_Kx(desc, rows, x_lattice):
    rows = np.ascontiguousarray(rows, dtype=np.int64)
    x = np.ascontiguousarray(x_lattice, dtype=np.float64)
    y = np.zeros(len(rows))
    st = lib().ora_sample_Kx(ctypes.byref(desc), len(rows), _lp(rows), _dp(x), _dp(y))
    return y, st


if __name__ == "__main__":
    print(build(force="--force" in sys.argv))
