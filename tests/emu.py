"""ctypes binding of the host emulation library (tests only)."""
import ctypes

import numpy as np

from paper_2410_05934_gb300 import build as B

U64P = ctypes.POINTER(ctypes.c_uint64)
_lib = None


def lib():
    global _lib
    if _lib is None:
        L = ctypes.CDLL(B.build_emulation())
        u32, u64, i32, vp = ctypes.c_uint32, ctypes.c_uint64, ctypes.c_int, ctypes.c_void_p
        L.nttemu_plan.argtypes = [ctypes.POINTER(vp), u32, U64P, u32, u32, u32]
        L.nttemu_plan.restype = i32
        L.nttemu_plan_destroy.argtypes = [vp]
        L.nttemu_schedule_count.argtypes = [u32]
        L.nttemu_transform.argtypes = [vp, u32, i32, U64P, U64P, u64, u64]
        L.nttemu_transform.restype = i32
        L.nttemu_pointwise.argtypes = [vp, U64P, U64P, U64P, u64]
        L.nttemu_status.argtypes = [vp]
        L.nttemu_debug_bounded_wait.argtypes = [vp, u32, u32, U64P]
        L.nttemu_debug_bounded_wait.restype = i32
        L.nttemu_batch_transform.argtypes = [vp, i32, U64P, U64P]
        L.nttemu_batch_transform.restype = i32
        L.nttemu_hmul_tensor.argtypes = [vp, u32, U64P, U64P, U64P]
        L.nttemu_hmul_tensor.restype = i32
        L.nttemu_tfhe_cmux.argtypes = [vp, U64P, ctypes.POINTER(ctypes.c_uint32), U64P, u32, u32, U64P, u64]
        L.nttemu_tfhe_cmux.restype = i32
        L.nttemu_bconv.argtypes = [U64P, u32, U64P, u32, U64P, U64P, u64, u64]
        L.nttemu_bconv.restype = i32
        L.nttemu_rescale.argtypes = [vp, u32, U64P, U64P, U64P, u32]
        L.nttemu_rescale.restype = i32
        U32P = ctypes.POINTER(ctypes.c_uint32)
        L.nttemu_inverse_mul.argtypes = [vp, u32, U64P, ctypes.POINTER(ctypes.c_uint32), U64P,
                                         ctypes.POINTER(ctypes.c_uint32), U64P]
        L.nttemu_inverse_mul.restype = i32
        L.nttemu_transform32.argtypes = [vp, i32, U32P, U32P, u64, u64]
        L.nttemu_transform32.restype = i32
        L.nttemu_forward_inverse32.argtypes = [vp, U32P, U32P, vp, U32P, U32P]
        L.nttemu_forward_inverse32.restype = i32
        L.nttemu_pointwise32.argtypes = [vp, U32P, U32P, U32P, u64]
        L.nttemu_pointwise32.restype = i32
        L.nttemu_reduce_65q.argtypes = [vp, u32, U64P, U64P, u64]
        L.nttemu_reduce_65q.restype = i32
        _lib = L
    return _lib


def _p(a):
    return a.ctypes.data_as(U64P)


class EmuPlan:
    def __init__(self, log2n, moduli, batch=1, flags=0):
        arr = np.ascontiguousarray(np.array(moduli, dtype=np.uint64))
        self.h = ctypes.c_void_p()
        rc = lib().nttemu_plan(ctypes.byref(self.h), log2n, _p(arr), arr.size, batch, flags)
        if rc:
            raise ValueError("nttemu_plan failed: %d" % rc)
        self.log2n, self.n, self.rows = log2n, 1 << log2n, batch * arr.size

    def __del__(self):
        if self.h:
            lib().nttemu_plan_destroy(self.h)

    def transform(self, x, sched, inverse=False, out=None, row_begin=0, n_rows=None):
        x = np.ascontiguousarray(x, dtype=np.uint64)
        out = np.zeros_like(x) if out is None else out
        n_rows = self.rows - row_begin if n_rows is None else n_rows
        rc = lib().nttemu_transform(self.h, sched, int(inverse), _p(x), _p(out), row_begin, n_rows)
        if rc:
            raise ValueError("nttemu_transform failed: %d" % rc)
        return out

    def batch_transform(self, x, inverse=False):
        """The mixed-batch kernel's configuration for this N (direct form)."""
        x = np.ascontiguousarray(x, dtype=np.uint64)
        out = np.zeros_like(x)
        rc = lib().nttemu_batch_transform(self.h, int(inverse), _p(x), _p(out))
        if rc:
            raise ValueError("nttemu_batch_transform failed: %d" % rc)
        return out

    def hmul_tensor(self, a, b, sched):
        a = np.ascontiguousarray(a, dtype=np.uint64)
        b = np.ascontiguousarray(b, dtype=np.uint64)
        n_mod = a.shape[0] // 2
        out = np.zeros((3 * n_mod, a.shape[1]), dtype=np.uint64)
        rc = lib().nttemu_hmul_tensor(self.h, sched, _p(a), _p(b), _p(out))
        if rc:
            raise ValueError("nttemu_hmul_tensor failed: %d" % rc)
        return out

    def tfhe(self, d, key, levels, log2_base, rot=None, out=None):
        """tfhe_external_product (rot None) or tfhe_cmux_rotate of d [n_ct][2][N]."""
        d = np.ascontiguousarray(d, dtype=np.uint64)
        key = np.ascontiguousarray(key, dtype=np.uint64)
        out = np.zeros_like(d) if out is None else out
        rp = None
        if rot is not None:
            rot = np.ascontiguousarray(rot, dtype=np.uint32)
            rp = rot.ctypes.data_as(ctypes.POINTER(ctypes.c_uint32))
        rc = lib().nttemu_tfhe_cmux(self.h, _p(d), rp, _p(key), levels, log2_base, _p(out), d.shape[0])
        if rc:
            raise ValueError("nttemu_tfhe_cmux failed: %d" % rc)
        return out

    def inverse_mul(self, a, b, sched, a_poly=None, b_poly=None):
        """ntt_inverse_mul with schedule sched: [batch][n_moduli][N] output."""
        U32P = ctypes.POINTER(ctypes.c_uint32)
        a = np.ascontiguousarray(a, dtype=np.uint64)
        b = np.ascontiguousarray(b, dtype=np.uint64)
        out = np.zeros((self.rows, self.n), dtype=np.uint64)
        am = bm = None
        if a_poly is not None:
            am = np.ascontiguousarray(a_poly, dtype=np.uint32)
            bm = np.ascontiguousarray(b_poly, dtype=np.uint32)
        rc = lib().nttemu_inverse_mul(self.h, sched, _p(a), None if am is None else am.ctypes.data_as(U32P), _p(b),
                                      None if bm is None else bm.ctypes.data_as(U32P), _p(out))
        if rc:
            raise ValueError("nttemu_inverse_mul failed: %d" % rc)
        return out

    def rescale(self, x, sched, n_polys):
        """ntt_rescale with schedule sched: x [n_polys][L][N] (NTT domain) -> [n_polys][L-1][N]."""
        x = np.ascontiguousarray(x, dtype=np.uint64)
        n_mod, n = x.shape[1], x.shape[2]
        out = np.zeros((n_polys, n_mod - 1, n), dtype=np.uint64)
        work = np.zeros((n_polys, n), dtype=np.uint64)
        rc = lib().nttemu_rescale(self.h, sched, _p(x), _p(out), _p(work), n_polys)
        if rc:
            raise ValueError("nttemu_rescale failed: %d" % rc)
        return out

    def transform32(self, x, inverse=False, out=None, row_begin=0, n_rows=None):
        """A NTT_FLAG_WORD32 plan's transform on uint32 rows."""
        U32P = ctypes.POINTER(ctypes.c_uint32)
        x = np.ascontiguousarray(x, dtype=np.uint32)
        out = np.zeros_like(x) if out is None else out
        n_rows = self.rows - row_begin if n_rows is None else n_rows
        rc = lib().nttemu_transform32(self.h, int(inverse), x.ctypes.data_as(U32P), out.ctypes.data_as(U32P),
                                      row_begin, n_rows)
        if rc:
            raise ValueError("nttemu_transform32 failed: %d" % rc)
        return out

    def forward_inverse32(self, xf, inv_plan, xi):
        """ntt_forward_inverse of this plan's rows (forward) and inv_plan's (inverse), N = 1024."""
        U32P = ctypes.POINTER(ctypes.c_uint32)
        xf = np.ascontiguousarray(xf, dtype=np.uint32)
        xi = np.ascontiguousarray(xi, dtype=np.uint32)
        of, oi = np.zeros_like(xf), np.zeros_like(xi)
        rc = lib().nttemu_forward_inverse32(self.h, xf.ctypes.data_as(U32P), of.ctypes.data_as(U32P), inv_plan.h,
                                            xi.ctypes.data_as(U32P), oi.ctypes.data_as(U32P))
        if rc:
            raise ValueError("nttemu_forward_inverse32 failed: %d" % rc)
        return of, oi

    def pointwise32(self, a, b):
        U32P = ctypes.POINTER(ctypes.c_uint32)
        a = np.ascontiguousarray(a, dtype=np.uint32)
        b = np.ascontiguousarray(b, dtype=np.uint32)
        c = np.zeros_like(a)
        rc = lib().nttemu_pointwise32(self.h, a.ctypes.data_as(U32P), b.ctypes.data_as(U32P),
                                      c.ctypes.data_as(U32P), self.rows)
        if rc:
            raise ValueError("nttemu_pointwise32 failed: %d" % rc)
        return c

    def pointwise(self, a, b, n_rows=None):
        a = np.ascontiguousarray(a, dtype=np.uint64)
        b = np.ascontiguousarray(b, dtype=np.uint64)
        c = np.zeros_like(a)
        lib().nttemu_pointwise(self.h, _p(a), _p(b), _p(c), self.rows if n_rows is None else n_rows)
        return c

    def reduce_65q(self, limb, x):
        x = np.ascontiguousarray(np.asarray(x, dtype=np.uint64))
        out = np.zeros_like(x)
        rc = lib().nttemu_reduce_65q(self.h, limb, _p(x), _p(out), x.size)
        if rc:
            raise ValueError("nttemu_reduce_65q failed: %d" % rc)
        return out

    def status(self):
        return lib().nttemu_status(self.h)

    def debug_bounded_wait(self, deliver, spin_limit):
        out = np.zeros(2, dtype=np.uint64)
        rc = lib().nttemu_debug_bounded_wait(self.h, 1 if deliver else 0, spin_limit, _p(out))
        return rc, out


def bconv(x, Q, P):
    """ntt_bconv's arithmetic on the host: x [n_polys][L][n] -> [n_polys][K][n]."""
    x = np.ascontiguousarray(x, dtype=np.uint64)
    q = np.ascontiguousarray(np.array(Q, dtype=np.uint64))
    p = np.ascontiguousarray(np.array(P, dtype=np.uint64))
    out = np.zeros((x.shape[0], len(P), x.shape[2]), dtype=np.uint64)
    rc = lib().nttemu_bconv(_p(q), len(Q), _p(p), len(P), _p(x), _p(out), x.shape[2], x.shape[0])
    if rc:
        raise ValueError("nttemu_bconv failed: %d" % rc)
    return out


def schedule_count(log2n):
    return lib().nttemu_schedule_count(log2n)
