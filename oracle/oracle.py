"""ctypes binding of the C oracle -- TEST INFRASTRUCTURE ONLY.

Only tests/, __graft_entry__.smoke() and bench.py's CPU baseline leg may use
this module.  Every function here is the plain O(N^2) definition of
arxiv 2410.05934 Sec. II-D, Eq. 1 (see ntt_oracle.c for the formulas).
"""
import ctypes
import os

import numpy as np

from . import build as _build

_lib = None
U64P = ctypes.POINTER(ctypes.c_uint64)
U32P = ctypes.POINTER(ctypes.c_uint32)


def lib():
    global _lib
    if _lib is None:
        _lib = bind(_build.build())
    return _lib


def bind(path):
    """Loads an oracle library from path and declares its C signatures."""
    L = ctypes.CDLL(path)
    u64, u32, i32 = ctypes.c_uint64, ctypes.c_uint32, ctypes.c_int
    L.oracle_mulmod.restype = u64
    L.oracle_mulmod.argtypes = [u64, u64, u64]
    L.oracle_powmod.restype = u64
    L.oracle_powmod.argtypes = [u64, u64, u64]
    L.oracle_is_prime.restype = i32
    L.oracle_is_prime.argtypes = [u64]
    L.oracle_psi.restype = u64
    L.oracle_psi.argtypes = [u64, u32]
    L.oracle_bitrev.restype = u32
    L.oracle_bitrev.argtypes = [u32, u32]
    L.oracle_ntt_forward_at.restype = i32
    L.oracle_ntt_forward_at.argtypes = [U64P, u32, u64, u64, U32P, u32, U64P]
    L.oracle_ntt_inverse_at.restype = i32
    L.oracle_ntt_inverse_at.argtypes = [U64P, u32, u64, u64, U32P, u32, U64P]
    L.oracle_pointwise.restype = None
    L.oracle_pointwise.argtypes = [U64P, U64P, U64P, u64, u64]
    L.oracle_negacyclic_schoolbook.restype = None
    L.oracle_negacyclic_schoolbook.argtypes = [U64P, U64P, U64P, u32, u64]
    L.oracle_negacyclic_schoolbook_at.restype = None
    L.oracle_negacyclic_schoolbook_at.argtypes = [U64P, U64P, u32, u64, U32P, u32, U64P]
    L.oracle_transform_rows.restype = i32
    L.oracle_transform_rows.argtypes = [i32, U64P, U64P, u32, u32, U64P, U64P, U32P, u32, i32]
    L.oracle_transform_rows_split.restype = i32
    L.oracle_transform_rows_split.argtypes = [i32, U64P, U64P, u32, u32, U64P, U64P, u32, i32]
    L.oracle_radix2_rows.restype = i32
    L.oracle_radix2_rows.argtypes = [i32, U64P, U64P, u32, u32, U64P, u32, i32]
    return L


def _u64(a):
    a = np.ascontiguousarray(np.asarray(a, dtype=np.uint64))
    return a, a.ctypes.data_as(U64P)


def _u32(a):
    a = np.ascontiguousarray(np.asarray(a, dtype=np.uint32))
    return a, a.ctypes.data_as(U32P)


def default_threads():
    return max(1, os.cpu_count() or 1)


# ---- scalars -------------------------------------------------------------

def mulmod(a, b, q):
    return int(lib().oracle_mulmod(a, b, q))


def powmod(a, e, q):
    return int(lib().oracle_powmod(a, e, q))


def is_prime(n):
    return bool(lib().oracle_is_prime(n))


def psi(q, log2n):
    """The fixed primitive 2N-th root: g^((q-1)/2N), g the least non-residue."""
    return int(lib().oracle_psi(q, log2n))


def bitrev(j, log2n):
    return int(lib().oracle_bitrev(j, log2n))


# ---- one row ---------------------------------------------------------------

def ntt_forward(a, q, log2n=None, psi_=None, idx=None):
    """Forward negacyclic NTT of one row (all outputs, or those at idx)."""
    a, ap = _u64(a)
    log2n = int(a.size).bit_length() - 1 if log2n is None else log2n
    psi_ = psi(q, log2n) if psi_ is None else psi_
    if idx is None:
        out = np.zeros(1 << log2n, dtype=np.uint64)
        rc = lib().oracle_ntt_forward_at(ap, log2n, q, psi_, None, 0, out.ctypes.data_as(U64P))
    else:
        idx, ip = _u32(idx)
        out = np.zeros(idx.size, dtype=np.uint64)
        rc = lib().oracle_ntt_forward_at(ap, log2n, q, psi_, ip, idx.size, out.ctypes.data_as(U64P))
    if rc:
        raise MemoryError("oracle_ntt_forward_at failed")
    return out


def ntt_inverse(A, q, log2n=None, psi_=None, idx=None):
    """Inverse negacyclic NTT of one row (all coefficients, or those at idx)."""
    A, Ap = _u64(A)
    log2n = int(A.size).bit_length() - 1 if log2n is None else log2n
    psi_ = psi(q, log2n) if psi_ is None else psi_
    if idx is None:
        out = np.zeros(1 << log2n, dtype=np.uint64)
        rc = lib().oracle_ntt_inverse_at(Ap, log2n, q, psi_, None, 0, out.ctypes.data_as(U64P))
    else:
        idx, ip = _u32(idx)
        out = np.zeros(idx.size, dtype=np.uint64)
        rc = lib().oracle_ntt_inverse_at(Ap, log2n, q, psi_, ip, idx.size, out.ctypes.data_as(U64P))
    if rc:
        raise MemoryError("oracle_ntt_inverse_at failed")
    return out


def pointwise(a, b, q):
    a, ap = _u64(a)
    b, bp = _u64(b)
    c = np.zeros(a.size, dtype=np.uint64)
    lib().oracle_pointwise(ap, bp, c.ctypes.data_as(U64P), a.size, q)
    return c


def schoolbook(a, b, q):
    """a*b mod (x^N + 1, q) by the O(N^2) schoolbook definition."""
    a, ap = _u64(a)
    b, bp = _u64(b)
    log2n = int(a.size).bit_length() - 1
    c = np.zeros(a.size, dtype=np.uint64)
    lib().oracle_negacyclic_schoolbook(ap, bp, c.ctypes.data_as(U64P), log2n, q)
    return c


def schoolbook_at(a, b, q, idx):
    """Coefficients idx of a*b mod (x^N + 1, q), each by its O(N) sum."""
    a, ap = _u64(a)
    b, bp = _u64(b)
    idx, ip = _u32(idx)
    log2n = int(a.size).bit_length() - 1
    out = np.zeros(idx.size, dtype=np.uint64)
    lib().oracle_negacyclic_schoolbook_at(ap, bp, log2n, q, ip, idx.size, out.ctypes.data_as(U64P))
    return out


# ---- many rows -------------------------------------------------------------

def transform_rows(x, q_row, inverse=False, idx=None, nthreads=None, split=False, chunk=64):
    """Transforms each row of x (rows x N) with its own modulus q_row[r].

    idx (rows x k) restricts row r to the outputs idx[r]; split=True spreads
    the (row, output) pairs over threads, for a few long rows.
    """
    x = np.ascontiguousarray(np.asarray(x, dtype=np.uint64))
    rows, n = x.shape
    log2n = n.bit_length() - 1
    q_row = np.ascontiguousarray(np.asarray(q_row, dtype=np.uint64))
    psi_row = np.array([psi(int(q), log2n) for q in q_row], dtype=np.uint64)
    if np.any(psi_row == 0):
        raise ValueError("a modulus is not a prime = 1 mod 2N")
    nthreads = default_threads() if nthreads is None else nthreads
    _, xp = _u64(x)
    _, qp = _u64(q_row)
    _, pp = _u64(psi_row)
    if split:
        assert idx is None
        out = np.zeros((rows, n), dtype=np.uint64)
        rc = lib().oracle_transform_rows_split(int(inverse), xp, out.ctypes.data_as(U64P), rows, log2n,
                                               qp, pp, chunk, nthreads)
    elif idx is None:
        out = np.zeros((rows, n), dtype=np.uint64)
        rc = lib().oracle_transform_rows(int(inverse), xp, out.ctypes.data_as(U64P), rows, log2n,
                                         qp, pp, None, 0, nthreads)
    else:
        idx = np.ascontiguousarray(np.asarray(idx, dtype=np.uint32))
        assert idx.shape[0] == rows
        out = np.zeros(idx.shape, dtype=np.uint64)
        _, ip = _u32(idx)
        rc = lib().oracle_transform_rows(int(inverse), xp, out.ctypes.data_as(U64P), rows, log2n,
                                         qp, pp, ip, idx.shape[1], nthreads)
    if rc:
        raise MemoryError("oracle transform failed")
    return out


# ---- the O(N log N) CPU baseline (ntt_radix2.c) -----------------------------

def radix2_rows(x, moduli, inverse=False, nthreads=None):
    """Rows of x ([rows][N], row r over moduli[r % len(moduli)]) through the
    plain radix-2 transforms: the same results as transform_rows, in
    O(N log N) per row.  A timing baseline; parity is checked against the
    O(N^2) definitions."""
    x = np.ascontiguousarray(np.asarray(x, dtype=np.uint64))
    rows, n = x.shape
    log2n = n.bit_length() - 1
    moduli = np.ascontiguousarray(np.asarray(moduli, dtype=np.uint64))
    nthreads = default_threads() if nthreads is None else nthreads
    out = np.zeros((rows, n), dtype=np.uint64)
    _, xp = _u64(x)
    _, mp = _u64(moduli)
    rc = lib().oracle_radix2_rows(int(inverse), xp, out.ctypes.data_as(U64P), rows, log2n, mp, moduli.size,
                                  nthreads)
    if rc:
        raise ValueError("radix-2 baseline: bad modulus or size")
    return out
