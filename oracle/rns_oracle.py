"""RNS basis conversion (BConv) and Rescale -- TEST INFRASTRUCTURE ONLY.

Only tests/, __graft_entry__.smoke() and bench.py's CPU baseline leg may use
this module.  These are the CKKS operators that sit around the NTT in key
switching and after a multiplication (Sec. II-A: Rescale brings the scale
back to Delta and drops one level; Sec. III Phase 1 lists BConv beside NTT,
ModMul, ModAdd and Automorph), written as their textbook definitions over
the residue number system of Q = q_0 ... q_(L-1):

  BConv_{Q -> P}(x)_j = sum_i [x_i * Qhat_i^-1]_{q_i} * Qhat_i  mod p_j,
      Qhat_i = Q / q_i  (the fast basis conversion: it equals X + alpha Q
      mod p_j for the integer X < Q with residues x_i and some 0 <= alpha < L)
  Rescale(x)_i = round(X / q_(L-1)) mod q_i  for i < L - 1
      computed per coefficient as (x_i + h - r) * q_(L-1)^-1 mod q_i with
      h = floor(q_(L-1) / 2), r = (x_(L-1) + h) mod q_(L-1)

Rescale of a ciphertext held in the NTT domain (the form the library keeps
CKKS limbs in) brings every limb to coefficients with the O(N^2) inverse
definition, rescales, and goes back with the forward definition.
"""
import numpy as np

from . import oracle as O


def prod(vals):
    out = 1
    for v in vals:
        out *= int(v)
    return out


def qhat_inv(Q):
    """[(Q / q_i)^-1 mod q_i]."""
    big = prod(Q)
    return [pow(big // int(q) % int(q), -1, int(q)) for q in Q]


def bconv(x, Q, P):
    """x [L][N] residues mod Q -> [K][N] residues mod P (fast basis conversion)."""
    x = np.asarray(x, dtype=np.uint64)
    big = prod(Q)
    inv = qhat_inv(Q)
    hats = [big // int(q) for q in Q]
    L, n = x.shape
    out = np.zeros((len(P), n), dtype=np.uint64)
    for k in range(n):
        a = [int(x[i, k]) * inv[i] % int(Q[i]) for i in range(L)]
        for j, p in enumerate(P):
            out[j, k] = sum(a[i] * (hats[i] % int(p)) for i in range(L)) % int(p)
    return out


def rescale(x, Q):
    """x [L][N] coefficient-domain residues -> [L-1][N]: round(X / q_(L-1)) mod q_i."""
    x = np.asarray(x, dtype=np.uint64)
    ql = int(Q[-1])
    h = ql // 2
    L, n = x.shape
    out = np.zeros((L - 1, n), dtype=np.uint64)
    for i in range(L - 1):
        qi = int(Q[i])
        inv = pow(ql % qi, -1, qi)
        for k in range(n):
            r = (int(x[L - 1, k]) + h) % ql
            out[i, k] = (int(x[i, k]) + h - r) % qi * inv % qi
    return out


def rescale_ntt(x_ntt, Q, idx=None):
    """Rescale of NTT-domain limbs [L][N] -> NTT-domain [L-1][N] (all outputs,
    or those at idx)."""
    x_ntt = np.asarray(x_ntt, dtype=np.uint64)
    L, n = x_ntt.shape
    ql = int(Q[-1])
    h = ql // 2
    last = O.transform_rows(x_ntt[L - 1:L], [ql], inverse=True, split=n >= 4096)[0]
    r = (last.astype(object) + h) % ql
    width = n if idx is None else len(idx)
    out = np.zeros((L - 1, width), dtype=np.uint64)
    for i in range(L - 1):
        qi = int(Q[i])
        inv = pow(ql % qi, -1, qi)
        # (x_i + h - r) in coefficients is x_i + c with c_k = (h - r_k) mod q_i
        c = np.array([(h - int(v)) % qi for v in r], dtype=np.uint64)
        cn = O.ntt_forward(c, qi, idx=idx)
        xi = x_ntt[i] if idx is None else x_ntt[i][np.asarray(idx)]
        out[i] = [(int(a) + int(b)) % qi * inv % qi for a, b in zip(xi, cn)]
    return out
