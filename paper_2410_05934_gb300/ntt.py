"""Python binding of the batched negacyclic NTT library (C ABI: ntt_gb300.h).

The names follow the C ABI: ``Plan`` wraps ``ntt_plan`` and its methods call
``ntt_forward``, ``ntt_inverse`` and ``poly_mul_pointwise``.  Data are CUDA
tensors of 64-bit integers (int64 or uint64 holding the uint64 coefficient
bits), laid out [batch][n_moduli][N] and contiguous; torch provides only the
memory and the stream.  Raw device pointers (ints) are accepted as well.
"""
import ctypes

from . import _native
from ._native import U32P, U64P, check, load

NTT_FLAG_HOST_ONLY = 1
NTT_FLAG_CHECK = 2
NTT_FLAG_NATURAL_ORDER = 4
NTT_FLAG_WORD32 = 8
NTT_FLAG_OTF_TWIDDLES = 16


def _stream_handle(stream):
    if stream is None:
        try:
            import torch
            if torch.cuda.is_available():
                return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
        except ImportError:
            pass
        return ctypes.c_void_p(0)
    if isinstance(stream, int):
        return ctypes.c_void_p(stream)
    return ctypes.c_void_p(stream.cuda_stream)


def _ptr(x, min_elems=None, what="tensor", word=8):
    if isinstance(x, int):
        return ctypes.c_void_p(x)
    if not x.is_cuda:
        raise ValueError("%s must be a CUDA tensor" % what)
    if x.element_size() != word or x.is_floating_point():
        raise ValueError("%s must hold %d-bit integers" % (what, 8 * word))
    if not x.is_contiguous():
        raise ValueError("%s must be contiguous" % what)
    if min_elems is not None and x.numel() < min_elems:
        raise ValueError("%s has %d elements, needs %d" % (what, x.numel(), min_elems))
    return ctypes.c_void_p(x.data_ptr())


def schedule_count(log2n):
    return load().ntt_schedule_count(log2n)


def schedule_name(log2n, sched_id):
    buf = ctypes.create_string_buffer(256)
    check(load().ntt_schedule_name(log2n, sched_id, buf, 256), "ntt_schedule_name")
    return buf.value.decode()


def schedule_params(log2n, sched_id):
    """dict of a schedule's raw parameters (see ntt_schedule_params)."""
    buf = (ctypes.c_int32 * 11)()
    check(load().ntt_schedule_params(log2n, sched_id, buf, 11), "ntt_schedule_params")
    v = list(buf)
    form_col = v[1] & 3
    form_row = v[1] if v[1] < 4 else (v[1] >> 2) & 3
    d = {"kernels": v[0], "form": v[1], "pipelined": form_col == 1 or form_row == 1,
         "staged_twiddles": form_col != 2 and form_row != 2, "log2n": v[2]}
    if v[0] == 1:
        d.update(logt=v[3], logrp=v[4], tpc=v[5])
    else:
        d.update(split=v[3], logp=v[4], logt_col=v[5], logrp_col=v[6], tpc_col=v[7],
                 logt_row=v[8], logrp_row=v[9], tpc_row=v[10])
    return d


class Plan:
    """ntt_plan(log2n, moduli, batch, flags): tables on the current device."""

    def __init__(self, log2n, moduli, batch=1, flags=0, schedule=None):
        L = load()
        moduli = [int(q) for q in moduli]
        arr = (ctypes.c_uint64 * len(moduli))(*moduli)
        h = ctypes.c_void_p()
        check(L.ntt_plan(ctypes.byref(h), log2n, arr, len(moduli), batch, flags), "ntt_plan")
        self._h = h
        self.log2n, self.n, self.moduli, self.batch = log2n, 1 << log2n, moduli, batch
        self.n_moduli = len(moduli)
        self.word = 4 if flags & NTT_FLAG_WORD32 else 8     # bytes per coefficient
        self.rows = batch * len(moduli)
        if schedule == "auto":
            from .costmodel import choose_schedule
            bits = max(int(q).bit_length() for q in moduli)
            self.schedule, self.schedule_source = choose_schedule(log2n, len(moduli), batch, bits)
        elif schedule is not None:
            self.schedule = schedule

    # -- lifetime --
    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            load().ntt_plan_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    @property
    def handle(self):
        return self._h

    # -- queries --
    def root(self, limb=0):
        v = ctypes.c_uint64()
        check(load().ntt_plan_root(self._h, limb, ctypes.byref(v)), "ntt_plan_root")
        return v.value

    @property
    def schedule(self):
        v = ctypes.c_uint32()
        check(load().ntt_plan_get_schedule(self._h, ctypes.byref(v)), "ntt_plan_get_schedule")
        return v.value

    @schedule.setter
    def schedule(self, sched_id):
        check(load().ntt_plan_set_schedule(self._h, int(sched_id)), "ntt_plan_set_schedule")

    def last_launches(self):
        v = ctypes.c_uint32()
        check(load().ntt_plan_last_launches(self._h, ctypes.byref(v)), "ntt_plan_last_launches")
        return v.value

    def status(self, stream=None):
        """Synchronises the stream; returns and clears the device status word."""
        return load().ntt_status(self._h, _stream_handle(stream))

    def debug_bounded_wait(self, deliver, spin_limit, out=None, stream=None):
        """ntt_debug_bounded_wait: one CTA waits (bounded) on an mbarrier that a
        16-byte copy completes only when `deliver`; otherwise the wait runs out
        and the status word records NTT_ERR_TIMEOUT.  `out` (2 uint64 on the
        device, optional) receives the copied pair."""
        ptr = None if out is None else _ptr(out, 2, "out")
        check(load().ntt_debug_bounded_wait(self._h, 1 if deliver else 0, spin_limit, ptr, _stream_handle(stream)),
              "ntt_debug_bounded_wait")

    # -- compute --
    def forward(self, x, out=None, stream=None):
        out = x if out is None else out
        need = self.rows * self.n
        check(load().ntt_forward(self._h, _ptr(x, need, "in", self.word), _ptr(out, need, "out", self.word),
                                 _stream_handle(stream)), "ntt_forward")
        return out

    def inverse(self, x, out=None, stream=None):
        out = x if out is None else out
        need = self.rows * self.n
        check(load().ntt_inverse(self._h, _ptr(x, need, "in", self.word), _ptr(out, need, "out", self.word),
                                 _stream_handle(stream)), "ntt_inverse")
        return out

    def forward_rows(self, x, out, row_begin, n_rows, stream=None):
        need = (row_begin + n_rows) * self.n
        check(load().ntt_forward_rows(self._h, _ptr(x, need, "in", self.word), _ptr(out, need, "out", self.word),
                                      row_begin, n_rows, _stream_handle(stream)), "ntt_forward_rows")
        return out

    def inverse_rows(self, x, out, row_begin, n_rows, stream=None):
        need = (row_begin + n_rows) * self.n
        check(load().ntt_inverse_rows(self._h, _ptr(x, need, "in", self.word), _ptr(out, need, "out", self.word),
                                      row_begin, n_rows, _stream_handle(stream)), "ntt_inverse_rows")
        return out

    def hmul_tensor(self, a, b, out, stream=None):
        """(d0, d1, d2) = INTT of the CKKS tensor product of NTT-domain
        ciphertexts a = [a0; a1], b = [b0; b1] ([2][n_moduli][N] each)."""
        per = self.n_moduli * self.n
        check(load().ntt_hmul_tensor(self._h, _ptr(a, 2 * per, "a"), _ptr(b, 2 * per, "b"),
                                     _ptr(out, 3 * per, "out"), _stream_handle(stream)), "ntt_hmul_tensor")
        return out

    def inverse_mul(self, a, b, out, a_poly=None, b_poly=None, stream=None):
        """out[p] = INTT(a[a_poly[p]] (.) b[b_poly[p]]) per limb, the product
        formed inside the inverse's first kernel (ntt_inverse_mul)."""
        per = self.n_moduli * self.n
        a_polys = a.numel() // per
        b_polys = b.numel() // per
        am = bm = None
        if a_poly is not None or b_poly is not None:
            am = (ctypes.c_uint32 * len(a_poly))(*[int(v) for v in a_poly])
            bm = (ctypes.c_uint32 * len(b_poly))(*[int(v) for v in b_poly])
        check(load().ntt_inverse_mul(self._h, _ptr(a, what="a"), am, a_polys, _ptr(b, what="b"), bm, b_polys,
                                     _ptr(out, self.batch * per, "out"), _stream_handle(stream)), "ntt_inverse_mul")
        return out

    def rescale(self, x, out, work, n_polys=0, stream=None):
        """Rescale by the plan's last modulus: x [n_polys][L][N] -> out
        [n_polys][L-1][N], both NTT domain; work [n_polys][N] scratch."""
        polys = n_polys or self.batch
        check(load().ntt_rescale(self._h, _ptr(x, polys * self.n_moduli * self.n, "in"),
                                 _ptr(out, polys * (self.n_moduli - 1) * self.n, "out"),
                                 _ptr(work, polys * self.n, "work"), n_polys, _stream_handle(stream)), "ntt_rescale")
        return out

    def tfhe_key_prepare(self, key, levels, out=None, stream=None):
        """RGSW key rows [2 levels][2][N] (NTT domain, canonical) -> the
        {w, floor(w 2^64 / q)} pair form the TFHE kernels read
        ([2 levels][2][N][2])."""
        if out is None:
            import torch
            out = torch.empty((2 * levels, 2, self.n, 2), dtype=torch.int64, device=key.device)
        check(load().tfhe_key_prepare(self._h, _ptr(key, 4 * levels * self.n, "key"),
                                      levels, _ptr(out, 8 * levels * self.n, "out"), _stream_handle(stream)),
              "tfhe_key_prepare")
        return out

    def tfhe_external_product(self, d, key, levels, log2_base, out=None, stream=None):
        """K [x] d for d = [n_ct][2][N] RLWE ciphertexts and one RGSW key
        prepared by tfhe_key_prepare (tfhe_external_product)."""
        n_ct = d.shape[0] if hasattr(d, "shape") else None
        out = d if out is None else out
        check(load().tfhe_external_product(self._h, _ptr(d, what="d"), _ptr(key, 8 * levels * self.n, "key"),
                                           levels, log2_base, _ptr(out, what="out"),
                                           n_ct, _stream_handle(stream)), "tfhe_external_product")
        return out

    def tfhe_cmux_rotate(self, acc, rot, key, levels, log2_base, out=None, stream=None):
        """acc + K [x] (x^rot acc - acc) per ciphertext (tfhe_cmux_rotate);
        rot: CUDA int32 tensor of exponents, one per ciphertext."""
        n_ct = acc.shape[0]
        out = acc if out is None else out
        if not rot.is_cuda or rot.element_size() != 4 or rot.numel() < n_ct or not rot.is_contiguous():
            raise ValueError("rot must be a contiguous CUDA tensor of 32-bit exponents, one per ciphertext")
        check(load().tfhe_cmux_rotate(self._h, _ptr(acc, what="acc"), ctypes.c_void_p(rot.data_ptr()),
                                      _ptr(key, 8 * levels * self.n, "key"), levels, log2_base,
                                      _ptr(out, what="out"), n_ct, _stream_handle(stream)), "tfhe_cmux_rotate")
        return out

    def pointwise(self, a, b, out=None, n_polys=0, stream=None):
        out = a if out is None else out
        need = (n_polys or self.batch) * self.n_moduli * self.n
        check(load().poly_mul_pointwise(self._h, _ptr(a, need, "a", self.word), _ptr(b, need, "b", self.word),
                                        _ptr(out, need, "c", self.word), n_polys, _stream_handle(stream)),
              "poly_mul_pointwise")
        return out


NTT_BATCH_GRAPH = 1
NTT_BATCH_GROUPED = 4


class Batch:
    """ntt_batch_plan: an uneven mixed batch run as one persistent launch.

    requests: list of dicts with log2n, n_moduli, n_polys, moduli_offset,
    inverse, schedule, in, out -- in/out CUDA tensors or device pointers;
    schedule 0 (default) makes the request work items of the persistent
    kernel, s + 1 runs it as its own launches with schedule s of its N
    (``costmodel.schedule_requests`` fills it in).
    """

    def __init__(self, requests, moduli_pool, flags=NTT_BATCH_GRAPH):
        L = load()
        self._reqs = self._pack(requests)
        pool = [int(q) for q in moduli_pool]
        arr = (ctypes.c_uint64 * len(pool))(*pool)
        h = ctypes.c_void_p()
        check(L.ntt_batch_plan(ctypes.byref(h), self._reqs, len(self._reqs), arr, len(pool), flags),
              "ntt_batch_plan")
        self._h = h

    @staticmethod
    def _pack(requests):
        arr = (_native.NttRequest * len(requests))()
        for i, r in enumerate(requests):
            d = arr[i]
            d.log2n, d.n_moduli, d.n_polys = int(r["log2n"]), int(r["n_moduli"]), int(r["n_polys"])
            d.moduli_offset, d.inverse = int(r.get("moduli_offset", 0)), int(r.get("inverse", 0))
            d.schedule = int(r.get("schedule", 0))
            d.in_ = _ptr(r["in"], what="in").value
            d.out = _ptr(r.get("out", r["in"]), what="out").value
        return arr

    def update(self, requests, stream=None):
        reqs = self._pack(requests)
        check(load().ntt_batch_update(self._h, reqs, len(reqs), _stream_handle(stream)), "ntt_batch_update")
        self._reqs = reqs

    def execute(self, stream=None):
        check(load().ntt_batch_execute(self._h, _stream_handle(stream)), "ntt_batch_execute")

    def execute_plain(self, schedules=None, stream=None):
        sched = None
        if schedules is not None:
            sched = (ctypes.c_uint32 * len(schedules))(*[int(s) for s in schedules])
        check(load().ntt_batch_execute_plain(self._h, sched, _stream_handle(stream)), "ntt_batch_execute_plain")

    def status(self, stream=None):
        return load().ntt_batch_status(self._h, _stream_handle(stream))

    def info(self):
        items, launches, coef = ctypes.c_uint64(), ctypes.c_uint32(), ctypes.c_uint64()
        check(load().ntt_batch_info(self._h, ctypes.byref(items), ctypes.byref(launches), ctypes.byref(coef)),
              "ntt_batch_info")
        return {"items": items.value, "last_launches": launches.value, "coefficients": coef.value}

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            load().ntt_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class BConv:
    """ntt_bconv_plan(Q, P): RNS basis conversion of [n_polys][L][N] residues
    mod Q into [n_polys][K][N] residues mod P (fast conversion)."""

    def __init__(self, q_from, p_to):
        L = load()
        q = (ctypes.c_uint64 * len(q_from))(*[int(v) for v in q_from])
        p = (ctypes.c_uint64 * len(p_to))(*[int(v) for v in p_to])
        h = ctypes.c_void_p()
        check(L.ntt_bconv_plan(ctypes.byref(h), q, len(q_from), p, len(p_to)), "ntt_bconv_plan")
        self._h = h
        self.L, self.K = len(q_from), len(p_to)

    def __call__(self, x, out, log2n, n_polys=None, stream=None):
        n_polys = x.shape[0] if n_polys is None else n_polys
        n = 1 << log2n
        check(load().ntt_bconv(self._h, _ptr(x, n_polys * self.L * n, "in"), _ptr(out, n_polys * self.K * n, "out"),
                               log2n, n_polys, _stream_handle(stream)), "ntt_bconv")
        return out

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            load().ntt_bconv_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# C-ABI names as plain functions
def forward_inverse(fwd_plan, x_fwd, x_inv, inv_plan, out_fwd=None, out_inv=None, stream=None):
    """ntt_forward_inverse: the forward transform of fwd_plan's rows and the
    inverse of inv_plan's rows, issued together (one launch for 32-bit words
    at N = 1024).  The two transforms' buffers must not overlap."""
    out_fwd = x_fwd if out_fwd is None else out_fwd
    out_inv = x_inv if out_inv is None else out_inv
    nf, ni = fwd_plan.rows * fwd_plan.n, inv_plan.rows * inv_plan.n
    check(load().ntt_forward_inverse(fwd_plan.handle, _ptr(x_fwd, nf, "fwd in", fwd_plan.word),
                                     _ptr(out_fwd, nf, "fwd out", fwd_plan.word), inv_plan.handle,
                                     _ptr(x_inv, ni, "inv in", inv_plan.word), _ptr(out_inv, ni, "inv out", inv_plan.word),
                                     _stream_handle(stream)), "ntt_forward_inverse")
    return out_fwd, out_inv


def ntt_plan(log2n, moduli, batch=1, flags=0):
    return Plan(log2n, moduli, batch, flags)


def ntt_forward(plan, d_in, d_out=None, stream=None):
    return plan.forward(d_in, d_out, stream)


def ntt_inverse(plan, d_in, d_out=None, stream=None):
    return plan.inverse(d_in, d_out, stream)


def poly_mul_pointwise(plan, d_a, d_b, d_c=None, n_polys=0, stream=None):
    return plan.pointwise(d_a, d_b, d_c, n_polys, stream)
