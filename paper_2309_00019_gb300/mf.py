"""ctypes binding of libmf (include/mf.h), same names as the C ABI.

Argument marshalling only: every step of the matched filter runs in the CUDA
kernels of libmf.so.  Device buffers are passed as integer addresses
(``torch.Tensor.data_ptr()``), streams as ``torch.cuda.Stream.cuda_stream``.
There is no CPU fallback: ``load()`` raises if the shared library is missing.
"""

from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libmf.so")

MF_OK, MF_EINVAL, MF_ENOMEM, MF_ECUDA, MF_ESTATE, MF_EOVERFLOW, MF_ETIMEOUT = range(7)
MF_F32, MF_F16, MF_BF16, MF_F16X2 = 0, 1, 2, 3  # MF_F16X2: intermediates only (FP16 pairs)
STATUS_NAMES = {0: "MF_OK", 1: "MF_EINVAL", 2: "MF_ENOMEM", 3: "MF_ECUDA", 4: "MF_ESTATE", 5: "MF_EOVERFLOW",
                6: "MF_ETIMEOUT"}


class mf_plan_desc(C.Structure):
    _fields_ = [("fs", C.c_double), ("n", C.c_int64), ("n_det", C.c_int32), ("f_low", C.c_double),
                ("f_high", C.c_double), ("dtype", C.c_int), ("snr_thr", C.c_double), ("window", C.c_int64),
                ("valid_begin", C.c_int64), ("valid_end", C.c_int64), ("max_triggers", C.c_int64),
                ("cuda_stream", C.c_void_p)]


class mf_trigger(C.Structure):
    _fields_ = [("det", C.c_int32), ("tmpl", C.c_int32), ("sample", C.c_int64), ("snr", C.c_float),
                ("phase", C.c_float)]


class mf_coinc_desc(C.Structure):
    _fields_ = [("shift_samples", C.c_int64), ("n_shifts", C.c_int32), ("window_samples", C.c_int64),
                ("rho_c_thr", C.c_double), ("rho_c_store", C.c_double), ("max_coincs", C.c_int64)]


class mf_coinc(C.Structure):
    _fields_ = [("tmpl", C.c_int32), ("shift", C.c_int32), ("sample0", C.c_int64), ("sample1", C.c_int64),
                ("snr0", C.c_float), ("snr1", C.c_float), ("rho_c", C.c_float), ("reserved", C.c_int32)]


class mf_plan_stats(C.Structure):
    _fields_ = [("launches", C.c_int64), ("pass1_launches", C.c_int64), ("pass1_series", C.c_int64),
                ("pass1_ms", C.c_double), ("pass2_launches", C.c_int64), ("pass2_series", C.c_int64),
                ("pass2_ms", C.c_double), ("impl", C.c_int32), ("batch", C.c_int32)]


class mf_batch_desc(C.Structure):
    _fields_ = [("fs", C.c_double), ("n_det", C.c_int32), ("n_samples", C.c_int64), ("f_low", C.c_double),
                ("f_high", C.c_double), ("snr_thr", C.c_double), ("window", C.c_int64), ("n_class", C.c_int32),
                ("class_len", C.POINTER(C.c_double)), ("max_triggers", C.c_int64), ("cuda_stream", C.c_void_p)]


class mf_batch_trigger(C.Structure):
    _fields_ = [("det", C.c_int32), ("cls", C.c_int32), ("tmpl", C.c_int32), ("reserved", C.c_int32),
                ("sample", C.c_int64), ("snr", C.c_float), ("phase", C.c_float)]


MF_RUN_SERIAL, MF_RUN_STREAMS, MF_RUN_GRAPH, MF_RUN_FUSED, MF_RUN_FUSED_GRAPH = 0, 1, 2, 3, 4
BATCH_TRIGGER_NP = np.dtype([("det", np.int32), ("cls", np.int32), ("tmpl", np.int32), ("reserved", np.int32),
                             ("sample", np.int64), ("snr", np.float32), ("phase", np.float32)])

TRIGGER_NP = np.dtype([("det", np.int32), ("tmpl", np.int32), ("sample", np.int64), ("snr", np.float32),
                       ("phase", np.float32)])
COINC_NP = np.dtype([("tmpl", np.int32), ("shift", np.int32), ("sample0", np.int64), ("sample1", np.int64),
                     ("snr0", np.float32), ("snr1", np.float32), ("rho_c", np.float32), ("reserved", np.int32)])
assert TRIGGER_NP.itemsize == C.sizeof(mf_trigger) == 24
assert COINC_NP.itemsize == C.sizeof(mf_coinc) == 40

_P = C.c_void_p
_I64 = C.c_int64
# name -> (restype, argtypes)
SIGNATURES = {
    "mf_plan": (C.c_int, [C.POINTER(_P), C.POINTER(mf_plan_desc)]),
    "mf_destroy": (None, [_P]),
    "mf_last_error": (C.c_char_p, [_P]),
    "mf_set_psd": (C.c_int, [_P, _P, _I64]),
    "mf_load_bank": (C.c_int, [_P, _P, C.c_int, _I64, _I64, _P, C.c_int]),
    "mf_bank_reserve": (C.c_int, [_P, C.c_int, _I64]),
    "mf_bank_set_rows": (C.c_int, [_P, _I64, _I64, _P, _I64, _P, C.c_int]),
    "mf_get_sigmasq": (C.c_int, [_P, _P, _I64]),
    "mf_bank_quantize_rows": (C.c_int, [_P, _I64, _I64, _P, _I64, C.c_int]),
    "mf_set_data_dtype": (C.c_int, [_P, C.c_int]),
    "mf_set_intermediate": (C.c_int, [_P, C.c_int]),
    "mf_taylorf2": (C.c_int, [_P, _P, C.c_int64, C.c_double, C.c_int64, C.c_double, _P, C.c_int64, _P]),
    "mf_bank_generate_taylorf2": (C.c_int, [_P, C.c_int64, C.c_int64, _P, _P, C.c_double]),
    "mf_set_row_valid": (C.c_int, [_P, _P]),
    "mf_selftest_wait": (C.c_int, [_P, C.POINTER(C.c_int32)]),
    "mf_chisq": (C.c_int, [_P, C.c_int32, _P, _P]),
    "mf_psd_welch": (C.c_int, [C.c_double, C.c_int32, _I64, _P, _I64, _I64, _I64, C.c_int32, _P, _P]),
    "mf_fma_probe": (C.c_int, [C.POINTER(C.c_double), _P]),
    "mf_far": (C.c_int, [_P, _I64, _P, _I64, C.c_double, C.c_double, C.c_double, _P, _P, _P, _P]),
    "mf_batch_create": (C.c_int, [C.POINTER(_P), C.POINTER(mf_batch_desc)]),
    "mf_batch_destroy": (None, [_P]),
    "mf_batch_last_error": (C.c_char_p, [_P]),
    "mf_batch_set_psd": (C.c_int, [_P, _P, _I64]),
    "mf_batch_set_segment": (C.c_int, [_P, C.c_int32, _I64, C.c_int32]),
    "mf_batch_autotune": (C.c_int, [_P, _P]),
    "mf_batch_autotune_fused": (C.c_int, [_P, _P]),
    "mf_batch_segment": (C.c_int, [_P, C.c_int32, C.POINTER(_I64), C.POINTER(_I64), C.POINTER(_I64),
                                   C.POINTER(_I64), C.POINTER(C.c_double), C.POINTER(C.c_double)]),
    "mf_batch_plan": (C.c_int, [_P, C.c_int32, C.POINTER(_P)]),
    "mf_batch_run": (C.c_int, [_P, _P, _I64, C.c_int32]),
    "mf_batch_get_triggers": (C.c_int, [_P, _P, _I64, C.POINTER(_I64)]),
    "mf_set_batch": (C.c_int, [_P, C.c_int32]),
    "mf_strain_to_fd": (C.c_int, [_P, _P, _I64, _P, _I64]),
    "mf_decimate": (C.c_int, [_P, _P, _I64, _P, _I64]),
    "mf_filter": (C.c_int, [_P, _P, _I64, _P, _I64]),
    "mf_get_triggers": (C.c_int, [_P, _P, _I64, C.POINTER(_I64)]),
    "mf_device_triggers": (C.c_int, [_P, C.POINTER(_P), C.POINTER(_P)]),
    "mf_load_gate_template": (C.c_int, [_P]),
    "mf_sgchisq": (C.c_int, [_P, _P, _P, C.c_float, C.c_float, C.c_int32, _P, C.c_double, _P, _P, _P]),
    "mf_gate_apply": (C.c_int, [_P, _I64, C.c_int32, _I64, C.c_double, _P, _P, _I64, C.c_double, C.c_double, _P,
                                _I64, _P]),
    "mf_coincide": (C.c_int, [_P, C.POINTER(mf_coinc_desc), _P]),
    "mf_get_coincs": (C.c_int, [_P, _P, _I64, C.POINTER(_I64)]),
    "mf_set_nbhd": (C.c_int, [_P, _P, _P, _I64, C.c_int]),
    "mf_nbhd_union": (C.c_int, [_P, _P, _P, C.POINTER(_I64)]),
    "mf_profile": (C.c_int, [_P, C.c_int]),
    "mf_mlp_create": (C.c_int, [C.POINTER(_P), C.c_int32, C.c_int32, C.c_int32, C.c_int32, _I64, _P]),
    "mf_mlp_destroy": (None, [_P]),
    "mf_mlp_num_params": (_I64, [_P]),
    "mf_mlp_set_params": (C.c_int, [_P, _P, _I64, C.c_int]),
    "mf_mlp_get_params": (C.c_int, [_P, _P, _I64]),
    "mf_mlp_forward": (C.c_int, [_P, _P, _I64, _P]),
    "mf_mlp_loss_grad": (C.c_int, [_P, _P, _P, _P, _I64, _P, _P]),
    "mf_mlp_adamw_step": (C.c_int, [_P, C.c_float, C.c_float, C.c_float, C.c_float, C.c_float]),
    "mf_mlp_topk": (C.c_int, [_P, _P, _P, _I64, C.c_int32, C.c_float, _P, _P]),
    "mf_mlp_last_error": (C.c_char_p, [_P]),
    "mf_filter_noalloc": (C.c_int, [C.c_double, _I64, C.c_int32, C.c_double, C.c_double, C.c_double, _I64, _P, _P,
                                    _I64, _I64, _P, _I64, _P, _I64, _P, _P]),
    "mf_get_stats": (C.c_int, [_P, C.POINTER(mf_plan_stats), C.c_int]),
}

_lib = None


class MFError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


def load(path=LIB_PATH):
    """Load libmf.so (built by ``__graft_entry__.build()``); raises if absent."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise FileNotFoundError(f"libmf.so not found at {path}: build it with __graft_entry__.build()")
    lib = C.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib


def _check(plan, st, ok=(MF_OK,)):
    if st not in ok:
        msg = load().mf_last_error(plan)
        raise MFError(st, msg.decode() if msg else "")
    return st


def _ptr(x):
    """Address of a torch tensor, numpy array or integer."""
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if hasattr(x, "data_ptr"):
        return x.data_ptr()
    if isinstance(x, np.ndarray):
        return x.ctypes.data
    raise TypeError(f"cannot take the address of {type(x)}")


class Plan:
    """Owner of one ``mf_plan_t``; methods mirror the C calls."""

    def __init__(self, fs, n, n_det, f_low, f_high, snr_thr, window, valid_begin=0, valid_end=None,
                 dtype=MF_F32, max_triggers=1 << 20, stream=None):
        lib = load()
        d = mf_plan_desc(fs=fs, n=n, n_det=n_det, f_low=f_low, f_high=f_high, dtype=dtype, snr_thr=snr_thr,
                         window=window, valid_begin=valid_begin, valid_end=n if valid_end is None else valid_end,
                         max_triggers=max_triggers, cuda_stream=stream)
        h = _P()
        _check(None, lib.mf_plan(C.byref(h), C.byref(d)))
        self.h = h
        self.desc = d
        self.n, self.nb, self.n_det, self.n_tmpl = n, n // 2 + 1, n_det, 0
        self.lib = lib

    @classmethod
    def borrowed(cls, handle, desc):
        """A view of a plan owned by someone else (a Batch): never destroyed here."""
        self = cls.__new__(cls)
        self.h, self.desc, self.lib = handle, desc, load()
        self.n, self.nb, self.n_det, self.n_tmpl = desc.n, desc.n // 2 + 1, desc.n_det, 0
        self._borrowed = True
        return self

    def close(self):
        if getattr(self, "h", None) and not getattr(self, "_borrowed", False):
            self.lib.mf_destroy(self.h)
        self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_psd(self, psd):
        psd = np.ascontiguousarray(psd, dtype=np.float64)
        _check(self.h, self.lib.mf_set_psd(self.h, psd.ctypes.data, len(psd)))

    def load_bank(self, htilde, dtype=MF_F32, ld=None, scales=None, on_device=None):
        n_tmpl = htilde.shape[0]
        ld = htilde.shape[1] if ld is None else ld
        if on_device is None:
            on_device = 0 if isinstance(htilde, np.ndarray) else int(htilde.is_cuda)
        sc = None if scales is None else np.ascontiguousarray(scales, dtype=np.float32)
        _check(self.h, self.lib.mf_load_bank(self.h, _ptr(htilde), dtype, n_tmpl, ld, _ptr(sc), on_device))
        self.n_tmpl = n_tmpl

    def bank_reserve(self, n_tmpl, dtype=MF_F32):
        _check(self.h, self.lib.mf_bank_reserve(self.h, dtype, n_tmpl))
        self.n_tmpl = n_tmpl

    def bank_set_rows(self, row0, rows, ld=None, scales=None, on_device=None):
        ld = rows.shape[1] if ld is None else ld
        if on_device is None:
            on_device = 0 if isinstance(rows, np.ndarray) else int(rows.is_cuda)
        sc = None if scales is None else np.ascontiguousarray(scales, dtype=np.float32)
        _check(self.h, self.lib.mf_bank_set_rows(self.h, row0, rows.shape[0], _ptr(rows), ld, _ptr(sc), on_device))

    def bank_quantize_rows(self, row0, rows, ld=None, on_device=None):
        """Quantise complex64 template rows into the plan's 16-bit bank."""
        ld = rows.shape[1] if ld is None else ld
        if on_device is None:
            on_device = 0 if isinstance(rows, np.ndarray) else int(rows.is_cuda)
        _check(self.h, self.lib.mf_bank_quantize_rows(self.h, row0, rows.shape[0], _ptr(rows), ld, on_device))

    def set_data_dtype(self, dtype):
        _check(self.h, self.lib.mf_set_data_dtype(self.h, dtype))

    def set_intermediate(self, dtype):
        _check(self.h, self.lib.mf_set_intermediate(self.h, dtype))

    def bank_generate_taylorf2(self, row0, m1, m2, f_low):
        m1 = np.ascontiguousarray(m1, dtype=np.float64)
        m2 = np.ascontiguousarray(m2, dtype=np.float64)
        _check(self.h, self.lib.mf_bank_generate_taylorf2(self.h, row0, len(m1), m1.ctypes.data, m2.ctypes.data,
                                                          f_low))

    def set_row_valid(self, ranges):
        """Per-row analysed ranges, int64 [n_det, 2] (None restores the plan's range)."""
        r = None if ranges is None else np.ascontiguousarray(ranges, dtype=np.int64)
        _check(self.h, self.lib.mf_set_row_valid(self.h, _ptr(r)))

    def chisq(self, n_bands, chi2, newsnr):
        """chi^2 and the re-weighted SNR of the last filter's triggers into device float arrays."""
        _check(self.h, self.lib.mf_chisq(self.h, n_bands, _ptr(chi2), _ptr(newsnr)))

    def sgchisq(self, f_final, mtotal, snr_in, chi2_r, snr_hat, m_min=30.0, snr_min=0.0,
                offsets=(15.0, 30.0, 45.0, 60.0, 75.0, 90.0, 105.0, 120.0), q=20.0):
        """Sine-Gaussian veto of the last filter's triggers (mf_sgchisq): f_final, mtotal device float
        [n_tmpl]; snr_in, chi2_r, snr_hat device float [max_triggers]."""
        off = np.ascontiguousarray(offsets, dtype=np.float64)
        _check(self.h, self.lib.mf_sgchisq(self.h, _ptr(f_final), _ptr(mtotal), float(m_min), float(snr_min),
                                           len(off), off.ctypes.data, float(q), _ptr(snr_in), _ptr(chi2_r),
                                           _ptr(snr_hat)))

    def selftest_wait(self):
        """Run the bounded-wait self-test; returns the number of threads that came back."""
        r = C.c_int32(0)
        _check(self.h, self.lib.mf_selftest_wait(self.h, C.byref(r)))
        return r.value

    def set_batch(self, batch):
        _check(self.h, self.lib.mf_set_batch(self.h, batch))

    def sigmasq(self, n=None):
        n = self.n_tmpl if n is None else n
        out = np.zeros(n, dtype=np.float64)
        _check(self.h, self.lib.mf_get_sigmasq(self.h, out.ctypes.data, n))
        return out

    def strain_to_fd(self, strain, dtilde, ld_strain=None, ld_dtilde=None):
        ld_strain = strain.shape[-1] if ld_strain is None else ld_strain
        ld_dtilde = dtilde.shape[-1] if ld_dtilde is None else ld_dtilde
        _check(self.h, self.lib.mf_strain_to_fd(self.h, _ptr(strain), ld_strain, _ptr(dtilde), ld_dtilde))

    def decimate(self, dtilde_in, dtilde_out, ld_in=None, ld_out=None):
        ld_in = dtilde_in.shape[-1] if ld_in is None else ld_in
        ld_out = dtilde_out.shape[-1] if ld_out is None else ld_out
        _check(self.h, self.lib.mf_decimate(self.h, _ptr(dtilde_in), ld_in, _ptr(dtilde_out), ld_out))

    def filter(self, dtilde, subset=None, n_subset=None, ld=None):
        ld = dtilde.shape[-1] if ld is None else ld
        if subset is None:
            n_subset = -1
        elif n_subset is None:
            n_subset = subset.shape[0]
        sp = _ptr(subset) if (subset is not None and n_subset > 0) else None
        _check(self.h, self.lib.mf_filter(self.h, _ptr(dtilde), ld, sp, n_subset))

    def _host_buffer(self, name, count, dtype, pinned):
        """Host array of `count` records: a fresh one, or (pinned) a view of a page-locked buffer the
        plan keeps and reuses (valid until the next call that uses it)."""
        if not pinned:
            return np.empty(count, dtype=dtype)
        import torch

        need = count * dtype.itemsize
        buf = getattr(self, name, None)
        if buf is None or buf.numel() < need:
            buf = torch.empty(max(need, 1), dtype=torch.uint8, pin_memory=True)
            setattr(self, name, buf)
        return buf.numpy()[:need].view(dtype)

    def triggers(self, cap=None, pinned=False):
        """Triggers of the last filter (mf_get_triggers).  pinned: read into a page-locked buffer
        of the plan (faster; the array is overwritten by the next pinned call)."""
        n = _I64(0)
        if cap is None:
            _check(self.h, self.lib.mf_get_triggers(self.h, None, 0, C.byref(n)), ok=(MF_OK, MF_EOVERFLOW))
            cap = n.value
        out = self._host_buffer("_pinned_trig", cap, TRIGGER_NP, pinned)
        st = self.lib.mf_get_triggers(self.h, out.ctypes.data if cap else None, cap, C.byref(n))
        _check(self.h, st, ok=(MF_OK, MF_EOVERFLOW))
        return out[: min(cap, n.value, self.desc.max_triggers)], n.value, st

    def load_gate_template(self):
        """One-row bank sqrt(S_n) on the band: filter() then finds the gates (mf_load_gate_template)."""
        _check(self.h, self.lib.mf_load_gate_template(self.h))

    def device_triggers(self):
        t, c = _P(), _P()
        _check(self.h, self.lib.mf_device_triggers(self.h, C.byref(t), C.byref(c)))
        return t.value, c.value

    def coincide(self, followed, shift_samples, n_shifts, window_samples, rho_c_thr, rho_c_store=None,
                 max_coincs=1 << 20):
        d = mf_coinc_desc(shift_samples=shift_samples, n_shifts=n_shifts, window_samples=window_samples,
                          rho_c_thr=rho_c_thr, rho_c_store=rho_c_thr if rho_c_store is None else rho_c_store,
                          max_coincs=max_coincs)
        _check(self.h, self.lib.mf_coincide(self.h, C.byref(d), _ptr(followed)))
        self.coinc_cap = max(getattr(self, "coinc_cap", 0), max_coincs)

    def coincs(self, cap=None, pinned=False):
        n = _I64(0)
        if cap is None:
            _check(self.h, self.lib.mf_get_coincs(self.h, None, 0, C.byref(n)), ok=(MF_OK, MF_EOVERFLOW))
            cap = n.value
        out = self._host_buffer("_pinned_coinc", cap, COINC_NP, pinned)
        st = self.lib.mf_get_coincs(self.h, out.ctypes.data if cap else None, cap, C.byref(n))
        _check(self.h, st, ok=(MF_OK, MF_EOVERFLOW))
        return out[: min(cap, n.value, getattr(self, "coinc_cap", cap))], n.value, st

    def set_nbhd(self, ptr, idx):
        ptr = np.ascontiguousarray(ptr, dtype=np.int64)
        idx = np.ascontiguousarray(idx, dtype=np.int32)
        _check(self.h, self.lib.mf_set_nbhd(self.h, ptr.ctypes.data, idx.ctypes.data if len(idx) else None,
                                            len(ptr) - 1, 0))

    def nbhd_union(self, followed, subset):
        n = _I64(0)
        _check(self.h, self.lib.mf_nbhd_union(self.h, _ptr(followed), _ptr(subset), C.byref(n)))
        return n.value

    def profile(self, enable=True):
        """mf_profile: False / 0 off, True / 1 every launch pair, k > 1 every k-th launch pair."""
        _check(self.h, self.lib.mf_profile(self.h, int(enable)))

    def stats(self, reset=False):
        st = mf_plan_stats()
        _check(self.h, self.lib.mf_get_stats(self.h, C.byref(st), int(reset)))
        return {f: getattr(st, f) for f, _ in mf_plan_stats._fields_}


class MLP:
    """Owner of one ``mf_mlp_t`` (learned proposal network); methods mirror the C calls."""

    def __init__(self, n_in, width, depth, n_out, max_batch, stream=None):
        lib = load()
        h = _P()
        _check(None, lib.mf_mlp_create(C.byref(h), n_in, width, depth, n_out, max_batch, stream))
        self.h, self.lib = h, lib
        self.dims = (n_in, width, depth, n_out)
        self.n_params = lib.mf_mlp_num_params(h)

    def _chk(self, st):
        if st != MF_OK:
            msg = self.lib.mf_mlp_last_error(self.h)
            raise MFError(st, msg.decode() if msg else "")

    def close(self):
        if getattr(self, "h", None):
            self.lib.mf_mlp_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_params(self, theta):
        if isinstance(theta, np.ndarray):
            t = np.ascontiguousarray(theta, dtype=np.float32)
            self._chk(self.lib.mf_mlp_set_params(self.h, t.ctypes.data, len(t), 0))
        else:
            self._chk(self.lib.mf_mlp_set_params(self.h, _ptr(theta), theta.numel(), 1))

    def get_params(self):
        out = np.zeros(self.n_params, dtype=np.float32)
        self._chk(self.lib.mf_mlp_get_params(self.h, out.ctypes.data, self.n_params))
        return out

    def forward(self, x, logits=None):
        self._chk(self.lib.mf_mlp_forward(self.h, _ptr(x), x.shape[0], _ptr(logits)))

    def loss_grad(self, x, n_valid, label, loss=None, grad=None):
        self._chk(self.lib.mf_mlp_loss_grad(self.h, _ptr(x), _ptr(n_valid), _ptr(label), x.shape[0], _ptr(loss),
                                            _ptr(grad)))

    def adamw_step(self, lr, beta1=0.9, beta2=0.999, eps=1e-8, weight_decay=0.0):
        self._chk(self.lib.mf_mlp_adamw_step(self.h, lr, beta1, beta2, eps, weight_decay))

    def topk(self, x, n_valid, k, out, p_mass=2.0, count=None):
        self._chk(self.lib.mf_mlp_topk(self.h, _ptr(x), _ptr(n_valid), x.shape[0], k, p_mass, _ptr(out),
                                       _ptr(count)))


def _bcheck(batch, st, ok=(MF_OK,)):
    if st not in ok:
        msg = load().mf_batch_last_error(batch)
        raise MFError(st, msg.decode() if msg else "")
    return st


class Batch:
    """Owner of one ``mf_batch_t``: long data in overlapping segments, one plan
    per template-length class (include/mf.h)."""

    def __init__(self, fs, n_det, n_samples, f_low, f_high, snr_thr, window, class_len, max_triggers=1 << 22,
                 stream=None):
        lib = load()
        self._len = (C.c_double * len(class_len))(*class_len)
        d = mf_batch_desc(fs=fs, n_det=n_det, n_samples=n_samples, f_low=f_low, f_high=f_high, snr_thr=snr_thr,
                          window=window, n_class=len(class_len), class_len=self._len, max_triggers=max_triggers,
                          cuda_stream=stream)
        h = _P()
        _bcheck(None, lib.mf_batch_create(C.byref(h), C.byref(d)))
        self.h, self.desc, self.lib = h, d, lib
        self.n_class = len(class_len)

    def close(self):
        if getattr(self, "h", None):
            self.lib.mf_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_psd(self, psd, n_psd):
        psd = np.ascontiguousarray(psd, dtype=np.float64)
        assert len(psd) == n_psd // 2 + 1
        _bcheck(self.h, self.lib.mf_batch_set_psd(self.h, psd.ctypes.data, n_psd))

    def set_segment(self, cls, n, per_launch=0):
        _bcheck(self.h, self.lib.mf_batch_set_segment(self.h, cls, n, per_launch))

    def autotune(self, n_tmpl, fused=False):
        """Segment length and launch batch per class (fused: one segment length for all, for MF_RUN_FUSED)."""
        a = np.ascontiguousarray(n_tmpl, dtype=np.int64)
        fn = self.lib.mf_batch_autotune_fused if fused else self.lib.mf_batch_autotune
        _bcheck(self.h, fn(self.h, a.ctypes.data))

    def segment(self, cls):
        v = [_I64() for _ in range(4)]
        e, r = C.c_double(), C.c_double()
        _bcheck(self.h, self.lib.mf_batch_segment(self.h, cls, *[C.byref(x) for x in v], C.byref(e), C.byref(r)))
        return dict(n=v[0].value, tmpl_len=v[1].value, stride=v[2].value, n_seg=v[3].value, est_ms=e.value,
                    run_ms=r.value)

    def plan(self, cls):
        """The class's plan (a borrowed Plan: load its bank with bank_reserve / bank_set_rows / ...)."""
        h = _P()
        _bcheck(self.h, self.lib.mf_batch_plan(self.h, cls, C.byref(h)))
        g = self.segment(cls)
        d = mf_plan_desc(fs=self.desc.fs, n=g["n"], n_det=g["n_seg"] * self.desc.n_det, f_low=self.desc.f_low,
                         f_high=self.desc.f_high, dtype=MF_F32, snr_thr=self.desc.snr_thr, window=self.desc.window,
                         valid_begin=g["tmpl_len"], valid_end=g["n"], max_triggers=self.desc.max_triggers,
                         cuda_stream=None)
        return Plan.borrowed(h, d)

    def run(self, strain, ld=None, mode=None):
        """mf_batch_run; mode None: the fused work queue under a captured graph (MF_RUN_FUSED_GRAPH) when every
        class with a plan has the same segment length (the fused queue also needs FP32 banks and data), else the
        classes one after another (MF_RUN_SERIAL)."""
        ld = strain.shape[-1] if ld is None else ld
        if mode is None:
            ns = {self.segment(ci)["n"] for ci in range(self.n_class)} - {0}
            mode = MF_RUN_FUSED_GRAPH if len(ns) == 1 else MF_RUN_SERIAL
        _bcheck(self.h, self.lib.mf_batch_run(self.h, _ptr(strain), ld, mode))

    def triggers(self):
        n = _I64(0)
        _bcheck(self.h, self.lib.mf_batch_get_triggers(self.h, None, 0, C.byref(n)), ok=(MF_OK, MF_EOVERFLOW))
        out = np.zeros(n.value, dtype=BATCH_TRIGGER_NP)
        st = self.lib.mf_batch_get_triggers(self.h, out.ctypes.data if n.value else None, n.value, C.byref(n))
        _bcheck(self.h, st, ok=(MF_OK, MF_EOVERFLOW))
        return out, n.value, st


def far(stat_fg, stat_bg, t_bg, scale=1.0, fit_min=None):
    """mf_far: (far_count, far_fit, alpha, beta) for foreground / background statistics."""
    lib = load()
    fg = np.ascontiguousarray(stat_fg, dtype=np.float32)
    bg = np.ascontiguousarray(stat_bg, dtype=np.float32)
    fc = np.zeros(len(fg))
    ff = np.zeros(len(fg))
    a, b = C.c_double(), C.c_double()
    fm = float(np.min(bg)) if fit_min is None and len(bg) else (0.0 if fit_min is None else fit_min)
    _check(None, lib.mf_far(_ptr(fg) if len(fg) else None, len(fg), _ptr(bg) if len(bg) else None, len(bg),
                            float(t_bg), float(scale), fm, _ptr(fc) if len(fg) else None,
                            _ptr(ff) if len(fg) else None, C.byref(a), C.byref(b)))
    return fc, ff, a.value, b.value


def psd_welch(strain, fs, seg_len, stride, average="median", out=None, stream=None):
    """mf_psd_welch on a device float32 tensor [n_det, n_samples]; returns the device float64 PSD [n_det, seg_len/2+1]."""
    import torch

    n_det, n_samples = strain.shape
    ld = strain.stride(0) if n_det > 1 else n_samples  # a single row's stride may be reported as 0
    if strain.stride(1) != 1:
        raise ValueError("psd_welch: rows must be contiguous")
    if out is None:
        out = torch.zeros((n_det, seg_len // 2 + 1), dtype=torch.float64, device=strain.device)
    _check(None, load().mf_psd_welch(float(fs), n_det, n_samples, _ptr(strain), ld, seg_len, stride,
                                     0 if average == "mean" else 1, _ptr(out), stream))
    return out


def gate_apply(strain, gate_plan, t_zero, t_taper, out=None, stream=None):
    """mf_gate_apply: device float32 strain [n_det, n] times the inverse Tukey windows of the
    gates found by gate_plan's last filter (a plan loaded with load_gate_template); returns out."""
    import torch

    n_det, n = strain.shape
    ld = strain.stride(0) if n_det > 1 else n
    if strain.stride(1) != 1:
        raise ValueError("gate_apply: rows must be contiguous")
    if out is None:
        out = torch.empty_like(strain)
    ld_out = out.stride(0) if n_det > 1 else n
    t, c = gate_plan.device_triggers()
    _check(None, load().mf_gate_apply(_ptr(strain), ld, n_det, n, float(gate_plan.desc.fs), t, c,
                                      gate_plan.desc.max_triggers, float(t_zero), float(t_taper), _ptr(out), ld_out,
                                      stream))
    return out


def fma_probe(stream=None):
    """Measured FP32 FMA throughput of the device, TFLOP/s (mf_fma_probe)."""
    t = C.c_double()
    _check(None, load().mf_fma_probe(C.byref(t), stream))
    return t.value
