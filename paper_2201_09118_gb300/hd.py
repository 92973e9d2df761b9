"""Thin ctypes binding of libhd.so (include/hd.h).

Argument marshalling only: every step of the decode path runs in the library's
CUDA kernels.  Device buffers and streams come from PyTorch.  If the library
cannot be loaded the import of any function here raises; there is no fallback.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass
from typing import Optional, Sequence

import numpy as np

from . import build as _build

HD_OK = 0
HD_PENDING = 1
HD_ERR_ARG = -1
HD_ERR_CAPACITY = -2
HD_ERR_SYMBOL = -3
HD_ERR_CORRUPT = -4
HD_ERR_NOSYNC = -5
HD_ERR_TIMEOUT = -6
HD_ERR_CUDA = -7
HD_ERR_NOMEM = -8
HD_ERR_BUSY = -9

_NAMES = {
    0: "HD_OK", 1: "HD_PENDING", -1: "HD_ERR_ARG", -2: "HD_ERR_CAPACITY", -3: "HD_ERR_SYMBOL",
    -4: "HD_ERR_CORRUPT", -5: "HD_ERR_NOSYNC", -6: "HD_ERR_TIMEOUT", -7: "HD_ERR_CUDA",
    -8: "HD_ERR_NOMEM", -9: "HD_ERR_BUSY",
}


class HDError(RuntimeError):
    def __init__(self, fn: str, code: int):
        super().__init__(f"{fn} returned {_NAMES.get(code, code)}")
        self.code = code


class hd_stream_info(ctypes.Structure):
    _fields_ = [("nbits", ctypes.c_uint64), ("nwords", ctypes.c_uint64),
                ("nsub", ctypes.c_uint64)]


class hd_field(ctypes.Structure):
    _fields_ = [("words", ctypes.c_void_p), ("nwords", ctypes.c_uint64),
                ("nbits", ctypes.c_uint64), ("gap", ctypes.c_void_p),
                ("subseq_bits", ctypes.c_uint32), ("lengths", ctypes.c_void_p),
                ("alphabet", ctypes.c_uint32), ("n", ctypes.c_uint64)]


class hd_config(ctypes.Structure):
    _fields_ = [("subseq_bits", ctypes.c_uint32), ("threads", ctypes.c_uint32),
                ("window", ctypes.c_uint32), ("lut_bits", ctypes.c_uint32),
                ("cr_classes", ctypes.c_uint32), ("decoder", ctypes.c_uint32)]


class hd_serve_config(ctypes.Structure):
    _fields_ = [("budget_bytes", ctypes.c_uint64), ("slots", ctypes.c_uint32),
                ("max_batch", ctypes.c_uint32), ("queue_cap", ctypes.c_uint32),
                ("direct", ctypes.c_uint32), ("watchdog_us", ctypes.c_uint32)]


class hd_result(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int32), ("d_out", ctypes.c_void_p), ("n", ctypes.c_uint64),
                ("queue_us", ctypes.c_double), ("latency_us", ctypes.c_double)]


class hd_serve_stats_t(ctypes.Structure):
    _fields_ = [(k, ctypes.c_uint64) for k in ("submitted", "completed", "batches", "pending",
                                                "in_flight", "budget_bytes", "used_bytes",
                                                "peak_bytes", "timed_out_batches",
                                                "retired_batches")]


class hd_lorenzo(ctypes.Structure):
    _fields_ = [("ndim", ctypes.c_uint32), ("radius", ctypes.c_uint32),
                ("dims", ctypes.c_uint64 * 3), ("eb", ctypes.c_double),
                ("out_idx", ctypes.c_void_p), ("out_val", ctypes.c_void_p),
                ("n_out", ctypes.c_uint64), ("chunk_slices", ctypes.c_uint32),
                ("band_rows", ctypes.c_uint32), ("separate", ctypes.c_uint32),
                ("pad", ctypes.c_uint32)]


def lorenzo_params(dims, radius: int, eb: float, out_idx=None, out_val=None,
                   chunk_slices: int = 0, band_rows: int = 0, separate: bool = False) -> hd_lorenzo:
    """hd_lorenzo for a grid (dims[0] fastest) and device outlier tensors."""
    L = hd_lorenzo()
    L.ndim = len(dims)
    for k, v in enumerate(dims):
        L.dims[k] = int(v)
    L.radius = int(radius)
    L.eb = float(eb)
    n_out = 0 if out_idx is None else int(out_idx.numel())
    L.out_idx = out_idx.data_ptr() if n_out else None
    L.out_val = out_val.data_ptr() if n_out else None
    L.n_out = n_out
    L.chunk_slices = int(chunk_slices)
    L.band_rows = int(band_rows)
    L.separate = 1 if separate else 0
    return L


# every exported symbol of include/hd.h with its ctypes signature
_P = ctypes.c_void_p
_SIGS = {
    "hd_build_codebook": ([_P, ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint32, _P],
                          ctypes.c_int),
    "hd_encode": ([_P, ctypes.c_uint64, _P, ctypes.c_uint32, ctypes.c_uint32, _P,
                   ctypes.c_uint64, _P, ctypes.c_uint64, ctypes.POINTER(hd_stream_info)],
                  ctypes.c_int),
    "hd_build_codebook_freq": ([_P, ctypes.c_uint32, ctypes.c_uint32, _P], ctypes.c_int),
    "hd_histogram_device": ([_P, _P, ctypes.c_uint64, ctypes.c_uint32, _P, _P], ctypes.c_int),
    "hd_encode_device": ([_P, _P, ctypes.c_uint64, _P, ctypes.c_uint32, ctypes.c_uint32, _P,
                          ctypes.c_uint64, _P, ctypes.c_uint64, ctypes.POINTER(hd_stream_info),
                          _P], ctypes.c_int),
    "hd_reconstruct_device": ([_P, _P, ctypes.POINTER(hd_lorenzo), _P, _P], ctypes.c_int),
    "hd_decompress_device": ([_P, ctypes.POINTER(hd_field), ctypes.POINTER(hd_lorenzo), _P, _P],
                             ctypes.c_int),
    "hd_ctx_create": ([ctypes.c_int, ctypes.POINTER(_P)], ctypes.c_int),
    "hd_ctx_destroy": ([_P], ctypes.c_int),
    "hd_set_config": ([_P, ctypes.POINTER(hd_config)], ctypes.c_int),
    "hd_get_config": ([_P, ctypes.POINTER(hd_config)], ctypes.c_int),
    "hd_decode": ([_P, ctypes.POINTER(hd_field), _P, _P], ctypes.c_int),
    "hd_status": ([_P, _P], ctypes.c_int),
    "hd_sync_points": ([_P, ctypes.POINTER(hd_field), _P, _P], ctypes.c_int),
    "hd_inspect_tables": ([_P, _P, ctypes.c_uint32, ctypes.c_uint32, _P, _P, _P, _P, _P],
                          ctypes.c_int),
    "hd_decode_batch": ([_P, ctypes.POINTER(hd_field), ctypes.c_uint32, _P, _P], ctypes.c_int),
    "hd_batch_status": ([_P, _P, ctypes.c_uint32, _P], ctypes.c_int),
    "hd_decode_host": ([_P, ctypes.POINTER(hd_field), _P, _P], ctypes.c_int),
    "hd_decode_static": ([ctypes.POINTER(hd_field), _P, _P], ctypes.c_int),
    "hd_profile": ([_P, ctypes.c_int], ctypes.c_int),
    "hd_phase_times": ([_P, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_uint64)],
                       ctypes.c_int),
    "hd_set_wait_limit": ([_P, ctypes.c_uint64], ctypes.c_int),
    "hd_autotune_save": ([_P, ctypes.c_char_p], ctypes.c_int),
    "hd_autotune_load": ([_P, ctypes.c_char_p, ctypes.POINTER(ctypes.c_uint32)], ctypes.c_int),
    "hd_kernel_time": ([_P, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_uint64)],
                       ctypes.c_int),
    "hd_launch_count": ([_P], ctypes.c_uint64),
    "hd_autotune": ([_P, ctypes.POINTER(hd_field), ctypes.c_uint32, _P, _P,
                     ctypes.POINTER(hd_config)], ctypes.c_int),
    "hd_graph_stats": ([_P, ctypes.POINTER(ctypes.c_uint64), ctypes.POINTER(ctypes.c_uint32)],
                       ctypes.c_int),
    "hd_serve_create": ([ctypes.c_int, ctypes.POINTER(hd_serve_config), ctypes.POINTER(hd_config),
                         ctypes.POINTER(_P)], ctypes.c_int),
    "hd_serve_destroy": ([_P], ctypes.c_int),
    "hd_serve_register": ([_P, ctypes.POINTER(hd_field), ctypes.POINTER(ctypes.c_uint32)],
                          ctypes.c_int),
    "hd_serve_submit": ([_P, ctypes.c_uint32, ctypes.POINTER(ctypes.c_uint64)], ctypes.c_int),
    "hd_serve_poll": ([_P, ctypes.c_uint64, ctypes.POINTER(hd_result)], ctypes.c_int),
    "hd_serve_release": ([_P, ctypes.c_uint64], ctypes.c_int),
    "hd_serve_drain": ([_P], ctypes.c_int),
    "hd_serve_completed": ([_P, _P, ctypes.c_uint32, ctypes.POINTER(ctypes.c_uint32)],
                           ctypes.c_int),
    "hd_serve_stats": ([_P, ctypes.POINTER(hd_serve_stats_t)], ctypes.c_int),
    "hd_version": ([], ctypes.c_char_p),
}

_lib = None


def library_path() -> str:
    return _build.LIB


def load(build_if_needed: bool = True):
    """Loads libhd.so (building it first when sources changed)."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.build() if build_if_needed else _build.LIB
    if not os.path.exists(path):
        raise ImportError(f"libhd.so not found at {path}; run paper_2201_09118_gb300.build")
    lib = ctypes.CDLL(path)
    for name, (args, res) in _SIGS.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = res
    _lib = lib
    return lib


def exported_symbols():
    return sorted(_SIGS)


def _check(fn: str, rc: int):
    if rc != HD_OK:
        raise HDError(fn, rc)
    return rc


def _np_ptr(a: np.ndarray):
    return ctypes.c_void_p(a.ctypes.data)


def _stream_handle(stream) -> ctypes.c_void_p:
    if stream is None:
        import torch
        stream = torch.cuda.current_stream()
    h = getattr(stream, "cuda_stream", stream)
    return ctypes.c_void_p(int(h) if h else 0)


# ---------------------------------------------------------------------------
# host-side codebook / encoder
# ---------------------------------------------------------------------------


def hd_build_codebook(codes: np.ndarray, alphabet: int, max_len: int = 32) -> np.ndarray:
    codes = np.ascontiguousarray(codes, dtype=np.uint16)
    out = np.zeros(alphabet, dtype=np.uint8)
    _check("hd_build_codebook",
           load().hd_build_codebook(_np_ptr(codes), codes.size, alphabet, max_len, _np_ptr(out)))
    return out


def hd_build_codebook_freq(freq: np.ndarray, max_len: int = 32) -> np.ndarray:
    freq = np.ascontiguousarray(freq, dtype=np.uint64)
    out = np.zeros(freq.size, dtype=np.uint8)
    _check("hd_build_codebook_freq",
           load().hd_build_codebook_freq(_np_ptr(freq), freq.size, max_len, _np_ptr(out)))
    return out


def hd_encode(codes: np.ndarray, lengths: np.ndarray, subseq_bits: int = 128,
              with_gap: bool = True) -> dict:
    """Returns {'words', 'gap' (or None), 'nbits', 'nwords', 'nsub'}."""
    codes = np.ascontiguousarray(codes, dtype=np.uint16)
    lengths = np.ascontiguousarray(lengths, dtype=np.uint8)
    lib = load()
    info = hd_stream_info()
    rc = lib.hd_encode(_np_ptr(codes), codes.size, _np_ptr(lengths), lengths.size, subseq_bits,
                       None, 0, None, 0, ctypes.byref(info))
    if rc not in (HD_OK, HD_ERR_CAPACITY):
        raise HDError("hd_encode", rc)
    words = np.zeros(max(1, info.nwords), dtype=np.uint32)
    gap = np.zeros(max(1, info.nsub), dtype=np.uint8) if with_gap else None
    _check("hd_encode", lib.hd_encode(_np_ptr(codes), codes.size, _np_ptr(lengths), lengths.size,
                                      subseq_bits, _np_ptr(words), words.size,
                                      _np_ptr(gap) if gap is not None else None,
                                      gap.size if gap is not None else 0, ctypes.byref(info)))
    return {"words": words[:info.nwords], "gap": None if gap is None else gap[:info.nsub],
            "nbits": int(info.nbits), "nwords": int(info.nwords), "nsub": int(info.nsub),
            "subseq_bits": subseq_bits}


# ---------------------------------------------------------------------------
# device fields and context
# ---------------------------------------------------------------------------


@dataclass
class DeviceField:
    """An encoded field resident on the GPU (torch tensors own the memory)."""
    words: "object"            # torch.int32 tensor (the uint32 units)
    nbits: int
    gap: Optional["object"]    # torch.uint8 tensor or None
    subseq_bits: int
    lengths: "object"          # torch.uint8 tensor [alphabet]
    alphabet: int
    n: int

    def c_struct(self) -> hd_field:
        return hd_field(self.words.data_ptr(), self.words.numel(), self.nbits,
                        self.gap.data_ptr() if self.gap is not None else None,
                        self.subseq_bits, self.lengths.data_ptr(), self.alphabet, self.n)

    @staticmethod
    def upload(enc: dict, lengths: np.ndarray, n: int, device="cuda", with_gap: bool = True):
        import torch
        words = torch.from_numpy(enc["words"].view(np.int32).copy()).to(device)
        gap = None
        if with_gap and enc.get("gap") is not None:
            g = enc["gap"] if enc["gap"].size else np.zeros(1, np.uint8)
            gap = torch.from_numpy(np.ascontiguousarray(g)).to(device)
        lt = torch.from_numpy(np.ascontiguousarray(lengths, dtype=np.uint8)).to(device)
        return DeviceField(words, int(enc["nbits"]), gap, int(enc["subseq_bits"]), lt,
                           int(lengths.size), int(n))


class Context:
    """Owns an hd_ctx for one device."""

    def __init__(self, device: int = 0):
        self._lib = load()
        h = ctypes.c_void_p()
        _check("hd_ctx_create", self._lib.hd_ctx_create(device, ctypes.byref(h)))
        self.handle = h
        self.device = device

    def close(self):
        if self.handle:
            self._lib.hd_ctx_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_config(self, subseq_bits=0, threads=0, window=0, lut_bits=0, cr_classes=0,
                   decoder=0):
        """decoder: 0 automatic, 1 two phases, 2 one pass (hd_config.decoder)."""
        cfg = hd_config(subseq_bits, threads, window, lut_bits, cr_classes, decoder)
        _check("hd_set_config", self._lib.hd_set_config(self.handle, ctypes.byref(cfg)))

    def reset_config(self):
        _check("hd_set_config", self._lib.hd_set_config(self.handle, None))

    def get_config(self) -> dict:
        cfg = hd_config()
        _check("hd_get_config", self._lib.hd_get_config(self.handle, ctypes.byref(cfg)))
        return {"subseq_bits": cfg.subseq_bits, "threads": cfg.threads, "window": cfg.window,
                "lut_bits": cfg.lut_bits, "cr_classes": cfg.cr_classes, "decoder": cfg.decoder}

    def decode(self, field: DeviceField, out, stream=None) -> None:
        f = field.c_struct()
        _check("hd_decode", self._lib.hd_decode(self.handle, ctypes.byref(f),
                                                 ctypes.c_void_p(out.data_ptr()),
                                                 _stream_handle(stream)))

    def status(self, stream=None) -> int:
        return self._lib.hd_status(self.handle, _stream_handle(stream))

    def reconstruct(self, codes, L: hd_lorenzo, out, stream=None) -> None:
        """Lorenzo reconstruction of device codes (uint16 as int16) into a
        float32 device tensor (hd_reconstruct_device)."""
        _check("hd_reconstruct_device", self._lib.hd_reconstruct_device(
            self.handle, ctypes.c_void_p(codes.data_ptr()), ctypes.byref(L),
            ctypes.c_void_p(out.data_ptr()), _stream_handle(stream)))

    def decompress(self, field: DeviceField, L: hd_lorenzo, out, stream=None) -> None:
        """Decode then reconstruct (hd_decompress_device)."""
        f = field.c_struct()
        _check("hd_decompress_device", self._lib.hd_decompress_device(
            self.handle, ctypes.byref(f), ctypes.byref(L), ctypes.c_void_p(out.data_ptr()),
            _stream_handle(stream)))

    def sync_points(self, field: DeviceField, gap_out, stream=None) -> None:
        f = field.c_struct()
        _check("hd_sync_points", self._lib.hd_sync_points(self.handle, ctypes.byref(f),
                                                           ctypes.c_void_p(gap_out.data_ptr()),
                                                           _stream_handle(stream)))

    def inspect_tables(self, lengths_dev, alphabet: int, K: int, stream=None) -> dict:
        """The per-prefix decode tables (hd_inspect_tables) of the code-length
        table `lengths_dev` (a uint8 device tensor): numpy arrays lut16, len8,
        run8 and pair of 2^K entries each."""
        n = 1 << K
        lut16 = np.zeros(n, np.uint16)
        len8 = np.zeros(n, np.uint8)
        run8 = np.zeros(n, np.uint8)
        pair = np.zeros(n, np.uint32)
        _check("hd_inspect_tables", self._lib.hd_inspect_tables(
            self.handle, ctypes.c_void_p(lengths_dev.data_ptr()), alphabet, K,
            lut16.ctypes.data, len8.ctypes.data, run8.ctypes.data, pair.ctypes.data,
            _stream_handle(stream)))
        return {"lut16": lut16, "len8": len8, "run8": run8, "pair": pair}

    def decode_batch(self, fields: Sequence[DeviceField], outs, stream=None) -> None:
        nf = len(fields)
        arr = (hd_field * max(1, nf))(*[f.c_struct() for f in fields])
        ptrs = (ctypes.c_void_p * max(1, nf))(*[o.data_ptr() for o in outs])
        _check("hd_decode_batch", self._lib.hd_decode_batch(self.handle, arr, nf, ptrs,
                                                             _stream_handle(stream)))

    def autotune(self, fields: Sequence[DeviceField], outs, stream=None) -> dict:
        """Times every candidate launch shape on this batch and keeps the fastest
        for the batch's class; returns it."""
        nf = len(fields)
        arr = (hd_field * max(1, nf))(*[f.c_struct() for f in fields])
        ptrs = (ctypes.c_void_p * max(1, nf))(*[o.data_ptr() for o in outs])
        cfg = hd_config()
        _check("hd_autotune", self._lib.hd_autotune(self.handle, arr, nf, ptrs,
                                                    _stream_handle(stream), ctypes.byref(cfg)))
        return {"subseq_bits": cfg.subseq_bits, "threads": cfg.threads, "window": cfg.window,
                "lut_bits": cfg.lut_bits, "cr_classes": cfg.cr_classes, "decoder": cfg.decoder}

    def autotune_save(self, path: str) -> None:
        """Writes this context's tuned launch shapes to `path` (hd_autotune_save)."""
        _check("hd_autotune_save", self._lib.hd_autotune_save(self.handle, path.encode()))

    def autotune_load(self, path: str) -> int:
        """Takes the tuned shapes of this GPU from `path`; returns how many."""
        n = ctypes.c_uint32()
        _check("hd_autotune_load", self._lib.hd_autotune_load(self.handle, path.encode(),
                                                              ctypes.byref(n)))
        return n.value

    def graph_stats(self):
        cap = ctypes.c_uint64()
        cached = ctypes.c_uint32()
        _check("hd_graph_stats", self._lib.hd_graph_stats(self.handle, ctypes.byref(cap),
                                                          ctypes.byref(cached)))
        return cap.value, cached.value

    def histogram(self, codes, alphabet: int, stream=None) -> np.ndarray:
        """Symbol counts of a device int16/uint16 tensor (hd_histogram_device)."""
        freq = np.zeros(alphabet, dtype=np.uint64)
        _check("hd_histogram_device", self._lib.hd_histogram_device(
            self.handle, codes.data_ptr(), codes.numel(), alphabet, _np_ptr(freq),
            _stream_handle(stream)))
        return freq

    def encode(self, codes, lengths: np.ndarray, subseq_bits: int = 128, with_gap: bool = True,
               stream=None) -> dict:
        """GPU encode of a device tensor of symbols (hd_encode_device); returns
        device tensors 'words' (int32 view of the uint32 units) and 'gap' (or
        None) with 'nbits', 'nwords', 'nsub'."""
        import torch
        lengths = np.ascontiguousarray(lengths, dtype=np.uint8)
        info = hd_stream_info()
        rc = self._lib.hd_encode_device(self.handle, codes.data_ptr(), codes.numel(),
                                        _np_ptr(lengths), lengths.size, subseq_bits, None, 0,
                                        None, 0, ctypes.byref(info), _stream_handle(stream))
        if rc not in (HD_OK, HD_ERR_CAPACITY):
            raise HDError("hd_encode_device", rc)
        words = torch.empty(max(1, info.nwords), dtype=torch.int32, device=codes.device)
        gap = (torch.empty(max(1, info.nsub), dtype=torch.uint8, device=codes.device)
               if with_gap else None)
        _check("hd_encode_device", self._lib.hd_encode_device(
            self.handle, codes.data_ptr(), codes.numel(), _np_ptr(lengths), lengths.size,
            subseq_bits, words.data_ptr(), words.numel(),
            gap.data_ptr() if gap is not None else None, gap.numel() if gap is not None else 0,
            ctypes.byref(info), _stream_handle(stream)))
        return {"words": words[:info.nwords], "gap": None if gap is None else gap[:info.nsub],
                "nbits": int(info.nbits), "nwords": int(info.nwords), "nsub": int(info.nsub),
                "subseq_bits": subseq_bits}

    def batch_status(self, nf: int, stream=None):
        st = np.zeros(max(1, nf), dtype=np.int32)
        rc = self._lib.hd_batch_status(self.handle, _np_ptr(st), nf, _stream_handle(stream))
        return rc, st[:nf]

    def decode_host(self, enc: dict, lengths: np.ndarray, n: int, out: np.ndarray = None,
                    stream=None, with_gap: bool = True) -> np.ndarray:
        """Host buffers in, host symbols out (copies inside the call)."""
        words = np.ascontiguousarray(enc["words"], dtype=np.uint32)
        gap = enc.get("gap") if with_gap else None
        if gap is not None:
            gap = np.ascontiguousarray(gap, dtype=np.uint8)
        lengths = np.ascontiguousarray(lengths, dtype=np.uint8)
        if out is None:
            out = np.empty(max(1, n), dtype=np.uint16)
        f = hd_field(words.ctypes.data, words.size, int(enc["nbits"]),
                     gap.ctypes.data if gap is not None and gap.size else None,
                     int(enc["subseq_bits"]), lengths.ctypes.data, lengths.size, n)
        _check("hd_decode_host", self._lib.hd_decode_host(self.handle, ctypes.byref(f),
                                                          _np_ptr(out), _stream_handle(stream)))
        return out[:n]

    def decode_host_ptrs(self, words_ptr: int, nwords: int, nbits: int, gap_ptr: int,
                         subseq_bits: int, lengths_ptr: int, alphabet: int, n: int,
                         out_ptr: int, stream=None) -> int:
        """Raw-pointer variant (e.g. pinned torch tensors); returns the status."""
        f = hd_field(words_ptr, nwords, nbits, gap_ptr or None, subseq_bits, lengths_ptr,
                     alphabet, n)
        return self._lib.hd_decode_host(self.handle, ctypes.byref(f), ctypes.c_void_p(out_ptr),
                                        _stream_handle(stream))

    def profile(self, enable: bool = True):
        _check("hd_profile", self._lib.hd_profile(self.handle, 1 if enable else 0))

    def kernel_time(self):
        ms = ctypes.c_double()
        n = ctypes.c_uint64()
        _check("hd_kernel_time", self._lib.hd_kernel_time(self.handle, ctypes.byref(ms),
                                                          ctypes.byref(n)))
        return ms.value, n.value

    def set_wait_limit(self, cycles: int) -> None:
        """Per-wait limit of the one-pass decoder's look-back (SM cycles; 0 = default)."""
        _check("hd_set_wait_limit", self._lib.hd_set_wait_limit(self.handle, cycles))

    def phase_times(self):
        """Per-phase ms of the profiled single-field decodes since the last
        call (hd_phase_times): dict sync / count / index / write, plus decodes."""
        ms = (ctypes.c_double * 4)()
        n = ctypes.c_uint64()
        _check("hd_phase_times", self._lib.hd_phase_times(self.handle, ms, ctypes.byref(n)))
        return {"sync": ms[0], "count": ms[1], "index": ms[2], "write": ms[3],
                "decodes": n.value}

    def launch_count(self) -> int:
        return int(self._lib.hd_launch_count(self.handle))


class Server:
    """A decode server (hd_serve_*): resident fields, requests admitted by a
    device-memory budget, continuous batching over `slots` streams."""

    def __init__(self, device: int = 0, budget_bytes: int = 40 << 30, slots: int = 2,
                 max_batch: int = 64, queue_cap: int = 0, direct: bool = False,
                 shape: Optional[dict] = None, watchdog_us: int = 0):
        self._lib = load()
        cfg = hd_serve_config(budget_bytes, slots, max_batch, queue_cap, 1 if direct else 0,
                              watchdog_us)
        sh = None
        if shape:
            sh = hd_config(shape.get("subseq_bits", 0), shape.get("threads", 0),
                           shape.get("window", 0), shape.get("lut_bits", 0),
                           shape.get("cr_classes", 0), shape.get("decoder", 0))
        h = ctypes.c_void_p()
        _check("hd_serve_create", self._lib.hd_serve_create(
            device, ctypes.byref(cfg), ctypes.byref(sh) if sh is not None else None,
            ctypes.byref(h)))
        self.handle = h
        self._fields = []  # keeps the registered fields' tensors alive

    def close(self):
        if self.handle:
            self._lib.hd_serve_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def register(self, field: DeviceField) -> int:
        fid = ctypes.c_uint32()
        f = field.c_struct()
        _check("hd_serve_register", self._lib.hd_serve_register(self.handle, ctypes.byref(f),
                                                                ctypes.byref(fid)))
        self._fields.append(field)
        return fid.value

    def submit(self, field_id: int) -> int:
        t = ctypes.c_uint64()
        _check("hd_serve_submit", self._lib.hd_serve_submit(self.handle, field_id,
                                                            ctypes.byref(t)))
        return t.value

    def poll(self, ticket: int):
        """None while pending, else a dict with status, d_out, n, queue_us, latency_us."""
        r = hd_result()
        rc = self._lib.hd_serve_poll(self.handle, ticket, ctypes.byref(r))
        if rc == HD_PENDING:
            return None
        _check("hd_serve_poll", rc)
        return {"status": r.status, "d_out": r.d_out, "n": r.n, "queue_us": r.queue_us,
                "latency_us": r.latency_us}

    def release(self, ticket: int) -> None:
        _check("hd_serve_release", self._lib.hd_serve_release(self.handle, ticket))

    def drain(self) -> None:
        _check("hd_serve_drain", self._lib.hd_serve_drain(self.handle))

    def completed(self, cap: int = 4096) -> np.ndarray:
        """Tickets completed since the last call (uint64 array)."""
        buf = np.empty(max(1, cap), dtype=np.uint64)
        k = ctypes.c_uint32()
        _check("hd_serve_completed", self._lib.hd_serve_completed(self.handle, _np_ptr(buf), cap,
                                                                  ctypes.byref(k)))
        return buf[:k.value]

    def stats(self) -> dict:
        s = hd_serve_stats_t()
        _check("hd_serve_stats", self._lib.hd_serve_stats(self.handle, ctypes.byref(s)))
        return {k: getattr(s, k) for k, _ in hd_serve_stats_t._fields_}


class _DeviceSpan:
    """A raw device range seen through the CUDA array interface (no copy)."""

    def __init__(self, ptr: int, n: int):
        self.__cuda_array_interface__ = {"shape": (n,), "typestr": "<i2", "data": (ptr, False),
                                         "version": 3, "strides": None}


def device_u16_view(ptr: int, n: int, device: int = 0):
    """The n uint16 symbols at a device pointer as an int16 torch tensor view
    (valid while the memory is; clone() to keep them)."""
    import torch
    if n == 0:
        return torch.empty(0, dtype=torch.int16, device=f"cuda:{device}")
    return torch.as_tensor(_DeviceSpan(ptr, n), device=f"cuda:{device}")


def hd_version() -> str:
    return load().hd_version().decode()
