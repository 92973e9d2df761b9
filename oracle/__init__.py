"""CPU oracle for the Huffman decoding path (test infrastructure only).

A plain C library (``oracle.c``) compiled with gcc and called through ctypes.
It is what the CUDA decoder is checked against, and it is pinned on its own by
the ``-m "not gpu"`` tests (worked examples of the paper, textbook cases, brute
force, invariants).  Only ``tests/``, the package smoke check and the CPU
baseline leg of ``bench.py`` may import this module; the product path never
does, and it shares no code with the CUDA path.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

OK = 0
ERR_ARG = -1
ERR_CAPACITY = -2
ERR_SYMBOL = -3
ERR_CORRUPT = -4
ERR_NOSYNC = -5
ERR_NOMEM = -8


class OracleError(RuntimeError):
    def __init__(self, fn: str, code: int):
        super().__init__(f"oracle {fn} failed with status {code}")
        self.code = code


def build(force: bool = False) -> str:
    """Compile liboracle.so with gcc (plain -O2, no target-specific flags)."""
    with _lock:
        stale = (not os.path.exists(_LIB_PATH)
                 or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC))
        if force or stale:
            tmp = _LIB_PATH + f".tmp{os.getpid()}"
            subprocess.check_call(["gcc", "-O2", "-std=c11", "-shared", "-fPIC",
                                   "-o", tmp, _SRC])
            os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    if _lib is not None:
        return _lib
    build()
    lib = ctypes.CDLL(_LIB_PATH)
    P = ctypes.c_void_p
    U64 = ctypes.c_uint64
    U32 = ctypes.c_uint32
    I = ctypes.c_int
    sig = {
        "or_histogram": [P, U64, U32, P],
        "or_huffman_depths": [P, U32, P],
        "or_package_merge": [P, U32, U32, P],
        "or_code_lengths": [P, U32, U32, P],
        "or_canonical_codes": [P, U32, P],
        "or_encode": [P, U64, P, P, U32, U32, P, U64, P, P],
        "or_gap_build": [P, U64, P, U32, U64, P, U64],
        "or_gap_paper": [P, U64, P, U32, U64, P, U64],
        "or_subseq_counts": [P, U64, P, U32, U64, P, U64],
        "or_decode": [P, U64, U64, U64, P, P, U32, P, U64, P],
        "or_sync_points": [P, U64, U64, P, P, U32, U32, P, U64, U32, P],
    }
    for name, args in sig.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = I
    lib.or_stream_size.argtypes = [U64, U32, P, P]
    lib.or_stream_size.restype = None
    _lib = lib
    return lib


def _p(a: np.ndarray):
    return ctypes.c_void_p(a.ctypes.data)


def _check(fn, rc):
    if rc != OK:
        raise OracleError(fn, rc)


def _u16(x):
    return np.ascontiguousarray(x, dtype=np.uint16)


def histogram(x, alphabet: int) -> np.ndarray:
    x = _u16(x)
    freq = np.zeros(alphabet, dtype=np.uint64)
    _check("histogram", _load().or_histogram(_p(x), x.size, alphabet, _p(freq)))
    return freq


def huffman_depths(freq) -> np.ndarray:
    freq = np.ascontiguousarray(freq, dtype=np.uint64)
    d = np.zeros(freq.size, dtype=np.uint32)
    _check("huffman_depths", _load().or_huffman_depths(_p(freq), freq.size, _p(d)))
    return d


def package_merge(freq, max_len: int) -> np.ndarray:
    freq = np.ascontiguousarray(freq, dtype=np.uint64)
    out = np.zeros(freq.size, dtype=np.uint8)
    _check("package_merge", _load().or_package_merge(_p(freq), freq.size, max_len, _p(out)))
    return out


def code_lengths(freq, max_len: int = 32) -> np.ndarray:
    freq = np.ascontiguousarray(freq, dtype=np.uint64)
    out = np.zeros(freq.size, dtype=np.uint8)
    _check("code_lengths", _load().or_code_lengths(_p(freq), freq.size, max_len, _p(out)))
    return out


def canonical_codes(lengths) -> np.ndarray:
    lengths = np.ascontiguousarray(lengths, dtype=np.uint8)
    codes = np.zeros(lengths.size, dtype=np.uint32)
    _check("canonical_codes", _load().or_canonical_codes(_p(lengths), lengths.size, _p(codes)))
    return codes


def stream_size(nbits: int, S: int):
    a = ctypes.c_uint64()
    b = ctypes.c_uint64()
    _load().or_stream_size(nbits, S, ctypes.byref(a), ctypes.byref(b))
    return a.value, b.value


def encode(x, lengths, codes, S: int):
    """Returns (words uint32, nbits)."""
    x = _u16(x)
    lengths = np.ascontiguousarray(lengths, dtype=np.uint8)
    codes = np.ascontiguousarray(codes, dtype=np.uint32)
    nbits = int(lengths[x].astype(np.uint64).sum()) if x.size else 0
    _, nwords = stream_size(nbits, S)
    words = np.zeros(nwords, dtype=np.uint32)
    nb = ctypes.c_uint64()
    nw = ctypes.c_uint64()
    _check("encode", _load().or_encode(_p(x), x.size, _p(lengths), _p(codes), lengths.size, S,
                                       _p(words), words.size, ctypes.byref(nb), ctypes.byref(nw)))
    assert nb.value == nbits and nw.value == nwords
    return words, nbits


def gap_build(x, lengths, S: int, nbits: int) -> np.ndarray:
    x = _u16(x)
    lengths = np.ascontiguousarray(lengths, dtype=np.uint8)
    nsub, _ = stream_size(nbits, S)
    gap = np.zeros(max(nsub, 1), dtype=np.uint8)
    _check("gap_build", _load().or_gap_build(_p(x), x.size, _p(lengths), S, nbits, _p(gap),
                                             gap.size))
    return gap[:nsub]


def gap_paper(x, lengths, S: int, nbits: int) -> np.ndarray:
    x = _u16(x)
    lengths = np.ascontiguousarray(lengths, dtype=np.uint8)
    nsub, _ = stream_size(nbits, S)
    gap = np.zeros(max(nsub, 1), dtype=np.int32)
    _check("gap_paper", _load().or_gap_paper(_p(x), x.size, _p(lengths), S, nbits, _p(gap),
                                             gap.size))
    return gap[:nsub]


def subseq_counts(x, lengths, S: int, nbits: int) -> np.ndarray:
    x = _u16(x)
    lengths = np.ascontiguousarray(lengths, dtype=np.uint8)
    nsub, _ = stream_size(nbits, S)
    c = np.zeros(max(nsub, 1), dtype=np.uint32)
    _check("subseq_counts", _load().or_subseq_counts(_p(x), x.size, _p(lengths), S, nbits,
                                                     _p(c), c.size))
    return c[:nsub]


def decode(words, nbits: int, codes, lengths, n_cap: int | None = None,
           start_bit: int = 0) -> np.ndarray:
    words = np.ascontiguousarray(words, dtype=np.uint32)
    lengths = np.ascontiguousarray(lengths, dtype=np.uint8)
    codes = np.ascontiguousarray(codes, dtype=np.uint32)
    if n_cap is None:
        n_cap = max(1, nbits - start_bit)
    out = np.zeros(max(1, n_cap), dtype=np.uint16)
    k = ctypes.c_uint64()
    _check("decode", _load().or_decode(_p(words), words.size, start_bit, nbits, _p(codes),
                                       _p(lengths), lengths.size, _p(out), n_cap,
                                       ctypes.byref(k)))
    return out[:k.value]


def sync_points(words, nbits: int, codes, lengths, S: int, max_rounds: int | None = None):
    """Returns (sync uint64 [nsub], rounds)."""
    words = np.ascontiguousarray(words, dtype=np.uint32)
    lengths = np.ascontiguousarray(lengths, dtype=np.uint8)
    codes = np.ascontiguousarray(codes, dtype=np.uint32)
    nsub, _ = stream_size(nbits, S)
    if max_rounds is None:
        max_rounds = nsub + 1
    sync = np.zeros(max(1, nsub), dtype=np.uint64)
    r = ctypes.c_uint32()
    _check("sync_points", _load().or_sync_points(_p(words), words.size, nbits, _p(codes),
                                                 _p(lengths), lengths.size, S, _p(sync),
                                                 sync.size, max_rounds, ctypes.byref(r)))
    return sync[:nsub], r.value


def compress(x, alphabet: int, S: int = 128, max_len: int = 32):
    """Convenience: lengths, canonical codes, packed stream and gap array of ``x``."""
    freq = histogram(x, alphabet)
    lengths = code_lengths(freq, max_len)
    codes = canonical_codes(lengths)
    words, nbits = encode(x, lengths, codes, S)
    gap = gap_build(x, lengths, S, nbits)
    return {"lengths": lengths, "codes": codes, "words": words, "nbits": nbits, "gap": gap,
            "S": S, "alphabet": alphabet, "n": int(np.asarray(x).size)}
