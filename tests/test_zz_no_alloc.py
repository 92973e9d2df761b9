"""hd_decode_static, the allocation-free gap-array decode entry point.

Some callers cannot call cudaMalloc when they decode (real-time loops that
cannot take its possible device-wide synchronisation, plugins whose host
framework's allocator already reserved the device memory).  For them the
library keeps its scratch in one fixed device array instead of a context's
workspace.  This test calls that entry point through the C ABI and checks its
output against the context-based hd_decode on the same inputs, on two calls in
a row: the array keeps the previous call's contents, so the second call also
shows that everything that must start from zero is cleared.  It lives in its
own file, collected last.
"""
import ctypes

import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

CANARY = 0xABCD


def test_decode_static_matches_hd_decode_twice():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2201_09118_gb300 import hd
    lib = hd.load()
    ctx = hd.Context(0)
    stream = torch.cuda.current_stream()
    try:
        # a large field first, then a smaller one: the second call starts from
        # the first call's leftover look-back states and table
        for n, scale, seed in ((3_000_017, 40.0, 31), (1_000_003, 2.0, 32)):
            x = synth.laplace_codes(n, scale=scale, seed=seed)
            c = oracle.compress(x, 1024, S=128)
            enc = {"words": c["words"], "gap": c["gap"], "nbits": c["nbits"], "subseq_bits": 128}
            f = hd.DeviceField.upload(enc, c["lengths"], n)
            ref = torch.empty(n, dtype=torch.int16, device="cuda")
            ctx.decode(f, ref, stream)
            assert ctx.status(stream) == hd.HD_OK
            out = torch.full((n + 16,), CANARY, dtype=torch.int32).to(torch.int16).cuda()
            cf = f.c_struct()
            rc = lib.hd_decode_static(ctypes.byref(cf), ctypes.c_void_p(out.data_ptr()),
                                      ctypes.c_void_p(stream.cuda_stream))
            assert rc == hd.HD_OK
            got = out.cpu().numpy().view(np.uint16)
            assert np.array_equal(got[:n], ref.cpu().numpy().view(np.uint16))
            assert np.array_equal(got[:n], x)
            assert np.all(got[n:] == np.uint16(CANARY))
    finally:
        ctx.close()


def test_decode_static_rejects_oversized_field_before_gpu_work():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2201_09118_gb300 import hd
    lib = hd.load()
    words = torch.zeros(8, dtype=torch.int32, device="cuda")
    gap = torch.zeros(8, dtype=torch.uint8, device="cuda")
    lengths = torch.ones(2, dtype=torch.uint8, device="cuda")
    out = torch.zeros(8, dtype=torch.int16, device="cuda")
    nbits = 1 << 40  # far more look-back states than the fixed scratch holds
    f = hd.hd_field(words.data_ptr(), nbits // 32 + 1, nbits, gap.data_ptr(), 128,
                    lengths.data_ptr(), 2, nbits)
    rc = lib.hd_decode_static(ctypes.byref(f), ctypes.c_void_p(out.data_ptr()), None)
    assert rc == hd.HD_ERR_CAPACITY
    torch.cuda.synchronize()


def test_decode_static_corrupt_call_then_clean_call():
    # the error word lives in the shared fixed array: a call that fails must not
    # leave its error bits to the next call on the same array
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2201_09118_gb300 import hd
    lib = hd.load()
    stream = torch.cuda.current_stream()
    x = synth.laplace_codes(400_009, scale=6.0, seed=33)
    c = oracle.compress(x, 1024, S=128)
    enc = {"words": c["words"], "gap": c["gap"], "nbits": c["nbits"], "subseq_bits": 128}
    good = hd.DeviceField.upload(enc, c["lengths"], c["n"])
    bad_gap = c["gap"].copy()
    bad_gap[len(bad_gap) // 3] = 200  # no codeword starts 200 bits into a subsequence
    bad = hd.DeviceField.upload(dict(enc, gap=bad_gap), c["lengths"], c["n"])
    n = c["n"]
    for field, want in ((bad, hd.HD_ERR_CORRUPT), (good, hd.HD_OK), (bad, hd.HD_ERR_CORRUPT),
                        (good, hd.HD_OK)):
        out = torch.full((n + 16,), CANARY, dtype=torch.int32).to(torch.int16).cuda()
        cf = field.c_struct()
        rc = lib.hd_decode_static(ctypes.byref(cf), ctypes.c_void_p(out.data_ptr()),
                                  ctypes.c_void_p(stream.cuda_stream))
        assert rc == want
        got = out.cpu().numpy().view(np.uint16)
        assert np.all(got[n:] == np.uint16(CANARY))
        if want == hd.HD_OK:
            assert np.array_equal(got[:n], x)
