"""Full-size parity of the skew sweep: a 1D field of 280,953,867 codes (the
HACC particle count) quantized at relative error bounds 1e-2, 1e-4 and 1e-6
with alphabets 256, 1024 and 4096, decoded with the gap array and by
self-synchronisation in the default launch shape; and 26 2D fields
of 1800 x 3600 at 1e-4 decoded as one batch.  Every output is compared with
the oracle's bit-serial decode of the oracle's encoding, element by element.
"""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

N_1D = 280_953_867


@pytest.fixture(scope="module")
def field_1d():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return synth.fourier_field((N_1D,), noise=1e-4, kmax=64, seed=1002)


@pytest.fixture(scope="module")
def ctx():
    from paper_2201_09118_gb300 import hd
    c = hd.Context(0)
    yield c
    c.close()


def upload(c, with_gap):
    from paper_2201_09118_gb300 import hd
    enc = {"words": c["words"], "gap": c["gap"], "nbits": c["nbits"], "subseq_bits": c["S"]}
    return hd.DeviceField.upload(enc, c["lengths"], c["n"], with_gap=with_gap)


@pytest.mark.parametrize("rel_eb,alphabet", [(1e-2, 256), (1e-4, 1024), (1e-6, 4096)])
def test_skew_sweep_280m_codes(field_1d, ctx, rel_eb, alphabet):
    codes, _, _ = synth.lorenzo_codes(field_1d, rel_eb, radius=alphabet // 2)
    c = oracle.compress(codes, alphabet, S=128)
    ref = oracle.decode(c["words"], c["nbits"], c["codes"], c["lengths"], n_cap=c["n"])
    assert np.array_equal(ref, codes)  # the oracle's own round trip
    bits = c["nbits"] / c["n"]
    if rel_eb == 1e-2:
        assert bits < 1.3 and np.count_nonzero(codes == alphabet // 2) > 0.95 * codes.size
    for with_gap in (True, False):
        f = upload(c, with_gap)
        out = torch.empty(c["n"] + 8, dtype=torch.int16, device="cuda")
        out[c["n"]:] = 0x1234
        ctx.decode(f, out)
        assert ctx.status() == 0
        got = out.cpu().numpy().view(np.uint16)
        assert np.array_equal(got[:c["n"]], ref), (rel_eb, with_gap)
        assert np.all(got[c["n"]:] == 0x1234)
        del f, out
        torch.cuda.empty_cache()


def test_2d_fields_26_variables_as_one_batch(ctx):
    from paper_2201_09118_gb300 import hd
    comps, fields, outs = [], [], []
    for v in range(26):
        f2 = synth.fourier_field((1800, 3600), noise=1e-4, kmax=8, seed=2000 + v)
        codes, _, _ = synth.lorenzo_codes(f2, 1e-4, radius=512)
        c = oracle.compress(codes, 1024, S=128)
        comps.append(c)
        fields.append(upload(c, v % 2 == 0))  # both strategies in the batch
        outs.append(torch.empty(c["n"], dtype=torch.int16, device="cuda"))
    ctx.decode_batch(fields, outs)
    rc, st = ctx.batch_status(len(fields))
    assert rc == hd.HD_OK and np.all(st == 0)
    for c, o in zip(comps, outs):
        ref = oracle.decode(c["words"], c["nbits"], c["codes"], c["lengths"], n_cap=c["n"])
        assert np.array_equal(o.cpu().numpy().view(np.uint16), ref)
