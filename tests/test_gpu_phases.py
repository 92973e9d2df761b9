"""Per-phase timing (hd_phase_times) of the decode paths, the breakdown the
paper reports for its decoders (Sec. V-B: synchronisation, output indices,
decode and write).  While profiling, the two-phase kernels are queued one phase
at a time; the output must be the oracle's all the same."""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def setup():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2201_09118_gb300 import hd
    ctx = hd.Context(0)
    x = synth.laplace_codes(1 << 21, scale=30.0, seed=61)
    c = oracle.compress(x, 1024, S=128)
    enc = {"words": c["words"], "gap": c["gap"], "nbits": c["nbits"], "subseq_bits": 128}
    yield hd, ctx, x, enc, c
    ctx.close()


@pytest.mark.parametrize("mode", ["gap-2phase", "gap-1pass", "selfsync"])
def test_phase_times_and_output(setup, mode):
    hd, ctx, x, enc, c = setup
    f = hd.DeviceField.upload(enc, c["lengths"], c["n"], with_gap=mode != "selfsync")
    out = torch.empty(c["n"], dtype=torch.int16, device="cuda")
    ctx.set_config(decoder={"gap-2phase": 1, "gap-1pass": 2, "selfsync": 0}[mode])
    try:
        ctx.profile(True)
        ctx.kernel_time()
        ctx.phase_times()
        for _ in range(3):
            out.fill_(0)
            ctx.decode(f, out)
            assert ctx.status() == hd.HD_OK
            assert np.array_equal(out.cpu().numpy().view(np.uint16), x)
        total, spans = ctx.kernel_time()
        ph = ctx.phase_times()
        ctx.profile(False)
    finally:
        ctx.reset_config()
    assert spans == 3 and ph["decodes"] == 3
    assert ph["write"] > 0
    if mode == "gap-2phase":
        assert ph["count"] > 0 and ph["index"] > 0 and ph["sync"] == 0
    elif mode == "gap-1pass":
        assert ph["count"] == 0 and ph["index"] == 0 and ph["sync"] == 0
    else:
        assert ph["sync"] > 0 and ph["index"] > 0 and ph["count"] == 0
    parts = ph["sync"] + ph["count"] + ph["index"] + ph["write"]
    # the phases tile the span between the decode's first and last event
    assert abs(parts - total) <= 0.05 * total + 0.01
