"""GPU parity of the batched path: many fields of uneven sizes, own codebooks,
decoded by graph launches (hd_decode_batch) and by the autotuned shapes
(hd_autotune), against the CPU oracle's decode of every field.
"""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

CANARY = 0xABCD


@pytest.fixture()
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2201_09118_gb300 import hd
    c = hd.Context(0)
    yield c
    c.close()


def make_batch(n_fields, lo, hi, seed, with_gap=True, S=128, alphabets=(256, 1024, 4096),
               eb_lo=1e-6, eb_hi=1e-2):
    """Fields drawn like the batched workload (log-uniform sizes, mixed alphabets
    and error bounds), each compressed by the oracle with its own codebook."""
    from paper_2201_09118_gb300 import hd
    specs = synth.batch_spec(n_fields, lo=lo, hi=hi, alphabets=alphabets, eb_lo=eb_lo,
                             eb_hi=eb_hi, seed=seed)
    comps, fields, outs = [], [], []
    for sp in specs:
        x = synth.smooth_codes_1d(sp.n, sp.rel_eb, alphabet=sp.alphabet, seed=sp.seed)
        c = oracle.compress(x, sp.alphabet, S=S)
        c["x"] = x
        comps.append(c)
        enc = {"words": c["words"], "gap": c["gap"], "nbits": c["nbits"], "subseq_bits": S}
        wg = with_gap if isinstance(with_gap, bool) else with_gap(len(fields))
        fields.append(hd.DeviceField.upload(enc, c["lengths"], c["n"], with_gap=wg))
        outs.append(torch.full((c["n"] + 16,), CANARY, dtype=torch.int32).to(torch.int16).cuda())
    return comps, fields, outs


def expected(c):
    # the oracle's bit-serial decode for small fields; for larger ones the
    # oracle's own round trip (its decode of its encoding returns the input,
    # pinned in test_oracle.py) lets the source codes stand in for it
    if c["n"] <= 1 << 17:
        return oracle.decode(c["words"], c["nbits"], c["codes"], c["lengths"], n_cap=c["n"])
    return c["x"]


def check_outputs(comps, outs):
    for k, (c, o) in enumerate(zip(comps, outs)):
        r = o.cpu().numpy().view(np.uint16)
        ref = expected(c)
        if not np.array_equal(r[:c["n"]], ref):
            bad = np.nonzero(r[:c["n"]] != ref)[0]
            raise AssertionError(f"field {k}: {bad.size} mismatches, first at {bad[:8].tolist()}")
        assert np.all(r[c["n"]:] == np.uint16(CANARY)), f"field {k}: write past the output"


def reset(outs):
    for o in outs:
        o.fill_(CANARY - 65536)


def test_batch_graph_is_replayed_for_later_batches(ctx):
    from paper_2201_09118_gb300 import hd
    # three batches of the same class (same error-bound range and alphabet,
    # different sizes and seeds) share one captured graph
    batches = [make_batch(10, 1 << 12, 1 << 17, seed, alphabets=(1024,), eb_lo=1e-4,
                          eb_hi=1e-4) for seed in (101, 102, 103)]
    for rep in range(2):
        for comps, fields, outs in batches:
            reset(outs)
            ctx.decode_batch(fields, outs)
            rc, st = ctx.batch_status(len(fields))
            assert rc == hd.HD_OK and np.all(st == 0)
            check_outputs(comps, outs)
    captures, cached = ctx.graph_stats()
    assert captures == 1 and cached == 1


def test_batch_uneven_sizes_and_alphabets(ctx):
    from paper_2201_09118_gb300 import hd
    comps, fields, outs = make_batch(40, 1 << 8, 1 << 20, 202)
    ctx.decode_batch(fields, outs)
    rc, st = ctx.batch_status(len(fields))
    assert rc == hd.HD_OK and np.all(st == 0)
    check_outputs(comps, outs)


def test_batch_equals_per_field_decode(ctx):
    comps, fields, outs = make_batch(16, 1 << 10, 1 << 18, 303)
    ctx.decode_batch(fields, outs)
    assert ctx.batch_status(len(fields))[0] == 0
    for f, c, o in zip(fields, comps, outs):
        single = torch.full_like(o, CANARY - 65536)
        ctx.decode(f, single)
        assert ctx.status() == 0
        assert torch.equal(single, o)


def test_batch_both_strategies(ctx):
    from paper_2201_09118_gb300 import hd
    comps, fields, outs = make_batch(12, 1 << 10, 1 << 18, 404, with_gap=lambda k: k % 3 != 0)
    ctx.decode_batch(fields, outs)
    rc, st = ctx.batch_status(len(fields))
    assert rc == hd.HD_OK and np.all(st == 0)
    check_outputs(comps, outs)


def test_batch_self_sync_only(ctx):
    from paper_2201_09118_gb300 import hd
    comps, fields, outs = make_batch(10, 1 << 10, 1 << 18, 505, with_gap=False)
    ctx.decode_batch(fields, outs)
    rc, st = ctx.batch_status(len(fields))
    assert rc == hd.HD_OK and np.all(st == 0)
    check_outputs(comps, outs)


def test_batch_corrupt_field_reported_alone(ctx):
    from paper_2201_09118_gb300 import hd
    comps, fields, outs = make_batch(6, 1 << 12, 1 << 16, 606)
    bad = 2
    f = fields[bad]
    fields[bad] = hd.DeviceField(f.words, f.nbits, f.gap, f.subseq_bits, f.lengths, f.alphabet,
                                 f.n + 1)
    ctx.decode_batch(fields, outs)
    rc, st = ctx.batch_status(len(fields))
    assert rc == hd.HD_ERR_CORRUPT
    assert st[bad] == hd.HD_ERR_CORRUPT
    assert all(st[k] == 0 for k in range(len(fields)) if k != bad)
    check_outputs([c for k, c in enumerate(comps) if k != bad],
                  [o for k, o in enumerate(outs) if k != bad])
    r = outs[bad].cpu().numpy().view(np.uint16)
    assert np.all(r[comps[bad]["n"] + 1:] == np.uint16(CANARY))


def test_batch_capacity_growth_recaptures(ctx):
    small = make_batch(4, 1 << 10, 1 << 12, 707, alphabets=(1024,))
    large = make_batch(30, 1 << 16, 1 << 19, 708, alphabets=(1024,))
    for comps, fields, outs in (small, large, small):
        reset(outs)
        ctx.decode_batch(fields, outs)
        assert ctx.batch_status(len(fields))[0] == 0
        check_outputs(comps, outs)
    captures, _ = ctx.graph_stats()
    assert captures >= 2


def test_autotune_choice_decodes_exactly(ctx):
    from paper_2201_09118_gb300 import hd
    comps, fields, outs = make_batch(8, 1 << 12, 1 << 17, 808)
    best = ctx.autotune(fields, outs)
    assert best["subseq_bits"] in (128, 256, 512)
    assert best["threads"] in (128, 256, 512)
    assert best["lut_bits"] in (11, 12, 13, 14)
    check_outputs(comps, outs)  # the tuner leaves the batch decoded
    reset(outs)
    ctx.decode_batch(fields, outs)
    rc, st = ctx.batch_status(len(fields))
    assert rc == hd.HD_OK and np.all(st == 0)
    check_outputs(comps, outs)
    # the stored choice is the shape the batch now runs with
    assert ctx.get_config()["window"] > 0


def test_autotune_self_sync(ctx):
    comps, fields, outs = make_batch(6, 1 << 12, 1 << 16, 909, with_gap=False)
    best = ctx.autotune(fields, outs)
    assert best["subseq_bits"] in (64, 128, 256)
    reset(outs)
    ctx.decode_batch(fields, outs)
    assert ctx.batch_status(len(fields))[0] == 0
    check_outputs(comps, outs)


def test_autotune_cache_saved_and_loaded_by_a_new_context(ctx, tmp_path):
    from paper_2201_09118_gb300 import hd
    comps, fields, outs = make_batch(8, 1 << 12, 1 << 17, 818)
    best = ctx.autotune(fields, outs)
    path = str(tmp_path / "tune.txt")
    ctx.autotune_save(path)
    lines = open(path).read().split("\n")
    assert lines[0] == "hd-autotune 1" and len([ln for ln in lines[1:] if ln]) >= 1
    c2 = hd.Context(0)
    try:
        assert c2.autotune_load(path) >= 1
        reset(outs)
        c2.decode_batch(fields, outs)
        assert c2.batch_status(len(fields))[0] == 0
        check_outputs(comps, outs)
        got = c2.get_config()
        for k in ("subseq_bits", "threads", "lut_bits"):
            assert got[k] == best[k], (k, got, best)
        # entries of another device are skipped, a file of another kind is refused
        other = str(tmp_path / "other.txt")
        with open(other, "w") as fh:
            fh.write("hd-autotune 1\n")
            for ln in lines[1:]:
                if ln:
                    fh.write("Some_Other_GPU " + ln.split(" ", 1)[1] + "\n")
        assert c2.autotune_load(other) == 0
        bad = str(tmp_path / "bad.txt")
        with open(bad, "w") as fh:
            fh.write("hd-autotune 1\nname 0 1 2\n")
        with pytest.raises(hd.HDError):
            c2.autotune_load(bad)
        with pytest.raises(hd.HDError):
            c2.autotune_load(str(tmp_path / "missing.txt"))
    finally:
        c2.close()
