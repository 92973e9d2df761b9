"""GPU tests of the serving loop (hd_serve_*): every request's output is the
same as decoding its field alone (and as the oracle's decode), whatever else
shares its batch or runs beside it; admission respects the memory budget."""
import random
import time

import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def pool():
    """Resident fields of uneven sizes, own codebooks, both strategies, with
    each field's output decoded alone through hd_decode."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2201_09118_gb300 import hd
    ctx = hd.Context(0)
    specs = synth.batch_spec(14, lo=1 << 8, hi=1 << 19, seed=1234)
    fields, alone, comps = [], [], []
    for k, sp in enumerate(specs):
        x = synth.smooth_codes_1d(sp.n, sp.rel_eb, alphabet=sp.alphabet, seed=sp.seed)
        c = oracle.compress(x, sp.alphabet, S=128)
        c["x"] = x
        enc = {"words": c["words"], "gap": c["gap"], "nbits": c["nbits"], "subseq_bits": 128}
        f = hd.DeviceField.upload(enc, c["lengths"], c["n"], with_gap=(k % 4 != 3))
        out = torch.empty(c["n"], dtype=torch.int16, device="cuda")
        ctx.decode(f, out)
        assert ctx.status() == 0
        fields.append(f)
        alone.append(out)
        comps.append(c)
    for c, o in zip(comps, alone):
        ref = c["x"] if c["n"] > 1 << 16 else oracle.decode(
            c["words"], c["nbits"], c["codes"], c["lengths"], n_cap=c["n"])
        assert np.array_equal(o.cpu().numpy().view(np.uint16), ref)
    yield fields, alone, comps
    ctx.close()


def result_tensor(res):
    from paper_2201_09118_gb300 import hd
    return hd.device_u16_view(res["d_out"], res["n"])


def collect(srv, tickets, release=True, timeout_s=60.0):
    got = {}
    t0 = time.time()
    while len(got) < len(tickets):
        for t in srv.completed():
            t = int(t)
            res = srv.poll(t)
            assert res is not None
            got[t] = (res, result_tensor(res).clone() if res["status"] == 0 else None)
            if release:
                srv.release(t)
        assert time.time() - t0 < timeout_s, "requests did not complete"
    return got


@pytest.mark.parametrize("slots,max_batch", [(2, 16), (4, 4), (1, 64)])
def test_each_result_same_alone_and_in_the_mix(pool, slots, max_batch):
    from paper_2201_09118_gb300 import hd
    fields, alone, _ = pool
    srv = hd.Server(0, budget_bytes=1 << 30, slots=slots, max_batch=max_batch)
    ids = [srv.register(f) for f in fields]
    rng = random.Random(slots * 100 + max_batch)
    order = [rng.randrange(len(ids)) for _ in range(120)]
    tickets = {}
    for k, fid in enumerate(order):
        tickets[srv.submit(ids[fid])] = fid
        if k % 7 == 0:
            time.sleep(rng.random() * 2e-4)  # arrivals while earlier batches run
    got = collect(srv, list(tickets))
    for t, fid in tickets.items():
        res, out = got[t]
        assert res["status"] == hd.HD_OK
        assert res["n"] == fields[fid].n
        assert res["latency_us"] >= res["queue_us"] >= 0
        assert torch.equal(out, alone[fid])
    st = srv.stats()
    assert st["completed"] == len(order) and st["pending"] == 0 and st["in_flight"] == 0
    assert st["used_bytes"] == 0
    if max_batch > 1:
        assert st["batches"] < len(order)  # requests shared launches
    srv.close()


def test_direct_one_launch_per_request(pool):
    from paper_2201_09118_gb300 import hd
    fields, alone, _ = pool
    srv = hd.Server(0, budget_bytes=1 << 30, slots=1, max_batch=1, direct=True)
    ids = [srv.register(f) for f in fields]
    tickets = {srv.submit(ids[k % len(ids)]): k % len(ids) for k in range(30)}
    got = collect(srv, list(tickets))
    for t, fid in tickets.items():
        assert got[t][0]["status"] == 0
        assert torch.equal(got[t][1], alone[fid])
    assert srv.stats()["batches"] == 30
    srv.close()


def test_budget_admission_waits_for_released_outputs(pool):
    from paper_2201_09118_gb300 import hd
    fields, alone, _ = pool
    big = max(range(len(fields)), key=lambda k: fields[k].n)
    need = 2 * fields[big].n
    budget = 2 * ((need + 255) // 256 * 256) + 256  # room for two of the largest
    srv = hd.Server(0, budget_bytes=budget, slots=2, max_batch=8)
    fid = srv.register(fields[big])
    tickets = [srv.submit(fid) for _ in range(9)]
    got = collect(srv, tickets, release=True)
    for t in tickets:
        assert got[t][0]["status"] == 0
        assert torch.equal(got[t][1], alone[big])
    st = srv.stats()
    assert st["peak_bytes"] <= st["budget_bytes"]
    assert st["batches"] >= 5  # at most two outputs could be live at once
    srv.close()


def test_submit_rejects_output_larger_than_budget(pool):
    from paper_2201_09118_gb300 import hd
    fields, _, _ = pool
    big = max(range(len(fields)), key=lambda k: fields[k].n)
    srv = hd.Server(0, budget_bytes=1 << 12, slots=1, max_batch=4)
    fid = srv.register(fields[big])
    with pytest.raises(hd.HDError) as e:
        srv.submit(fid)
    assert e.value.code == hd.HD_ERR_NOMEM
    srv.close()


def test_corrupt_request_reported_alone(pool):
    from paper_2201_09118_gb300 import hd
    fields, alone, _ = pool
    srv = hd.Server(0, budget_bytes=1 << 30, slots=1, max_batch=32)
    ids = [srv.register(f) for f in fields[:4]]
    f = fields[1]
    bad = srv.register(hd.DeviceField(f.words, f.nbits, f.gap, f.subseq_bits, f.lengths,
                                      f.alphabet, f.n + 3))
    tickets = [srv.submit(i) for i in ids] + [srv.submit(bad)]
    got = collect(srv, tickets)
    for k, t in enumerate(tickets[:-1]):
        assert got[t][0]["status"] == 0
        assert torch.equal(got[t][1], alone[k])
    assert got[tickets[-1]][0]["status"] == hd.HD_ERR_CORRUPT
    srv.close()


def test_destroy_with_requests_waiting_for_memory(pool):
    from paper_2201_09118_gb300 import hd
    fields, _, _ = pool
    big = max(range(len(fields)), key=lambda k: fields[k].n)
    srv = hd.Server(0, budget_bytes=(2 * fields[big].n + 255) // 256 * 256, slots=2,
                    max_batch=4)
    fid = srv.register(fields[big])
    for _ in range(6):
        srv.submit(fid)  # only one output fits and none is released
    time.sleep(0.05)
    t0 = time.time()
    srv.close()
    assert time.time() - t0 < 10


def test_watchdog_times_out_batches_without_handing_out_their_memory():
    # a 1-microsecond limit on batches of one large gap-array field (hundreds
    # of microseconds on the GPU, queued asynchronously): the worker finds each
    # batch still running at its first look, so the requests complete with
    # HD_ERR_TIMEOUT and no output, while the slot and the output memory stay
    # held until the work really ends; nothing hangs, the budget comes back in
    # full, and with the default limit the same requests decode exactly
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2201_09118_gb300 import hd
    x = synth.laplace_codes(1 << 24, scale=30.0, seed=91)
    c = oracle.compress(x, 1024, S=128)
    enc = {"words": c["words"], "gap": c["gap"], "nbits": c["nbits"], "subseq_bits": 128}
    f = hd.DeviceField.upload(enc, c["lengths"], c["n"], with_gap=True)
    ref = torch.from_numpy(x.view(np.int16)).cuda()
    srv = hd.Server(0, budget_bytes=1 << 30, slots=2, max_batch=1, watchdog_us=1)
    fid = srv.register(f)
    tickets = {srv.submit(fid): 0 for _ in range(8)}
    got = collect(srv, tickets)
    statuses = [res["status"] for res, _ in got.values()]
    assert set(statuses) <= {hd.HD_OK, hd.HD_ERR_TIMEOUT}
    assert statuses.count(hd.HD_ERR_TIMEOUT) > 0
    for res, out in got.values():
        if res["status"] == hd.HD_ERR_TIMEOUT:
            assert res["d_out"] in (None, 0)
        else:
            assert torch.equal(out, ref)
    srv.drain()
    t0 = time.time()
    while True:  # timed-out batches retire once their work has ended
        st = srv.stats()
        if st["timed_out_batches"] == 0 and st["used_bytes"] == 0:
            break
        assert time.time() - t0 < 30, st
        time.sleep(0.01)
    assert st["retired_batches"] > 0
    assert st["completed"] == st["submitted"] == 8
    srv.close()
    srv = hd.Server(0, budget_bytes=1 << 30, slots=2, max_batch=1)
    fid = srv.register(f)
    tickets = {srv.submit(fid): 0 for _ in range(8)}
    for res, out in collect(srv, tickets).values():
        assert res["status"] == hd.HD_OK
        assert torch.equal(out, ref)
    assert srv.stats()["timed_out_batches"] == 0
    srv.close()
