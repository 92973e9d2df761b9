"""CPU-side checks of the C-ABI library: it builds for sm_103a, loads, exports
every symbol include/hd.h declares, and its host-side codebook builder and
encoder agree with the oracle.  No GPU work is issued here."""
import os
import re

import numpy as np
import pytest

import oracle
import synth
from paper_2201_09118_gb300 import hd

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_symbols():
    src = open(os.path.join(ROOT, "include", "hd.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(hd_[a-z_]+)\s*\(", src)))


def test_library_loads_and_exports_every_declared_symbol():
    lib = hd.load()
    declared = _declared_symbols()
    assert declared, "no declarations parsed"
    for name in declared:
        assert hasattr(lib, name), name
    # the binding wraps exactly the declared entry points
    assert sorted(hd.exported_symbols()) == declared
    assert hd.hd_version().startswith("hd-gb300")


@pytest.mark.parametrize("A,scale,seed", [(1024, 2.0, 1), (1024, 40.0, 2), (256, 8.0, 3),
                                          (4096, 300.0, 4)])
def test_codebook_cost_equals_oracle(A, scale, seed):
    x = synth.laplace_codes(50000, scale=scale, center=A // 2, alphabet=A, seed=seed)
    freq = oracle.histogram(x, A).astype(np.int64)
    L = hd.hd_build_codebook(x, A)
    Lo = oracle.code_lengths(freq.astype(np.uint64))
    assert int((freq * L).sum()) == int((freq * Lo).sum())
    assert all((L > 0) == (freq > 0))
    assert sum(2.0 ** -int(l) for l in L if l) == pytest.approx(1.0, abs=0)


def test_codebook_length_limit_matches_package_merge_cost():
    fib = [1, 1]
    while len(fib) < 40:
        fib.append(fib[-1] + fib[-2])
    x = np.repeat(np.arange(40, dtype=np.uint16), fib)
    freq = np.array(fib, np.int64)
    for limit in (32, 20, 8):
        L = hd.hd_build_codebook(x, 64, max_len=limit)[:40]
        Lo = oracle.package_merge(freq.astype(np.uint64), limit)
        assert int(L.max()) <= limit
        assert int((freq * L).sum()) == int((freq * Lo).sum())


@pytest.mark.parametrize("S", [64, 128, 256])
def test_encoder_bit_exact_with_oracle(S):
    x = synth.laplace_codes(123457, scale=5.0, seed=9)
    L = hd.hd_build_codebook(x, 1024)
    enc = hd.hd_encode(x, L, S)
    words, nbits = oracle.encode(x, L, oracle.canonical_codes(L), S)
    assert enc["nbits"] == nbits
    assert np.array_equal(enc["words"], words)
    assert np.array_equal(enc["gap"], oracle.gap_build(x, L, S, nbits))


def test_encoder_errors():
    x = np.array([1, 2, 3], np.uint16)
    L = np.zeros(8, np.uint8)
    L[1] = L[2] = 1
    with pytest.raises(hd.HDError) as e:
        hd.hd_encode(x, L, 128)
    assert e.value.code == hd.HD_ERR_SYMBOL
    with pytest.raises(hd.HDError) as e:
        hd.hd_encode(x, np.array([0, 1, 1, 1], np.uint8), 128)
    assert e.value.code == hd.HD_ERR_ARG
    with pytest.raises(hd.HDError) as e:
        hd.hd_encode(x, np.array([0, 2, 2, 2], np.uint8), 96)
    assert e.value.code == hd.HD_ERR_ARG
    with pytest.raises(hd.HDError) as e:
        hd.hd_build_codebook(np.array([9], np.uint16), 8)
    assert e.value.code == hd.HD_ERR_SYMBOL


def test_codebook_from_counts_matches_codebook_from_symbols():
    x = synth.laplace_codes(100000, scale=12.0, seed=9)
    freq = np.bincount(x, minlength=1024).astype(np.uint64)
    assert np.array_equal(hd.hd_build_codebook_freq(freq, 32), hd.hd_build_codebook(x, 1024, 32))
    with pytest.raises(hd.HDError):
        hd.hd_build_codebook_freq(np.zeros(1, np.uint64), 32)  # alphabet < 2


def test_struct_layouts_match_the_header(tmp_path):
    """Every ABI struct the binding declares has the header's size and field
    offsets (compiled from include/hd.h with the host C compiler)."""
    import ctypes
    import shutil
    import subprocess
    cc = shutil.which("gcc") or shutil.which("cc")
    if not cc:
        pytest.skip("no C compiler")
    exe = str(tmp_path / "abi_layout")
    subprocess.run([cc, "-O0", "-I", os.path.join(ROOT, "include"),
                    os.path.join(ROOT, "tests", "native", "abi_layout.c"), "-o", exe], check=True)
    out = subprocess.run([exe], capture_output=True, text=True, check=True).stdout
    got = dict(line.rsplit(" ", 1) for line in out.strip().splitlines())
    from paper_2201_09118_gb300 import hd
    for name, cls in [("hd_stream_info", hd.hd_stream_info), ("hd_field", hd.hd_field),
                      ("hd_config", hd.hd_config), ("hd_serve_config", hd.hd_serve_config),
                      ("hd_result", hd.hd_result), ("hd_serve_stats_t", hd.hd_serve_stats_t),
                      ("hd_lorenzo", hd.hd_lorenzo)]:
        assert int(got[name]) == ctypes.sizeof(cls), name
        for field, _ in cls._fields_:
            key = f"{name}.{field}"
            if key in got:
                assert int(got[key]) == getattr(cls, field).offset, key
