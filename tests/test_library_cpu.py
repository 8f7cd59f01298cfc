"""Host-side checks of the C-ABI library that need no GPU: it loads, exports
every entry point include/messi.h declares, rejects invalid arguments before
touching the device, and its breakpoints agree with the oracle's."""
import ctypes
import os
import re
import subprocess

import numpy as np
import pytest

import oracle

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "messi.h")


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__

    __graft_entry__.build()
    return ctypes.CDLL(os.path.join(ROOT, "paper_2110_07519_gb300", "libmessi.so"))


def declared():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(messi_[a-z_]+)\s*\(", text)))


def test_header_declares_the_abi():
    names = declared()
    for must in ("messi_build", "messi_query", "messi_query_batched", "messi_free", "messi_query_stats",
                 "messi_lower_bounds", "messi_summarize", "messi_last_error", "messi_check"):
        assert must in names


def test_library_exports_every_declared_symbol(lib):
    path = os.path.join(ROOT, "paper_2110_07519_gb300", "libmessi.so")
    out = subprocess.run(["nm", "-D", "--defined-only", path], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\bT (messi_\w+)", out))
    missing = [n for n in declared() if n not in exported]
    assert not missing, missing
    for n in declared():
        assert hasattr(lib, n)
    # nothing but the C ABI leaks out (the static CUDA runtime stays private)
    assert all(s.startswith("messi_") for s in re.findall(r"\bT (\w+)", out))


def test_python_binding_names_match_header():
    import paper_2110_07519_gb300 as m

    for n in declared():
        assert callable(getattr(m, n)), n


@pytest.mark.parametrize("card", [2, 4, 8, 16, 32, 64, 128, 256])
def test_breakpoints_match_oracle(card):
    # both sides compute the double nearest each quantile (each by its own
    # method): the tables agree bit for bit, so a PAA value gets the same
    # symbol from either
    import paper_2110_07519_gb300 as m

    lib_b = m.messi_breakpoints(card)
    orc_b = oracle.breakpoints(card)
    assert np.array_equal(lib_b.view(np.uint64), orc_b.view(np.uint64))
    assert np.all(np.diff(lib_b) > 0)


@pytest.mark.parametrize("card", [4, 16, 64, 256])
def test_library_breakpoints_correctly_rounded(card):
    # against a 300-bit evaluation of the quantile (mpmath), independently
    # of the oracle
    mpmath = pytest.importorskip("mpmath")
    import paper_2110_07519_gb300 as m

    mpmath.mp.prec = 300
    lib_b = m.messi_breakpoints(card)
    for j in range(1, card):
        exact = mpmath.sqrt(2) * mpmath.erfinv(2 * mpmath.mpf(j) / card - 1)
        got = lib_b[j - 1]
        gap = abs(mpmath.mpf(got) - exact)
        for nb in (np.nextafter(got, -np.inf), np.nextafter(got, np.inf)):
            assert gap < abs(mpmath.mpf(nb) - exact), (card, j)


def test_invalid_arguments_rejected_without_gpu(lib):
    import paper_2110_07519_gb300 as m

    out = ctypes.c_void_p()
    x = np.zeros((4, 256), np.float32)
    p = x.ctypes.data
    bad = [
        (p, 4, 250, 16, 256),     # len not a multiple of segments
        (p, 4, 256, 17, 256),     # too many segments
        (p, 4, 256, 16, 100),     # cardinality not a power of two
        (p, 4, 256, 16, 512),     # cardinality above 256
        (p, 0, 256, 16, 256),     # empty collection
        (p, 4, 48, 16, 256),      # segment length 3, not a power of two >= 4
        (None, 4, 256, 16, 256),  # null series
    ]
    for args in bad:
        st = lib.messi_build(ctypes.c_void_p(args[0]) if args[0] else None, ctypes.c_uint64(args[1]),
                             ctypes.c_uint32(args[2]), ctypes.c_uint32(args[3]), ctypes.c_uint32(args[4]),
                             None, None, ctypes.byref(out))
        assert st == 1, args
        assert m.messi_last_error() != ""
    assert lib.messi_breakpoints(ctypes.c_uint32(3), None) == 1
    assert lib.messi_query(None, None, 1, 1, 0, 0, None, None, None) == 1
    assert lib.messi_query_stats(None, None) == 1
    lib.messi_free(None)


def test_every_declared_entry_point_is_documented():
    # each C-ABI declaration is preceded by a comment block stating what it
    # does (the passage it implements, or that the paper has no counterpart)
    text = open(HEADER).read()
    decls = list(re.finditer(r"\n(?:messi_status|void|const char \*)\s+\*?(messi_\w+)\s*\(", text))
    assert decls
    undocumented = []
    for d in decls:
        before = text[: d.start()].rstrip()
        # an enum line may sit between the comment and the declaration
        before = re.sub(r"\n\s*enum\s*\{[^}]*\};\s*$", "", before).rstrip()
        if not before.endswith("*/"):
            undocumented.append(d.group(1))
    assert not undocumented, undocumented


def test_windows_arguments_rejected_without_gpu(lib):
    # messi_windows validates before touching the device: null, empty or
    # oversize windows, zero stride, a series shorter than one window, and
    # host pointers are EINVAL
    P, U32, U64 = ctypes.c_void_p, ctypes.c_uint32, ctypes.c_uint64
    f = lib.messi_windows
    f.argtypes = [P, U64, U32, U32, ctypes.c_int32, P, ctypes.POINTER(U64), P]
    x = np.zeros(100, np.float32)
    o = np.zeros(37 * 64, np.float32)
    cnt = U64(0)
    xs, os_ = P(x.ctypes.data), P(o.ctypes.data)
    assert f(None, 100, 64, 1, 1, os_, ctypes.byref(cnt), None) == 1
    assert f(xs, 100, 64, 1, 1, None, ctypes.byref(cnt), None) == 1
    assert f(xs, 100, 0, 1, 1, os_, ctypes.byref(cnt), None) == 1
    assert f(xs, 100, 70_000, 1, 1, os_, ctypes.byref(cnt), None) == 1
    assert f(xs, 100, 64, 0, 1, os_, ctypes.byref(cnt), None) == 1
    assert f(xs, 50, 64, 1, 1, os_, ctypes.byref(cnt), None) == 1
    assert f(xs, 100, 64, 1, 1, os_, ctypes.byref(cnt), None) == 1     # host buffers
    assert cnt.value == 0


def test_bench_traffic_gate_follows_the_kernel_source(tmp_path, monkeypatch):
    # bench.py reports the ncu DRAM traffic only while the kernel's sources
    # hash to the value recorded beside it; scaled by the number of series
    import importlib.util

    spec = importlib.util.spec_from_file_location("bench_gate", os.path.join(ROOT, "bench.py"))
    b = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(b)
    csrc = tmp_path / "paper_2110_07519_gb300" / "csrc"
    csrc.mkdir(parents=True)
    for name in ("screen.cu", "tc.cuh", "device_common.cuh"):
        (csrc / name).write_text(f"// {name}\n")
    (tmp_path / "profiles").mkdir()
    monkeypatch.setattr(b, "ROOT", str(tmp_path))
    sha = b.scan_source_sha("k_tc_screen")
    (tmp_path / "profiles" / "k_tc_screen_traffic.txt").write_text(
        f"# test\nsource_sha: {sha}\ndram_bytes_per_series: 520.5\n")
    assert b.profiled_traffic(1000, "k_tc_screen") == pytest.approx(520_500.0)
    (csrc / "screen.cu").write_text("// changed\n")
    assert b.profiled_traffic(1000, "k_tc_screen") is None
    assert b.profiled_traffic(1000, "k_lb_scan") is None          # no summary for it here


def test_autotune_cache_reuses_a_stored_choice(tmp_path, monkeypatch):
    # the binding's cache: the first call times the shapes and stores the
    # choice under (collection shape, batch mode, k, device); the next call
    # applies it without timing; an unreadable cache counts as empty
    import types

    import paper_2110_07519_gb300 as m

    calls = {"tune": 0, "set": []}
    choice = {"batch": 128, "chunk_tiles": 16, "ctas_per_sm": 2, "mode": 0, "ms_per_query": 1.5}

    def fake_tune(index, queries, k=1, stream=None):
        calls["tune"] += 1
        return dict(choice)

    monkeypatch.setattr(m, "messi_index_get_info", lambda ix: {"n_series": 1000, "len": 256})
    monkeypatch.setattr(m, "messi_autotune", fake_tune)
    monkeypatch.setattr(m, "messi_set_tuning", lambda ix, b, c, s: calls["set"].append((b, c, s)))
    ix = types.SimpleNamespace(_batch_mode=0)
    cache = tmp_path / "tune.json"
    cache.write_text("not json")
    assert m.autotune_cached(ix, None, k=1, cache=str(cache)) == choice
    assert calls == {"tune": 1, "set": []}
    assert m.autotune_cached(ix, None, k=1, cache=str(cache)) == choice
    assert calls["tune"] == 1 and calls["set"] == [(128, 16, 2)]
    m.autotune_cached(ix, None, k=10, cache=str(cache))            # another k: timed again
    assert calls["tune"] == 2


def test_bench_clock_sampler_parses_reasons():
    # the timed region's clock record: median SM clock, the highest max
    # clock, and every throttle reason seen active in any sample
    import importlib.util

    spec = importlib.util.spec_from_file_location("bench_clk", os.path.join(ROOT, "bench.py"))
    b = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(b)

    class FakeProc:
        def terminate(self):
            pass

        def communicate(self, timeout=None):
            return ("1965, 2070, 1100.5, 0x0, Not Active, Not Active, Not Active, Not Active\n"
                    "1650, 2070, 1398.0, 0x4, Not Active, Not Active, Not Active, Active\n"
                    "garbage line\n"
                    "1700, 2070, 1390.0, 0x4, Not Active, Not Active, Not Active, Active\n", "")

    s = b.ClockSampler.__new__(b.ClockSampler)
    s.proc = FakeProc()
    rec = s.stop()
    assert rec == {"sm_mhz": 1700.0, "sm_max_mhz": 2070.0, "reasons": ["sw_power_cap"], "samples": 3}
    s.proc = None
    assert s.stop()["reasons"] == ["nvidia-smi unavailable"]
