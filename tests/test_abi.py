"""CPU-side checks of the C ABI: the library builds, loads, and exports every
symbol include/vbdr.h declares; argument validation needs no GPU."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_symbols():
    txt = open(os.path.join(ROOT, "include", "vbdr.h")).read()
    return sorted(set(re.findall(r"VBDR_API\s+[\w\s\*]*?\b(vbdr_\w+)\s*\(", txt)))


@pytest.fixture(scope="module")
def lib():
    from paper_1810_13132_gb300 import vbdr
    return vbdr.load()


def test_header_declares_the_five_call_contract():
    syms = _declared_symbols()
    for s in ("vbdr_create", "vbdr_scan_slice", "vbdr_slide", "vbdr_estimate",
              "vbdr_destroy"):
        assert s in syms


def test_library_exports_every_declared_symbol(lib):
    from paper_1810_13132_gb300 import vbdr
    for s in _declared_symbols():
        assert hasattr(lib, s), s
    assert sorted(vbdr.exported_symbols()) == _declared_symbols()


def test_strerror(lib):
    from paper_1810_13132_gb300 import vbdr
    for code in range(0, -7, -1):
        assert lib.vbdr_strerror(code)
    assert lib.vbdr_strerror(-99) == b"unknown status"


def _cfg(**kw):
    from paper_1810_13132_gb300.vbdr import vbdr_config
    base = dict(k=10, log2_g=7, log2_g_min=0, group_rule=0, layout=0, reserved=0,
                num_bdr=1 << 16, seed=1)
    base.update(kw)
    return vbdr_config(**base)


@pytest.mark.parametrize("bad", [
    dict(k=0), dict(k=256), dict(layout=3), dict(reserved=1), dict(group_rule=2),
    dict(log2_g=0), dict(log2_g=17), dict(num_bdr=0), dict(num_bdr=(1 << 32) + 1),
    dict(num_bdr=1 << 32),  # the exact pool sum must fit 64 bits
    dict(num_bdr=128),  # Z must exceed g = 128
    dict(group_rule=1, log2_g_min=7),  # b_min + 3 > 9
    dict(log2_g=5, log2_g_min=6),
])
def test_create_rejects_invalid_config_without_touching_the_gpu(lib, bad):
    h = ctypes.c_void_p()
    c = _cfg(**bad)
    assert lib.vbdr_create(ctypes.byref(c), ctypes.byref(h)) == -1
    assert not h.value


def test_null_handle_calls(lib):
    assert lib.vbdr_create(None, None) == -1
    assert lib.vbdr_destroy(None) == 0
    assert lib.vbdr_scan_slice(None, None, 0, None) == -1
    assert lib.vbdr_slide(None, None) == -1
    assert lib.vbdr_estimate(None, None, 0, None, None) == -1
    assert lib.vbdr_estimate_alt(None, None, 0, None, 1, None) == -1
    assert lib.vbdr_copy_pool_sums_alt(None, None, None, None) == -1
    assert lib.vbdr_copy_pcsa(None, None, None) == -1
    assert lib.vbdr_selftest_bounded_wait(0, None) == -1  # refused before any CUDA call
    assert lib.vbdr_plan_create(None, None, 0, None, None) == -1
    assert lib.vbdr_plan_destroy(None) == 0
    assert lib.vbdr_plan_info(None, None, None, None) == -1
    assert lib.vbdr_plan_status(None) == -1
    assert lib.vbdr_estimate_planned(None, None, None, None) == -1
    assert lib.vbdr_estimate_planned_host(None, None, None, None) == -1
    assert lib.vbdr_estimate_planned_compact(None, None, None, ctypes.c_float(0.0), None,
                                             None) == -1


def test_noalloc_rejects_invalid_sizes_without_touching_the_gpu(lib):
    f = lib.vbdr_estimate_registers_noalloc
    dummy = ctypes.c_void_p(16)  # never dereferenced: the sizes are refused first
    assert f(dummy, 1 << 32, 8, 1, dummy, 1, dummy, None) == -1  # Z = 2^32
    assert f(dummy, 256, 8, 1, dummy, 1, dummy, None) == -1      # Z must exceed g
    assert f(dummy, 1 << 20, 0, 1, dummy, 1, dummy, None) == -1  # log2_g < 1
    assert f(dummy, 1 << 20, 10, 1, dummy, 1, dummy, None) == -4  # g above 512
    assert f(None, 1 << 20, 8, 1, dummy, 1, dummy, None) == -1


def test_oracle_and_library_share_no_source():
    """The oracle and the CUDA path are independent: no file of one includes,
    imports or links the other."""
    def code_refs(path):
        refs = []
        for line in open(path):
            t = line.strip()
            if t.startswith(("#include", "import ", "from ")) or "CDLL(" in t:
                refs.append(t)
        return " ".join(refs)

    pkg = os.path.join(ROOT, "paper_1810_13132_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".cu", ".cuh", ".py", ".h", ".cpp")):
                assert "oracle" not in code_refs(os.path.join(dirpath, f)), f
    for f in os.listdir(os.path.join(ROOT, "oracle")):
        if f.endswith((".c", ".py")):
            refs = code_refs(os.path.join(ROOT, "oracle", f))
            assert "paper_1810_13132_gb300" not in refs and "vbdr.h" not in refs, f


def test_compact_net_parameters(tmp_path):
    """CompactNet holds exactly the 465 FP32 parameters of the compact
    correction (host memory, passed with every launch) and its nmax."""
    import numpy as np
    from paper_1810_13132_gb300 import CompactNet
    with pytest.raises(ValueError):
        CompactNet(np.zeros(464), 1.0)
    theta = np.arange(465, dtype=np.float64) / 7.0
    path = tmp_path / "net.npz"
    np.savez(path, params=theta.astype(np.float32), nmax=np.float32(123.5))
    net = CompactNet.load(str(path))
    assert net.theta.dtype == np.float32 and net.theta.flags["C_CONTIGUOUS"]
    np.testing.assert_array_equal(net.theta, theta.astype(np.float32))
    assert net.nmax == 123.5
    from oracle import learned
    assert CompactNet.N_PARAMS == learned.C_N_PARAMS
