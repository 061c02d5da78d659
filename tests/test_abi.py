"""The C-ABI library builds, loads without a GPU, and exports every entry
point that include/ljsel.h declares (no compute calls: CPU only)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "ljsel.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(ljsel_[a-z_0-9]+)\s*\(", src)))


@pytest.fixture(scope="module")
def built():
    import __graft_entry__
    __graft_entry__.build()
    import paper_2505_03438_gb300 as lj
    return lj


def test_every_declared_symbol_is_exported(built):
    names = _declared()
    assert len(names) >= 18
    L = ctypes.CDLL(built.LIB_PATH)
    for n in names:
        assert hasattr(L, n), n
    # the binding wraps each of them under the same name
    assert set(names) == set(built.EXPORTED)
    for n in names:
        assert hasattr(built, n), n


def test_abi_version_and_error_string(built):
    L = built.lib()
    assert L.ljsel_abi_version() == 1
    assert isinstance(L.ljsel_last_error(), bytes)


def test_struct_layouts_match_header(built):
    # the ctypes mirrors must have the C sizes (checked against a C compile)
    import subprocess
    import tempfile
    code = r'''
    #include <stdio.h>
    #include "ljsel.h"
    int main(void){printf("%zu %zu %zu %zu %zu %zu %zu\n", sizeof(ljsel_params), sizeof(ljsel_config),
      sizeof(ljsel_stats), sizeof(ljsel_counters), sizeof(ljsel_tuner_opts), sizeof(ljsel_tuner_report),
      sizeof(ljsel_profile));printf("%zu\n", sizeof(ljsel_peaks));return 0;}
    '''
    with tempfile.TemporaryDirectory() as d:
        c = os.path.join(d, "s.c")
        open(c, "w").write(code)
        exe = os.path.join(d, "s")
        subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), c, "-o", exe], check=True)
        out = subprocess.run([exe], capture_output=True, text=True, check=True).stdout.split()
    sizes = [ctypes.sizeof(t) for t in (built.ljsel_params, built.ljsel_config, built.ljsel_stats,
                                        built.ljsel_counters, built.ljsel_tuner_opts, built.ljsel_tuner_report,
                                        built.ljsel_profile, built.ljsel_peaks)]
    assert [int(s) for s in out] == sizes


def test_invalid_arguments_fail_without_gpu(built):
    import numpy as np
    # a box below 2 (r_c + skin) is rejected before any device call
    p = built.make_params(box=5.0, rcut=2.5, skin=0.3)
    x = np.zeros((4, 3))
    with pytest.raises(built.LjselError) as e:
        built.ljsel_create(p, 4, x, x)
    assert e.value.status == 5
    p = built.make_params(box=20.0, eps=[[1.0, 1.5], [1.2, 0.5]], sigma=[[1, 1], [1, 1]])
    with pytest.raises(built.LjselError) as e:
        built.ljsel_create(p, 4, x, x)
    assert e.value.status == 1
    # more particles than a 27-bit list index can name
    p = built.make_params(box=20.0)
    with pytest.raises(built.LjselError) as e:
        built.ljsel_create(p, 1 << 27, x, x)
    assert e.value.status == 1
    # batches: one species only; every replica box at least 2 (r_c + skin); counts >= 0
    boxes = np.full((2, 3), 20.0)
    with pytest.raises(built.LjselError) as e:
        built.ljsel_batch_create(built.make_params(20.0, eps=[[1, 1], [1, 1]], sigma=[[1, 1], [1, 1]]), boxes,
                                 [2, 2], x, x)
    assert e.value.status == 9
    with pytest.raises(built.LjselError) as e:
        built.ljsel_batch_create(built.make_params(20.0), np.array([[20.0] * 3, [5.0] * 3]), [2, 2], x, x)
    assert e.value.status == 5
    with pytest.raises(built.LjselError) as e:
        built.ljsel_batch_create(built.make_params(20.0), boxes, [5, -1], x, x)
    assert e.value.status == 1
    with pytest.raises(built.LjselError) as e:
        built.ljsel_batch_create(built.make_params(20.0, walls=(1, 0, 0)), boxes, [2, 2], x, x)
    assert e.value.status == 9
    # a wall flag is 0 or 1
    p = built.make_params(20.0)
    p.walls[0] = 2
    with pytest.raises(built.LjselError) as e:
        built.ljsel_create(p, 4, x, x)
    assert e.value.status == 1


def test_batch_tile_layout(built):
    assert ctypes.sizeof(built.ljsel_batch_tile) == 16


def test_missing_library_fails_loudly(monkeypatch, built):
    import paper_2505_03438_gb300 as lj
    monkeypatch.setattr(lj, "LIB_PATH", "/nonexistent/libljsel.so")
    monkeypatch.setattr(lj, "_lib", None)
    with pytest.raises(RuntimeError):
        lj.lib()
