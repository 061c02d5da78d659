"""Run by tests/test_gpu_checked.py in a child process with
LJSEL_LIBRARY=checked: the process loaded the bounds-checked library and
not the plain one.  Skipped in a normal run."""
import os

import pytest

pytestmark = pytest.mark.gpu


@pytest.mark.skipif(os.environ.get("LJSEL_LIBRARY") != "checked", reason="only in the checked-build child run")
def test_the_checked_library_is_loaded():
    import paper_2505_03438_gb300 as lj
    lj.lib()
    assert lj.LIB_PATH.endswith("libljsel_checked.so")
    maps = open("/proc/self/maps").read()
    assert "libljsel_checked.so" in maps and "/libljsel.so" not in maps
