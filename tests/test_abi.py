"""CPU checks of the C ABI: the library builds, loads and exports every symbol
that include/vie.h declares; the ctypes structs match the header's layout."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "vie.h")).read()
    return sorted(set(re.findall(r"\b(vie_[a-z_0-9]+)\s*\(", src)))


def test_library_exports_every_declared_symbol():
    from paper_1809_05334_gb300 import build, vie
    build.build()
    lib = vie.load()
    names = _declared()
    assert len(names) >= 10
    for n in names:
        assert hasattr(lib, n), n
    assert sorted(vie.EXPORTS) == names


def test_struct_layout_matches_header():
    from paper_1809_05334_gb300 import vie
    # vie_options: 4 int32 + 2 double + 2 int32
    assert ctypes.sizeof(vie.Options) == 4 * 4 + 2 * 8 + 2 * 4
    # vie_request: 3 double + 16 double + pointer + int32 (+ padding)
    assert ctypes.sizeof(vie.Request) == 3 * 8 + 16 * 8 + 8 + 8
    assert vie.Result.absorbed.offset % 8 == 0


def test_status_strings_and_no_gpu_error():
    from paper_1809_05334_gb300 import vie
    lib = vie.load()
    assert lib.vie_status_str(-4) == b"VIE_RAYLEIGH_ANOMALY"
    assert lib.vie_status_str(12345) == b"VIE_UNKNOWN"
    assert lib.vie_last_error(None) == b""
    import torch
    if not torch.cuda.is_available():
        with pytest.raises(vie.VIEError):
            vie.Solver()
