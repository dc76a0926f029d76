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
    # vie_options: 4 int32 + 2 double + 4 int32
    assert ctypes.sizeof(vie.Options) == 4 * 4 + 2 * 8 + 4 * 4
    # vie_request: 3 double + 16 double + pointer + 2 int32 + pointer
    assert ctypes.sizeof(vie.Request) == 3 * 8 + 16 * 8 + 8 + 8 + 8
    assert vie.Result.absorbed.offset % 8 == 0


def test_struct_layout_compiled_against_header(tmp_path):
    """sizeof/offsetof of every ABI struct, as the C compiler lays them out from
    include/vie.h, equal the ctypes mirrors of the binding."""
    import shutil
    import subprocess
    from paper_1809_05334_gb300 import vie
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    structs = {"vie_options": vie.Options, "vie_request": vie.Request, "vie_result": vie.Result,
               "vie_mesh": vie.Mesh, "vie_server_stats": vie.ServerStats, "vie_tune_report": vie.TuneReport}
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "vie.h"', "int main(void) {"]
    for cname, cls in structs.items():
        lines.append('printf("%s size %%zu\\n", sizeof(%s));' % (cname, cname))
        for f, _ in cls._fields_:
            lines.append('printf("%s %s %%zu\\n", offsetof(%s, %s));' % (cname, f, cname, f))
    lines.append("return 0; }")
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run([cc, "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    got = {tuple(l.split()[:2]): int(l.split()[2]) for l in out if l.strip()}
    for cname, cls in structs.items():
        assert got[(cname, "size")] == ctypes.sizeof(cls), cname
        for f, _ in cls._fields_:
            assert got[(cname, f)] == getattr(cls, f).offset, (cname, f)


def test_status_strings_and_no_gpu_error():
    from paper_1809_05334_gb300 import vie
    lib = vie.load()
    assert lib.vie_status_str(-4) == b"VIE_RAYLEIGH_ANOMALY"
    for code, name in vie.STATUS.items():
        assert lib.vie_status_str(code).decode() == name
    assert lib.vie_status_str(12345) == b"VIE_UNKNOWN"
    assert lib.vie_last_error(None) == b""
    import torch
    if not torch.cuda.is_available():
        with pytest.raises(vie.VIEError):
            vie.Solver()
        with pytest.raises(vie.VIEError):
            vie.Server()
