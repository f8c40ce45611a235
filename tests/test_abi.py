"""The C-ABI library builds for sm_103a, loads, and exports every entry point
declared in include/vmo.h (no compute calls: no GPU needed)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "vmo.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(vmo_[a-z_0-9]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    from paper_1105_4490_gb300 import _build_lib
    path = _build_lib.build()
    return ctypes.CDLL(path)


def test_every_declared_symbol_is_exported(lib):
    names = _declared()
    assert len(names) >= 20
    missing = [n for n in names if not hasattr(lib, n)]
    assert missing == []


def test_binding_covers_header():
    from paper_1105_4490_gb300 import vmo
    assert sorted(vmo.SYMBOLS) == _declared()


def test_status_strings_and_defaults(lib):
    from paper_1105_4490_gb300 import vmo
    L = vmo.load()
    assert L.vmo_status_string(0) == b"ok"
    assert L.vmo_status_string(6) == b"unsupported"
    p = vmo.default_params()
    assert (p.d, p.iters, p.km_iters, p.min_part, p.occupancy) == (3, 100, 20, 64, 8)
    assert abs(p.decay - 0.9) < 1e-6 and p.sigma == 1.0


def test_params_struct_layout():
    """The ctypes mirror matches the C struct (field order and size)."""
    from paper_1105_4490_gb300 import vmo
    assert ctypes.sizeof(vmo._Params) == 4 * 14 + 8  # 14 x 4-byte fields, uint64 seed
    assert ctypes.sizeof(vmo._Tree) == 8 + 7 * 8
    assert ctypes.sizeof(vmo._Stats) == 6 * 8


def test_struct_layouts_match_c(tmp_path):
    """sizeof / offsetof of every ABI struct, compiled from include/vmo.h with
    the host C compiler, equal the ctypes mirrors of the binding."""
    import shutil
    import subprocess
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no host C compiler")
    from paper_1105_4490_gb300 import vmo
    structs = {"vmo_params": vmo._Params, "vmo_csr": vmo._Csr, "vmo_tree": vmo._Tree, "vmo_stats": vmo._Stats,
               "vmo_server_config": vmo._ServerConfig, "vmo_request_info": vmo._RequestInfo,
               "vmo_server_stats": vmo._ServerStats, "vmo_tuning": vmo._Tuning}
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "vmo.h"', "int main(void) {"]
    for cname, ct in structs.items():
        lines.append(f'  printf("{cname} sizeof %zu\\n", sizeof({cname}));')
        for f, _ in ct._fields_:
            lines.append(f'  printf("{cname} {f} %zu\\n", offsetof({cname}, {f}));')
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run([cc, "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    got = {}
    for ln in out:
        if ln:
            s, f, v = ln.split()
            got[(s, f)] = int(v)
    for cname, ct in structs.items():
        assert got[(cname, "sizeof")] == ctypes.sizeof(ct), cname
        for f, _ in ct._fields_:
            assert got[(cname, f)] == getattr(ct, f).offset, (cname, f)


def test_tuning_host_calls():
    """The launch-shape setting is host state: read, set, refused out of range
    (unchanged then), restored."""
    import paper_1105_4490_gb300 as V
    t0 = V.get_tuning()
    assert t0 == {"small_step_threads": 19456, "radix_max_bits": 10, "assign_items": 4, "small_bin_points": 2048}
    V.set_tuning(0, 8, 2, 0)
    got = {"small_step_threads": 0, "radix_max_bits": 8, "assign_items": 2, "small_bin_points": 0}
    assert V.get_tuning() == got
    for bad in ((-1, 10, 8), (0, 7, 8), (0, 11, 8), (0, 10, 3), (0, 10, 16), (0, 10, 8, -1), (0, 10, 8, 2049)):
        with pytest.raises(V.VmoError):
            V.set_tuning(*bad)
        assert V.get_tuning() == got
    V.set_tuning(**t0)
    assert V.get_tuning() == t0
