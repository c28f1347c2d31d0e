"""The C-ABI library builds for sm_103a, loads, and exports every entry point its headers declare."""
import os
import re
import ctypes

import paper_1506_05741_b300 as dm

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            src = open(os.path.join(ROOT, "include", fn)).read()
            names |= set(re.findall(r"^DIAM_API [^(]*?\b(diam_\w+)\(", src, flags=re.M))
    return names


def test_library_exports_every_declared_symbol():
    lib = ctypes.CDLL(dm.lib_path() if os.path.exists(dm.lib_path()) else dm._build.build())
    names = declared()
    assert len(names) >= 19
    for n in sorted(names):
        assert hasattr(lib, n), n


def test_config_defaults_follow_algorithm_1():
    cfg = dm.default_config(64, 3)
    assert abs(cfg["beta0"] - 0.3) < 1e-15          # min(2.4 / sqrt(d), 0.5)
    assert dm.default_config(4, 1)["beta0"] == 0.5
    assert cfg["acc_lo"] == 0.3 and cfg["acc_hi"] == 0.5 and cfg["infl"] == 1.0


def test_struct_layouts_match_header(tmp_path):
    """Every field offset and size of the ctypes mirrors equals the C compiler's layout of include/diam.h."""
    import subprocess
    probes = []
    for cname, cls in [("diam_config", dm.DiamConfig), ("diam_target", dm.DiamTarget), ("diam_stats", dm.DiamStats)]:
        probes.append(f'printf("{cname} size %zu\\n", sizeof({cname}));')
        for f, _ in cls._fields_:
            probes.append(f'printf("{cname} {f} %zu\\n", offsetof({cname}, {f}));')
    src = tmp_path / "probe.c"
    src.write_text('#include <stdio.h>\n#include <stddef.h>\n#include "diam.h"\nint main(void){' + "".join(probes)
                   + "return 0;}\n")
    exe = tmp_path / "probe"
    subprocess.check_call(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)])
    out = subprocess.check_output([str(exe)]).decode().split("\n")
    got = {tuple(l.split()[:2]): int(l.split()[2]) for l in out if l.strip()}
    for cname, cls in [("diam_config", dm.DiamConfig), ("diam_target", dm.DiamTarget), ("diam_stats", dm.DiamStats)]:
        assert got[(cname, "size")] == ctypes.sizeof(cls), cname
        for f, _ in cls._fields_:
            assert got[(cname, f)] == getattr(cls, f).offset, (cname, f)
