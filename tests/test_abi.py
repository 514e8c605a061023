"""The C-ABI library builds, loads and exports what include/lcf.h declares (CPU only)."""
import ctypes as C
import os
import re
import subprocess
import tempfile

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "lcf.h")


def declared_symbols():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(lcf_[a-z_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    from paper_2405_11105_b300 import build
    path = build.build()
    return C.CDLL(path)


def test_every_declared_symbol_is_exported(lib):
    names = declared_symbols()
    assert len(names) >= 10
    for n in names:
        assert hasattr(lib, n), n


def test_config_struct_layout_matches_header():
    """Every field of the ctypes mirror sits at the C struct's offset, and the sizes agree."""
    import paper_2405_11105_b300 as L
    cfg = L.lcf_config
    names = [f[0] for f in cfg._fields_]
    prints = "".join('      printf("%%zu\\n", offsetof(lcf_config, %s));\n' % n for n in names)
    prog = (
        "#include <stdio.h>\n#include <stddef.h>\n#include \"lcf.h\"\n"
        "int main(void) {\n"
        '      printf("%zu\\n", sizeof(lcf_config));\n' + prints + "      return 0;\n}\n")
    with tempfile.TemporaryDirectory() as d:
        c = os.path.join(d, "t.c")
        open(c, "w").write(prog)
        exe = os.path.join(d, "t")
        subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), "-I", "/usr/local/cuda/include", c,
                        "-o", exe], check=True)
        out = list(map(int, subprocess.run([exe], capture_output=True, text=True, check=True).stdout.split()))
    assert C.sizeof(cfg) == out[0]
    for n, off in zip(names, out[1:]):
        assert getattr(cfg, n).offset == off, n


def test_config_default_and_status_strings():
    import paper_2405_11105_b300 as L
    c = L.lcf_config_default(256, 128, 100, 8, 8)
    assert (c.nz, c.nx, c.nt, c.wz, c.wx) == (256, 128, 100, 8, 8)
    assert c.sigma_scale == 1.0 and c.support_sigmas == 3.0
    assert c.thresh_mode == L.LCF_T_CURVATURE
    for s in range(8):
        assert L.lcf_status_string(s)
    with pytest.raises(L.LcfError):
        L._check(L.LCF_EINVAL, "x")


def test_library_has_no_oracle_dependency():
    # the product library must not link or embed the CPU oracle
    from paper_2405_11105_b300 import build
    path = build.build()
    out = subprocess.run(["nm", "-D", path], capture_output=True, text=True).stdout
    assert "ora_" not in out
    src_dir = os.path.join(ROOT, "paper_2405_11105_b300")
    for dp, _, files in os.walk(src_dir):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                txt = open(os.path.join(dp, f)).read()
                assert "import oracle" not in txt and "from oracle" not in txt, f
