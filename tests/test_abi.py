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
    import paper_2405_11105_b300 as L
    prog = r"""
    #include <stdio.h>
    #include <stddef.h>
    #include "lcf.h"
    int main(void) {
      printf("%zu %zu %zu %zu\n", sizeof(lcf_config), offsetof(lcf_config, beta),
             offsetof(lcf_config, gram_path), offsetof(lcf_config, max_sweeps));
      return 0;
    }"""
    with tempfile.TemporaryDirectory() as d:
        c = os.path.join(d, "t.c")
        open(c, "w").write(prog)
        exe = os.path.join(d, "t")
        subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), "-I", "/usr/local/cuda/include", c,
                        "-o", exe], check=True)
        out = subprocess.run([exe], capture_output=True, text=True, check=True).stdout.split()
    size, beta, gp, ms = map(int, out)
    cfg = L.lcf_config
    assert C.sizeof(cfg) == size
    assert cfg.beta.offset == beta and cfg.gram_path.offset == gp and cfg.max_sweeps.offset == ms


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
