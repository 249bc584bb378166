"""CPU checks of the boundary: the C-ABI library builds, loads and exports every
symbol include/memd.h declares; the product path never touches the oracle and
the oracle never touches the product."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for h in os.listdir(os.path.join(ROOT, "include")):
        if not h.endswith(".h"):
            continue
        txt = open(os.path.join(ROOT, "include", h)).read()
        txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
        for m in re.finditer(r"\b(memd_\w+)\s*\(", txt):
            names.add(m.group(1))
    return names


def test_library_exports_every_declared_symbol():
    from paper_1309_7859_gb300 import build
    path = build.build()
    lib = ctypes.CDLL(path)           # loads without a GPU (no compute calls here)
    names = declared_functions()
    assert len(names) >= 20
    for n in sorted(names):
        assert hasattr(lib, n), n
    out = subprocess.run(["nm", "-D", "--defined-only", path], capture_output=True, text=True).stdout
    exported = {l.split()[-1] for l in out.splitlines() if " T " in l}
    assert names <= exported


def test_binding_covers_the_abi():
    from paper_1309_7859_gb300 import memd
    assert set(memd.EXPORTS) == declared_functions()


def test_kernels_are_built_for_sm103a():
    from paper_1309_7859_gb300 import build
    assert build.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]


def test_product_and_oracle_share_no_code():
    pkg = os.path.join(ROOT, "paper_1309_7859_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h", ".cpp")):
                txt = open(os.path.join(dirpath, f)).read()
                assert not re.search(r"^\s*(import|from)\s+oracle|oracle/|memd_oracle", txt, re.M), f
    for f in os.listdir(os.path.join(ROOT, "oracle")):
        if f.endswith((".c", ".h", ".py")):
            txt = open(os.path.join(ROOT, "oracle", f)).read()
            assert "paper_1309_7859_gb300" not in txt, f
            assert "memd.h" not in txt and "memd_internal" not in txt, f


def test_binding_fails_loudly_without_gpu():
    import torch
    if torch.cuda.is_available():
        pytest.skip("GPU present")
    from paper_1309_7859_gb300.memd import Memd
    with pytest.raises(RuntimeError):
        Memd((4, 4, 4), (4.0, 4.0, 4.0))
