"""The C-ABI library builds, loads without a GPU, and exports every entry point include/zsmiles.h declares."""
import ctypes
import os
import re
import subprocess

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    text = open(os.path.join(ROOT, "include", "zsmiles.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(zs_[a-z_0-9]+)\s*\(", text)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ["zs_load_dictionary", "zs_free_dictionary", "zs_compress", "zs_decompress",
                     "zs_build_line_index", "zs_decompress_lines", "zs_last_error"]:
        assert required in names


def test_library_exports_every_declared_symbol():
    from paper_2404_19391_gb300 import build
    lib = build.build()
    out = subprocess.run(["nm", "-D", "--defined-only", lib], capture_output=True, text=True, check=True).stdout
    exported = set(re.findall(r"\bT (zs_[a-z_0-9]+)", out))
    missing = [n for n in declared_functions() if n not in exported]
    assert not missing, missing
    h = ctypes.CDLL(lib)
    for n in declared_functions():
        assert hasattr(h, n)
    h.zs_version.restype = ctypes.c_char_p
    assert b"sm_103a" in h.zs_version()
    h.zs_compress_bound.restype = ctypes.c_size_t
    h.zs_compress_bound.argtypes = [ctypes.c_size_t]
    assert h.zs_compress_bound(100) == 316


def test_product_path_does_not_reference_the_oracle():
    pkg = os.path.join(ROOT, "paper_2404_19391_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".cpp", ".h")):
                text = open(os.path.join(dirpath, f), errors="replace").read()
                assert "import oracle" not in text and "from oracle" not in text and "zs_oracle" not in text, f


def test_no_cpu_fallback():
    """Without a CUDA device the binding refuses to work: a dictionary cannot be loaded and host tensors are
    rejected, so no call can quietly run anywhere but the GPU kernels."""
    import pytest
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a CUDA device is present")
    from paper_2404_19391_gb300 import zsmiles as zs
    zs.load_library()
    with pytest.raises(Exception):
        zs.Dictionary()
    with pytest.raises(ValueError):
        zs._ptr(torch.zeros(16, dtype=torch.uint8))
