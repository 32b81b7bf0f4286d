"""CPU checks of the boundary: the C-ABI library builds, loads and exports
every entry point declared in include/sft.h; the ctypes structure layouts
match the C header (sizes and offsets compiled by gcc); the package fails
loudly without the library. No GPU work."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "sft.h")


@pytest.fixture(scope="module")
def built():
    from paper_2603_00538_gb300 import _build
    _build.build()
    import paper_2603_00538_gb300 as sft
    return sft


def _declared():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(sft_[a-z_0-9]+)\s*\(", text)))


def test_header_declares_entry_points():
    names = _declared()
    for must in ("sft_source_create", "sft_target_create", "sft_transfer", "sft_conservation_error"):
        assert must in names


def test_library_exports_every_declared_symbol(built):
    lib = ctypes.CDLL(built.LIB_PATH)
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing
    out = subprocess.run(["nm", "-D", "--defined-only", built.LIB_PATH], capture_output=True, text=True).stdout
    for n in _declared():
        assert re.search(rf"\bT {n}$", out, re.M), n
    assert set(_declared()) == set(built.EXPORTS)


def test_status_strings(built):
    lib = built.lib()
    assert lib.sft_status_str(0) == b"SFT_OK"
    assert lib.sft_status_str(5) == b"SFT_ERR_NOT_CONVERGED"


def test_null_arguments_rejected_without_gpu(built):
    lib = built.lib()
    assert lib.sft_source_create(None, None) == 1          # SFT_ERR_ARG
    assert lib.sft_transfer(None, None, None, None, None, None, None) == 1
    assert b"null" in lib.sft_last_error()


def test_ctypes_layout_matches_header(tmp_path):
    import paper_2603_00538_gb300 as sft
    src = tmp_path / "lay.c"
    src.write_text(f'#include <stdio.h>\n#include <stddef.h>\n#include "{HEADER}"\n'
                   "int main(){printf(\"%zu %zu %zu %zu %zu %zu %zu %zu %zu %zu\\n\", sizeof(sft_mesh_desc),"
                   " sizeof(sft_options), sizeof(sft_stats), offsetof(sft_options, cuda_stream),"
                   " offsetof(sft_stats, ms_setup), offsetof(sft_mesh_desc, grid_scale_L),"
                   " sizeof(sft_surrogate_opts), offsetof(sft_surrogate_opts, exact_cost),"
                   " offsetof(sft_surrogate_opts, sample_f_out), sizeof(sft_surrogate_stats));}\n")
    exe = tmp_path / "lay"
    subprocess.run(["gcc", str(src), "-o", str(exe)], check=True)
    got = [int(v) for v in subprocess.run([str(exe)], capture_output=True, text=True).stdout.split()]
    want = [ctypes.sizeof(sft.sft_mesh_desc), ctypes.sizeof(sft.sft_options), ctypes.sizeof(sft.sft_stats),
            sft.sft_options.cuda_stream.offset, sft.sft_stats.ms_setup.offset,
            sft.sft_mesh_desc.grid_scale_L.offset, ctypes.sizeof(sft.sft_surrogate_opts),
            sft.sft_surrogate_opts.exact_cost.offset, sft.sft_surrogate_opts.sample_f_out.offset,
            ctypes.sizeof(sft.sft_surrogate_stats)]
    assert got == want


def test_product_path_fails_loudly_without_library(monkeypatch):
    import paper_2603_00538_gb300 as sft
    monkeypatch.setattr(sft, "LIB_PATH", "/nonexistent/libsft.so")
    monkeypatch.setattr(sft, "_lib", None)
    with pytest.raises(sft.SftUnavailable):
        sft.lib()


def test_package_never_imports_oracle():
    pkg = os.path.join(ROOT, "paper_2603_00538_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".hpp", ".h")):
                text = open(os.path.join(dirpath, f)).read()
                assert "oracle" not in re.sub(r"(#|//).*", "", text), f
