"""The C-ABI library builds, loads and exports every symbol include/sy.h declares;
host-only entry points (no GPU needed) agree with the oracle bit for bit."""
import ctypes as C
import re
import subprocess

import pytest

import oracle
import paper_2505_06022_gb300 as sy

ROOT = __file__.rsplit("/tests/", 1)[0]


def declared_symbols():
    text = open(ROOT + "/include/sy.h").read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:const\s+)?[a-z_0-9]+\s*\**\s*(sy_[a-z0-9_]+)\s*\(", text, flags=re.M)))


def test_header_declares_the_boundary():
    names = declared_symbols()
    for must in ["sy_queue_create", "sy_saxpy", "sy_stencil_step", "sy_split_rows", "sy_energy_read",
                 "sy_kernel_energy", "sy_device_energy", "sy_wave_energy", "sy_status_string", "sy_last_error"]:
        assert must in names


def test_library_exports_every_declared_symbol():
    path = sy.lib().__dict__.get("_name") or sy.lib_path()
    out = subprocess.run(["nm", "-D", "--defined-only", path], capture_output=True, text=True, check=True).stdout
    exported = set(re.findall(r"\bT\s+(sy_[a-z0-9_]+)", out))
    missing = [n for n in declared_symbols() if n not in exported]
    assert not missing, f"declared but not exported: {missing}"
    # and nothing C++ leaks: every exported symbol is a C name from the header
    assert exported <= set(declared_symbols())


def test_status_strings_and_version():
    L = sy.lib()
    assert sy.sy_abi_version() == 1
    for code, name in sy.STATUS.items():
        assert L.sy_status_string(code).decode() == name


@pytest.mark.parametrize("n,k", [(8192, 4), (10, 3), (7, 7), (5, 1), (100, 9), (0, 1), (3, 5)])
def test_split_rows_matches_oracle(n, k):
    assert sy.sy_split_rows(n, k) == oracle.split_rows(n, k)


def test_range_mappers_match_oracle():
    for ny in (1, 6, 19):
        for r in (0, 1, 2, 4):
            for a in range(ny):
                for b in range(a + 1, ny + 1):
                    assert sy.sy_rm_neighbourhood((a, b), r, ny) == oracle.rm_neighbourhood(a, b, r, ny)
                    assert sy.sy_rm_one_to_one((a, b)) == oracle.rm_one_to_one(a, b)


@pytest.mark.parametrize("chunks,n", [([(0, 5), (6, 10)], 10), ([(0, 6), (5, 10)], 10), ([(0, 5), (5, 9)], 10),
                                      ([(0, 0), (0, 10)], 10), ([(5, 10), (0, 5)], 10), ([(0, 1), (1, 10)], 10),
                                      ([(0, 10)], 10), ([], 0)])
def test_chunk_validation_matches_oracle(chunks, n):
    ok = oracle.chunks_valid(n, chunks) if chunks else False
    if ok:
        sy.sy_chunks_validate(n, chunks)
    else:
        with pytest.raises(sy.SyError) as e:
            sy.sy_chunks_validate(n, chunks)
        assert e.value.name == "SY_ERR_BAD_CHUNKS"


def test_errors_are_reported_not_raised_across_the_abi():
    with pytest.raises(sy.SyError) as e:
        sy.sy_split_rows(10, 0)
    assert e.value.name == "SY_ERR_INVALID_ARGUMENT" and "chunks" in str(e.value)
    L = sy.lib()
    assert L.sy_split_rows(5, 2, None) == 2  # SY_ERR_NULL_POINTER
    assert L.sy_saxpy(None, 4, C.c_float(1.0), None, None, None, None) == 2


def test_no_oracle_in_the_product_library():
    out = subprocess.run(["nm", "-D", sy.lib_path()], capture_output=True, text=True, check=True).stdout
    assert "oracle" not in out
    deps = subprocess.run(["ldd", sy.lib_path()], capture_output=True, text=True).stdout
    assert "liboracle" not in deps


def test_product_package_never_imports_the_oracle():
    import ast
    import os

    pkg = os.path.dirname(sy.__file__)
    for name in os.listdir(pkg):
        if not name.endswith(".py"):
            continue
        tree = ast.parse(open(os.path.join(pkg, name)).read())
        for node in ast.walk(tree):
            if isinstance(node, ast.Import):
                assert all(not a.name.startswith("oracle") for a in node.names), name
            elif isinstance(node, ast.ImportFrom):
                assert not (node.module or "").startswith("oracle"), name
    csrc = os.path.join(pkg, "csrc")
    for name in os.listdir(csrc):
        assert "oracle" not in open(os.path.join(csrc, name), errors="ignore").read().lower(), name
    # and the oracle uses nothing of the product: no package import, no repository header
    odir = os.path.join(os.path.dirname(pkg), "oracle")
    for name in os.listdir(odir):
        path = os.path.join(odir, name)
        if name.endswith(".py"):
            for node in ast.walk(ast.parse(open(path).read())):
                if isinstance(node, (ast.Import, ast.ImportFrom)):
                    mods = [a.name for a in node.names] if isinstance(node, ast.Import) else [node.module or ""]
                    assert all("paper_2505_06022_gb300" not in m for m in mods), name
        elif name.endswith(".c"):
            includes = [l for l in open(path) if l.startswith("#include")]
            assert all("<" in l for l in includes), (name, includes)


def test_binding_refuses_strided_views():
    import torch

    base = torch.zeros(6, 8)
    assert sy._ptr(base) == base.data_ptr() and sy._ptr(base[2:]) == base[2:].data_ptr()
    for view in (base.t(), base[:, :5], base[::2]):
        with pytest.raises(ValueError):
            sy._ptr(view)


def test_stencil_variant_table_and_default():
    """Host-side variant table: 12 tile forms for FP32 storage, 15 for 16-bit (the narrow forms
    and the march form); variant 0 stands for a listed variant with the same description; tile
    widths are 32 vectors (register tiles) or 30 (halo-lane, narrow and march strips); the march
    form reports its nominal 32-row segment; out-of-range ids are refused."""
    for dtype, count in ((sy.SY_F32, 12), (sy.SY_BF16, 15), (sy.SY_F16, 15)):
        es = 4 if dtype == sy.SY_F32 else 2
        V = 16 // es
        for r in (1, 2, 3, 4):
            assert sy.sy_stencil_variant_count(r, dtype) == count
            d = sy.sy_stencil_default_variant(r, dtype)
            assert 1 <= d <= count
            assert sy.sy_stencil_variant_info(r, dtype, 0) == sy.sy_stencil_variant_info(r, dtype, d)
            for v in range(1, count + 1):
                rows, cols, thr = sy.sy_stencil_variant_info(r, dtype, v)
                assert rows in (2, 4, 8, 16, 32) and thr in (128, 256)
                if v <= 8:
                    assert cols == 32 * V
                elif v <= 12:
                    assert cols == 30 * V and rows in (4, 8)
                elif v <= 14:
                    assert cols == 30 * 4 and thr == 128
                else:
                    assert (rows, cols, thr) == (32, 30 * V, 128)
            with pytest.raises(sy.SyError):
                sy.sy_stencil_variant_info(r, dtype, count + 1)
    with pytest.raises(sy.SyError):
        sy.sy_stencil_default_variant(5, sy.SY_F32)
