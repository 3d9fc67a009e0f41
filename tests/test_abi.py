"""The C-ABI library builds, loads and exports every function include/*.h
declares (CPU only: no compute calls)."""
import glob
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        for mt in re.finditer(r"^[A-Za-z_][\w \*]*?\b(ruqlp_\w+)\s*\(", src, flags=re.M):
            names.add(mt.group(1))
    return names


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__ as g
    g.build()
    from paper_2209_12464_gb300 import ruqlp
    return ruqlp


def test_header_declares_entry_points():
    names = _declared()
    for must in ["ruqlp_create", "ruqlp_destroy", "ruqlp_decompose", "ruqlp_decompose_host",
                 "ruqlp_last_error"]:
        assert must in names


def test_library_exports_every_declared_symbol(lib):
    out = subprocess.run(["nm", "-D", "--defined-only", lib.LIB_PATH], capture_output=True,
                         text=True, check=True).stdout
    exported = set(re.findall(r"\b(ruqlp_\w+)\b", out))
    missing = _declared() - exported
    assert not missing, f"declared but not exported: {sorted(missing)}"
    for name in _declared():
        assert hasattr(lib.lib(), name)


def test_binding_signatures_cover_header(lib):
    assert set(lib.exported_symbols()) <= _declared()


def test_workspace_bytes_host_logic(lib):
    assert lib.ruqlp_workspace_bytes(1000, 800, 30, lib.F64) > 0
    assert lib.ruqlp_workspace_bytes(0, 800, 30, lib.F64) == 0
    assert lib.ruqlp_workspace_bytes(1000, 800, 513, lib.F64) == 0
    a = lib.ruqlp_workspace_bytes(20000, 20000, 220, lib.BF16)
    b = lib.ruqlp_workspace_bytes(20000, 20000, 220, lib.F64)
    assert 0 < a < b
    # CSR: the CSC copy grows with nnz; FP64 values are not supported
    c0 = lib.ruqlp_workspace_bytes(200000, 100000, 110, lib.F32, 0)
    c1 = lib.ruqlp_workspace_bytes(200000, 100000, 110, lib.F32, 20000000)
    assert 0 < c0 < c1 and c1 - c0 >= 20000000 * 8 - 1024
    assert lib.ruqlp_workspace_bytes(200, 100, 10, lib.F64, 50) == 0


def test_version(lib):
    assert "sm_103a" in lib.ruqlp_version()


def test_missing_library_raises_with_no_fallback(tmp_path):
    """Without the built library every entry point raises (there is no CPU
    or PyTorch path to fall back on)."""
    code = "\n".join([
        "import sys",
        f"sys.path.insert(0, {ROOT!r})",
        "from paper_2209_12464_gb300 import ruqlp",
        f"ruqlp.LIB_PATH = {str(tmp_path / 'absent.so')!r}",
        "for call in (lambda: ruqlp.lib(), lambda: ruqlp.Handle(0, 0),",
        "             lambda: ruqlp.ruqlp_version()):",
        "    try:",
        "        call()",
        "    except RuntimeError as e:",
        "        print('raised', 'not built' in str(e))",
        "    else:",
        "        print('returned')",
    ])
    r = subprocess.run([__import__("sys").executable, "-c", code], capture_output=True, text=True,
                       timeout=300)
    assert r.returncode == 0, r.stderr
    assert r.stdout.split() == ["raised", "True"] * 3, r.stdout
