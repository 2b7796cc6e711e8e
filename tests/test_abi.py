"""Host-side checks of the C-ABI library (no GPU needed): it builds, loads, and exports
every entry point declared in include/fcgno.h; the oracle and the library stay separate."""
import ctypes
import re
from pathlib import Path

import pytest

ROOT = Path(__file__).resolve().parents[1]


def declared_symbols():
    text = (ROOT / "include" / "fcgno.h").read_text()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(fcgno_[A-Za-z_0-9]+)\s*\(", text)))


@pytest.fixture(scope="module")
def libpath():
    from paper_2402_05598_gb300 import build
    return build.build()


def test_library_exports_every_declared_symbol(libpath):
    lib = ctypes.CDLL(str(libpath))
    syms = declared_symbols()
    assert len(syms) >= 15
    missing = [s for s in syms if not hasattr(lib, s)]
    assert not missing, missing


def test_binding_covers_header(libpath):
    from paper_2402_05598_gb300 import fcgno
    assert sorted(fcgno.EXPORTS) == declared_symbols()


def test_host_only_calls(libpath):
    """Calls that need no GPU: status strings, weight counts, argument validation."""
    from paper_2402_05598_gb300 import fcgno
    from paper_2402_05598_gb300 import inputs as I
    assert fcgno.status_str(fcgno.FCGNO_OK) == "ok"
    assert "breakdown" in fcgno.status_str(fcgno.FCGNO_EBREAKDOWN)
    for C, M in ((16, 8), (32, 12)):
        d = fcgno.make_desc(width=C, layers=4, modes=M)
        assert fcgno.weight_count(d) == I.weight_count(I.ModelDesc(width=C, layers=4, modes=M, proj_width=C))
    bad = fcgno.make_desc(width=0)
    assert fcgno.weight_count(bad) == 0
    # invalid arguments are rejected before any CUDA call
    h = ctypes.c_void_p()
    assert fcgno.lib.fcgno_assemble(1, 1, None, None, ctypes.byref(h)) == fcgno.FCGNO_EINVAL
    opts = fcgno.fcgno_solve_opts(1e-6, 9, 10, 0, 1)
    assert fcgno.lib.fcgno_solve(None, None, None, None, ctypes.byref(opts), 1, None, None) == fcgno.FCGNO_EINVAL
    assert fcgno.workspace_bytes(64, 256, 1, fcgno.make_desc(32, 4, 12)) > 256 * 64 * 64 * 8 * 8


def test_oracle_and_library_do_not_import_each_other():
    for f in (ROOT / "oracle").rglob("*.py"):
        src = f.read_text()
        assert "paper_2402_05598_gb300" not in src, f
    for f in (ROOT / "paper_2402_05598_gb300").rglob("*.py"):
        src = f.read_text()
        assert not re.search(r"^\s*(from|import)\s+oracle", src, flags=re.M), f
    for f in (ROOT / "paper_2402_05598_gb300" / "csrc").glob("*"):
        assert "oracle" not in f.read_text().lower(), f
