"""The C-ABI library builds, loads without a GPU and exports every entry
point that include/mss.h declares (no compute calls)."""
import ctypes
import re
import shutil
import subprocess
from pathlib import Path

import pytest

ROOT = Path(__file__).resolve().parents[1]


def _declared():
    text = (ROOT / "include" / "mss.h").read_text()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(mss_[a-z_0-9]+)\s*\(", text)) - {"mss_alloc_fn", "mss_free_fn"})


@pytest.fixture(scope="module")
def lib_path():
    if shutil.which("nvcc") is None and not Path("/usr/local/cuda/bin/nvcc").exists():
        pytest.skip("nvcc not available")
    from paper_1912_04385_gb300 import build
    return build.build()


def test_header_declares_the_boundary():
    names = _declared()
    for n in ("mss_setup", "mss_apply", "mss_fgmres_solve", "mss_create", "mss_destroy"):
        assert n in names


def test_library_exports_every_declared_symbol(lib_path):
    from paper_1912_04385_gb300 import mss
    lib = mss.load()
    declared = _declared()
    for name in declared:
        assert hasattr(lib, name), name
    assert sorted(mss.EXPORTS) == declared
    out = subprocess.run(["nm", "-D", "--defined-only", str(lib_path)], capture_output=True,
                         text=True, check=True).stdout
    exported = set(re.findall(r" T (mss_[a-z_0-9]+)$", out, flags=re.M))
    assert set(declared) <= exported


def test_status_strings_without_gpu(lib_path):
    from paper_1912_04385_gb300 import mss
    lib = mss.load()
    assert lib.mss_status_string(0) == b"MSS_OK"
    assert lib.mss_status_string(-3) == b"MSS_ERR_NOT_CONVERGED"
    o = mss.Options()
    assert lib.mss_options_default(ctypes.byref(o)) == 0
    assert o.amg_max_coarse == 1000 and o.restart == 30 and abs(o.amg_theta - 0.25) < 1e-15


def test_binding_fails_loudly_without_library(tmp_path):
    from paper_1912_04385_gb300 import mss
    with pytest.raises(RuntimeError):
        mss.load(tmp_path / "missing.so")
