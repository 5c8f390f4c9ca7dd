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


# library field -> oracle field, for the settings both implement
_SHARED = {"scheme": "scheme", "stage_order": "stage_order", "stage3": "stage3",
           "ilu_order": "ilu_order", "smoother": "smoother", "nu_pre": "nu_pre",
           "nu_post": "nu_post", "cheb_degree": "cheb_degree",
           "amg_max_coarse": "max_coarse", "amg_max_levels": "max_levels",
           "interp_max_elems": "interp_max", "restart": "restart", "ilu_strip": "ilu_strip",
           "amg_theta": "theta", "jacobi_omega": "omega", "cheb_lo_ratio": "cheb_lo_ratio",
           "cheb_hi_factor": "cheb_hi_factor", "seed": "seed"}


def test_library_and_oracle_defaults_agree(lib_path):
    # the two sides are written separately; parity runs on the defaults, so a
    # default that drifts on one side only would surface as a GPU mismatch
    import oracle
    from paper_1912_04385_gb300 import mss
    lo, oo = mss.options(), oracle.options()
    for lk, ok in _SHARED.items():
        assert getattr(lo, lk) == getattr(oo, ok), (lk, getattr(lo, lk), getattr(oo, ok))
    for name in ("cptr3", "cpr", "ilu0", "cptr"):
        assert mss.SCHEMES[name] == oracle.oracle.SCHEME[name]
    for name in ("jacobi", "chebyshev", "mcsgs"):
        assert mss.SMOOTHERS[name] == oracle.oracle.SMOOTHER[name]


def test_options_names_and_unknown_keys(lib_path):
    from paper_1912_04385_gb300 import mss
    o = mss.options(scheme="cpr", smoother="chebyshev", precision="mixed", driver="graph",
                    restart=50, amg_theta=0.5)
    assert (o.scheme, o.smoother, o.precision, o.driver) == (1, 1, 1, 1)
    assert o.restart == 50 and o.amg_theta == 0.5
    with pytest.raises(KeyError):
        mss.options(no_such_option=1)
    with pytest.raises(KeyError):
        mss.options(scheme="no_such_scheme")
