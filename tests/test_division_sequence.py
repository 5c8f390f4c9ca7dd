"""The interpolation kernels divide by a shared reciprocal: one division
y = 1/b per divisor, then per quotient q0 = a y, one remainder correction
and a second (Markstein's theorem), which must give the bits of a / b. This
restates the sequence on the host (C, correctly rounded fma) and compares it
with the division on seeded pairs: random, near-1, near-2 and short
mantissas with binary exponents in [-400, 400]; plus a planted variant
(the product with the reciprocal, uncorrected), which the same pairs must
catch."""
import ctypes
import shutil
import subprocess
from pathlib import Path

import pytest

HERE = Path(__file__).resolve().parent
SRC = HERE / "csrc" / "division_sequence.c"


@pytest.fixture(scope="module")
def lib(tmp_path_factory):
    if shutil.which("gcc") is None:
        pytest.skip("gcc not found")
    out = tmp_path_factory.mktemp("divseq") / "libdivseq.so"
    subprocess.run(["gcc", "-O2", "-ffp-contract=off", "-fPIC", "-shared", str(SRC), "-o",
                    str(out), "-lm"], check=True, capture_output=True)
    L = ctypes.CDLL(str(out))
    L.count_mismatches.restype = ctypes.c_longlong
    L.count_mismatches.argtypes = [ctypes.c_longlong, ctypes.c_uint64, ctypes.c_int,
                                   ctypes.POINTER(ctypes.c_double)]
    L.shared_reciprocal_quotient.restype = ctypes.c_double
    L.shared_reciprocal_quotient.argtypes = [ctypes.c_double] * 3
    return L


@pytest.mark.parametrize("seed", [0x1234567, 0x9e3779b9, 42])
def test_shared_reciprocal_division_is_correctly_rounded(lib, seed):
    first = (ctypes.c_double * 2)()
    bad = lib.count_mismatches(2_000_000, seed, 1, first)
    assert bad == 0, (bad, first[0], first[1])


def test_planted_uncorrected_quotient_is_caught(lib):
    first = (ctypes.c_double * 2)()
    assert lib.count_mismatches(200_000, 0x1234567, 0, first) > 1000


def test_sequence_examples(lib):
    for a, b in [(1.0, 3.0), (2.0, 3.0), (-7.5, 0.1), (1e-100, 3e50), (123456789.0, 1e-7)]:
        y = 1.0 / b
        assert lib.shared_reciprocal_quotient(a, b, y) == a / b
