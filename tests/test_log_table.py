"""The constants of the FP64 logarithm of the step kernels (log_table.h,
written by paper_1611_00907_gb300/csrc/gen_log_table.py): the committed
header is what the script writes, and its values agree with the host libm
(an independent implementation) to the last bit."""
import importlib.util
import math
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1611_00907_gb300", "csrc")


def _gen():
    spec = importlib.util.spec_from_file_location(
        "gen_log_table", os.path.join(CSRC, "gen_log_table.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def _header_values():
    text = open(os.path.join(CSRC, "log_table.h")).read()
    rows = re.findall(r"\{(\S+), (\S+)\},\s*// (\d+)", text)
    lows = re.findall(r"^\s+(\S+),\s*// (\d+)$", text.split("kLogTableLo")[1], re.M)
    assert [int(j) for _, j in lows] == list(range(129))
    hi = float.fromhex(re.search(r"LN2_HI = (\S+);", text).group(1))
    lo = float.fromhex(re.search(r"LN2_LO = (\S+);", text).group(1))
    return [(int(j), float.fromhex(a), float.fromhex(b), float.fromhex(c))
            for (a, b, j), (c, _) in zip(rows, lows)], hi, lo


def _is_multiple_of_2_32(v):
    return (v * 2.0 ** 32).is_integer()


def test_header_is_what_the_script_writes():
    assert open(os.path.join(CSRC, "log_table.h")).read() == _gen().header()


def test_breakpoints_match_libm():
    rows, _, _ = _header_values()
    assert [j for j, _, _, _ in rows] == list(range(129))
    for j, inv, hi, lo in rows:
        F = 1.0 + j / 128.0
        assert inv == 1.0 / F                     # IEEE division rounds correctly
        # hi on the 2^-32 grid, lo the rest: hi + lo is ln F to the last bit
        # of libm's log (within an ulp of its own)
        assert _is_multiple_of_2_32(hi) and abs(lo) <= 2.0 ** -33
        assert abs((hi + lo) - math.log(F)) <= math.ulp(math.log(F) or 1e-300), j


def test_ln2_split():
    _, hi, lo = _header_values()
    # on the 2^-32 grid: m * hi + hi(ln F) is exact for every binary exponent m
    assert _is_multiple_of_2_32(hi)
    assert hi + lo == math.log(2.0)
    assert abs(lo) <= 2.0 ** -33
