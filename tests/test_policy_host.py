"""Host-side checks of the precision-policy table and error metrics (no GPU).

The 13 configurations must be the ones Table 2 lists (Sec. 4): Group A with
rp = fp64 storage, one block lowered to fp32 in A-2..A-4; Group B with rp =
fp32 storage, one block raised to fp64 in B-2..B-4 and one fp16 kernel
override in B-5..B-7 (adv_dealias in the SEM block, ax_helm in the velocity
and the pressure block).  The metrics follow Sec. 4.2: e_max takes the largest
pointwise difference over the largest reference value, e_peak the difference of
the two maxima over the largest reference value.
"""
import ctypes
import os
import re

import pytest

from paper_2608_24348_gb300 import policy, sem

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
BLOCKS = ("sem", "vel", "pres")


def test_table2_has_the_papers_thirteen_configurations():
    assert list(policy.TABLE2) == [f"A-{k}" for k in range(5)] + [f"B-{k}" for k in range(8)]
    for name, r in policy.TABLE2.items():
        assert r["storage"] == ("f64" if name.startswith("A") else "f32")


@pytest.mark.parametrize("name,lowered", [("A-1", BLOCKS), ("A-2", ("sem",)), ("A-3", ("vel",)),
                                          ("A-4", ("pres",)), ("A-0", ())])
def test_group_a_lowers_the_named_blocks_to_fp32(name, lowered):
    r = policy.TABLE2[name]
    for b in BLOCKS:
        assert r[b] == ("f32" if b in lowered else "f64"), (name, b)


@pytest.mark.parametrize("name,raised", [("B-1", BLOCKS), ("B-2", ("sem",)), ("B-3", ("vel",)),
                                         ("B-4", ("pres",)), ("B-0", ())])
def test_group_b_raises_the_named_blocks_to_fp64(name, raised):
    r = policy.TABLE2[name]
    for b in BLOCKS:
        assert r[b] == ("f64" if b in raised else "f32"), (name, b)


@pytest.mark.parametrize("name,block", [("B-5", "sem"), ("B-6", "vel"), ("B-7", "pres")])
def test_group_b_fp16_kernel_overrides(name, block):
    r = policy.TABLE2[name]
    for b in BLOCKS:
        assert r[b] == ("f16_tc" if b == block else "f32"), (name, b)


def test_rule_adds_the_first_step_and_copies():
    r = policy.rule("B-6", first_step=101)
    assert r["first_step"] == 101 and r["vel"] == "f16_tc"
    r["vel"] = "f64"
    assert policy.TABLE2["B-6"]["vel"] == "f16_tc"


def test_error_metrics_on_a_worked_example():
    ref = [1.0, 4.0, 2.0]
    mxp = [1.2, 3.5, 2.0]
    # largest pointwise difference 0.5 (at the second sample) over max |ref| = 4
    assert policy.e_max(mxp, ref) == pytest.approx(0.125)
    # maxima 3.5 and 4.0 (same sample here)
    assert policy.e_peak(mxp, ref) == pytest.approx(0.125)
    # peaks at different samples: e_peak compares the maxima, not the samples
    late = [1.0, 2.0, 4.4]
    assert policy.e_peak(late, ref) == pytest.approx(0.1)
    assert policy.e_max(late, ref) == pytest.approx(0.6)
    assert policy.e_max(ref, ref) == 0.0


def test_policy_struct_matches_the_c_header():
    text = open(os.path.join(ROOT, "include", "sem.h")).read()
    body = re.search(r"typedef struct \{([^}]*)\} sem_tgv_policy;", text).group(1)
    fields = re.findall(r"\b(\w+)\s*[,;]", re.sub(r"/\*.*?\*/", "", body, flags=re.S))
    assert fields == [f for f, _ in sem.TgvPolicy._fields_]
    assert ctypes.sizeof(sem.TgvPolicy) == 5 * ctypes.sizeof(ctypes.c_int)
    m = re.search(r"#define SEM_TGV_MAX_RULES (\d+)", text)
    assert m and int(m.group(1)) == 8


def test_peak_is_the_vertex_of_the_parabola_through_the_top_samples():
    t = [0.1 * i for i in range(20)]
    # an exact parabola: the vertex is recovered between samples
    tp, yp = policy.peak(t, [3 - (x - 0.537) ** 2 for x in t])
    assert tp == pytest.approx(0.537, abs=1e-12) and yp == pytest.approx(3.0, abs=1e-12)
    # a smooth non-parabolic peak: error of the three-point vertex is O(dt^3) in time
    import math
    tp, yp = policy.peak(t, [math.exp(-(x - 1.234) ** 2) for x in t])
    assert abs(tp - 1.234) < 2e-3 and abs(yp - 1.0) < 1e-4
    # a maximum at the end of the record stays the last sample
    assert policy.peak(t, t) == (pytest.approx(1.9), pytest.approx(1.9))
