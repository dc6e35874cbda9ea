"""The stored reference values under tests/golden/.

* ``paper_tables.txt`` holds the Nusselt numbers the paper prints (Tables 1
  and 2).  The transcription is checked against the paper's own internal
  consistency: Case 2 at Da = 1e-3 is Case 1 at n = 0.6, and Case 3 at
  Ra = 1e5 repeats Case 2 at Da = 1e-2 (the paper's values differ by 7.7e-5,
  its run-to-run scatter).
* ``oracle_golden.txt`` holds values of the FP64 oracle on small seeded runs,
  written by ``make_oracle_golden.py`` (which calls only ``oracle/``).  The
  oracle must still produce them, so that a change of its arithmetic is a
  deliberate one.
"""
import math
import os
import sys

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))


def test_paper_fixture_is_consistent():
    from golden.paper import paper_tables
    rows = paper_tables()
    assert len(rows) == 12
    t1 = [r for r in rows if r["table"] == "table1"]
    assert [r["n"] for r in t1] == [0.6, 1.0, 1.4] and all(r["Pr"] == 100 and r["Da"] is None for r in t1)
    by = {(r["case"], r["n"], r["Da"], r["Ra"]): r["nu"] for r in rows if r["table"] == "table2"}
    assert by[("case2", 0.6, 1e-3, 1e5)] == by[("case1", 0.6, 1e-3, 1e5)]
    assert abs(by[("case3", 0.6, 1e-2, 1e5)] / by[("case2", 0.6, 1e-2, 1e5)] - 1) < 1e-4
    # the validation values lie between the two benchmark solutions or within 2 % of them
    for r in t1:
        lo, hi = min(r["nu_matin"], r["nu_turan"]), max(r["nu_matin"], r["nu_turan"])
        assert lo * 0.98 <= r["nu"] <= hi * 1.08


def _golden():
    out = {}
    with open(os.path.join(HERE, "golden", "oracle_golden.txt")) as fh:
        for line in fh:
            if line.startswith("#") or not line.strip():
                continue
            run, key, val = line.split()
            out.setdefault(run, {})[key] = float(val)
    return out


@pytest.mark.parametrize("i", range(4))
def test_oracle_reproduces_its_golden_values(orc, i):
    sys.path.insert(0, os.path.join(HERE, "golden"))
    import make_oracle_golden as mk
    from paper_2011_15073_gb300 import inputs
    spec = mk.RUNS[i]
    got = mk.run(orc, inputs, spec)
    want = _golden()[spec[0]]
    assert set(got) == set(want)
    for k, v in got.items():
        assert math.isclose(v, want[k], rel_tol=1e-12, abs_tol=1e-15), (spec[0], k, v, want[k])
