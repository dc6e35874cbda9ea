"""Write tests/golden/oracle_golden.txt: reference values of the FP64 oracle
on small seeded runs, so that a change of the oracle's arithmetic shows up as
a failing CPU test (tests/test_golden_cpu.py) and has to be made on purpose.

Calls only oracle/ and the seeded inputs; run it from the repository root:
    python tests/golden/make_oracle_golden.py
"""
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

# (name, nx, ny, params, map options, steps, perturbation seed, Darcy-field seed or None)
RUNS = [
    ("thinning_literal", 24, 17, dict(n=0.6, Da=1e-2, Ra=1e5, Pr=6.2), dict(porosity=0.6, clamp_mode=0), 60, 1, None),
    ("newtonian_pr10", 16, 16, dict(n=1.0, Da=1e-1, Ra=1e3, Pr=10.0), dict(porosity=0.6), 80, 2, None),
    ("thickening_darcy_model", 20, 14, dict(n=1.4, Da=1e-3, Ra=1e5, Pr=6.2),
     dict(porosity=1.0, porous_model=0, clamp_mode=1), 60, 3, None),
    ("field_implicit_tau", 18, 12, dict(n=0.8, Da=1e-2, Ra=1e4, Pr=6.2),
     dict(porosity=0.6, clamp_mode=1, tau_iters=4), 40, 4, 5),
]


def run(orc, inputs, spec):
    name, nx, ny, prm, kw, steps, seed, field = spec
    c = orc.Cavity.from_params(nx, ny, prm["n"], prm["Da"], prm["Ra"], prm["Pr"], **kw)
    c.set_state(*inputs.perturbed_state(c.get_state(), seed=seed, amp=1e-2))
    if field is not None:
        c.set_darcy_field(inputs.darcy_field(field, nx, ny))
    c.step(steps)
    f, g, tau = c.get_state()
    hot, cold, _ = c.nusselt()
    w = np.arange(1, f[0].size + 1, dtype=np.float64).reshape(f[0].shape) / f[0].size
    return {"nu_hot": hot, "nu_cold": cold, "f_weighted": float(np.sum(f * w)), "g_weighted": float(np.sum(g * w)),
            "tau_mean": float(tau.mean()), "f_max": float(f.max()), "g_min": float(g.min())}


def main():
    import oracle
    from paper_2011_15073_gb300 import inputs
    oracle.build()
    lines = ["# Reference values of the FP64 oracle (oracle/oracle.c) on small seeded runs, written by",
             "#   python tests/golden/make_oracle_golden.py",
             "# Columns: run quantity value.  A change of these numbers is a change of the oracle's",
             "# arithmetic and names the passage of the paper that justifies it."]
    for spec in RUNS:
        for k, v in run(oracle, inputs, spec).items():
            lines.append(f"{spec[0]} {k} {v!r}")
    with open(os.path.join(HERE, "oracle_golden.txt"), "w") as fh:
        fh.write("\n".join(lines) + "\n")


if __name__ == "__main__":
    main()
