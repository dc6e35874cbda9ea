"""Reader of the paper's printed Nusselt numbers (tests/golden/paper_tables.txt)."""
import os

HERE = os.path.dirname(os.path.abspath(__file__))


def paper_tables():
    """Rows of the paper's Tables 1 and 2 as dicts: table, case, n, Da (None
    for the clear fluid), Ra, Pr, nu, and for Table 1 nu_matin, nu_turan."""
    rows = []
    with open(os.path.join(HERE, "paper_tables.txt")) as fh:
        for line in fh:
            if not line.strip() or line.startswith("#"):
                continue
            p = line.split()
            r = dict(table=p[0], case=p[1], n=float(p[2]), Da=None if p[3] == "-" else float(p[3]),
                     Ra=float(p[4]), Pr=float(p[5]), nu=float(p[6]))
            if len(p) > 7:
                r["nu_matin"], r["nu_turan"] = float(p[7]), float(p[8])
            rows.append(r)
    return rows
