"""Write tests/golden/cf_nu14.json from the oracle's CF construction (oracle.cf only).

Test infrastructure.  Run:  python -m oracle.make_cf_table
The table is the nu = 14 Caratheodory-Fejer approximant of e^x on (-inf, 0] used in the
paper's experiments (Section 5: nu = 14; Section 2 for the construction).
"""
import json
import time

from oracle import cf


def main():
    t0 = time.time()
    tab = cf.cf_table()
    tab["source"] = ("Section 2 (CF approximation, partial fractions, eq. (11)); nu = 14 "
                     "as in Section 5.  Poles from the Hankel eigenvector, residues by the "
                     "least-squares reading; computed by oracle/cf.py at 50 digits.")
    tab["seconds"] = round(time.time() - t0, 1)
    out = {k: v for k, v in tab.items() if k not in ("tau", "omega")}
    with open(cf.GOLDEN, "w") as f:
        json.dump(out, f, indent=1)
    print(json.dumps(out, indent=1))


if __name__ == "__main__":
    main()
