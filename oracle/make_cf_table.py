"""Write tests/golden/cf_nu<nu>.json from the oracle's CF construction (oracle.cf only).

Test infrastructure.  Run:  python -m oracle.make_cf_table [nu ...]   (default: 14)
nu = 14 is the Caratheodory-Fejer approximant of e^x on (-inf, 0] used in the paper's
experiments (Section 5: nu = 14; Section 2 for the construction); other even degrees pin the
library's table for a plan's nu_cf option.
"""
import json
import sys
import time

from oracle import cf


def write(nu):
    t0 = time.time()
    tab = cf.cf_table(nu=nu)
    tab["source"] = ("Section 2 (CF approximation, partial fractions, eq. (11)); nu = %d "
                     "(Section 5 uses 14).  Poles from the Hankel eigenvector, residues by the "
                     "least-squares reading; computed by oracle/cf.py at 50 digits." % nu)
    tab["seconds"] = round(time.time() - t0, 1)
    out = {k: v for k, v in tab.items() if k not in ("tau", "omega")}
    with open(cf.golden_path(nu), "w") as f:
        json.dump(out, f, indent=1)
    print(json.dumps(out, indent=1))


def main():
    for nu in [int(a) for a in sys.argv[1:]] or [cf.NU_DEFAULT]:
        write(nu)


if __name__ == "__main__":
    main()
