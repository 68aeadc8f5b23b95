"""Write the stored expected values under tests/golden/ from the oracle alone.

bruteforce_n16.json: the exhaustive optimum of |d_eff|^2 over all 2^16 sign
patterns for N = 16 unit domains at dk1 w = 2pi/7.0, dk2 w = 2pi/1.6 (the
small correctness workload); d_eff is the Sec. 2.1 double integral.
Run:  python tests/golden/make_golden.py
"""
import json
import math
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402


def main():
    k1, k2 = 2 * math.pi / 7.0, 2 * math.pi / 1.6
    best, mask = oracle.bruteforce(16, k1, k2)
    out = {"source": "oracle.bruteforce (Sec. 2.1 d_eff, exhaustive over 2^16 patterns)",
           "N": 16, "kappa1": k1, "kappa2": k2, "best_f": best, "best_mask": mask,
           "best_mask_twin": mask ^ 0xFFFF}
    with open(os.path.join(HERE, "bruteforce_n16.json"), "w") as fh:
        json.dump(out, fh, indent=1)
    print(out)


if __name__ == "__main__":
    main()
