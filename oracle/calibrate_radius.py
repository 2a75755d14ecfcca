"""Calibrate the connection radius r_n of the synthetic workloads with the oracle.

TEST INFRASTRUCTURE.  For a sample count n (start + goal + samples, seed 0, no
obstacles) it computes every ordered pair's steering cost with the CPU oracle
and picks r so that the mean out-degree of {v -> u : Cost(v,u) < r} is
40 ln(n) / ln(4000): about 33 at n = 1002 and 40 at n = 4002.  The printed
values are the ones stored in paper_1607_06886_gb300/inputs.py RADIUS_TABLE.

    python oracle/calibrate_radius.py 1002 4002
"""
import math
import os
import sys

import numpy as np

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
from oracle import cpu  # noqa: E402
from paper_1607_06886_gb300 import inputs  # noqa: E402


def calibrate(n_total: int) -> float:
    states = inputs.sample_states(n_total - 2, seed=0)
    c = np.sort(cpu.pair_costs(states).ravel())
    target = 40.0 * math.log(n_total) / math.log(4000.0)
    k = int(round(target * n_total))
    return float(0.5 * (c[k - 1] + c[k]))


if __name__ == "__main__":
    for arg in sys.argv[1:] or ["1002", "4002"]:
        n = int(arg)
        r = calibrate(n)
        print(f"{n}: {r:.4f}")
