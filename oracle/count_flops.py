"""Floating-point operation counts of the oracle's plain restatement of one
RK stage (3 levels of 256^2, TOV K=100, Gamma=2, rho_c=1.28e-3), per face or
cell and per phase, from the op-counting build of the oracle (opcount.cpp).
These count the oracle's loops as written (zero-weight taps, the 49-term
mixed derivative, the triple-loop Christoffel terms); the roofline's
numerators are the method's own counts, derived by hand and from the
library's executed instructions.  Test infrastructure; run by hand, prints a
table and the raw JSON:
    python oracle/count_flops.py
"""
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import oracle as O  # noqa: E402
from paper_2502_03223_gb300 import workloads as W  # noqa: E402


def main():
    cfg, tov = W.config_tov_stable()
    datas = [W.tov_level_data(cfg, tov, l) for l in range(cfg.n_levels)]
    c = O.opcount(cfg, datas)
    print("Oracle operation counts per unit, TOV 3 x 256^2 (level 1), one RK stage")
    print("(add, mul, div, sqrt, pow/exp = 1 each; comparisons, fabs = 0)")
    for k, unit in (("flux_face", "x-face (PPM 5 prims + 6-pt metric + tetrad HLLC)"),
                    ("hydro_div_cell", "cell (flux divergence + sources)"),
                    ("cartoon_cell", "cell of the plane patch (9-pt interp + rotation, 7 planes, 25 fields)"),
                    ("z4c_derivs_cell", "cell (central/mixed/lopsided/KO differences of 25 fields)"),
                    ("z4c_point_cell", "cell (pointwise Z4c algebra + matter)"),
                    ("rk_update_cell", "cell (RK combination, algebraic constraints, recovery)")):
        print("  %-16s %10.1f  per %s" % (k, c[k], unit))
    print("mean Illinois iterations per cell: %.3f" % c["c2p_iters_mean"])
    print(json.dumps(c))


if __name__ == "__main__":
    main()
