"""Algorithmic FLOP counts of the benchmark workload (3 levels of 256^2, TOV
K=100, Gamma=2, rho_c=1.28e-3), per face / cell and per phase of one RK
stage, from the op-counting build of the oracle.  Writes
profiles/flops_tov_stable_3x256.md.  Test infrastructure; run by hand:
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
    path = os.path.join(ROOT, "profiles", "flops_tov_stable_3x256.md")
    with open(path, "w") as f:
        f.write("# Algorithmic FLOPs per unit, TOV 3 x 256^2 (level 1), one RK stage\n\n")
        f.write("Counted by `python oracle/count_flops.py` (the oracle's C sources compiled with a counting\n")
        f.write("scalar: add, mul, div, sqrt, pow/exp = 1 FLOP each; comparisons, fabs = 0).\n\n")
        f.write("| phase | unit | FLOPs per unit |\n|---|---|---|\n")
        for k, unit in (("flux_face", "x-face (PPM 5 prims + 6-pt metric + tetrad HLLC)"),
                        ("hydro_div_cell", "cell (flux divergence + sources)"),
                        ("cartoon_cell", "cell of the plane patch (9-pt interp + rotation, 7 planes, 25 fields)"),
                        ("z4c_derivs_cell", "cell (central/mixed/lopsided/KO differences of 25 fields)"),
                        ("z4c_point_cell", "cell (pointwise Z4c algebra + matter)"),
                        ("rk_update_cell", "cell (RK combination, algebraic constraints, recovery)")):
            f.write("| %s | %s | %.1f |\n" % (k, unit, c[k]))
        f.write("\nmean Illinois iterations per cell: %.3f\n\n" % c["c2p_iters_mean"])
        f.write("```json\n%s\n```\n" % json.dumps(c))
    print(json.dumps(c))


if __name__ == "__main__":
    main()
