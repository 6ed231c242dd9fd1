"""Shared by the Bondi tests: the paper's L1 measure of the rest-mass density
(Sec. III, Bondi accretion) between the initial and the evolved state,
weighted by sqrt(-g) dV = alpha W^-3 (2 pi x dx dz) over the interior cells
of every level not covered by a finer one."""
import numpy as np

from paper_2502_03223_gb300 import workloads as W

G = 8


def bondi_l1(cfg, datas, read_rho):
    """read_rho(level) -> the padded rho plane of the evolved state."""
    num = den = 0.0
    for l in range(cfg.n_levels):
        sl = (slice(G, G + cfg.nz), slice(G, G + cfg.nx))
        X, _ = W.cell_centres(cfg, l)
        d = datas[l]
        rho0 = d[25][sl]
        rho = read_rho(l)[sl]
        wgt = (d[18] * d[0] ** -3.0 * X)[sl] * cfg.dx(l) * cfg.dz(l)
        if l < cfg.n_levels - 1:
            wgt = wgt.copy()
            wgt[:cfg.nz // 2, :cfg.nx // 2] = 0.0
        num += float(np.sum(np.abs(rho - rho0) * wgt))
        den += float(np.sum(rho0 * wgt))
    return num / den
