"""ORACLE -- test infrastructure only (see oracle/__init__.py).

The density-fitting object operations of the paper's section "Density fitting utilities", eqs. (1)-(3),
on a three-index tensor I[g, r, s] (g: auxiliary index) with arbitrary two- and four-index tensors M, G,
written out as plain einsum definitions in FP64:

(1) index transformations:  I'_{g,ts} = sum_r I_{g,rs} M_rt   (transform_first)
                            I'_{g,rt} = sum_s I_{g,rs} M_st   (transform_second)
                            I'_{g,rs} = sum_d M'_gd I_{d,rs}  (transform_aux)
(2) contractions of two objects:
                            M_st = sum_{g r} I_{g,rs} I'_{g,rt}       (contract_first)
                            G_{rs,tu} = sum_g I_{g,rs} I'_{g,tu}      (contract_aux)
                            M_gd = sum_{rs} I_{g,rs} I'_{d,rs}        (contract_pairs)
(3) contractions with density matrices:
                            D_g = sum_{rs} I_{g,rs} M_rs              (density_fit)
                            M_rs = sum_g D_g I_{g,rs}                 (density_back)
                            I'_{g,tu} = sum_{rs} I_{g,rs} G_{rs,tu}   (apply_four_index)
"""
from __future__ import annotations

import numpy as np


def transform_first(I, M):
    return np.einsum("grs,rt->gts", I, M)


def transform_second(I, M):
    return np.einsum("grs,st->grt", I, M)


def transform_aux(I, Mp):
    return np.einsum("gd,drs->grs", Mp, I)


def contract_first(I, I2):
    return np.einsum("grs,grt->st", I, I2)


def contract_aux(I, I2):
    """G as a matrix over (rs) x (tu)."""
    g = np.einsum("grs,gtu->rstu", I, I2)
    return g.reshape(I.shape[1] * I.shape[2], I2.shape[1] * I2.shape[2])


def contract_pairs(I, I2):
    return np.einsum("grs,drs->gd", I, I2)


def density_fit(I, M):
    return np.einsum("grs,rs->g", I, M)


def density_back(I, D):
    return np.einsum("g,grs->rs", D, I)


def apply_four_index(I, G, nt, nu):
    """G: (rs) x (tu) matrix."""
    G4 = G.reshape(I.shape[1], I.shape[2], nt, nu)
    return np.einsum("grs,rstu->gtu", I, G4)
