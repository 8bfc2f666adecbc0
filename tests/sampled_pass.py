"""Oracle output of one SG-WLS pass at chosen across-offsets (test helper).

The output of a pass at across-offset o (a column for the column direction)
is the mean, over the centres k with |k - o| <= r, of subsystem k's exact
solution at o (Sec. 2.3, steps 1-4); only those 2r + 1 subsystems are
solved, so full-size images can be checked on sampled offsets."""
import numpy as np

from oracle import COLUMN
from oracle.sgwls import centre_indices, neighbourhood_construction, solve_subsystem, subsystem_band


def oracle_pass_offsets(U, G, lam, prm, direction, offsets):
    """Pass output at the given across-offsets: (C, len(offsets), lines)."""
    U = U.astype(np.float64)
    G = G.astype(np.float64)
    C, H, W = U.shape
    dim, L = (W, H) if direction == COLUMN else (H, W)
    ks = centre_indices(dim, prm.r, prm.step)
    out = np.zeros((C, len(offsets), L))
    for n_o, o in enumerate(offsets):
        acc = np.zeros((C, L))
        cnt = np.zeros(L)
        for k in ks:
            if abs(k - o) > prm.r:
                continue
            rows, cols = neighbourhood_construction(direction, k, prm.r, H, W)
            u = solve_subsystem(subsystem_band(rows, cols, G, lam, prm), U[:, rows, cols].T, prm.r)
            across, line = (cols, rows) if direction == COLUMN else (rows, cols)
            m = across == o
            acc[:, line[m]] += u[m].T
            cnt[line[m]] += 1.0
        out[:, n_o] = acc / cnt
    return out
