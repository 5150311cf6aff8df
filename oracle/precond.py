"""Block-diagonal preconditioner (Sec. 3.2.1), FP64.

Test infrastructure only (see the package docstring).

Steps (Sec. 3.2.1):
 1. divide the spheres into subsets G_j by an array of cuboids and renumber the
    spheres so that each subset is one consecutive run of indices;
 2. form the block M_j = M^{ii'} restricted to i, i' in G_j;
 3. factor P_j M_j = L_j U_j (LU with partial pivoting) and store the factors;
 4. apply x = M_j^{-1} y per block by solving L_j U_j x = P_j y.

The paper does not fix the cuboid grid.  Reading used here: the grid is
anchored at the minimum corner of the bounding box of the sphere centres, a
sphere belongs to the cuboid floor((r - r_min)/edge) that holds its centre,
empty cuboids are dropped, cuboids are ordered lexicographically by their
(z, y, x) index and spheres keep their original relative order inside a
cuboid.
"""

import numpy as np
import scipy.linalg as sla

from .solve import master_matrix
from .translation import coupling_matrix


def partition(positions, edge):
    """Return (perm, offsets): ``perm[new] = old`` sphere index, and block
    offsets into the permuted order (length n_blocks + 1)."""
    pos = np.asarray(positions, dtype=float)
    lo = pos.min(axis=0)
    cell = np.floor((pos - lo) / edge).astype(np.int64)
    keys = [(int(c[2]), int(c[1]), int(c[0]), i) for i, c in enumerate(cell)]
    keys.sort()
    perm = np.array([kk[3] for kk in keys], dtype=np.int64)
    offsets = [0]
    for q in range(1, len(keys)):
        if keys[q][:3] != keys[q - 1][:3]:
            offsets.append(q)
    offsets.append(len(keys))
    return perm, np.array(offsets, dtype=np.int64)


class BlockPreconditioner:
    """Dense-LU block-diagonal preconditioner in the ORIGINAL sphere order."""

    def __init__(self, positions, k, lmax, tdiag, edge):
        pos = np.asarray(positions, dtype=float)
        self.nm = 2 * lmax * (lmax + 2)
        self.perm, self.offsets = partition(pos, edge)
        t = np.asarray(tdiag).reshape(pos.shape[0], self.nm)
        self.blocks = []
        for q in range(len(self.offsets) - 1):
            ids = self.perm[self.offsets[q]:self.offsets[q + 1]]
            W = coupling_matrix(pos[ids], k, lmax)
            M = master_matrix(t[ids].reshape(-1), W)
            self.blocks.append((ids, sla.lu_factor(M)))

    def apply(self, y):
        """x = blockdiag(M_j)^{-1} y, y shaped (N, nmax) (or flat)."""
        shp = np.shape(y)
        yy = np.asarray(y, dtype=complex).reshape(-1, self.nm)
        x = np.zeros_like(yy)
        for ids, lu in self.blocks:
            x[ids] = sla.lu_solve(lu, yy[ids].reshape(-1)).reshape(-1, self.nm)
        return x.reshape(shp)
