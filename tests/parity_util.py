"""Comparison helpers for GPU-vs-oracle parity tests.

Factors U_k are unique only up to column sign, and a column is determined by
the data only when its singular value is separated from its neighbours; the
helpers align signs, compare well-separated columns element by element, and
compare clusters of close singular values through their subspace projectors.
"""

import numpy as np

U_TOL = 1e-4          # factors, max-abs after sign alignment (float32 path)
RELERR_TOL = 1e-5     # |relerr_gpu - relerr_oracle|
GAP_MIN = 1e-3        # columns with (sigma gap)/sigma_1 below this are compared as subspaces


def to_np(t):
    return t.detach().cpu().double().numpy()


def align_signs(Ug, Ur):
    s = np.sign((Ug * Ur).sum(axis=0))
    s[s == 0] = 1.0
    return Ug * s, s


def clusters(sigma, r, gap_min=GAP_MIN):
    """Split columns 0..r-1 into runs whose consecutive relative gaps < gap_min."""
    sigma = np.asarray(sigma, dtype=np.float64)
    s1 = sigma[0] if sigma[0] > 0 else 1.0
    out, cur = [], [0]
    for j in range(1, r):
        if (sigma[j - 1] - sigma[j]) / s1 < gap_min:
            cur.append(j)
        else:
            out.append(cur)
            cur = [j]
    out.append(cur)
    # a cluster touching column r-1 is only determined if sigma_{r-1} is separated from sigma_r
    tail_ok = len(sigma) <= r or (sigma[r - 1] - sigma[r]) / s1 >= gap_min
    return out, tail_ok


def compare_factor(Ug, Ur, sigma_ref, tol=U_TOL, gap_min=GAP_MIN, min_covered=1):
    """Returns (signs, max-abs deviation over determined columns, #strict columns,
    #covered columns).  Strict columns are compared element by element, columns of
    a cluster of close singular values through the cluster's projector; a trailing
    cluster that is not separated from sigma_r is undetermined and not covered.
    Fails unless at least ``min_covered`` columns were compared."""
    Ug = np.asarray(Ug, dtype=np.float64)
    r = Ur.shape[1]
    Ua, s = align_signs(Ug, Ur)
    cl, tail_ok = clusters(sigma_ref, r, gap_min)
    worst, strict, covered = 0.0, 0, 0
    for ci, c in enumerate(cl):
        if ci == len(cl) - 1 and not tail_ok:
            continue
        covered += len(c)
        if len(c) == 1:
            worst = max(worst, np.abs(Ua[:, c[0]] - Ur[:, c[0]]).max())
            strict += 1
        else:
            Pg = Ua[:, c] @ Ua[:, c].T
            Pr = Ur[:, c] @ Ur[:, c].T
            worst = max(worst, np.abs(Pg - Pr).max())
    assert covered >= min_covered, ("compared %d of %d columns" % (covered, r), min_covered)
    return s, worst, strict, covered


def orthonormality(U):
    U = np.asarray(U, dtype=np.float64)
    return np.abs(U.T @ U - np.eye(U.shape[1])).max()


def flip_core(G, signs):
    G = np.array(G, dtype=np.float64, copy=True)
    for k, s in enumerate(signs):
        shape = [1] * G.ndim
        shape[k] = -1
        G = G * s.reshape(shape)
    return G
