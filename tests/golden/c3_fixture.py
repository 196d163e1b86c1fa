"""The stored oracle SVD of the complex 4096 x 2048 workload
(c3_oracle_4096x2048.npz, written by make_c3_oracle.py from the oracle
alone) and the error of another SVD of the same input against it, output by
output: the singular values, and the sampled columns of U and V after the
one unit phase per singular triplet that the SVD leaves free."""
import hashlib
import os

import numpy as np

PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "c3_oracle_4096x2048.npz")


def load():
    """The stored oracle result as a dict, or None when it has not been
    written."""
    if not os.path.exists(PATH):
        return None
    z = np.load(PATH)
    return {k: z[k] for k in z.files}


def input_matches(A, fx):
    """Whether A is bit-equal to the input the oracle ran on."""
    h = hashlib.sha256(np.ascontiguousarray(A).tobytes()).hexdigest()
    return h == str(fx["input_sha256"])


def errors(sigma, U_cols, V_cols, fx):
    """Errors of (sigma, U[:, cols], V[:, cols]) against the oracle's:
    singular values normwise (max |d sigma| / sigma_1) and relatively (max
    |d sigma_j| / sigma_j); for each sampled column j the 2-norm distances
    ||u_j - e^{i t} u_j'|| and ||v_j - e^{i t} v_j'|| with the phase t that
    aligns u_j with the oracle's u_j'.  Also the per-column bound
    64 n eps sigma_1 / gap_j (gap_j: distance to the nearest other singular
    value), the normwise perturbation bound for singular vectors."""
    so = fx["sigma"]
    sigma = np.asarray(sigma, dtype=np.float64)
    n = so.size
    d = np.abs(sigma - so)
    out = {"sigma_max_err_normwise": float(d.max() / so[0]),
           "sigma_max_err_relative": float((d / so).max())}
    cols = fx["cols"]
    Uo, Vo = fx["U_cols"], fx["V_cols"]
    eu, ev, bound = [], [], []
    eps = np.finfo(np.float64).eps
    for k, j in enumerate(cols):
        ph = np.vdot(Uo[:, k], U_cols[:, k])
        ph = ph / abs(ph) if ph != 0 else 1.0
        eu.append(float(np.linalg.norm(U_cols[:, k] - ph * Uo[:, k])))
        ev.append(float(np.linalg.norm(V_cols[:, k] - ph * Vo[:, k])))
        others = np.delete(so, j)
        bound.append(float(64 * n * eps * so[0] / np.abs(others - so[j]).min()))
    out.update({"cols": [int(c) for c in cols], "U_col_err": eu, "V_col_err": ev,
                "col_bound_64neps_over_gap": bound,
                "U_cols_max_err": max(eu), "V_cols_max_err": max(ev)})
    return out
