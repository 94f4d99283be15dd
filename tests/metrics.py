"""Error metrics of the parity tests (reading R13).

max_rel_per_cell: max over cells and components of |U - U_ref| divided by the
cell's T^00 of U_ref (|M| < E, so it is the natural scale of every
component), floored at 1e-12 max |E_ref| so that vacuum cells (E_ref = 0)
are compared on that absolute scale.
rel_l1: per field, sum |a - b| / sum |b|; a field with sum |b| = 0 (a
momentum component that is zero everywhere) is divided by sum |E_ref|.
"""
import numpy as np


def max_rel_per_cell(U, Uref):
    U = np.asarray(U, dtype=np.float64)
    Uref = np.asarray(Uref, dtype=np.float64)
    scale = np.maximum(np.abs(Uref[0]), 1e-12 * np.abs(Uref[0]).max())
    return float((np.abs(U - Uref) / scale[None]).max())


def rel_l1(U, Uref):
    U = np.asarray(U, dtype=np.float64)
    Uref = np.asarray(Uref, dtype=np.float64)
    out = []
    for q in range(Uref.shape[0]):
        den = np.abs(Uref[q]).sum()
        if den == 0.0:
            den = np.abs(Uref[0]).sum()
        out.append(float(np.abs(U[q] - Uref[q]).sum() / den))
    return out
