"""Error metrics of the parity tests (reading R13).

max_rel_per_cell: max over cells and components of |U - U_ref| divided by the
cell's T^00 of U_ref (|M| < E, so it is the natural scale of every
component), floored at 1e-12 max |E_ref| so that vacuum cells (E_ref = 0)
are compared on that absolute scale.
rel_l1: per field, sum |a - b| / max(sum |b|, 1e-3 sum |E_ref|).  A field's
own sum is the denominator wherever the field carries at least a thousandth
of the energy; below that the energy scale is.  The floor is what makes the
FP32 bound meaningful for fields that are (nearly) zero: the FP32 rounding of
a momentum component is set by the energy-scale terms of its flux (the
pressure p = E/3 in M_n v_n + p), not by the component's own size, so a
pencil at rest next to a blast, whose momentum is a few cells of 1e-9 E,
would otherwise be judged by FP32 noise over a vanishing denominator.
"""
import numpy as np

L1_FLOOR = 1e-3


def max_rel_per_cell(U, Uref):
    U = np.asarray(U, dtype=np.float64)
    Uref = np.asarray(Uref, dtype=np.float64)
    scale = np.maximum(np.abs(Uref[0]), 1e-12 * np.abs(Uref[0]).max())
    return float((np.abs(U - Uref) / scale[None]).max())


def rel_l1(U, Uref, floor=L1_FLOOR):
    """floor = 0: the bare ratio, with sum |E_ref| only where sum |b| = 0."""
    U = np.asarray(U, dtype=np.float64)
    Uref = np.asarray(Uref, dtype=np.float64)
    esum = np.abs(Uref[0]).sum()
    out = []
    for q in range(Uref.shape[0]):
        den = max(np.abs(Uref[q]).sum(), floor * esum)
        if den == 0.0:
            den = esum
        out.append(float(np.abs(U[q] - Uref[q]).sum() / den))
    return out
