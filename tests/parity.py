"""Field comparison used by every GPU parity test.

A field passes when both
* the norm-wise error ||got - ref||_2 / ||ref||_2 <= tol, and
* the element-wise error max |got - ref| / max |ref| <= ELEM_FACTOR * tol
(complex entries; max over all entries compared).  The element-wise bound
catches a wrong value confined to a few sites (a boundary slab, a ragged
tail) that the norm would average away; for a correct field the two ratios
are about equal (rounding errors spread like the values), hence the factor
of 5.  Every comparison is recorded, and the worst ratios of each test are
printed at the end of the run (conftest.py).
"""

import numpy as np

ELEM_FACTOR = 5.0
RECORDS = []   # (test id, what, tol, norm-wise, element-wise)
CURRENT = {"test": ""}


def errors(got, ref):
    got = np.asarray(got)
    ref = np.asarray(ref)
    d = got - ref
    nrm = float(np.linalg.norm(d) / np.linalg.norm(ref))
    elem = float(np.abs(d).max() / np.abs(ref).max())
    return nrm, elem


def assert_close(got, ref, tol, what=""):
    nrm, elem = errors(got, ref)
    RECORDS.append((CURRENT["test"], str(what), tol, nrm, elem))
    assert nrm <= tol and elem <= ELEM_FACTOR * tol, (
        f"{what}: norm-wise {nrm:.3e}, element-wise {elem:.3e} (tol {tol:g}, element-wise {ELEM_FACTOR * tol:g})")
    return nrm, elem
