"""The library's fully symmetric simplex rules (host code, no GPU) against the oracle's, derived independently
(scipy variable projection there, the library's own Gauss-Newton here): same points and weights at every degree."""
import numpy as np
import pytest

from oracle import symmetric

mfa = pytest.importorskip("paper_1903_08243_gb300")


def canon(pts, w):
    return np.array(sorted(map(tuple, np.round(np.column_stack([pts, w]), 10))))


@pytest.mark.parametrize("cell, dim", [("tri", 2), ("tet", 3)])
@pytest.mark.parametrize("degree", range(7))
def test_library_rule_equals_oracle_rule(cell, dim, degree):
    try:
        lpts, lw = mfa.mfa_simplex_rule(mfa.MFA_CELL_TRI3 if dim == 2 else mfa.MFA_CELL_TET4, degree)
    except OSError as e:  # the library could not be loaded on this machine
        pytest.skip(str(e))
    opts, ow = symmetric.rule(dim, degree)
    assert lw.shape == ow.shape
    a, b = canon(lpts, lw), canon(opts, ow)
    assert np.abs(a - b).max() <= 1e-9
    # unrounded: match every library point with its oracle point
    for p, w in zip(lpts, lw):
        d = np.abs(opts - p).max(axis=1)
        j = int(np.argmin(d))
        assert d[j] <= 1e-13 and abs(ow[j] - w) <= 1e-14


def test_bad_arguments():
    try:
        lib = mfa.lib()
    except OSError as e:
        pytest.skip(str(e))
    with pytest.raises(mfa.MfaError):
        mfa.mfa_simplex_rule(mfa.MFA_CELL_HEX8, 2)
    with pytest.raises(mfa.MfaError):
        mfa.mfa_simplex_rule(mfa.MFA_CELL_TET4, 7)
    import ctypes
    n = ctypes.c_int()
    buf = np.empty(64)
    assert lib.mfa_simplex_rule(mfa.MFA_CELL_TET4, 6, 10, buf.ctypes.data, buf.ctypes.data, ctypes.byref(n)) != 0
    assert n.value == 24  # the count is reported even when the buffers are too small
