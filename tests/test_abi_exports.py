"""The C-ABI library loads on a machine without a GPU and exports every
function that the headers under include/ declare (no compute calls)."""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared(header):
    text = open(os.path.join(ROOT, "include", header)).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(elbm[a-z0-9]*_[a-z0-9_]+)\s*\(", text)))


def test_library_exports_every_declared_symbol():
    from paper_2605_01774_gb300 import build, elbm
    build.build()
    L = elbm.lib()
    names = []
    for h in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if h.endswith(".h"):
            names += _declared(h)
    assert len(names) > 20
    missing = [n for n in names if not hasattr(L, n)]
    assert not missing, missing


def test_host_only_validation():
    from paper_2605_01774_gb300 import elbm as E
    assert E.elbm_check_tensor([0.1, 0, 0, 0.1, 0, 0.1]) == 0
    assert E.elbm_check_tensor([0.1, 0.2, 0, 0.1, 0, 0.1]) == 2
    assert E.elbm_check_tensor([0.1, 0, 0, 0.1, 0, float("nan")]) == 2
    assert E.elbm_check_velocity([0.05, 0.03, 0.02]) == 0
    assert E.elbm_check_velocity([0.9, 0, 0]) == 3
    import numpy as np
    d = np.array([0.1, 1e-3, 1e-5])
    T = E.elbm_relaxation_complement([d[0], 0, 0, d[1], 0, d[2]])
    # T = 2I - S has eigenvalues 2 - 2/(1 + 6 d) = 12 d / (1 + 6 d), full relative precision at d = 1e-5
    assert np.allclose(T[[0, 3, 5]], 12 * d / (1 + 6 * d), rtol=1e-15)


def test_bulk_copy_rate_rejects_bad_arguments():
    from paper_2605_01774_gb300 import elbm as E
    for size, bps in ((8, 1), (24, 1), (32768, 1), (512, 0), (512, 5)):
        with pytest.raises(E.ElbmError) as ei:
            E.elbm_bulk_copy_rate(size, bps)
        assert ei.value.status == 1


def test_host_only_validation_2d():
    import numpy as np
    from paper_2605_01774_gb300 import elbm as E
    assert E.elbm2d_check_velocity([0.05, -0.03]) == 0
    assert E.elbm2d_check_velocity([0.9, 0.0]) == 3
    assert E.elbm2d_check_velocity([float("nan"), 0.0]) == 3
    d = np.array([0.05, 1e-6])
    T = E.elbm2d_relaxation_complement([d[0], 0.0, d[1]])
    assert np.allclose(T[[0, 2]], 12 * d / (1 + 6 * d), rtol=1e-15) and T[1] == 0.0
    # rotated: T shares D's principal axes
    c, s = np.cos(0.4), np.sin(0.4)
    R = np.array([[c, -s], [s, c]])
    D = R @ np.diag(d) @ R.T
    T = E.elbm2d_relaxation_complement([D[0, 0], D[0, 1], D[1, 1]])
    Tm = np.array([[T[0], T[1]], [T[1], T[2]]])
    assert np.allclose(R.T @ Tm @ R, np.diag(12 * d / (1 + 6 * d)), atol=1e-15)
    with pytest.raises(E.ElbmError):
        E.elbm2d_relaxation_complement([1e-2, 2e-2, 1e-2])
