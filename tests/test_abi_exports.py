"""The C-ABI library loads on a machine without a GPU and exports every
function that include/elbm.h declares (no compute calls)."""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared(header):
    text = open(os.path.join(ROOT, "include", header)).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(elbm_[a-z0-9_]+)\s*\(", text)))


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
