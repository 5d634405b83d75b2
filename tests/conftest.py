import os
import sys

import pytest

ROOT = os.path.abspath(os.path.join(os.path.dirname(__file__), ".."))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a) and the built library")


@pytest.fixture(scope="session")
def golden_pedigree():
    import json
    from fractions import Fraction
    import numpy as np

    with open(os.path.join(ROOT, "tests", "golden", "pedigree_exact.json")) as f:
        d = json.load(f)

    def arr(x):
        return np.vectorize(lambda s: float(Fraction(s)))(np.array(x, dtype=object)).astype(np.float64)

    return dict(
        Phi=arr(d["Phi"]), XL=arr(d["XL"]), XR=np.array(d["XR"], dtype=np.int8),
        Y=arr(d["Y"]), h2=arr(d["h2"]), s2=arr(d["s2"]), B=arr(d["B"]), Vd=arr(d["Vdiag"]),
        W=arr(d["W"]), raw=d,
    )
