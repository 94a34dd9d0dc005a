import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a) and the built library")
    config.addinivalue_line("markers", "slow: longer CPU oracle runs")


def pytest_collection_modifyitems(config, items):
    try:
        import torch
        has_gpu = torch.cuda.is_available()
    except Exception:  # pragma: no cover
        has_gpu = False
    if has_gpu:
        return
    skip = pytest.mark.skip(reason="no CUDA GPU in this environment")
    for it in items:
        if "gpu" in it.keywords:
            it.add_marker(skip)


# One-sided checks on mixed-precision bounds: the upper bound must not fall
# below the oracle's by more than a relative slack, the lower bound not rise
# above it by more.  The target is 1e-13.  It is what every lower bound and
# every upper bound up to contrast 1e3 get: their measured margins against the
# oracle stay below 5e-14.  Above contrast 1e3 the oracle's own upper bound
# moves between admissible double grids by up to the spread measured by
# tests/golden/make_spread.py (7.8e-13 at contrast ~1e4: FP64 rounding of the
# large double-grid values A_M), so no check can resolve the upper bound more
# finely than that; those upper bounds get twice the measured spread (the
# GPU's evaluation carries rounding of the same size).
ONE_SIDED_SLACK = 1e-13


def _measured_spread():
    import json
    p = os.path.join(ROOT, "tests", "golden", "oracle_spread.json")
    with open(p) as f:
        return float(json.load(f)["max_spread"])


def contrast(m):
    vals = [m["a0"]] + [inc[3] for inc in m["inclusions"]]
    return max(vals) / min(vals)


def one_sided_slack(m):
    """(upper slack, lower slack) of the one-sided checks for microstructure m."""
    if contrast(m) <= 1e3:
        return ONE_SIDED_SLACK, ONE_SIDED_SLACK
    return max(ONE_SIDED_SLACK, 2.0 * _measured_spread()), ONE_SIDED_SLACK


def one_sided_margins(U, L, Uo, Lo):
    """(upper margin, lower margin): min_i (U_ii - Uo_ii) / Uo_ii and
    min_i (Lo_ii - L_ii) / Lo_ii; both are >= 0 when the bounds are on the
    guaranteed side of the oracle's."""
    import numpy as np
    U, L, Uo, Lo = (np.asarray(a) for a in (U, L, Uo, Lo))
    d = U.shape[0]
    mu = min((U[i, i] - Uo[i, i]) / Uo[i, i] for i in range(d))
    ml = min((Lo[i, i] - L[i, i]) / Lo[i, i] for i in range(d))
    return float(mu), float(ml)
