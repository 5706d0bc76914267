import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)
HERE = os.path.dirname(os.path.abspath(__file__))
if HERE not in sys.path:
    sys.path.insert(0, HERE)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")
    config.addinivalue_line("markers", "slow: takes more than a few seconds")


@pytest.fixture(autouse=True)
def _parity_record_scope(request):
    import parity

    parity.CURRENT["test"] = request.node.nodeid
    yield


def pytest_terminal_summary(terminalreporter):
    """Worst norm-wise and element-wise parity errors of each GPU test
    (relative to its tolerance), when any field was compared."""
    try:
        import parity
    except ImportError:
        return
    if not parity.RECORDS:
        return
    worst = {}
    for test, what, tol, nrm, elem in parity.RECORDS:
        w = worst.setdefault(test, [0.0, 0.0, 0.0, 0.0])
        w[0] = max(w[0], nrm)
        w[1] = max(w[1], elem)
        w[2] = max(w[2], nrm / tol)
        w[3] = max(w[3], elem / tol)
    terminalreporter.section("parity errors (worst per test: norm-wise, element-wise, both / tol)")
    for test, (n, e, rn, re_) in sorted(worst.items()):
        terminalreporter.write_line(f"{test}: norm {n:.2e} elem {e:.2e} | /tol {rn:.2f} {re_:.2f}")


@pytest.fixture(scope="session")
def oracle_mod():
    import oracle

    oracle.build()
    return oracle
