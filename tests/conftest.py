import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (sm_103a) and the built libmw")
    config.addinivalue_line("markers", "slow: longer CPU test")


@pytest.fixture(scope="session")
def orc():
    import oracle
    oracle.build()
    return oracle


@pytest.fixture(scope="session")
def mwlib():
    """The CUDA library binding; builds libmw.so if needed.  GPU tests only."""
    import torch
    if not torch.cuda.is_available():
        pytest.fail("GPU test collected without a CUDA device")
    from paper_0809_2811_gb300 import build, mw
    build.build()
    mw.lib()
    return mw


def pytest_terminal_summary(terminalreporter, exitstatus, config):
    """Prints each parity comparison's errors as fractions of its tolerances
    (force, energy, virial; 1.0 = at the tolerance) and the strict per-atom
    relative force error."""
    try:
        import _parity
    except ImportError:
        return
    if not _parity.MARGINS:
        return
    tr = terminalreporter
    tr.section("parity margins (error / tolerance; strict = max |dF|/|F| over |F| >= eps/sigma)")
    for case, m in _parity.MARGINS:
        tr.write_line(f"{case:48s} force {m.get('force', float('nan')):.3f}  energy {m.get('energy', float('nan')):.3f}"
                      f"  virial {m.get('virial', float('nan')):.3f}  strict {m.get('strict_force_rel', float('nan')):.2e}")
