import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA device (GB300) and the compiled sacra2d library")
    config.addinivalue_line("markers", "slow: longer CPU runs")


import pytest  # noqa: E402


@pytest.fixture(autouse=True)
def _parity_stats(request):
    """For GPU tests: reset the parity statistics of gpu_common.compare_level
    before the test and print them after it (seen with pytest -rP)."""
    if request.node.get_closest_marker("gpu") is None:
        yield
        return
    import gpu_common
    gpu_common.reset_stats()
    yield
    if gpu_common.STATS["cells"]:
        print("parity: " + gpu_common.stats_line())
