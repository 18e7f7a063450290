import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")
    config.addinivalue_line("markers", "slow: longer CPU-only runs")
    # compile the CUDA library (when its sources changed) before any test module
    # loads it, so that no module keeps an older build mapped
    from paper_0912_3824_gb300 import build
    build.build()
