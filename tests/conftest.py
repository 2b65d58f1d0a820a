import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (B300, sm_103a) and the built libnvdb.so")
    config.addinivalue_line("markers", "slow: long-running CPU test")
    # libnvdb.so is a build output (not in version control): compile it if missing or stale
    from paper_2208_04448_b300 import _build as b
    b.build()
