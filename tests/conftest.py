import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a) and the built libreg")


def pytest_sessionfinish(session, exitstatus):
    """With REG_PARITY_LOG set, write every recorded parity error (measured error against
    the FP64 oracle and the tolerance it was held to) to that JSON file."""
    path = os.environ.get("REG_PARITY_LOG")
    if not path:
        return
    from tests import gpu_util
    if gpu_util.RECORDS:
        os.makedirs(os.path.dirname(os.path.abspath(path)), exist_ok=True)
        gpu_util.write_records(path)
