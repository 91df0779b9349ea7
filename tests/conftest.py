import os
import sys
import tempfile

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

# the autotuner's choices go to a cache file of this test session, not the
# user's (tests that check the file set their own path)
os.environ["INTERGRAMS_TUNE_CACHE"] = os.path.join(tempfile.mkdtemp(prefix="ig_tune_"), "autotune.txt")


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")
    config.addinivalue_line("markers", "slow: long-running CPU test")
