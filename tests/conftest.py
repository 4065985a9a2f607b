import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")
    # Build (incrementally) the CUDA library and the C oracle before collection; nvcc
    # cross-compiles sm_103a without a GPU.
    from paper_1709_00178_gb300 import build as pbuild
    from oracle.build import build_oracle

    pbuild.build()
    build_oracle()
