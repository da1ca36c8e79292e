import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    # temporary files of the tests stay inside the repository (git-ignored)
    if not config.option.basetemp:
        config.option.basetemp = os.path.join(ROOT, ".pytest_tmp")
    config.addinivalue_line("markers", "gpu: needs a CUDA device (B300, sm_103a)")
    config.addinivalue_line("markers", "slow: long-running CPU test")


def pytest_sessionstart(session):
    # A fresh checkout has no built library (build artefacts are not committed): build it
    # once, as __graft_entry__.build() would, so that the ABI tests can load it.  An
    # existing library is used as it is.
    from paper_2509_10722_b300 import build as B
    if not os.path.exists(B.LIB):
        B.build()
