import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def _build_library():
    """Build libafqmc.so if it is missing or older than its sources (build.py is
    loaded by path: importing the package needs the library)."""
    import importlib.util
    spec = importlib.util.spec_from_file_location("_afqmc_build", os.path.join(ROOT, "paper_2609_14668_b300", "build.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    mod.build()


_build_library()


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (B300) and the built libafqmc.so")
    config.addinivalue_line("markers", "slow: CPU test that takes tens of seconds")
    config.addinivalue_line("markers", "paper: long GPU physics run against the paper's tables (opt-in: -m paper)")
