import glob
import importlib.util
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

PKG = os.path.join(ROOT, "paper_2608_06466_b300")
LIB = os.path.join(PKG, "libmc.so")
LIB_CHECK = os.path.join(PKG, "libmc_check.so")


def _library_is_current(lib):
    if not os.path.exists(lib):
        return False
    srcs = glob.glob(os.path.join(PKG, "csrc", "*")) + glob.glob(os.path.join(ROOT, "include", "*.h"))
    return os.path.getmtime(lib) >= max(os.path.getmtime(p) for p in srcs)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (B300, sm_103a)")


def pytest_sessionstart(session):
    # A fresh checkout has no libmc.so nor its bounds-check build
    # libmc_check.so (built files are not committed): build them first (nvcc
    # cross-compiles without a GPU). The build script is loaded by path,
    # because importing the package needs the library.
    stale = [check for check, lib in ((False, LIB), (True, LIB_CHECK)) if not _library_is_current(lib)]
    if stale:
        spec = importlib.util.spec_from_file_location("_mc_build", os.path.join(PKG, "build.py"))
        mod = importlib.util.module_from_spec(spec)
        spec.loader.exec_module(mod)
        for check in stale:
            mod.build(check=check)
