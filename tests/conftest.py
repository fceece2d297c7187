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


def _library_is_current():
    if not os.path.exists(LIB):
        return False
    srcs = glob.glob(os.path.join(PKG, "csrc", "*")) + glob.glob(os.path.join(ROOT, "include", "*.h"))
    return os.path.getmtime(LIB) >= max(os.path.getmtime(p) for p in srcs)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (B300, sm_103a)")


def pytest_sessionstart(session):
    # A fresh checkout has no libmc.so (built files are not committed): build it
    # first (nvcc cross-compiles without a GPU). The build script is loaded by
    # path, because importing the package needs the library.
    if not _library_is_current():
        spec = importlib.util.spec_from_file_location("_mc_build", os.path.join(PKG, "build.py"))
        mod = importlib.util.module_from_spec(spec)
        spec.loader.exec_module(mod)
        mod.build()
