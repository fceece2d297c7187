"""CPU-side checks of the C-ABI library: it loads without a GPU and exports
every function include/mc.h declares (no compute calls here)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            src = open(os.path.join(ROOT, "include", fn)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"\b(mc_[a-z0-9_]+)\s*\(", src))
    return names


@pytest.mark.parametrize("name", ["libmc.so", "libmc_check.so"])
def test_library_exports_every_declared_symbol(name):
    # both builds are made at session start (tests/conftest.py)
    lib = ctypes.CDLL(os.path.join(ROOT, "paper_2608_06466_b300", name))
    missing = [n for n in sorted(_declared()) if not hasattr(lib, n)]
    assert not missing, f"declared in include/ but not exported: {missing}"
    assert lib.mc_version() >= 1


def test_normal_build_checks_nothing_without_gpu():
    import paper_2608_06466_b300 as mc
    rep = mc.mc_bounds_report(0)
    assert rep["enabled"] == 0 and rep["refused"] == 0 and rep["calls_checked"] == 0


def test_opts_default_and_last_error_without_gpu():
    import paper_2608_06466_b300 as mc
    o = mc.mc_burn_opts_default()
    assert o.rtol == 1e-6 and o.atol == 1e-10 and o.max_order == 5 and o.max_steps == 100000
    assert o.lu_precision == 64
    assert isinstance(mc.mc_last_error(), str)


def test_network_create_rejects_bad_descriptions_without_gpu():
    """Validation happens before any device call."""
    import numpy as np
    import paper_2608_06466_b300 as mc
    from mc_inputs import robertson_network
    net = robertson_network()
    net.react = net.react.copy()
    net.react[0, 0] = 7  # species index out of range
    try:
        mc.Network(net)
        raised = False
    except mc.MCError as e:
        raised = "MC_E_INVALID" in str(e)
    assert raised
    big = robertson_network()
    big.n_species = 41
    try:
        mc.Network(big)
        raised = False
    except mc.MCError as e:
        raised = "MC_E_UNSUPPORTED" in str(e)
    assert raised


@pytest.mark.parametrize("field,value,message", [
    ("staging", 3, "staging must be"), ("staging", -1, "staging must be"),
    ("jacobian", 2, "jacobian must be"), ("lu_precision", 16, "lu_precision must be"),
    ("max_order", 6, "max_order must be"), ("rtol", 0.0, "rtol and atol"),
    ("straggler_steps", -2, "straggler_steps"), ("block_threads", 48, "block_threads"),
])
def test_burn_options_are_checked_before_any_device_call(field, value, message):
    """Option validation runs first: a bad field is refused with its own message
    on a machine without a GPU (no network is needed to get there)."""
    import types
    import paper_2608_06466_b300 as mc
    o = mc.mc_burn_opts_default()
    setattr(o, field, value)
    dummy = types.SimpleNamespace(handle=None)
    with pytest.raises(mc.MCError, match="MC_E_INVALID") as err:
        mc.mc_burn_batch(dummy, o, 0, 1.0, None, 0, None, None, None, None, None)
    assert message in str(err.value) or message in mc.mc_last_error()
