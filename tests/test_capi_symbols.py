"""The C ABI library builds for sm_103a, loads without a GPU and exports every
function include/vlb.h declares (no compute call is made here)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared(header):
    text = open(header).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(vlb_[a-z_0-9]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    from paper_2410_23802_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_every_declared_symbol_is_exported(lib):
    names = []
    for h in os.listdir(os.path.join(ROOT, "include")):
        if h.endswith(".h"):
            names += _declared(os.path.join(ROOT, "include", h))
    assert "vlb_step" in names and "vlb_create" in names
    for n in names:
        assert hasattr(lib, n), n


def test_binding_struct_matches_header(lib):
    from paper_2410_23802_gb300 import vlb as V
    lib.vlb_params_size.restype = ctypes.c_size_t
    assert lib.vlb_params_size() == ctypes.sizeof(V.vlb_params)
    p = V.vlb_params_default()
    assert p.abi_version == 1 and abs(p.lambda_q_flow - 1 / 12) < 1e-16 and p.s_e == 1.25


def test_parameter_validation_without_gpu():
    from paper_2410_23802_gb300 import vlb as V
    for bad in (dict(nx=1), dict(tau_f=0.5), dict(precision=7), dict(rho_ratio=0.0), dict(thermal_rates_mode=3)):
        with pytest.raises(V.VlbError) as e:
            V.vlb_create(V.vlb_params_default(**bad))
        assert e.value.status == V.VLB_EINVAL
