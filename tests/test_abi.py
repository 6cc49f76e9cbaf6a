"""Host-side checks of the C ABI: the library loads on a machine without a
GPU, exports every entry point include/net.h declares, and rejects invalid
descriptors before touching the device."""
import ctypes
import os
import re

import pytest

from paper_1811_03882_gb300 import binding, build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def L():
    build.build()
    return binding.lib()


def declared_symbols():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", fn)).read()
            txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
            names |= set(re.findall(r"\b(net_[a-z_0-9]+)\s*\(", txt))
    return sorted(names)


def test_every_declared_symbol_is_exported(L):
    syms = declared_symbols()
    assert "net_forward" in syms and "net_create" in syms and len(syms) >= 15
    for s in syms:
        assert hasattr(L, s), s
    assert set(syms) <= set(binding._SIGS), set(syms) - set(binding._SIGS)


def test_version_and_error_string(L):
    assert b"sm_103a" in L.net_version()
    assert isinstance(binding.last_error(), str)


def test_create_rejects_bad_descriptors(L):
    h = ctypes.c_void_p()
    assert L.net_create(None, ctypes.byref(h)) == binding.NET_E_INVAL
    layers = (binding.net_layer * 1)(binding.net_layer(5, 8, 1, 1, 0))  # k = 5
    d = binding.net_desc(3, 1, ctypes.cast(layers, ctypes.POINTER(binding.net_layer)), 0, None,
                         1, 64, 0, None, 0)
    assert L.net_create(ctypes.byref(d), ctypes.byref(h)) == binding.NET_E_INVAL
    assert "k=5" in binding.last_error()
    layers[0] = binding.net_layer(3, 8, 1, 1, 0)
    d.max_batch = 0
    assert L.net_create(ctypes.byref(d), ctypes.byref(h)) == binding.NET_E_INVAL
    d.max_batch, d.prec = 1, 7
    assert L.net_create(ctypes.byref(d), ctypes.byref(h)) == binding.NET_E_INVAL


def test_free_null_is_ok(L):
    assert L.net_free(None) == binding.NET_OK
