"""The C-ABI library loads without a GPU and exports every function include/gx.h declares."""
import ctypes
import os
import re

import paper_2512_12615_gb300 as gx

HEADER = os.path.join(os.path.dirname(os.path.dirname(__file__)), "include", "gx.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = re.findall(r"^[A-Za-z_][\w \t\*]*?\b(gx_\w+)\s*\(", text, flags=re.M)
    return sorted(set(names))


def test_header_parses():
    names = declared_functions()
    assert "gx_verify_load" in names and "gx_run_batch" in names and "gx_ringbuf_drain" in names
    assert len(names) >= 30


def test_every_declared_symbol_is_exported():
    lib = ctypes.CDLL(gx.lib()._name)
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_the_header():
    assert set(declared_functions()) <= set(gx.exported_symbols())


def test_no_device_is_reported_cleanly_or_device_is_gb300():
    import ctypes as C
    h = C.c_void_p()
    rc = gx.lib().gx_init(0, 0, C.byref(h))
    if rc == 0:
        assert gx.lib().gx_shutdown(h) == 0
    else:
        assert rc == gx.E_NODEV
    assert gx.lib().gx_strerror(gx.E_VERIFY).decode().startswith("program rejected")
