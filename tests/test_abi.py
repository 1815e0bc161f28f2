"""CPU-side checks of the C ABI: the library loads, exports every declared
entry point, and fails cleanly (no crash) without a GPU."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "tci_b300.h")


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:const\s+)?\w+\**\s+\**(tci_\w+)\s*\(", src, flags=re.M)))


def test_header_declares_entry_points():
    names = declared_functions()
    for n in ("tci_create_context", "tci_contract", "tci_heff_apply", "tci_lanczos", "tci_version"):
        assert n in names


def test_library_exports_every_declared_symbol():
    import paper_2512_23917_b300 as tci
    out = subprocess.run(["nm", "-D", "--defined-only", tci.LIB_PATH], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\bT (tci_\w+)", out))
    missing = [n for n in declared_functions() if n not in exported]
    assert not missing, missing
    # and the binding knows every one of them
    bound = {s[0] for s in tci.SIGNATURES}
    assert set(declared_functions()) <= bound, set(declared_functions()) - bound


def test_version_and_status_strings():
    import paper_2512_23917_b300 as tci
    assert tci.version() == "1.0"
    assert tci.lib.tci_status_string(3).decode() == "TCI_ERR_LABEL"


def test_null_arguments_are_rejected_without_a_device():
    import paper_2512_23917_b300 as tci
    # destroying a NULL context is an error, not a crash
    h = ctypes.c_void_p()
    assert tci.lib.tci_destroy_context(ctypes.byref(h)) == 9
    assert tci.lib.tci_create_context(None, 0, None) == 1
    assert b"NULL" in tci.lib.tci_last_error(None)
    # free of a NULL tensor
    assert tci.lib.tci_tensor_free(ctypes.byref(ctypes.c_void_p())) == 1
    # plan-level setters reject a NULL plan before touching a device
    cfg = (ctypes.c_int * 4)(256, 1024, 0, 4)
    assert tci.lib.tci_heff_set_config(None, cfg) == 1
    assert tci.lib.tci_heff_get_config(None, cfg) == 1
    assert tci.lib.tci_heff_set_lanczos_arith(None, 2) == 1
    assert tci.lib.tci_heff_set_gram_schmidt(None, 1) == 1


@pytest.mark.skipif(os.path.exists("/dev/nvidia0"), reason="only meaningful without a GPU")
def test_context_creation_fails_cleanly_without_gpu():
    import paper_2512_23917_b300 as tci
    h = ctypes.c_void_p()
    st = tci.lib.tci_create_context(ctypes.byref(h), 0, None)
    assert st in (1, 7) and not h.value
