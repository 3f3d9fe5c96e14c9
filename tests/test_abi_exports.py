"""The C-ABI library loads and exports every function include/pwave.h
declares (no GPU needed: nothing is called)."""
import ctypes
import os
import re

from tests._lib import ROOT, ensure_built


def declared_functions():
    src = open(os.path.join(ROOT, "include", "pwave.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(pw_[a-z0-9_]+)\s*\(", src)))


def test_header_declares_the_core_calls():
    names = declared_functions()
    for n in ("pw_ctx_create", "pw_model_load", "pw_encode_image", "pw_decode_image",
              "pw_decode_batch", "pw_cdf_bank", "pw_rans_decode", "pw_context_params",
              "pw_lift_inverse"):
        assert n in names


def test_library_exports_every_declared_symbol():
    lib = ctypes.CDLL(ensure_built())
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_python_binding_covers_the_abi():
    ensure_built()
    import paper_2405_12631_gb300 as pw
    missing = [n for n in declared_functions() if n not in pw.EXPORTED]
    assert not missing, missing
