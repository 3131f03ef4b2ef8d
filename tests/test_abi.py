"""The C-ABI library builds, loads and exports every entry point its header
declares; host-side argument handling needs no GPU."""
import ctypes
import os
import re

import pytest

from paper_2203_08263_gb300 import build as nbuild
from paper_2203_08263_gb300 import nbody as nb

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _header_functions():
    text = open(os.path.join(ROOT, "include", "nbody.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(nb_[a-z_]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    nbuild.build()
    return nb.load()


def test_every_declared_symbol_is_exported_and_bound(lib):
    declared = _header_functions()
    assert len(declared) >= 18
    for name in declared:
        assert hasattr(lib, name), name
        assert name in nb.SIGNATURES, f"binding lacks {name}"
    assert set(nb.SIGNATURES) == set(declared)


def test_version_and_status_strings(lib):
    assert lib.nb_abi_version() == 1
    names = [lib.nb_status_string(s).decode() for s in range(6)]
    assert names == ["NB_OK", "NB_ERR_INVALID", "NB_ERR_CUDA", "NB_ERR_NOMEM",
                     "NB_ERR_TIMEOUT", "NB_ERR_UNSUPPORTED"]
    assert lib.nb_status_string(99).decode() == "NB_ERR_UNKNOWN"


def test_null_and_invalid_arguments_are_rejected_without_a_device(lib):
    p = nb.nb_params(1.0, 0.01, 1e-3, 0, 0, (ctypes.c_int * 4)(0, 0, 0, 0))
    assert lib.nb_create(None, 0, ctypes.byref(p)) == nb.NB_ERR_INVALID
    h = ctypes.c_void_p()
    assert lib.nb_create(ctypes.byref(h), 0, None) == nb.NB_ERR_INVALID
    for bad in (nb.nb_params(1.0, 0.0, 1e-3, 0, 0), nb.nb_params(1.0, -1.0, 1e-3, 0, 0),
                nb.nb_params(float("nan"), 0.01, 1e-3, 0, 0), nb.nb_params(1.0, 0.01, 1e-3, 7, 0),
                nb.nb_params(1.0, 0.01, 1e-3, 0, 5)):
        assert lib.nb_create(ctypes.byref(h), 0, ctypes.byref(bad)) == nb.NB_ERR_INVALID
        assert not h.value
    # calls on a NULL context fail cleanly
    assert lib.nb_accel(None, 4, None, None, None, None) == nb.NB_ERR_INVALID
    assert lib.nb_run(None, 4, None, None, None, 1, None, 0, None) == nb.NB_ERR_INVALID
    assert lib.nb_sync(None, None) == nb.NB_ERR_INVALID
    assert lib.nb_launch_count(None) == 0
    assert lib.nb_last_error(None) == b""
    lib.nb_destroy(None)
    assert lib.nb_batched_max_n() >= 8192


def _header_enum(prefix):
    text = open(os.path.join(ROOT, "include", "nbody.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return {m.group(1): int(m.group(2)) for m in re.finditer(r"\b(" + prefix + r"[A-Z0-9_]+)\s*=\s*(\d+)", text)}


def test_binding_constants_match_the_header():
    """Debug keys, force forms and statuses: the values the binding passes
    and decodes are the header's."""
    dbg = _header_enum("NB_DBG_")
    assert dbg and all(getattr(nb, k) == v for k, v in dbg.items())
    forms = _header_enum("NB_FORM_")
    assert sorted(forms.values()) == sorted(nb.FORMS)
    for k, v in forms.items():
        assert nb.FORMS[v] == k[len("NB_FORM_"):].lower(), (k, nb.FORMS[v])
    st = _header_enum("NB_ERR_")
    assert all(getattr(nb, k) == v for k, v in st.items())
