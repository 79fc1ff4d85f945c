"""The C-ABI library builds, loads without a GPU, and exports every entry point
that include/helrm.h declares (no compute calls here)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "helrm.h")


def declared():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(helrm_[a-z0-9_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def libpath():
    from paper_2506_18150_gb300 import build
    return build.build()


def test_header_declares_the_boundary():
    """The calls of the hot path's boundary: keys, encryption, the matvec and
    the lookup, the inference, import/export, the client's packing, the NTT,
    and bootstrapping."""
    names = declared()
    for must in ["helrm_keygen", "helrm_encrypt", "helrm_decrypt", "helrm_rotate", "helrm_ptct_matvec",
                 "helrm_embedding_lookup", "helrm_infer", "helrm_ct_export", "helrm_ct_import",
                 "helrm_query_pack", "helrm_emb_prepare", "helrm_ptmat_prepare", "helrm_free",
                 "helrm_last_error", "helrm_ntt", "helrm_bootstrap", "helrm_boot_create", "helrm_keygen_ex",
                 "helrm_conjugate"]:
        assert must in names


def test_library_exports_every_declared_symbol(libpath):
    lib = ctypes.CDLL(libpath)
    missing = [n for n in declared() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_the_header(libpath):
    from paper_2506_18150_gb300 import helrm
    assert set(helrm.declared_symbols()) == set(declared())


def test_status_strings_without_gpu(libpath):
    from paper_2506_18150_gb300 import helrm
    lib = helrm.lib()
    assert lib.helrm_status_string(-5) == b"missing key"
    assert lib.helrm_last_error(None) == b"invalid context"
    lib.helrm_free(None)                                 # NULL is a no-op


def test_param_errors_need_no_gpu(libpath):
    from paper_2506_18150_gb300 import helrm
    with pytest.raises(helrm.HelrmError) as e:
        helrm.helrm_ctx_create(9, [40], 1, 40, 1, 30.0)  # log_n below the supported range
    assert e.value.name == "HELRM_E_PARAM"
