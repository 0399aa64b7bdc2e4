"""The C-ABI library builds, loads without a GPU, and exports every function
that include/igp.h declares (no compute call is made here)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_functions():
    names = []
    for f in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if not f.endswith(".h"):
            continue
        text = open(os.path.join(ROOT, "include", f)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        names += re.findall(r"^\s*(?:const\s+)?[A-Za-z_][\w\s\*]*?\b(igp_\w+)\s*\(", text, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def libigp():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2508_19737_gb300 import api
    return api.lib()


def test_header_declares_the_boundary():
    names = _declared_functions()
    for n in ("igp_graph_build", "igp_embed", "igp_graph_export", "igp_degree_factors", "igp_generate_x",
              "igp_last_error", "igp_graph_free"):
        assert n in names


def test_every_declared_symbol_is_exported(libigp):
    for n in _declared_functions():
        assert hasattr(libigp, n), f"{n} declared in include/ but not exported"


def test_binding_covers_the_header():
    from paper_2508_19737_gb300 import api
    assert sorted(api.exported_symbols()) == sorted(_declared_functions())


def test_host_only_calls(libigp):
    from paper_2508_19737_gb300 import api
    assert api.version().startswith("igp-gb300")
    o = api.embed_opts()
    assert (o.alpha, o.theta, o.eps, o.znorm_ddof, o.storage, o.out_row_l2) == (1.0, 0.1, 1e-3, 1, 0, 0)
    # argument checks happen before any CUDA call
    h = ctypes.c_void_p()
    st = libigp.igp_graph_build(None, None, 5, 0, None, ctypes.byref(h))
    assert st == api.IGP_E_INVAL and h.value is None
    assert b"N" in libigp.igp_last_error()
    assert libigp.igp_embed(None, -0.5, 10, 32, 0, None, None, None) == api.IGP_E_INVAL


def test_product_path_does_not_import_the_oracle():
    pkg = os.path.join(ROOT, "paper_2508_19737_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h", ".cpp")):
                text = open(os.path.join(dirpath, f)).read()
                assert not re.search(r"^\s*(import|from)\s+oracle", text, flags=re.M), f


def test_missing_library_fails_loudly(monkeypatch, tmp_path):
    """Without the built library every call raises: there is no CPU or PyTorch fallback."""
    import numpy as np
    from paper_2508_19737_gb300 import api
    monkeypatch.setattr(api, "LIB_PATH", str(tmp_path / "libigp.so"))
    monkeypatch.setattr(api, "_lib", None)
    with pytest.raises(RuntimeError, match="missing"):
        api.lib()
    with pytest.raises(RuntimeError, match="missing"):
        api.graph_build(np.zeros(1, np.int32), np.zeros(1, np.int32), 2)
    with pytest.raises(RuntimeError, match="missing"):
        api.embed_opts()
