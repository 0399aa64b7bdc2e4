"""The ctypes mirrors of the C-ABI structs in the Python binding have the layout the C compiler
gives the declarations of include/igp.h: the same size and the same offset for every field. A
field added on one side only would otherwise shift every later field silently."""
import ctypes
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

STRUCTS = {"igp_embed_opts": "EmbedOpts", "igp_server_opts": "ServerOpts", "igp_request": "Request",
           "igp_server_stats": "ServerStats"}


def _c_layout(tmp_path):
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no host C compiler")
    from paper_2508_19737_gb300 import api
    lines = ["#include <stddef.h>", "#include <stdio.h>", '#include "igp.h"', "int main(void) {"]
    for cname, pyname in STRUCTS.items():
        lines.append(f'  printf("{cname} sizeof %zu\\n", sizeof({cname}));')
        for f, _ in getattr(api, pyname)._fields_:
            lines.append(f'  printf("{cname} {f} %zu\\n", offsetof({cname}, {f}));')
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run([cc, "-std=c99", "-Wall", "-Werror", "-I", os.path.join(ROOT, "include"), str(src), "-o",
                    str(exe)], check=True, capture_output=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout
    layout = {}
    for ln in out.splitlines():
        s, f, v = ln.split()
        layout[(s, f)] = int(v)
    return layout


def test_ctypes_structs_match_the_c_header(tmp_path):
    from paper_2508_19737_gb300 import api
    layout = _c_layout(tmp_path)
    for cname, pyname in STRUCTS.items():
        py = getattr(api, pyname)
        assert ctypes.sizeof(py) == layout[(cname, "sizeof")], cname
        for f, _ in py._fields_:
            assert getattr(py, f).offset == layout[(cname, f)], (cname, f)


def test_embed_opts_defaults_and_host_async():
    """igp_embed_opts_init (host code, no GPU needed) leaves host_async at 0: a host output is
    final when igp_embed returns unless the caller asks otherwise; the binding sets it on request."""
    from paper_2508_19737_gb300 import api
    assert api.embed_opts().host_async == 0
    o = api.embed_opts(host_async=True, storage="bf16")
    assert o.host_async == 1 and o.storage == api.STORAGE["bf16"] and o.alpha == 1.0 and o.theta == 0.1
