"""The C ABI without a GPU: the library loads, exports every symbol that
include/tabnet.h declares, and validates blobs on the host (tabnet_create's
loading step, Sec. III-B cold start) with the documented error codes."""
import ctypes
import os
import re
import struct

import numpy as np
import pytest

from paper_2510_19689_b300 import synth, tabnet

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "tabnet.h")).read()
    return sorted(set(re.findall(r"\b(tabnet_[a-z_0-9]+)\s*\(", src)))


def test_library_exports_every_declared_symbol():
    L = tabnet.lib()
    declared = _declared()
    assert declared, "no declarations found"
    for name in declared:
        assert hasattr(L, name), name
    assert set(declared) == set(tabnet.EXPORTS)
    assert L.tabnet_abi_version() == 1


def test_blob_inspect_reads_shape():
    for name in ("c1", "c2", "c3"):
        spec = synth.SPECS[name]
        blob = synth.to_blob(synth.make_params(spec, 1))
        d = tabnet.blob_inspect(blob)
        assert (d.n_num, d.n_cat, d.d_emb, d.n_feat) == (spec.n_num, spec.n_cat, spec.d_emb, spec.n_feat)
        assert (d.n_d, d.n_a, d.n_steps, d.n_classes) == (spec.n_d, spec.n_a, spec.n_steps, spec.n_classes)
        assert abs(d.gamma - spec.gamma) < 1e-12


@pytest.fixture(scope="module")
def blob():
    return synth.to_blob(synth.make_params(synth.SPECS["c1"], 3))


def _code(b):
    try:
        tabnet.blob_inspect(b)
        return 0
    except tabnet.TabnetError as e:
        return e.code


def test_blob_errors(blob):
    assert _code(blob) == 0
    assert _code(b"XXXX" + blob[4:]) == -2                     # magic
    assert _code(blob[:4] + struct.pack("<I", 7) + blob[8:]) == -3   # version
    assert _code(blob[:-4]) == -4                              # truncated
    assert _code(blob + b"\0\0\0\0") == -4                     # trailing bytes
    bad = bytearray(blob)
    bad[200] ^= 0x40
    assert _code(bytes(bad)) == -5                             # hash
    dims = bytearray(blob)
    struct.pack_into("<i", dims, 32 + 4 * 4, 0)                # n_steps = 0
    assert _code(bytes(dims)) == -6
    assert _code(blob[:10]) == -4


def test_create_without_gpu_fails_cleanly(blob):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(tabnet.TabnetError) as e:
        tabnet.Model(blob, "bf16")
    assert e.value.code == -7
    # argument errors come before any device work
    h = ctypes.c_void_p()
    assert tabnet.lib().tabnet_create(None, 0, 1, 0, ctypes.byref(h)) == -1
    assert tabnet.lib().tabnet_forward(None, None, None, 1, None, None, None, None) == -1
    assert tabnet.lib().tabnet_status_string(-6) == b"model shape not supported"


# The binding's ctypes mirrors of the header's structs, field by field: the
# same names in the same order, each the size the C type has, so that a
# field added to one side only (the server's config and statistics grow)
# fails here rather than shifting every later field on the GPU machine.
_STRUCTS = {"tabnet_dims": "Dims", "tabnet_segment": "Segment", "tabnet_server_config": "ServerConfig",
            "tabnet_server_stats": "ServerStats", "tabnet_server_request": "ServerRequest"}
_C_SIZES = {"int32_t": 4, "int": 4, "double": 8, "uint64_t": 8, "int64_t": 8, "size_t": 8}


def _header_structs():
    src = open(os.path.join(ROOT, "include", "tabnet.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    src = re.sub(r"//[^\n]*", "", src)
    out = {}
    for body, name in re.findall(r"typedef struct \{(.*?)\}\s*(\w+)\s*;", src, flags=re.S):
        fields = []
        for decl in body.split(";"):
            decl = " ".join(decl.split())
            if not decl:
                continue
            decl = decl.replace("const ", "")
            m = re.match(r"(\w+)\s*(\**)\s*(.*)", decl)
            ctype, stars, names = m.group(1), m.group(2), m.group(3)
            for nm in names.split(","):
                nm = nm.strip()
                ptr = bool(stars) or nm.startswith("*")
                nm = nm.lstrip("*").strip()
                fields.append((nm, 8 if ptr else _C_SIZES[ctype]))
        out[name] = fields
    return out


def test_ctypes_structs_match_the_header():
    structs = _header_structs()
    for cname, pyname in _STRUCTS.items():
        assert cname in structs, cname
        want = structs[cname]
        py = getattr(tabnet, pyname)
        got = [(f[0], ctypes.sizeof(f[1])) for f in py._fields_]
        assert got == want, (cname, got, want)
        # natural alignment: the C struct's size
        off = 0
        for _, sz in want:
            off = (off + sz - 1) // sz * sz + sz
        align = max(sz for _, sz in want)
        assert ctypes.sizeof(py) == (off + align - 1) // align * align, cname
