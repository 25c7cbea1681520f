"""The C-ABI library builds for sm_103a, loads, and exports every entry point include/orrb.h declares.

No compute calls here: this runs without a GPU.  The host-only entry points
(status strings, the mesh arena size of the clustering pass) are exercised.
"""

import ctypes as C
import os
import re

import numpy as np
import pytest

from paper_1906_11633_b300 import build, lib
from paper_1906_11633_b300 import scenegen as sg

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def so():
    build.build()
    return lib.load()


def declared_symbols():
    text = open(os.path.join(ROOT, "include", "orrb.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(orrb_[a-z_0-9]+)\s*\(", text)))


def test_every_declared_symbol_is_exported(so):
    names = declared_symbols()
    assert len(names) >= 12
    for n in names:
        assert hasattr(so, n), n
    assert set(names) == set(lib.EXPORTS)


def test_status_strings(so):
    for s in range(8):
        assert so.orrb_status_string(s)
    assert so.orrb_status_string(0) == b"ok"


def test_create_without_device_fails_cleanly(so):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    ctx = C.c_void_p()
    assert so.orrb_create(0, C.byref(ctx)) != 0


def test_mesh_arena_size_and_validation(so):
    meshes = sg.hand_meshes()
    from paper_1906_11633_b300.render import _mesh_descs
    descs, keep = _mesh_descs(meshes)
    n = lib.orrb_mesh_arena_size(descs)
    tris = sum(m.n_tris for m in meshes)
    assert n >= tris * 4 + sum(m.n_verts for m in meshes) * 32
    bad = sg.Mesh(meshes[0].pos, meshes[0].nrm, meshes[0].idx.copy(), meshes[0].tri_mat)
    bad.idx[0, 0] = 99
    d2, k2 = _mesh_descs([bad])
    with pytest.raises(lib.OrrbError):
        lib.orrb_mesh_arena_size(d2)
