"""The C-ABI library builds for sm_103a, loads and exports every symbol the
header declares; host-side validation errors need no GPU."""
import ctypes
import os
import re

import numpy as np
import pytest

from paper_2603_28475_b300 import scenes as S

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _header_symbols():
    src = open(os.path.join(ROOT, "include", "tac.h")).read()
    return sorted(set(re.findall(r"^\s*(?:int|const char\*)\s+(tac_\w+)\s*\(", src, flags=re.M)))


@pytest.fixture(scope="module")
def lib():
    from paper_2603_28475_b300 import build
    build.build()
    from paper_2603_28475_b300 import tac
    return tac.load_library()


def test_header_declares_the_boundary():
    syms = _header_symbols()
    for s in ("tac_create_batch", "tac_destroy_batch", "tac_set_indenter", "tac_step", "tac_markers",
              "tac_get_state", "tac_set_state", "tac_set_params", "tac_broadphase", "tac_last_error"):
        assert s in syms


def test_library_exports_every_declared_symbol(lib):
    for s in _header_symbols():
        assert hasattr(lib, s), s


def test_binding_covers_every_symbol():
    from paper_2603_28475_b300 import tac
    assert sorted(tac.SYMBOLS) == _header_symbols()


def test_library_is_built_for_sm_103a(lib):
    from paper_2603_28475_b300 import build
    assert "compute_103a,code=sm_103a" in build.ARCH


def _create(lib, pad, ind):
    from paper_2603_28475_b300 import tac
    pd = tac.PadDesc(pad.rest.shape[0], pad.tets.shape[0], pad.fixed.shape[0], pad.markers.shape[0],
                     pad.rest.ctypes.data, pad.tets.ctypes.data, pad.fixed.ctypes.data, pad.markers.ctypes.data)
    idesc = tac.IndenterDesc(ind.verts.shape[0], ind.tris.shape[0], ind.verts.ctypes.data, ind.tris.ctypes.data)
    prm = tac.make_params(S.Material())
    h = ctypes.c_void_p()
    rc = lib.tac_create_batch(ctypes.byref(pd), ctypes.byref(prm), 1, ctypes.byref(idesc), 1, 1, None, None,
                              ctypes.byref(h))
    return rc, lib.tac_last_error().decode()


def test_inverted_tet_is_rejected_before_any_device_work(lib):
    pad = S.hex_pad((4e-3, 4e-3, 2e-3), (2, 2, 1))
    pad.tets = pad.tets.copy()
    pad.tets[3, [2, 3]] = pad.tets[3, [3, 2]]
    ind = S.icosphere(1e-3, 0)
    rc, msg = _create(lib, pad, ind)
    assert rc == -2 and "tet 3" in msg


def test_out_of_range_index_is_rejected(lib):
    pad = S.hex_pad((4e-3, 4e-3, 2e-3), (2, 2, 1))
    pad.tets = pad.tets.copy()
    pad.tets[0, 0] = 10 ** 6
    rc, msg = _create(lib, pad, S.icosphere(1e-3, 0))
    assert rc == -2 and "out of range" in msg


def test_marker_off_the_top_face_is_rejected(lib):
    pad = S.hex_pad((4e-3, 4e-3, 2e-3), (2, 2, 1))
    pad.markers = np.array([[5e-3, 1e-3]], dtype=np.float32)
    rc, msg = _create(lib, pad, S.icosphere(1e-3, 0))
    assert rc == -2 and "marker 0" in msg


def test_null_arguments_are_rejected(lib):
    assert lib.tac_step(None, None, None, None) == -1
    assert lib.tac_markers(None, None, None) == -1
    h = ctypes.c_void_p()
    assert lib.tac_create_batch(None, None, 0, None, 0, 0, None, None, ctypes.byref(h)) == -1
    assert lib.tac_set_block_shape(None, 256) == -1
    th = ctypes.c_int()
    assert lib.tac_autotune_block_shape(None, None, 1, ctypes.byref(th), None, None) == -1
