"""The C-ABI library builds, loads and exports every function include/grmhd.h declares (no GPU needed)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    txt = open(os.path.join(ROOT, "include", "grmhd.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?(?:[a-z_0-9]+[\s*]+)+(grmhd_[a-z_0-9]+)\s*\(", txt, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__
    __graft_entry__.build()
    import paper_2510_13965_gb300 as g
    return g.load()


def test_header_declares_the_boundary():
    names = _declared()
    for n in ("grmhd_init_patches", "grmhd_rhs_substep", "grmhd_con2prim", "grmhd_rk_update"):
        assert n in names
    assert len(names) >= 15


def test_every_declared_symbol_is_exported(lib):
    for n in _declared():
        assert hasattr(lib, n), n


def test_binding_covers_the_header():
    import paper_2510_13965_gb300 as g
    assert sorted(g.exported_symbols()) == _declared()


def test_abi_version_and_argument_checks(lib):
    assert lib.grmhd_abi_version() == 1
    ctx = ctypes.c_void_p(1)
    # Host-side argument validation needs no GPU: NULL params are rejected before any CUDA call.
    assert lib.grmhd_init_patches(ctypes.byref(ctx), None, 1, None, None, None) == -1
    assert not ctx.value
    assert lib.grmhd_init_state(None, 0, None) == -1
    assert lib.grmhd_rhs_substep(None, 0, 0.1) == -1
    assert lib.grmhd_c2p_flat(None, None, 1, None, None, None, None, None) == -1


def test_struct_layouts_match_header():
    import paper_2510_13965_gb300 as g
    assert ctypes.sizeof(g.Params) == 22 * 8 + 4 * 4
    assert ctypes.sizeof(g.PatchDesc) == 6 * 4 + 4 * 8 + 6 * 8
    assert ctypes.sizeof(g.EosTable) == 4 * 4 + 6 * 8 + 3 * 8
