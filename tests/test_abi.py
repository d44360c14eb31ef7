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
    assert lib.grmhd_abi_version() == 2
    ctx = ctypes.c_void_p(1)
    # Host-side argument validation needs no GPU: NULL params are rejected before any CUDA call.
    assert lib.grmhd_init_patches(ctypes.byref(ctx), None, 1, None, None, None) == -1
    assert not ctx.value
    assert lib.grmhd_init_state(None, 0, None) == -1
    assert lib.grmhd_rhs_substep(None, 0, 0.1) == -1
    assert lib.grmhd_c2p_flat(None, None, 1, None, None, None, None, None) == -1
    assert lib.grmhd_set_subcycling(None, 1) == -1


def test_hybrid_eos_parameters_rejected_on_the_host(lib):
    """eos_kind 2 with an unusable piece list fails with GRMHD_ERR_ARG before any CUDA call."""
    import paper_2510_13965_gb300 as g
    import synth
    good = synth.hybrid_params()
    bad = [dict(npoly=0), dict(npoly=5), dict(K_poly=0.0), dict(gamma_poly=(2.0, 1.0, 3.0, 0.0)),
           dict(rho_poly=(9e-4, 4e-4, 0.0)), dict(rho_poly=(0.0, 9e-4, 0.0)), dict(eos_kind=3)]
    for b in bad:
        p = g.make_params({**good, **b})
        assert lib.grmhd_c2p_flat(ctypes.byref(p), None, 0, None, None, None, None, None) == -1, b
        assert lib.grmhd_prim2con_flat(ctypes.byref(p), None, 0, None, None, None, None) == -1, b


def test_struct_layouts_match_header(tmp_path):
    import shutil
    import subprocess
    import paper_2510_13965_gb300 as g
    assert ctypes.sizeof(g.Params) == 22 * 8 + 4 * 4 + 2 * 4 + 8 + 3 * 8 + 4 * 8 + 4 * 8 + 8
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    # Every field offset of the binding's Params equals the C header's.
    names = [f[0] for f in g.Params._fields_]
    src = tmp_path / "off.c"
    src.write_text("#include <stddef.h>\n#include <stdio.h>\n#include \"grmhd.h\"\nint main(void) {\n" +
                   "".join(f'  printf("%zu\\n", offsetof(grmhd_params, {n}));\n' for n in names) +
                   '  printf("%zu\\n", sizeof(grmhd_params));\n  return 0;\n}\n')
    exe = tmp_path / "off"
    inc = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include")
    subprocess.run([cc, "-I", inc, str(src), "-o", str(exe)], check=True)
    out = [int(x) for x in subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split()]
    assert out[:-1] == [getattr(g.Params, n).offset for n in names]
    assert out[-1] == ctypes.sizeof(g.Params)
    assert ctypes.sizeof(g.PatchDesc) == 6 * 4 + 4 * 8 + 6 * 8
    assert ctypes.sizeof(g.EosTable) == 4 * 4 + 6 * 8 + 3 * 8


def test_les_rejected_by_the_allocation_free_entry(lib):
    """grmhd_rhs_eval_static has no scratch for the LES point values: any LES
    coefficient is refused before a pointer is touched."""
    import paper_2510_13965_gb300 as g
    import synth
    p = g.make_params({**synth.ideal_params(bc=1), "les_c": (0.0, 0.0, 0.0, 8.0)})
    d = g.PatchDesc()
    assert lib.grmhd_rhs_eval_static(ctypes.byref(p), ctypes.byref(d), None, 0, ctypes.c_void_p(8), None,
                                     None) == -1
