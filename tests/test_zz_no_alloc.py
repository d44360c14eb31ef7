"""The allocation-free entry point grmhd_rhs_eval_static against the context path.

grmhd_rhs_eval_static exists for callers that must not have the library call
cudaMalloc (device memory owned by their own pool allocator, code paths that
cannot afford the synchronisation an allocation may imply, hosts that only allow
their own allocator).  It keeps its working memory in a static device array.
This test calls it through the C ABI twice in a row, on two different patches,
and checks each result against grmhd_con2prim + grmhd_rhs_eval on a context:
right-hand side within the 1e-11 normwise tolerance of the parity tests,
primitives within 1e-10, status codes equal.  It also checks that a patch
larger than the static array is rejected before any work is enqueued.
The file is named to be collected last.
"""
import ctypes

import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import __graft_entry__  # noqa: E402

__graft_entry__.build()
import paper_2510_13965_gb300 as g  # noqa: E402

NF, NP = 32, 10


def _err(got, want):
    gg = got.reshape(got.shape[0], -1)
    ww = want.reshape(want.shape[0], -1)
    return np.abs(gg - ww).max(axis=1) / np.maximum(np.abs(ww).max(axis=1), 1e-30)


def _context_result(P, n, dx, U0):
    """Reference: the context entry points on a copy of the state."""
    pt = g.Patches(P, [dict(n=n, dx=dx)])
    pt.U[0][0].copy_(U0)
    torch.cuda.synchronize()
    pt.con2prim(0)
    rhs = pt.rhs_eval(0)[0]
    pt.synchronize()
    return rhs.cpu().numpy(), pt.prim[0].cpu().numpy(), pt.status[0].cpu().numpy(), pt.U[0][0].cpu().numpy()


def _static_call(P, n, dx, U0):
    """The allocation-free entry point; every buffer here belongs to the caller."""
    U = U0.clone()
    shp = tuple(U.shape[1:])
    prim = torch.zeros((NP,) + shp, dtype=torch.float64, device="cuda")
    status = torch.zeros(shp, dtype=torch.int8, device="cuda")
    rhs = torch.zeros_like(U)
    d = g.PatchDesc()
    d.n[:] = list(n)
    d.px = shp[2]
    d.dx = dx
    d.U[0] = U.data_ptr()
    d.prim = prim.data_ptr()
    d.status = status.data_ptr()
    params = g.make_params(P)
    stream = torch.cuda.current_stream()
    torch.cuda.synchronize()
    rc = g.load().grmhd_rhs_eval_static(ctypes.byref(params), ctypes.byref(d), None, 0,
                                        ctypes.c_void_p(rhs.data_ptr()), ctypes.c_void_p(stream.cuda_stream))
    assert rc == 0, rc
    torch.cuda.synchronize()
    return rhs.cpu().numpy(), prim.cpu().numpy(), status.cpu().numpy(), U.cpu().numpy()


def _state(P, n, dx, ID):
    pt = g.Patches(P, [dict(n=n, dx=dx)])
    pt.init_state(0, torch.as_tensor(ID, device="cuda"))
    pt.synchronize()
    return pt.U[0][0].clone()


def test_static_scratch_entry_point_matches_context_path_twice():
    cases = [
        (synth.ideal_params(bc=0), (16, 16, 16), 1 / 16, synth.config0_id(n=(16, 16, 16), seed=7)),
        (synth.ideal_params(bc=1), (20, 14, 17), 0.5,
         synth.tov_id(n=(20, 14, 17), x0=(-4.0, -3.0, 2.0), dx=0.5, seed=1)),
    ]
    for P, n, dx, ID in cases:
        U0 = _state(P, n, dx, ID)
        r_ref, p_ref, s_ref, u_ref = _context_result(P, n, dx, U0)
        r, p, s, u = _static_call(P, n, dx, U0)
        sl = (slice(None), slice(3, 3 + n[2]), slice(3, 3 + n[1]), slice(3, 3 + n[0]))
        assert np.all(_err(r[sl], r_ref[sl]) < 1e-11)
        assert np.array_equal(s, s_ref)
        ok = s_ref == 0
        assert np.all(np.abs(p[0][ok] - p_ref[0][ok]) <= 1e-10 * p_ref[0][ok])
        assert np.all(np.abs(p[1][ok] - p_ref[1][ok]) <= 1e-10 * np.abs(p_ref[1][ok]) + 1e-300)
        assert np.all(_err(u[22:], u_ref[22:]) < 1e-13)


def test_static_entry_point_rejects_patches_above_its_maximum():
    P = synth.ideal_params()
    big = torch.zeros((NF, 46, 46, 46), dtype=torch.float64, device="cuda")
    d = g.PatchDesc()
    d.n[:] = [40, 40, 40]
    d.px = 46
    d.dx = 0.1
    d.U[0] = big.data_ptr()
    d.prim = big.data_ptr()
    d.status = big.data_ptr()
    rc = g.load().grmhd_rhs_eval_static(ctypes.byref(g.make_params(P)), ctypes.byref(d), None, 0,
                                        ctypes.c_void_p(big.data_ptr()), None)
    assert rc == -7  # GRMHD_ERR_SIZE
