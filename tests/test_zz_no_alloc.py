"""The allocation-free entry point grmhd_rhs_eval_static.

grmhd_rhs_eval_static exists for callers that must not have the library call
cudaMalloc (device memory owned by their own pool allocator, code paths that
cannot afford the synchronisation an allocation may imply, hosts that only allow
their own allocator).  It keeps its working memory in a static device array.
This test calls it through the C ABI twice in a row, on two different patches,
and checks each result

* against grmhd_con2prim + grmhd_rhs_eval on a context (right-hand side within
  the 1e-11 normwise tolerance of the parity tests, primitives within 1e-10,
  status codes equal), and
* against the CPU oracle on the same input state (all ten primitives with the
  primitive tolerances of the parity tests, the right-hand side within 1e-11
  normwise per field, status codes equal),

that its device error flags are clear, and that the second call changes neither
torch's allocated bytes nor the device's free memory.  It also checks that a
patch larger than the static array is rejected before any work is enqueued.
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
import oracle  # noqa: E402
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


def _static_call(P, n, dx, U0, check_no_alloc=False):
    """The allocation-free entry point; every buffer here belongs to the caller."""
    U = U0.clone()
    shp = tuple(U.shape[1:])
    prim = torch.zeros((NP,) + shp, dtype=torch.float64, device="cuda")
    status = torch.zeros(shp, dtype=torch.int8, device="cuda")
    rhs = torch.zeros_like(U)
    flags = torch.full((1,), -1, dtype=torch.int32, device="cuda")
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
    before = (torch.cuda.memory_allocated(), torch.cuda.mem_get_info()[0])
    rc = g.load().grmhd_rhs_eval_static(ctypes.byref(params), ctypes.byref(d), None, 0,
                                        ctypes.c_void_p(rhs.data_ptr()), ctypes.c_void_p(flags.data_ptr()),
                                        ctypes.c_void_p(stream.cuda_stream))
    assert rc == 0, rc
    torch.cuda.synchronize()
    after = (torch.cuda.memory_allocated(), torch.cuda.mem_get_info()[0])
    if check_no_alloc:
        assert after == before, (before, after)
    assert int(flags.item()) == 0
    return rhs.cpu().numpy(), prim.cpu().numpy(), status.cpu().numpy(), U.cpu().numpy()


def _state(P, n, dx, ID):
    pt = g.Patches(P, [dict(n=n, dx=dx)])
    pt.init_state(0, torch.as_tensor(ID, device="cuda"))
    pt.synchronize()
    return pt.U[0][0].clone()


def _check_prims(p, p_ref, ok):
    """Primitive tolerances of the parity tests: rho, Ye relative 1e-10; W v^i
    absolute 1e-10; eps, p scaled by max(1, (1 + |q|) / |eps|) (q = tau / D)."""
    for f in (0, 7):
        assert np.all(np.abs(p[f][ok] - p_ref[f][ok]) <= 1e-10 * np.abs(p_ref[f][ok]) + 1e-300), f
    for a in range(3):
        wv, wv_ref = p[6] * p[3 + a], p_ref[6] * p_ref[3 + a]
        assert np.all(np.abs(wv[ok] - wv_ref[ok]) <= 1e-10), a
    assert np.all(np.abs(p[6][ok] - p_ref[6][ok]) <= 1e-10 * p_ref[6][ok])
    for f in (1, 2, 9):
        assert np.all(np.abs(p[f][ok] - p_ref[f][ok]) <= 1e-10 * (np.abs(p_ref[f][ok]) + 1e-12)), f


def test_static_scratch_entry_point_matches_context_path_and_oracle_twice():
    cases = [
        (synth.ideal_params(bc=0), (16, 16, 16), 1 / 16, synth.config0_id(n=(16, 16, 16), seed=7)),
        (synth.ideal_params(bc=1), (20, 14, 17), 0.5,
         synth.tov_id(n=(20, 14, 17), x0=(-4.0, -3.0, 2.0), dx=0.5, seed=1)),
    ]
    for call, (P, n, dx, ID) in enumerate(cases):
        U0 = _state(P, n, dx, ID)
        r_ref, p_ref, s_ref, u_ref = _context_result(P, n, dx, U0)
        r, p, s, u = _static_call(P, n, dx, U0, check_no_alloc=call > 0)
        sl = (slice(None), slice(3, 3 + n[2]), slice(3, 3 + n[1]), slice(3, 3 + n[0]))
        assert np.all(_err(r[sl], r_ref[sl]) < 1e-11)
        assert np.array_equal(s, s_ref)
        ok = s_ref == 0
        _check_prims(p, p_ref, ok)
        assert np.all(_err(u[22:], u_ref[22:]) < 1e-13)

        # The oracle on the same input state.
        O = oracle.Oracle(P)
        Uo = np.ascontiguousarray(U0.cpu().numpy())
        prim_o, st_o, _, _ = O.con2prim_patch(Uo, n)
        rhs_o = O.rhs_patch(Uo, prim_o, n, dx)
        assert np.array_equal(s, st_o)
        _check_prims(p, prim_o, st_o == 0)
        scale = np.maximum(np.abs(rhs_o[sl]).reshape(NF, -1).max(axis=1), 1e-300)
        err = np.abs(r[sl] - rhs_o[sl]).reshape(NF, -1).max(axis=1)
        # fields whose right-hand side vanishes analytically (the flat shift of
        # the static data) hold rounding only: 1e-14 absolute there
        assert np.all((err <= 1e-11 * scale) | (err <= 1e-14)), err / scale


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
                                        ctypes.c_void_p(big.data_ptr()), None, None)
    assert rc == -7  # GRMHD_ERR_SIZE
