"""GPU test of hz_residual_noalloc, the one entry point that allocates no device memory.

It serves callers that cannot call cudaMalloc: code that issues work while its stream is
being captured into a CUDA graph, allocators that own one fixed arena, hosts that control the
GPU memory budget.  Its scratch is a static device array shared by all calls, so the test makes
two calls in a row (the second reuses what the first left there) and checks both against the
existing entry points: the relative residual hz_solve reports for its solution, and the
residual field built from hz_apply_shifted.  Tolerances: 1e-12 on the norm, 1e-14 on the
field relative to ||s f|| (float64, as in the parity tests).  This file is collected last on purpose.
"""
import ctypes as C

import numpy as np
import pytest

import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1811_12378_gb300 as hzpkg  # noqa: E402
from paper_1811_12378_gb300.hz import HzGrid  # noqa: E402

DEV = "cuda:0"


def _ptr(t):
    return C.c_void_p(t.data_ptr()) if t is not None else None


def test_noalloc_residual_matches_existing_entry_points():
    lib = hzpkg.load()
    wl = W.small_case(3, 13, 9, 7, nrhs=2, layer=2, J=4)
    n = wl.n
    with hzpkg.Problem(wl.c, wl.h, wl.omega, wl.layer_cells, wl.sigma_max, wl.J, wl.t, wl.eps,
                       nrhs_max=2, restart_max=10, inner_k_max=3) as P:
        f = torch.from_numpy(wl.f.reshape(2, n).copy()).to(DEV)
        u, stats = P.solve(f, restart=10, inner_k=3, rtol=1e-8, max_cycles=20)
        s = P.info["s"]
        Au = P.apply_shifted(u)
        r_ref = (s * f - Au).cpu().numpy()
        sf_norm = float(torch.linalg.vector_norm(s * f))
    grid = HzGrid(wl.nx, wl.ny, wl.nz, wl.h, wl.omega, wl.layer_cells, wl.sigma_max)
    c_dev = torch.from_numpy(np.ascontiguousarray(wl.c)).to(DEV)
    c_min = float(wl.c.min())
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    for call in range(2):
        r = torch.full_like(f, float("nan"))
        norm2 = torch.full((2,), float("nan"), dtype=torch.float64, device=DEV)
        norm2_f = torch.full((2,), float("nan"), dtype=torch.float64, device=DEV)
        st = lib.hz_residual_noalloc(C.byref(grid), _ptr(c_dev), c_min, _ptr(f), s, _ptr(u),
                                     _ptr(r), _ptr(norm2), 2, stream)
        assert st == 0, lib.hz_last_error()
        st = lib.hz_residual_noalloc(C.byref(grid), _ptr(c_dev), c_min, _ptr(f), s, None, None,
                                     _ptr(norm2_f), 2, stream)
        assert st == 0, lib.hz_last_error()
        torch.cuda.synchronize()
        rel = torch.sqrt(norm2 / norm2_f).cpu().numpy()
        for v in range(2):
            assert rel[v] == pytest.approx(stats[v].rel_res_true, rel=1e-12), (call, v)
        # r = s f - A u is a cancellation (relative residual ~1e-8): compare it to the
        # existing entry point's s f - A u on the scale of the operands
        rn = r.cpu().numpy()
        assert np.linalg.norm(rn - r_ref) <= 1e-14 * sf_norm


def test_noalloc_rejects_sizes_beyond_its_scratch():
    lib = hzpkg.load()
    grid = HzGrid(256, 256, 256, 1.0 / 257, 200.0, 8, 1.0)
    dummy = torch.zeros(1, dtype=torch.float64, device=DEV)
    # 256^3 has 16384 blocks of 1024 points: 5 fields need 81920 > 65536 partials
    st = lib.hz_residual_noalloc(C.byref(grid), _ptr(dummy), 1.0, _ptr(dummy), 1.0, None, None,
                                 _ptr(dummy), 5, None)
    assert st == 1 and b"65536" in lib.hz_last_error()
    st = lib.hz_residual_noalloc(C.byref(grid), _ptr(dummy), 1.0, _ptr(dummy), 1.0, None, None,
                                 _ptr(dummy), 65, None)
    assert st == 1
