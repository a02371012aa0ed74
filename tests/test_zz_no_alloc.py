"""The allocation-free entry point, hj_solve_fixed_static.

Some callers cannot allocate device memory once they are running.  One
example is a safety filter in a real-time control loop: cudaMalloc/cudaFree
can stall the whole device.  Another is a process whose device memory is
owned by another framework's pool.  For them the library keeps its scratch
in a static device array.  These tests check that the entry point gives the
same result as the allocating path (hj_grid_create + hj_solve with fixed
steps), over two calls in a row, and that repeated calls leave the device's
free memory unchanged.  This file is named so that pytest collects it last.
"""
import numpy as np
import pytest

from paper_2101_05916_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

REL = 1e-4  # the parity tolerance used by the other GPU tests


@pytest.fixture(scope="module")
def hj():
    import torch
    assert torch.cuda.is_available()
    from paper_2101_05916_gb300 import build, hj as hjmod
    build.build()
    hjmod.lib()
    return hjmod


def reference(hj, spec, scheme, steps, mode, prior=None):
    g = hj.Grid.from_spec(spec)
    if prior is not None:
        g.set_value(prior)
    st = g.solve(mode, scheme=scheme, fixed_steps=steps)
    out = g.value()
    g.close()
    return out, st


def static_call(hj, spec, scheme, steps, mode, prior=None):
    import torch
    if prior is not None:
        W = torch.from_numpy(prior.reshape(-1).copy()).cuda()
    else:
        W = torch.full((spec.npts,), 123.0, device="cuda", dtype=torch.float32)
    hj.hj_solve_fixed_static(spec, W, mode=mode, scheme=scheme, steps=steps)
    torch.cuda.synchronize()
    return W.cpu().numpy().reshape(spec.n)


def close(a, b):
    return np.abs(a.astype(np.float64) - b).max() <= REL * np.abs(b).max()


def test_static_entry_matches_allocating_path_two_calls_in_a_row(hj):
    cases = [(wl.quad_x4(21, 0.5), 5, 12, hj.HJ_COLD),
             (wl.quad_z(101, 0.7), 2, 40, hj.HJ_COLD)]
    for spec, scheme, steps, mode in cases:
        ref, _ = reference(hj, spec, scheme, steps, mode)
        got = static_call(hj, spec, scheme, steps, mode)
        assert close(got, ref), spec.name
    # a warm call right after, on a different grid: stale scratch must not leak in
    spec = wl.quad_x4(17, 0.3, 3.5, "y")
    prior = (wl.seeded_field(spec, 3, 0.1) + 2.0).astype(np.float32)
    ref, _ = reference(hj, spec, 5, 9, hj.HJ_WARM, prior)
    got = static_call(hj, spec, 5, 9, hj.HJ_WARM, prior)
    assert close(got, ref)


def test_static_entry_allocates_nothing_on_repeat_calls(hj):
    import torch
    spec = wl.quad_z(61, 0.5)
    W = torch.zeros(spec.npts, device="cuda", dtype=torch.float32)
    hj.hj_solve_fixed_static(spec, W, scheme=2, steps=3)  # first call: address set-up
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for _ in range(2):
        hj.hj_solve_fixed_static(spec, W, scheme=2, steps=3)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0


def test_static_entry_rejects_oversized_grids(hj):
    spec = wl.quad_x4(46, 0.5)  # 46^4 = 4,477,456 nodes > 4,194,304
    import torch
    W = torch.zeros(1, device="cuda", dtype=torch.float32)
    with pytest.raises(ValueError):
        hj.hj_solve_fixed_static(spec, W, steps=1)  # binding checks the tensor size
    L = hj.lib()
    import ctypes
    n = (ctypes.c_int * 4)(46, 46, 46, 46)
    rc = L.hj_solve_fixed_static(4, n, hj._darr(spec.lo), hj._darr(spec.hi), hj.HJ_QUAD_X4,
                                 hj._darr(spec.params), 7, hj._darr(spec.d_lo),
                                 hj._darr(spec.d_hi), 1, hj._darr(spec.con_a),
                                 hj._darr(spec.con_b), 0, 5, 0.0, 1, 0, W.data_ptr(), None)
    assert rc == hj.HJ_ERR_ARG
    assert "allocation-free limit" in hj.hj_last_error()


def raw_call(hj, spec, ptr, dt=0.0, steps=1, scheme=2):
    import ctypes
    n = (ctypes.c_int * spec.ndim)(*[int(v) for v in spec.n])
    return hj.lib().hj_solve_fixed_static(
        spec.ndim, n, hj._darr(spec.lo), hj._darr(spec.hi), hj.MODELS[spec.model],
        hj._darr(spec.params), len(spec.params), hj._darr(spec.d_lo), hj._darr(spec.d_hi),
        len(spec.d_lo), hj._darr(spec.con_a), hj._darr(spec.con_b), hj.HJ_COLD, scheme,
        float(dt), int(steps), hj.HJ_CLAMP_VI, ptr, None)


def test_static_entry_rejects_host_memory_before_any_launch(hj):
    """A C caller that hands over a host pointer gets HJ_ERR_ARG, and no kernel
    runs on that memory."""
    spec = wl.quad_z(21, 0.5)
    host = np.zeros(spec.npts, dtype=np.float32)
    launches = hj.hj_kernel_launches()
    rc = raw_call(hj, spec, host.ctypes.data)
    assert rc == hj.HJ_ERR_ARG
    assert "device memory" in hj.hj_last_error() or "CUDA pointer" in hj.hj_last_error()
    assert hj.hj_kernel_launches() == launches
    assert np.all(host == 0.0)


def test_static_entry_dt_zero_is_cfl_and_negative_dt_is_rejected(hj):
    import torch
    spec = wl.quad_z(41, 0.5)
    W = torch.zeros(spec.npts, device="cuda", dtype=torch.float32)
    launches = hj.hj_kernel_launches()
    assert raw_call(hj, spec, W.data_ptr(), dt=-1e-3) == hj.HJ_ERR_ARG
    assert raw_call(hj, spec, W.data_ptr(), dt=float("nan")) == hj.HJ_ERR_ARG
    assert hj.hj_kernel_launches() == launches
    # dt == 0: the CFL step, the same as the allocating path's default dt
    assert raw_call(hj, spec, W.data_ptr(), dt=0.0, steps=7) == hj.HJ_OK
    torch.cuda.synchronize()
    ref, st = reference(hj, spec, 2, 7, hj.HJ_COLD)
    assert st["dt"] > 0.0
    assert close(W.cpu().numpy().reshape(spec.n), ref)
