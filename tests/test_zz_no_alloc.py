"""The allocation-free operator entry point, for callers that cannot call
cudaMalloc (code inside a pre-reserved memory pool, allocators that forbid
device allocation): on consecutive calls that reuse its fixed device scratch
array, its FP32 result must match dw_apply's FP32 result and the FP64 oracle's
D, and a call after the first must leave the device's free memory unchanged.
(Collected last on purpose: it shares one device array across calls.)"""

import numpy as np
import pytest

import fieldgen as fg
import oracle

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

TOL_F32 = 1e-5  # relative max-norm tolerance of the FP32 operator tests


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.complex128).view(np.float64).reshape(-1).copy()).cuda()


def _host(t, shape):
    return t.cpu().numpy().view(np.complex128).reshape(shape)


def test_noalloc_matches_dw_apply_and_oracle_on_two_calls():
    import paper_1204_5463_gb300 as dw

    dims = (4, 4, 6, 8)  # 768 sites: several thread blocks and a ragged tail
    m0 = -0.3
    U = fg.gauge_field(dims, 0.5, seed=31)
    Ud = _dev(U)
    stream = torch.cuda.current_stream().cuda_stream
    ctx = dw.dw_create(dims, (2, 2, 3, 4), m0, stream)
    try:
        dw.dw_set_gauge(ctx, Ud, True)
        for seed in (41, 42):  # two calls in a row through the same scratch
            psi = fg.gaussian_source(dims, seed)
            pin = _dev(psi)
            ref = torch.empty_like(pin)
            got = torch.empty_like(pin)
            dw.dw_apply(ctx, pin, ref, dw.DW_F32, 1)
            dw.dw_apply_f32_noalloc(dims, m0, Ud, pin, got, stream)
            a, b = _host(got, psi.shape), _host(ref, psi.shape)
            assert np.abs(a - b).max() <= TOL_F32 * np.abs(b).max()
            exact = oracle.dw(U, psi, dims, m0)
            assert np.abs(a - exact).max() <= TOL_F32 * np.abs(exact).max()
    finally:
        dw.dw_destroy(ctx)


def test_noalloc_call_leaves_free_device_memory_unchanged():
    import paper_1204_5463_gb300 as dw

    dims = (4, 4, 4, 8)
    m0 = 0.1
    U = fg.gauge_field(dims, 0.4, seed=5)
    psi = fg.gaussian_source(dims, 6)
    Ud, pin = _dev(U), _dev(psi)
    out = torch.empty_like(pin)
    stream = torch.cuda.current_stream().cuda_stream
    dw.dw_apply_f32_noalloc(dims, m0, Ud, pin, out, stream)  # set-up call on this device
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    for _ in range(3):
        dw.dw_apply_f32_noalloc(dims, m0, Ud, pin, out, stream)
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0
    exact = oracle.dw(U, psi, dims, m0)
    assert np.abs(_host(out, psi.shape) - exact).max() <= TOL_F32 * np.abs(exact).max()


def test_noalloc_rejects_lattices_beyond_its_scratch():
    import paper_1204_5463_gb300 as dw

    dims = (8, 8, 8, 16)  # 8192 sites > 4096
    x = torch.zeros(8, dtype=torch.float64, device="cuda")
    with pytest.raises(dw.DwError) as e:
        dw.dw_apply_f32_noalloc(dims, 0.0, x, x, x)
    assert e.value.code == dw.DW_EINVAL
