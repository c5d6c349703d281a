"""The allocation-free operator entry point, for callers that cannot call
cudaMalloc: its FP32 result must match dw_apply's FP32 result on the same
inputs, on consecutive calls that reuse its fixed device scratch array.
(Collected last on purpose: it shares one device array across calls.)"""

import numpy as np
import pytest

import fieldgen as fg

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

TOL_F32 = 1e-5  # relative max-norm tolerance of the FP32 operator tests


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.complex128).view(np.float64).reshape(-1).copy()).cuda()


def _host(t, shape):
    return t.cpu().numpy().view(np.complex128).reshape(shape)


def test_noalloc_matches_dw_apply_on_two_calls():
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
    finally:
        dw.dw_destroy(ctx)


def test_noalloc_rejects_lattices_beyond_its_scratch():
    import paper_1204_5463_gb300 as dw

    dims = (8, 8, 8, 16)  # 8192 sites > 4096
    x = torch.zeros(8, dtype=torch.float64, device="cuda")
    with pytest.raises(dw.DwError) as e:
        dw.dw_apply_f32_noalloc(dims, 0.0, x, x, x)
    assert e.value.code == dw.DW_EINVAL
