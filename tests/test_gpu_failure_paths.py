"""Failure paths that can be exercised without faulting or hanging a GPU: a host-side
deadline that runs out while a render is still on the stream, and a tensor-core kernel whose
bounded waits are given a tiny limit (a test hook), so that they give up, raise the device
flag and return.  In both cases the context stays usable and the next call succeeds."""
import numpy as np
import pytest

from paper_1601_02063_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def tracer():
    import torch
    from paper_1601_02063_gb300 import binding as B
    from paper_1601_02063_gb300 import build

    build.build()
    assert torch.cuda.is_available()
    tr = B.Tracer(0)
    yield tr
    tr.close()


def test_sync_deadline_runs_out_then_completes(tracer):
    """A 2048x2048 FP64 thin-disk render (about a second of GPU work) is still running when
    odx_sync is asked to wait 0 s: ODX_ERR_TIMEOUT, the work goes on; a second odx_sync with
    a generous deadline returns OK and every ray has a final status."""
    import torch
    from paper_1601_02063_gb300 import binding as B

    sc = W.scene(n_alpha=2048, n_beta=2048, precision="fp64")
    stream = torch.cuda.Stream()
    torch.cuda.synchronize()
    rec, _ = tracer.render(sc, stream=stream)
    with pytest.raises(B.OdxError) as info:
        B.odx_sync(tracer.ctx, stream.cuda_stream, 0.0)
    assert info.value.code == B.ERR_TIMEOUT
    assert "not done" in B.odx_last_error(tracer.ctx)
    B.odx_sync(tracer.ctx, stream.cuda_stream, 120.0)
    st = B.records_to_numpy(rec)[:2048 * 2048]["status"]
    assert np.all((st >= 1) & (st <= 5))


def test_tensor_core_wait_limit_raises_the_flag(tracer):
    """Inference with the in-loop tensor-core waits limited to one poll: the kernel gives up
    at its first waits (for the first tile's input, the weights' bulk copy or the first
    MMAs, none of which is done one poll after it is issued), raises the flag, waits for its
    own copies and MMAs with the default limit and frees its tensor memory.  The next
    synchronous call reports ODX_ERR_DEVICE_FLAG and clears it; with the limit restored the
    same inference returns the same outputs as before."""
    import torch
    from paper_1601_02063_gb300 import binding as B

    mlp = B.odx_mlp_create(tracer.ctx, 65536, W.SEED + 11)
    try:
        n = 1 << 16
        g = torch.Generator(device="cuda").manual_seed(5)
        x = torch.rand((n, 4), dtype=torch.float32, device="cuda", generator=g)
        y0 = torch.empty((n, 4), dtype=torch.float32, device="cuda")
        B.odx_mlp_forward(mlp, x.data_ptr(), n, y0.data_ptr())
        torch.cuda.synchronize()
        B.odx_mlp_get_params(mlp)  # no flag yet

        B.odx_mlp_set_wait_limit(mlp, 1)
        y1 = torch.full((n, 4), float("nan"), dtype=torch.float32, device="cuda")
        B.odx_mlp_forward(mlp, x.data_ptr(), n, y1.data_ptr())
        torch.cuda.synchronize()
        with pytest.raises(B.OdxError) as info:
            B.odx_mlp_get_params(mlp)
        assert info.value.code == B.ERR_DEVICE_FLAG
        B.odx_mlp_get_params(mlp)  # the flag was cleared by the report

        B.odx_mlp_set_wait_limit(mlp, 0)
        y2 = torch.empty((n, 4), dtype=torch.float32, device="cuda")
        B.odx_mlp_forward(mlp, x.data_ptr(), n, y2.data_ptr())
        torch.cuda.synchronize()
        B.odx_mlp_get_params(mlp)
        assert torch.equal(y2, y0)
    finally:
        B.odx_mlp_destroy(mlp)
