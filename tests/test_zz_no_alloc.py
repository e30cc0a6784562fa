"""odx_render_static: rendering without any device allocation by the library.

Some callers cannot let a library call cudaMalloc: their device memory is owned by another
allocator (a framework's caching pool, or a fixed budget reserved at start-up), as for a
renderer embedded as a plug-in in a host application or a serving loop that forbids
allocation after warm-up.  This entry point keeps its scratch in a fixed static device
array instead.  The tests check it against odx_render, the entry point with a context, on
two calls in a row (the second reuses the array the first left behind), in FP64 and in the
mixed path's three launches; that a request beyond the array's capacity is refused without
launching anything; and that a call on a capturing stream is refused.

This file is collected last; it passes alone in a fresh process and after the other tests.
"""
import numpy as np
import pytest

from paper_1601_02063_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _records(rec, n):
    from paper_1601_02063_gb300 import binding as B
    return B.records_to_numpy(rec)[:n]


def _check_equal(got, ref, img_got, img_ref):
    # same kernel, same per-ray arithmetic: the FP64 parity tolerance (1e-10 relative on
    # crossing radius, disk radius and redshift) is met exactly
    assert np.array_equal(got["status"], ref["status"])
    for f in ("r_cross", "r_hit", "g", "intensity", "H_end", "Q_drift"):
        a, b = got[f], ref[f]
        ok = ~np.isnan(b)
        assert np.array_equal(np.isnan(a), ~ok)
        assert np.all(np.abs(a[ok] - b[ok]) <= 1e-10 * np.abs(b[ok]))
    assert np.allclose(img_got, img_ref, rtol=1e-10, atol=0)


def _scenes(case):
    if case == "fp64_thin_disk":
        return [W.scene(n_alpha=48, n_beta=40),
                W.scene(a=0.5, theta_obs=1.3, n_alpha=33, n_beta=17)]
    # the mixed path's three launches (init, FP32 tracer, finish) on a transfer emitter
    base = dict(W.torus_512("mixed"), n_alpha=40, n_beta=32)
    return [base, dict(base, theta_obs=1.1, n_alpha=24, n_beta=19)]


@pytest.mark.parametrize("case", ["fp64_thin_disk", "mixed_torus"])
def test_static_entry_matches_render_on_two_calls(case):
    import torch
    from paper_1601_02063_gb300 import binding as B
    from paper_1601_02063_gb300 import build

    build.build()
    torch.cuda.set_device(0)
    scenes = _scenes(case)
    n, ni = B.n_rays(scenes), B.n_image(scenes)
    tr = B.Tracer(0)  # the default launch shape, the one the static entry point uses
    rec_ref, img_ref = tr.render(scenes)
    torch.cuda.synchronize()
    ref = _records(rec_ref, n)
    img_ref = img_ref[:ni].cpu().numpy()
    tr.close()

    stream = torch.cuda.current_stream().cuda_stream
    for call in range(2):
        rec = torch.full((n, B.RECORD_BYTES // 8), float("nan"), dtype=torch.float64,
                         device="cuda")
        img = torch.full((ni,), float("nan"), dtype=torch.float64, device="cuda")
        rc = B.odx_render_static(scenes, rec.data_ptr(), img.data_ptr(), stream)
        assert rc == B.OK, (call, rc, B.error_string(rc))
        torch.cuda.synchronize()
        _check_equal(_records(rec, n), ref, img.cpu().numpy(), img_ref)


def test_static_entry_refuses_stream_capture():
    """The scene table is copied from the call's own stack frame, which a graph replay could
    not read: while the stream captures, the call returns ODX_ERR_UNSUPPORTED and records
    nothing into the graph."""
    import torch
    from paper_1601_02063_gb300 import binding as B

    torch.cuda.set_device(0)
    scenes = [W.scene(n_alpha=8, n_beta=8)]
    rec = torch.zeros((64, B.RECORD_BYTES // 8), dtype=torch.float64, device="cuda")
    # the first call on the device (the symbol lookup) comes before any capture
    assert B.odx_render_static(scenes, rec.data_ptr(), None, None) == B.OK
    torch.cuda.synchronize()
    side = torch.cuda.Stream()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.stream(side):
        graph.capture_begin()
        try:
            rc = B.odx_render_static(scenes, rec.data_ptr(), None, side.cuda_stream)
        finally:
            graph.capture_end()
    assert rc == B.ERR_UNSUPPORTED
    torch.cuda.synchronize()


def test_static_entry_refuses_beyond_capacity():
    import torch
    from paper_1601_02063_gb300 import binding as B

    scenes = [W.scene(n_alpha=2, n_beta=2)] * (B.STATIC_MAX_SCENES + 1)
    rec = torch.full((4 * len(scenes), B.RECORD_BYTES // 8), 3.0, dtype=torch.float64,
                     device="cuda")
    rc = B.odx_render_static(scenes, rec.data_ptr(), None, None)
    assert rc == B.ERR_TOO_LARGE
    assert "capacity" in B.error_string(rc)
    torch.cuda.synchronize()
    assert torch.all(rec == 3.0)
    # invalid scenes are rejected the same way as by odx_render
    bad = W.scene(n_alpha=2, n_beta=2, a=1.5)
    assert B.odx_render_static([bad], rec.data_ptr(), None, None) == B.ERR_INVALID_ARG
