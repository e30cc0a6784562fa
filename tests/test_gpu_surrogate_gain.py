"""What the learned transfer function gains over the method without it, measured.

The network is trained briefly on rays the integrator traces (2^22 rays), then renders a
1024x1024 thin-disk image (a = 0.7, i = 45 deg) with integrator fallback near the critical
curve.  The same image is rendered by the mixed-precision integrator alone at the default
and at looser FP32 tolerances; the gain is the integrator's time at an image error no larger
than the surrogate's, divided by the surrogate's time.  The test reports that ratio and the
error-against-fallback curve (the critical-curve band widened until every pixel falls back,
which reproduces the integrator's image), and holds the briefly trained network to an image
error below 25 % (the images are compared with the plain FP64 integrator's; the benchmark
trains on 2^24 rays and reports the full curve)."""
import time

import numpy as np
import pytest

from paper_1601_02063_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def test_surrogate_gain_at_equal_image_error():
    import torch
    from paper_1601_02063_gb300 import binding as B
    from paper_1601_02063_gb300 import build
    from paper_1601_02063_gb300.surrogate import Surrogate, image_error

    build.build()
    tr = B.Tracer(0)
    sg = Surrogate(tr, max_batch=65536)
    try:
        sc = W.surrogate_scene_2048()
        sc.update(n_alpha=1024, n_beta=1024)
        n = 1024 * 1024
        _, ref = tr.render(dict(sc, precision="fp64"))
        torch.cuda.synchronize()
        ref = ref[:n].clone()

        def timed(fn, reps=3):
            fn()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            for _ in range(reps):
                out = fn()
            torch.cuda.synchronize()
            return (time.perf_counter() - t0) / reps * 1e3, out

        x, t = sg.make_data(1 << 22)
        sg.train(x, t, epochs=24, batch=65536, lr=2e-3, lr_final=2e-5)
        del x, t
        bufs = sg.render(sc)[:3]
        ms_s, out = timed(lambda: sg.render(sc, out=bufs))
        err_s = image_error(out[0], ref)
        print(f"surrogate: {ms_s:.2f} ms, fallback {out[3] / n:.2%}, image error {err_s:.3e}")
        assert err_s < 0.25
        curve = []
        for band in (0.5, 2.0, 8.0, 32.0):
            ms_b, ob = timed(lambda: sg.render(sc, band=band, out=bufs), 2)
            curve.append((band, ob[3] / n, image_error(ob[0], ref), ms_b))
            print(f"  band {band:5.1f} M: fallback {ob[3] / n:7.2%}, image error "
                  f"{curve[-1][2]:.3e}, {ms_b:.2f} ms")
        assert curve[-1][1] == 1.0 and curve[-1][2] < 1e-5  # everything on the integrator
        rec, img = tr.alloc(n, n)
        best = None
        for rt32 in (1e-6, 1e-4, 1e-3):
            sc_l = dict(sc, rtol_fp32=rt32)
            ms_l, _ = timed(lambda: tr.render(sc_l, out=(rec, img)))
            err_l = image_error(img[:n], ref)
            print(f"  integrator rtol_fp32 {rt32:g}: {ms_l:.2f} ms, image error {err_l:.3e}")
            if err_l <= err_s and (best is None or ms_l < best):
                best = ms_l
        assert best is not None  # the default tolerance is far more accurate than the network
        print(f"gain at equal image error: {best / ms_s:.2f}x")
        assert np.isfinite(best / ms_s)
    finally:
        sg.close()
        tr.close()
