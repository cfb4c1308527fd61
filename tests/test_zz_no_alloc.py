"""The allocation-free distance grid (slr_distance_grid_noalloc).

Callers that may not allocate device memory (another framework owns the
device memory, a real-time loop that must not allocate, a plug-in that only
gets pre-allocated buffers) use this entry point; its scratch is a fixed
array inside the library. Here its output must equal that of the context
path, slr_build_distance, exactly as every distance test demands (argmin and
d bit-identical), on two calls in a row: the second call reuses the scratch
left by the first. This file is collected last, so that a failure here
leaves every other test already run.
"""
import numpy as np
import pytest

from paper_2410_22205_gb300 import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _reference(dim, n, prec, pts):
    from paper_2410_22205_gb300 import slr

    shape = tuple(n) + ((1,) if dim == 2 else ())
    rec = slr.Reconstruction(dim=dim, n=shape, lo=(-1.0,) * dim,
                             hi=tuple(-1.0 + 2.0 * (shape[a] - 1) / (shape[0] - 1) for a in range(dim)),
                             precision=prec, interp=0, band=1)
    rec.load_cloud(pts)
    rec.build_distance()
    d, a = rec.d(), rec.argmin()
    rec.close()
    return shape, d, a


@pytest.mark.parametrize("dim,n,npts", [(3, (37, 41, 33), 20000), (2, (129, 97), 5000), (3, (24, 24, 24), 65536)])
@pytest.mark.parametrize("prec", [32, 64])
def test_noalloc_distance_grid_matches_context_path(dim, n, npts, prec):
    from paper_2410_22205_gb300 import slr

    pts = (synth.sphere_cloud(npts, 0.55, 0.01, 11) if dim == 3 else synth.circle_noisy(npts, 0.6, 0.01, 11))
    pts[::97] = pts[1::97][: pts[::97].shape[0]]  # exact duplicates: ties
    shape, d_ref, a_ref = _reference(dim, n, prec, pts)
    N = int(np.prod(shape))
    h = 2.0 / (shape[0] - 1)
    pts_dev = torch.tensor(pts, dtype=torch.float64, device="cuda")
    d_dev = torch.empty(N, dtype=torch.float32 if prec == 32 else torch.float64, device="cuda")
    a_dev = torch.empty(N, dtype=torch.int32, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    for call in range(2):
        d_dev.fill_(float("nan"))
        a_dev.fill_(-7)
        torch.cuda.synchronize()
        slr.slr_distance_grid_noalloc(dim, shape, (-1.0,) * dim, h, prec, pts_dev.data_ptr(), npts,
                                      d_dev.data_ptr(), a_dev.data_ptr(), stream)
        torch.cuda.synchronize()
        assert np.array_equal(a_dev.cpu().numpy(), a_ref), f"argmin differs on call {call}"
        assert np.array_equal(d_dev.cpu().numpy().astype(np.float64), d_ref), f"d differs on call {call}"


def test_noalloc_rejects_clouds_beyond_its_scratch():
    from paper_2410_22205_gb300 import slr

    pts_dev = torch.zeros((65537, 3), dtype=torch.float64, device="cuda")
    d_dev = torch.empty(8 ** 3, dtype=torch.float32, device="cuda")
    a_dev = torch.empty(8 ** 3, dtype=torch.int32, device="cuda")
    with pytest.raises(slr.SlrError) as e:
        slr.slr_distance_grid_noalloc(3, (8, 8, 8), (-1.0, -1.0, -1.0), 2.0 / 7, 32, pts_dev.data_ptr(), 65537,
                                      d_dev.data_ptr(), a_dev.data_ptr())
    assert e.value.status == slr.SLR_E_INVALID
    assert "65536" in str(e.value)


def test_noalloc_refuses_a_capturing_stream():
    """The call reads results back to the host and waits on its stream, so it
    cannot be recorded into a CUDA graph: on a capturing stream it returns
    SLR_E_INVALID with nothing enqueued, and the capture stays valid."""
    from paper_2410_22205_gb300 import slr

    pts_dev = torch.zeros((16, 3), dtype=torch.float64, device="cuda")
    d_dev = torch.empty(8 ** 3, dtype=torch.float32, device="cuda")
    a_dev = torch.empty(8 ** 3, dtype=torch.int32, device="cuda")
    x = torch.zeros(4, device="cuda")
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    err = None
    with torch.cuda.graph(g):
        x.add_(1.0)
        try:
            slr.slr_distance_grid_noalloc(3, (8, 8, 8), (-1.0,) * 3, 2.0 / 7, 32, pts_dev.data_ptr(), 16,
                                          d_dev.data_ptr(), a_dev.data_ptr(), torch.cuda.current_stream().cuda_stream)
        except slr.SlrError as e:
            err = e
    g.replay()
    torch.cuda.synchronize()
    assert err is not None and err.status == slr.SLR_E_INVALID
    assert "captured" in str(err)
    assert float(x[0].item()) == 1.0
