"""The allocation-free metrics entry point (ddgi_image_metrics_static) must
give the same result as ddgi_image_metrics, through the C ABI, on two calls
in a row with different images (the shared scratch array keeps the previous
call's partial sums, which must not leak into the next result).

Callers of the allocation-free form are those that must not call
cudaMalloc; this test allocates its own images with torch only to have
something to measure."""
import ctypes as C

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2108_05263_gb300 import build
    build.build()
    from paper_2108_05263_gb300 import ddgi
    return ddgi.load()


def _images(n, seed):
    import torch
    rng = np.random.default_rng(seed)
    img = rng.exponential(1.0, (n, 4)).astype(np.float32)
    ref = rng.exponential(2.0, (n, 4)).astype(np.float32)
    ref[: n // 4, :3] = 0.0
    return torch.from_numpy(img).cuda(), torch.from_numpy(ref).cuda()


def _metrics(lib, img, ref, scratch, out):
    rc = lib.ddgi_image_metrics(C.c_void_p(img.data_ptr()), C.c_void_p(ref.data_ptr()),
                                img.shape[0], C.c_void_p(scratch.data_ptr()), scratch.numel(),
                                C.c_void_p(out.data_ptr()), None)
    assert rc == 0
    return out.cpu().numpy().copy()


def _metrics_static(lib, img, ref, out):
    rc = lib.ddgi_image_metrics_static(C.c_void_p(img.data_ptr()), C.c_void_p(ref.data_ptr()),
                                       img.shape[0], C.c_void_p(out.data_ptr()), None)
    assert rc == 0
    return out.cpu().numpy().copy()


def test_static_metrics_match_the_allocating_form_on_two_calls(lib):
    import torch
    scratch = torch.empty(2048, dtype=torch.float64, device="cuda")
    out_a = torch.empty(2, dtype=torch.float64, device="cuda")
    out_b = torch.empty(2, dtype=torch.float64, device="cuda")
    # a large image first (many partial sums), then a small one (few): the
    # second call must not pick up partial sums left by the first
    for n, seed in ((1920 * 1080 + 3, 1), (5000, 2)):
        img, ref = _images(n, seed)
        want = _metrics(lib, img, ref, scratch, out_a)
        got = _metrics_static(lib, img, ref, out_b)
        np.testing.assert_allclose(got, want, rtol=1e-12)
        assert np.all(np.isfinite(got)) and got[0] > 0


def test_static_metrics_reject_oversized_images(lib):
    import torch
    out = torch.empty(2, dtype=torch.float64, device="cuda")
    img = torch.empty((1, 4), dtype=torch.float32, device="cuda")
    rc = lib.ddgi_image_metrics_static(C.c_void_p(img.data_ptr()), C.c_void_p(img.data_ptr()),
                                       (1 << 26) + 1, C.c_void_p(out.data_ptr()), None)
    assert rc == -1


def test_static_metrics_of_an_empty_image_are_zero(lib):
    """n = 0: the second kernel still runs and must write zeros (and not
    whatever the shared array or the output held before)."""
    import torch
    out = torch.full((2,), 7.0, dtype=torch.float64, device="cuda")
    img = torch.ones((4, 4), dtype=torch.float32, device="cuda")
    got = _metrics_static(lib, img[:0], img[:0], out)
    np.testing.assert_array_equal(got, [0.0, 0.0])


def test_static_metrics_reject_a_misaligned_image(lib):
    """Image rows are 16-byte records: a pointer 4 bytes into one is refused
    on the host, before anything is launched, and the output is untouched."""
    import torch
    out = torch.full((2,), 7.0, dtype=torch.float64, device="cuda")
    img, ref = _images(1024, 3)
    rc = lib.ddgi_image_metrics_static(C.c_void_p(img.data_ptr() + 4), C.c_void_p(ref.data_ptr()),
                                       1000, C.c_void_p(out.data_ptr()), None)
    assert rc == -1
    rc = lib.ddgi_image_metrics_static(C.c_void_p(img.data_ptr()), C.c_void_p(ref.data_ptr()),
                                       1000, C.c_void_p(out.data_ptr() + 4), None)
    assert rc == -1
    np.testing.assert_array_equal(out.cpu().numpy(), [7.0, 7.0])
