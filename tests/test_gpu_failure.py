"""Failure detection of the traversal, in the form this library supports:
a device-side limit that runs out sets the context's error word, the kernel
reports "no hit" for the rays concerned and the frame finishes; the host
learns of it from ddgi_get_status.  Nothing here faults, traps or hangs the
GPU: the limit is a configuration field (traversal_visit_cap), set low
enough that every ray reaches it."""
import dataclasses
import types

import numpy as np
import pytest

import scenegen

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dd():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2108_05263_gb300 import build
    build.build()
    from paper_2108_05263_gb300 import ddgi
    ddgi.load()
    return ddgi


def _with_cap(settings, cap):
    return types.SimpleNamespace(**dataclasses.asdict(settings), traversal_visit_cap=cap)


def test_traversal_visit_cap_is_reported_and_the_frame_completes(dd):
    # the apartment's BVH is many levels deep: a cap of one node stops every
    # ray at the root
    sc = scenegen.apartment(width=64, height=48, frames=2)
    cam = sc.cameras[0]
    capped = dd.Context.from_scene(sc, _with_cap(sc.settings, 1))
    assert capped.get_info().bvh_depth > 1
    fr = dd.Frame(capped, cam.width, cam.height, sc.settings.spatial_passes)
    rad = fr.render(0, cam).cpu().numpy()
    assert capped.get_status() == dd.ERR_TRAVERSAL_LIMIT
    assert "traversal" in capped.last_error()
    # every primary ray gave up: no valid pixel, black (and finite) radiance
    g1 = fr.g[0].g1.cpu().numpy()
    assert np.all(g1[:, 3].view(np.uint32) == 0xFFFFFFFF)
    assert np.all(np.isfinite(rad)) and np.all(rad[:, :3] == 0.0)
    # the word was cleared by the read: no launch since, so it stays clear
    assert capped.get_status() == dd.OK
    # the same frame again hits the limit again (the cap stays configured)
    fr.render(1, sc.cameras[1 % len(sc.cameras)])
    assert capped.get_status() == dd.ERR_TRAVERSAL_LIMIT

    # the default cap renders the same frames without an error
    free = dd.Context.from_scene(sc)
    fr2 = dd.Frame(free, cam.width, cam.height, sc.settings.spatial_passes)
    for f in range(2):
        rad2 = fr2.render(f, sc.cameras[f % len(sc.cameras)]).cpu().numpy()
        assert free.get_status() == dd.OK
    assert np.all(np.isfinite(rad2)) and rad2[:, :3].max() > 0.0
    g1 = fr2.g[1].g1.cpu().numpy()
    assert np.mean(g1[:, 3].view(np.uint32) != 0xFFFFFFFF) > 0.9


def test_traversal_visit_cap_out_of_range_is_refused(dd):
    sc = scenegen.tiny_room(width=16, height=16, frames=1)
    with pytest.raises(dd.DDGIError):
        dd.Context.from_scene(sc, _with_cap(sc.settings, (1 << 30) + 1))
