"""Checkpoint / resume through the C ABI: a context restored from a snapshot
continues exactly like the one that wrote it."""
import dataclasses

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


def _scene(learned):
    sc = scenegen.tiny_room_dynamic(width=64, height=48, frames=8)
    if learned:
        sc.settings = dataclasses.replace(sc.settings, learned_target=1, train_samples=4096)
    return sc


def _step(ctx, sc, f):
    ctx.scene_update(sc.instance_transforms(f), sc.emitter_radiance(f))
    ctx.probe_update(f)
    if sc.settings.learned_target:
        ctx.mlp_train(f)


def _render(dd, ctx, sc, f):
    cam = sc.cameras[f]
    fr = dd.Frame(ctx, cam.width, cam.height, sc.settings.spatial_passes)
    return fr.render(f, cam, probe_update=False).cpu().numpy()


def test_resumed_context_continues_bit_for_bit(dd):
    """Probe form with moving instances, toggling emitters and relocation:
    every later update and frame of the restored context is identical."""
    sc = _scene(False)
    a = dd.Context.from_scene(sc)
    for f in range(5):
        _step(a, sc, f)
    blob = a.state_save()
    b = dd.Context.from_scene(sc)
    b.state_load(blob)
    assert b.state_save() == blob
    for f in (5, 6):
        _step(a, sc, f)
        _step(b, sc, f)
    for x, y in zip(a.probe_state_get(), b.probe_state_get()):
        np.testing.assert_array_equal(x, y)
    np.testing.assert_array_equal(_render(dd, a, sc, 6), _render(dd, b, sc, 6))
    assert a.get_status() == dd.OK and b.get_status() == dd.OK


def test_resumed_learned_context(dd):
    """Learned target: the restored network, moments, average and state are
    the saved ones exactly; training continues alike up to the order of the
    gradient sums' floating-point atomics."""
    sc = _scene(True)
    a = dd.Context.from_scene(sc)
    for f in range(4):
        _step(a, sc, f)
    blob = a.state_save()
    b = dd.Context.from_scene(sc)
    b.state_load(blob)
    assert b.state_save() == blob
    np.testing.assert_array_equal(a.mlp_params_served(), b.mlp_params_served())
    assert a.mlp_status() == b.mlp_status()
    _step(a, sc, 4)
    _step(b, sc, 4)
    np.testing.assert_allclose(a.mlp_params(), b.mlp_params(), rtol=1e-4, atol=1e-6)
    assert a.mlp_status()["step"] == b.mlp_status()["step"]
    ra, rb = _render(dd, a, sc, 4), _render(dd, b, sc, 4)
    np.testing.assert_allclose(ra, rb, rtol=1e-3, atol=1e-4)


def test_snapshot_of_another_configuration_is_refused(dd):
    sc = _scene(True)
    a = dd.Context.from_scene(sc)
    _step(a, sc, 0)
    blob = a.state_save()
    other = dataclasses.replace(sc, settings=dataclasses.replace(sc.settings, learned_target=0, train_samples=0))
    c = dd.Context.from_scene(other)
    with pytest.raises(dd.DDGIError):
        c.state_load(blob)
    with pytest.raises(dd.DDGIError):
        a.state_load(blob[:-4])
    bad = bytearray(blob)
    bad[0] ^= 0xFF
    with pytest.raises(dd.DDGIError):
        a.state_load(bytes(bad))
    assert a.get_status() == dd.OK
