"""The BVH4 builder on the host (no GPU): compiles csrc/bvh_build.cpp with the
checker tests/bvh_check.cpp and runs it on seeded scenes, with and without
split references.  The checker verifies the tree's structure, that every
triangle is referenced, that boxes nest, and that closest hits of random rays
through the tree equal brute force over all triangles."""
import os
import shutil
import subprocess

import numpy as np
import pytest

import scenegen

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def checker(tmp_path_factory):
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no C++ compiler")
    out = str(tmp_path_factory.mktemp("bvh") / "bvh_check")
    subprocess.run([cxx, "-O2", "-std=c++17", "-o", out, os.path.join(ROOT, "tests", "bvh_check.cpp"),
                    os.path.join(ROOT, "paper_2108_05263_gb300", "csrc", "bvh_build.cpp")], check=True)
    return out


def _run(checker, tmp_path, verts, split, rays=1500):
    """split: False (every triangle fixed), True (none) or "half" (every other
    pair of triangles fixed: moving quads among static ones)."""
    path = str(tmp_path / "tris.bin")
    np.ascontiguousarray(verts, np.float32).tofile(path)
    mode = "2" if split == "half" else ("1" if split else "0")
    r = subprocess.run([checker, path, mode, str(rays)], capture_output=True, text=True)
    return r.returncode, r.stdout


def _big_and_small(seed=3):
    """Large quads (boxes of whole walls: split candidates) among many small
    random triangles."""
    rng = np.random.default_rng(seed)
    big = []
    for k in range(6):
        c = rng.uniform(-4, 4, 3)
        a, b = np.zeros(3), np.zeros(3)
        a[k % 3], b[(k + 1) % 3] = 4.0, 3.0
        p = [c - a - b, c + a - b, c + a + b, c - a + b]
        big += [[p[0], p[1], p[2]], [p[0], p[2], p[3]]]
    small = rng.uniform(-5, 5, (3000, 1, 3)) + rng.normal(0, 0.05, (3000, 3, 3))
    return np.concatenate([np.array(big), small]).astype(np.float32)


@pytest.mark.parametrize("split", [False, True])
def test_tiny_room(checker, tmp_path, split):
    rc, out = _run(checker, tmp_path, scenegen.tiny_room().verts, split)
    assert rc == 0, out


@pytest.mark.parametrize("split", [False, True, "half"])
def test_big_and_small_triangles(checker, tmp_path, split):
    rc, out = _run(checker, tmp_path, _big_and_small(), split)
    assert rc == 0, out
    if split:   # the large (free) quads were entered as several references
        slots = int(out.split("slots ")[1].split()[0])
        assert slots > 3012


def test_apartment_with_split_references(checker, tmp_path):
    rc, out = _run(checker, tmp_path, scenegen.apartment(frames=1).verts, True, rays=300)
    assert rc == 0, out
