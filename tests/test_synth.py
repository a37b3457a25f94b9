"""The synthetic scene generator's geometry, checked against point tests (CPU).

The interior of a union of boxes (the corridor opening into the room) must stop a ray exactly where it
leaves the union; rendering with bounding-sphere culling must equal rendering without it.
"""
import numpy as np

from synth.scenes import Box, Camera, Interior, Sphere, look_at, render


def _inside(boxes, q):
    return any(np.all(q > lo) and np.all(q < hi) for lo, hi in boxes)


def test_interior_of_a_union_stops_at_its_boundary():
    corr = (np.array([0.1, 4.0, 0.1]), np.array([6.1, 6.2, 2.8]))
    room = (np.array([6.0, 0.1, 0.1]), np.array([10.14, 10.14, 3.6]))
    scene = Interior([corr, room])
    rng = np.random.default_rng(0)
    checked = 0
    for _ in range(40):
        lo, hi = corr if rng.random() < 0.5 else room
        p = rng.uniform(lo + 0.05, hi - 0.05)
        d = rng.normal(size=(64, 3))
        d /= np.linalg.norm(d, axis=1, keepdims=True)
        t = scene.hit(p, d)
        for k in range(len(d)):
            assert np.isfinite(t[k]) and t[k] > 0
            assert _inside([corr, room], p + (t[k] - 1e-6) * d[k])       # still inside just before
            assert not _inside([corr, room], p + (t[k] + 1e-6) * d[k])   # outside just after
            checked += 1
    assert checked == 40 * 64


def test_culled_rendering_equals_plain_rendering():
    rng = np.random.default_rng(1)
    prims = [Box(lo, lo + rng.uniform(0.1, 0.5, 3)) for lo in rng.uniform(0, 3, (20, 3))]
    prims += [Sphere(c, r) for c, r in zip(rng.uniform(0, 3, (20, 3)), rng.uniform(0.05, 0.4, 20))]
    room = Interior([(np.array([-1.0, -1.0, -1.0]), np.array([4.0, 4.0, 4.0]))])
    cam = Camera(48, 36, 40.0, 40.0, 24.0, 18.0, look_at((3.5, -0.5, 2.0), (1.5, 1.5, 1.0)))
    a = render(cam, [room] + prims)
    b = render(cam, [room] + prims, cull=True)
    assert np.array_equal(a, b)
    assert np.isfinite(a).all()
