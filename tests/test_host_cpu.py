"""Host-side helpers of the binding, on the CPU: argument checks of
`Primitives`, the packed-image views, the camera structure and the camera
extent that scales the optimiser's rates and the population thresholds."""
import math

import numpy as np
import pytest

import scenes
from paper_2501_16312_gb300 import OCTAHEDRON, TETRAHEDRON, Primitives, _native, split_images, train


def _arrays(torch, n=5, kind=OCTAHEDRON, K=16):
    return (torch.zeros(n, 3), torch.zeros(n, kind, 3), torch.zeros(n), torch.zeros(n, K, 3))


def test_primitives_rejects_bad_arguments():
    torch = pytest.importorskip("torch")
    c, v, o, s = _arrays(torch)
    with pytest.raises(ValueError, match="kind"):
        Primitives(5, c, v, o, s)
    with pytest.raises(ValueError, match="verts has shape"):
        Primitives(TETRAHEDRON, c, v, o, s)                  # 6 vertices given for a tetrahedron
    with pytest.raises(ValueError, match="opacity has shape"):
        Primitives(OCTAHEDRON, c, v, torch.zeros(4), s)
    with pytest.raises(ValueError, match="sh has shape"):
        Primitives(OCTAHEDRON, c, v, o, s, sh_degree=2)      # 16 coefficients are degree 3
    # right shapes, but host memory or the wrong type: the library needs float32 device arrays
    with pytest.raises(ValueError, match="float32 CUDA"):
        Primitives(OCTAHEDRON, c, v, o, s)
    with pytest.raises(ValueError, match="float32 CUDA"):
        Primitives(OCTAHEDRON, c.double(), v, o, s)


def test_split_images_views_alias_the_packed_buffer():
    torch = pytest.importorskip("torch")
    cams = [scenes.Camera(np.eye(4, dtype=np.float32), 10.0, 10.0, 3.0, 2.0, w, h)
            for w, h in ((7, 3), (2, 5), (1, 1))]
    flat = torch.arange(3 * sum(c.width * c.height for c in cams), dtype=torch.float32)
    views = split_images(flat, cams)
    assert [tuple(v.shape) for v in views] == [(3, 3, 7), (3, 5, 2), (3, 1, 1)]
    # camera 1, channel 2, row 4, column 1 sits after camera 0's 63 values
    assert views[1][2, 4, 1].item() == 63 + 2 * 10 + 4 * 2 + 1
    views[2][0, 0, 0] = -1.0
    assert flat[-3].item() == -1.0


def test_camera_struct_packs_row_major_fields():
    M = np.arange(16, dtype=np.float32).reshape(4, 4)
    cams = [scenes.Camera(M, 1.5, 2.5, 3.5, 4.5, 640, 480), scenes.Camera(M.T.copy(), 1, 1, 0, 0, 1, 2)]
    arr = _native.camera_struct(cams)
    assert list(arr[0].viewmat) == list(range(16))
    assert (arr[0].fx, arr[0].fy, arr[0].cx, arr[0].cy, arr[0].width, arr[0].height) == \
        (1.5, 2.5, 3.5, 4.5, 640, 480)
    assert list(arr[1].viewmat) == list(M.T.reshape(16))
    assert len(_native.camera_struct([])) == 1                 # a valid pointer even for no camera


def test_camera_extent_is_the_largest_distance_from_the_mean_centre():
    # cameras on a circle of radius 4 around (1, 2, 3), looking at its centre
    rng = np.random.default_rng(0)
    centre = np.array([1.0, 2.0, 3.0])
    cams = []
    for a in np.linspace(0.0, 2.0 * math.pi, 8, endpoint=False) + rng.uniform(0, 0.1):
        eye = centre + 4.0 * np.array([math.cos(a), 0.0, math.sin(a)])
        cams.append(scenes.Camera(scenes.look_at(eye, centre).astype(np.float32), 1, 1, 0, 0, 4, 4))
    assert train.camera_extent(cams) == pytest.approx(4.0, rel=1e-5)
    # one camera has no spread: the extent defaults to 1
    assert train.camera_extent(cams[:1]) == 1.0
    # two cameras: half their distance
    assert train.camera_extent(cams[::4]) == pytest.approx(4.0, rel=1e-5)
