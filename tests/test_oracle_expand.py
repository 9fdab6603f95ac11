"""Pins of the FP64 map-expansion point selection (CPU): a hand-built case
whose answer is read off the picture, the near plane, the image border and
the threshold's strict inequality."""
import numpy as np

from oracle import expand as E


def _cam():
    return dict(R=np.eye(3), t=np.zeros(3), fx=10.0, fy=10.0, cx=2.0, cy=1.5, width=4, height=3)


def test_hand_built_selection():
    # 4 x 3 image; opacity below tau only in pixel (x=1, y=0) and (x=3, y=2)
    opac = np.array([[1.0, 0.2, 1.0, 1.0],
                     [1.0, 1.0, 1.0, 1.0],
                     [1.0, 1.0, 1.0, 0.98]])
    # points at z = 10 project to (x + 2, y + 1.5) pixels for camera-frame (x, y) = 10 * (world x, y) / 10
    pts = np.array([
        [-0.5, -1.0, 10.0],   # u = 1.5, v = 0.5 -> pixel (1, 0): selected
        [1.5, 1.0, 10.0],     # u = 3.5, v = 2.5 -> pixel (3, 2): 0.98 < 0.99, selected
        [0.5, 0.0, 10.0],     # pixel (2, 1): opacity 1, not selected
        [-0.5, -1.0, -10.0],  # behind the camera
        [-0.5, -1.0, 0.1],    # in front but nearer than the near plane
        [5.0, 0.0, 10.0],     # right of the image
        [-2.5, 0.0, 10.0],    # u = -0.5: left of the image
    ]).T
    idx, _ = E.select_points(pts, _cam(), opac, tau=0.99)
    assert idx.tolist() == [0, 1]
    # the threshold is strict: an opacity equal to tau is not selected
    idx, _ = E.select_points(pts, _cam(), opac, tau=0.98)
    assert idx.tolist() == [0]


def test_pixel_of_a_projection_is_the_one_containing_it():
    opac = np.ones((3, 4))
    opac[1, 2] = 0.0
    eps = 1e-6
    # u just below / above 3 (pixel border between x = 2 and x = 3), v = 1.5
    pts = np.array([[1.0 - eps, -0.05, 10.0], [1.0 + eps, -0.05, 10.0]]).T
    idx, border = E.select_points(pts, _cam(), opac)
    assert idx.tolist() == [0]
    assert np.all(border < 1e-4)
