"""Pins of the oracle's pooled observation (the policy input of the RL
rollout): closed forms on constructed frames, so that a wrong cell size, a
swapped width and height, a transposed cell index or a wrong block order
fails a case."""
import numpy as np
import pytest

import oracle
from paper_2605_01352_b300 import scene as S


def _scene(W=8, H=4, cams=2, envs=2):
    return S.generate(envs, 3, 5, kinds="mixed", res=W, height=H, cams_per_env=cams)


def _blank(sc):
    P = int(sc.cam_pix_off()[-1])
    return np.zeros((P, 3), np.uint8), np.zeros(P, np.float32)


def test_uniform_frame_gives_its_values_everywhere():
    sc = _scene()
    rgb, dep = _blank(sc)
    rgb[:] = (200, 100, 50)
    dep[:] = 2.5
    got = oracle.observe(sc, rgb, dep, 2, 0.25)
    n = 4
    lum = (0.299 * 200 + 0.587 * 100 + 0.114 * 50) / 255.0
    assert got.shape == (2, 2 * 2 * n)
    np.testing.assert_allclose(got[:, :2 * n], 2.5 * 0.25, rtol=0, atol=1e-15)
    np.testing.assert_allclose(got[:, 2 * n:], lum, rtol=0, atol=1e-15)


@pytest.mark.parametrize("c,y,x", [(0, 0, 0), (1, 3, 7), (2, 1, 5), (3, 2, 2), (3, 3, 0)])
def test_one_pixel_lands_in_its_cell(c, y, x):
    """A camera of 8 x 4 pixels in 2 x 2 cells of 4 x 2: the pixel (y, x)
    belongs to cell (y // 2, x // 4) of its camera; the depth block of the
    environment's cameras comes first, then the luminance block."""
    sc = _scene(W=8, H=4)
    rgb, dep = _blank(sc)
    p = int(sc.cam_pix_off()[c]) + y * 8 + x
    rgb[p] = (255, 255, 255)
    dep[p] = 6.0
    got = oracle.observe(sc, rgb, dep, 2, 2.0)
    want = np.zeros_like(got)
    e, k = c // 2, c % 2
    cell = (y // 2) * 2 + x // 4
    want[e, k * 4 + cell] = 6.0 / 8 * 2.0
    want[e, (2 + k) * 4 + cell] = 1.0 / 8
    np.testing.assert_allclose(got, want, rtol=0, atol=1e-15)


def test_one_cell_is_the_image_mean():
    sc = _scene(W=8, H=8, cams=1, envs=3)
    rng = np.random.default_rng(3)
    rgb, dep = _blank(sc)
    rgb[:] = rng.integers(0, 256, rgb.shape)
    dep[:] = rng.random(dep.shape)
    got = oracle.observe(sc, rgb, dep, 1, 1.0)
    off = sc.cam_pix_off()
    for c in range(3):
        sl = slice(off[c], off[c + 1])
        assert got[c, 0] == pytest.approx(dep[sl].astype(np.float64).mean(), rel=1e-14)
        y = rgb[sl].astype(np.float64) @ np.array([0.299, 0.587, 0.114]) / 255.0
        assert got[c, 1] == pytest.approx(y.mean(), rel=1e-14)


def test_cells_must_divide_the_camera():
    sc = _scene(W=8, H=4)
    rgb, dep = _blank(sc)
    with pytest.raises(ValueError):
        oracle.observe(sc, rgb, dep, 3, 1.0)
