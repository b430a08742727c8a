"""Rendering of voxel data as lattice cells (fcc_render_cells; Sec. 5, Fig. 4):
against a numpy restatement of the same ray marcher, and against the
geometry of the cells (the silhouette of one opaque cell seen along a
lattice axis: a unit square for the cube, the diamond |y| + |z| <= 1 of area
2 for the FCC lattice's rhombic dodecahedron)."""
import numpy as np
import pytest
import torch

from paper_1807_10058_gb300 import binding, inputs

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


def render_numpy(vol, n, cells, az, el, kappa, step, W, H):
    """The marcher's definition in FP64: camera, nearest lattice point
    (rounding; for D3 the odd-sum correction of the worst coordinate), voxel
    index, emission-absorption front to back."""
    lo, hi = (-0.5, n - 0.5) if cells == "cube" else (-1.0, 2.0 * n - 1.0)
    c, r = 0.5 * (lo + hi), 0.5 * (hi - lo) * np.sqrt(3.0)
    v = np.array([np.cos(el) * np.cos(az), np.cos(el) * np.sin(az), np.sin(el)])
    right = np.array([-np.sin(az), np.cos(az), 0.0])
    up = np.cross(v, right)
    sx = 2 * (np.arange(W) + 0.5) / W - 1
    sy = 1 - 2 * (np.arange(H) + 0.5) / H
    SX, SY = np.meshgrid(sx, sy)
    o = c + r * v + r * (SX[..., None] * right + SY[..., None] * up)
    d = -v
    C = np.zeros((H, W))
    A = np.zeros((H, W))
    for s in range(int(2 * r / step)):
        t = (s + 0.5) * step
        x = o + t * d
        f = np.rint(x)
        if cells == "cube":
            idx = f.astype(np.int64)
        else:
            err = np.abs(x - f)
            worst = np.argmax(err, axis=-1)
            odd = (f.sum(-1).astype(np.int64) % 2) != 0
            sel = np.take_along_axis(x, worst[..., None], -1)[..., 0] >= np.take_along_axis(f, worst[..., None], -1)[..., 0]
            corr = np.where(sel, 1.0, -1.0) * odd
            np.put_along_axis(f, worst[..., None], np.take_along_axis(f, worst[..., None], -1) + corr[..., None], -1)
            z = f.astype(np.int64)
            idx = np.stack([(z[..., 0] + z[..., 1] - z[..., 2]) // 2, (z[..., 1] + z[..., 2] - z[..., 0]) // 2,
                            (z[..., 0] + z[..., 2] - z[..., 1]) // 2], -1)
        inside = np.all((idx >= 0) & (idx < n), -1)
        val = np.zeros((H, W))
        ii = np.clip(idx, 0, n - 1)
        val[inside] = np.clip(vol[ii[..., 0], ii[..., 1], ii[..., 2]][inside], 0, 1)
        a = 1 - np.exp(-kappa * val * step)
        live = A < 0.999
        C += np.where(live, (1 - A) * a * val, 0)
        A += np.where(live, (1 - A) * a, 0)
    return C


# views: oblique, along an axis (rays parallel to two faces of the box the
# kernel clips them to), along a body diagonal, from below
VIEWS = [(0.7, 0.35), (0.0, 0.0), (np.pi / 4, 0.6154797), (2.5, -0.8)]


@pytest.mark.parametrize("view", VIEWS)
@pytest.mark.parametrize("cells", ["cube", "rhombic_dodecahedron"])
def test_render_matches_numpy_restatement(cells, view):
    """The kernel marches each ray only through the region its cells can
    occupy; the restatement marches the whole bounding sphere."""
    az, el = view
    n, W, H = 8, 48, 40
    vol = inputs.phantom(n, 1, seed=3)[0]
    vol = np.clip(vol / max(vol.max(), 1e-9), 0, 1)
    vol[vol < 0.2] = 0.0
    x = torch.from_numpy(vol.astype(np.float32).reshape(-1)).to(DEV)
    img = binding.render_cells(x, n, cells, azimuth=az, elevation=el, kappa=3.0, step=0.05, width=W, height=H)
    got = img.cpu().numpy().reshape(H, W)
    want = render_numpy(vol.astype(np.float32).astype(np.float64), n, cells, az, el, 3.0, 0.05, W, H)
    diff = np.abs(got - want)
    # a sample within rounding distance of a cell face may land in the
    # neighbouring cell on one side only: a few pixels may differ
    assert want.max() > 0.1
    assert np.mean(diff > 1e-3) < 0.02, (np.mean(diff > 1e-3), diff.max())
    assert np.mean(diff) < 2e-3 * want.max(), np.mean(diff)


@pytest.mark.parametrize("cells,area", [("cube", 1.0), ("rhombic_dodecahedron", 2.0)])
def test_single_cell_silhouette_along_an_axis(cells, area):
    n, W = 3, 256
    vol = np.zeros((n, n, n), dtype=np.float32)
    vol[1, 1, 1] = 1.0
    x = torch.from_numpy(vol.reshape(-1)).to(DEV)
    img = binding.render_cells(x, n, cells, azimuth=0.0, elevation=0.0, kappa=400.0, step=0.01, width=W, height=W)
    got = img.cpu().numpy().reshape(W, W)
    lo, hi = (-0.5, n - 0.5) if cells == "cube" else (-1.0, 2.0 * n - 1.0)
    r = 0.5 * (hi - lo) * np.sqrt(3.0)
    px = (2 * r / W) ** 2
    covered = (got > 0.5).sum() * px
    assert abs(covered - area) < 0.05 * area, (covered, area)


def test_render_rejects_bad_arguments():
    L = binding.lib()
    x = torch.zeros(8, device=DEV)
    img = torch.zeros(16, device=DEV)
    import ctypes
    for n, cells, kappa, step, w in ((0, 1, 1.0, 0.1, 4), (2, 5, 1.0, 0.1, 4), (2, 1, 0.0, 0.1, 4), (2, 1, 1.0, 0.0, 4),
                                     (2, 1, 1.0, 0.1, 0)):
        assert L.fcc_render_cells(ctypes.c_void_p(x.data_ptr()), n, cells, 0.0, 0.0, kappa, step, w, 4,
                                  ctypes.c_void_p(img.data_ptr()), None) == binding.FCC_ERR_INVALID_ARG
