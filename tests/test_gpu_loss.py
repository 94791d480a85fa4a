"""Loss on the fused SDF and the hand-written adjoint (extension): GPU vs the FP64 oracle's
loss, analytic gradient and frozen-decision central differences."""
import numpy as np
import pytest
import torch

import oracle
from gpu_helpers import cuda, gpu_volume, oracle_volume
from paper_1709_03763_b300 import synthetic
from paper_1709_03763_b300.autograd import surface_loss

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def setup(tiny):
    w = tiny
    D, C = cuda(w.kf_depth), cuda(w.kf_rgba)
    it = w.intr.as_tuple()
    V = gpu_volume(w)
    O = oracle_volume(w)
    for k in range(10):
        V.integrate(k, D[k], C[k], w.intr, w.kf_poses[k])
        O.integrate(k, w.kf_depth[k], w.kf_rgba[k], it, w.kf_poses[k])
    pts = synthetic.surface_points(w.scene, 20000, 1).astype(np.float32).astype(np.float64)
    _, _, pflag = O.loss(pts)
    pts = pts[pflag == 0]
    return w, D, C, V, O, pts


def test_loss_matches_oracle(setup):
    w, D, C, V, O, pts = setup
    out, gD = V.sdf_loss(torch.tensor(pts, dtype=torch.float32).cuda(), 0.1)
    L, P = out[0].item(), out[1].item()
    Lo, Po, _ = O.loss(pts, 0.1)
    # points with a marginal corner were removed, so the valid set is the same
    assert P == Po
    assert abs(L - Lo) <= 1e-4 * abs(Lo)


def test_adjoint_matches_oracle_gradient_and_finite_differences(setup):
    w, D, C, V, O, pts = setup
    it = w.intr.as_tuple()
    kfs = list(range(10))
    out, gD = V.sdf_loss(torch.tensor(pts, dtype=torch.float32).cuda(), 0.1)
    gx, gd = V.sdf_adjoint(kfs, [D[k] for k in kfs], w.kf_poses[kfs], w.intr, gD)
    gx = gx.cpu().numpy()
    ox, od, ex, ed = O.grad(kfs, w.kf_depth[kfs], w.kf_poses[kfs], it, pts, 0.1, with_budget=True)
    # 1e-4 of the largest keyframe gradient, plus the oracle's budget for contributions
    # whose pixel / band / clamp decision is within the float32 margin
    scale = np.abs(ox).max()
    for k in kfs:
        assert np.all(np.abs(gx[k] - ox[k]) <= 1e-4 * scale + 1.01 * ex[k]), (k, gx[k], ox[k], ex[k])
        # keyframes with a large gradient and a small budget: 1e-4 relative
        if np.abs(ox[k]).max() > 0.1 * scale and ex[k].max() < 1e-5 * np.abs(ox[k]).max():
            assert np.abs(gx[k] - ox[k]).max() <= 1e-4 * np.abs(ox[k]).max(), (k, gx[k], ox[k])
    # central differences of the oracle's frozen-decision loss, eps = 1e-4 rad / 1e-4 m
    eps = 1e-4
    for k in (0, 5):
        fd = np.zeros(6)
        for j in range(6):
            e = np.zeros(6)
            e[j] = eps
            fd[j] = (O.loss_perturbed(k, w.kf_depth[k], w.kf_poses[k], it, e, pts)
                     - O.loss_perturbed(k, w.kf_depth[k], w.kf_poses[k], it, -e, pts)) / (2 * eps)
        assert np.all(np.abs(gx[k] - fd) <= 1e-4 * np.abs(fd).max() + 1.01 * ex[k]), (k, gx[k], fd, ex[k])
    # depth-pixel gradient
    gd = gd.cpu().numpy()
    for k in kfs:
        dscale = np.abs(od).max()
        assert np.all(np.abs(gd[k] - od[k]) <= 1e-4 * dscale + 1.01 * ed[k]), k


def test_autograd_function_matches_adjoint(setup):
    w, D, C, V, O, pts = setup
    kfs = list(range(10))
    xi = torch.zeros((10, 6), dtype=torch.float64, requires_grad=True)
    dep = D.clone().requires_grad_(True)
    L = surface_loss(xi, dep, V, kfs, w.kf_poses, C, w.intr, torch.tensor(pts, dtype=torch.float32).cuda())
    L.backward()
    out, gD = V.sdf_loss(torch.tensor(pts, dtype=torch.float32).cuda(), 0.1)
    gx, gd = V.sdf_adjoint(kfs, [D[k] for k in kfs], w.kf_poses, w.intr, gD)
    assert abs(L.item() - out[0].item()) <= 1e-9 * abs(out[0].item())
    assert torch.allclose(xi.grad, gx.cpu(), rtol=1e-5, atol=1e-12)
    assert torch.allclose(dep.grad, gd, rtol=1e-4, atol=1e-9)
