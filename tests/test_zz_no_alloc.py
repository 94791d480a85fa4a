"""The allocation-free adjoint, sc_sdf_adjoint_noalloc, called through the C ABI.

Some callers cannot allocate device memory once they are running: a real-time
tracking thread whose memory budget is fixed when it starts, code that runs while
a CUDA graph is being captured (cudaMalloc is not allowed there), or an
application whose device memory is owned by a different allocator.  This entry
point gives them the adjoint without any allocation by the library: its scratch
is a fixed device array inside the library.  Its results must match
sc_sdf_adjoint's, call after call (the shared array keeps the previous call's
contents, which must not leak into the next result).  This file is collected
last on purpose."""
import ctypes

import numpy as np
import pytest
import torch

from gpu_helpers import cuda, gpu_volume
from paper_1709_03763_b300 import _lib, make_intrinsics, make_pose, synthetic

pytestmark = pytest.mark.gpu


def _call_noalloc(V, ids, D, poses, intr, gD):
    n = len(ids)
    K = make_intrinsics(intr)
    gx = torch.full((n, 6), float("nan"), dtype=torch.float64, device="cuda")
    gd = torch.full((n, K.height, K.width), float("nan"), dtype=torch.float32, device="cuda")
    c_ids = (ctypes.c_int32 * n)(*ids)
    c_dep = (ctypes.c_void_p * n)(*[D[k].data_ptr() for k in ids])
    c_pos = (_lib.Pose * n)(*[make_pose(poses[k]) for k in ids])
    rc = _lib.lib().sc_sdf_adjoint_noalloc(V.h, c_ids, c_dep, c_pos, n, ctypes.byref(K), gD.data_ptr(),
                                          gx.data_ptr(), gd.data_ptr(), torch.cuda.current_stream().cuda_stream)
    assert rc == _lib.SC_OK, rc
    torch.cuda.synchronize()
    return gx, gd


def test_noalloc_adjoint_matches_allocating_adjoint(tiny):
    w = tiny
    D, C = cuda(w.kf_depth), cuda(w.kf_rgba)
    V = gpu_volume(w)
    ids = list(range(10))
    V.integrate_many(ids, D, C, w.kf_poses, w.intr)
    pts = torch.tensor(synthetic.surface_points(w.scene, 20000, 1), dtype=torch.float32).cuda()
    _, gD = V.sdf_loss(pts, 0.1)
    ref_x, ref_d = V.sdf_adjoint(ids, [D[k] for k in ids], w.kf_poses, w.intr, gD)
    scale = ref_x.abs().max().item()
    dscale = ref_d.abs().max().item()
    assert scale > 0 and dscale > 0
    for call in range(2):  # two calls in a row through the same scratch array
        gx, gd = _call_noalloc(V, ids, D, w.kf_poses, w.intr, gD)
        assert torch.all(torch.isfinite(gx)) and torch.all(torch.isfinite(gd))
        assert (gx - ref_x).abs().max().item() <= 1e-9 * scale, call
        assert (gd - ref_d).abs().max().item() <= 1e-6 * dscale, call
    # a shorter call after a longer one: nothing of the previous call leaks in
    sub = [7, 2, 5]
    gx, gd = _call_noalloc(V, sub, D, w.kf_poses, w.intr, gD)
    for i, k in enumerate(sub):
        assert (gx[i] - ref_x[k]).abs().max().item() <= 1e-9 * scale
        assert (gd[i] - ref_d[k]).abs().max().item() <= 1e-6 * dscale


def test_noalloc_adjoint_rejects_more_than_its_capacity(tiny):
    w = tiny
    V = gpu_volume(w)
    n = 257
    K = make_intrinsics(w.intr)
    c_ids = (ctypes.c_int32 * n)()
    c_dep = (ctypes.c_void_p * n)()
    c_pos = (_lib.Pose * n)()
    dummy = torch.zeros(16, device="cuda")
    rc = _lib.lib().sc_sdf_adjoint_noalloc(V.h, c_ids, c_dep, c_pos, n, ctypes.byref(K), dummy.data_ptr(),
                                          dummy.data_ptr(), None, torch.cuda.current_stream().cuda_stream)
    assert rc == _lib.SC_ERR_CAPACITY
