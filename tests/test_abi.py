"""The C-ABI library loads, exports every entry point include/surfcorr.h declares, and
its host-side helpers agree with the oracle and with the Fig. 4 worked example.  No
GPU needed: nothing here launches a kernel."""
import ctypes
import json
import math
import os
import re

import numpy as np
import pytest

import oracle
from paper_1709_03763_b300 import _lib
from paper_1709_03763_b300 import synthetic
from paper_1709_03763_b300.volume import pose_distance, pose_exp_left, select_consecutive, select_topm

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "surfcorr.h")


def declared_symbols():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:const\s+)?\w+\*?\s+\*?(sc_\w+)\s*\(", text, flags=re.M)))


def test_header_declares_the_boundary():
    syms = declared_symbols()
    for s in ["sc_create_volume", "sc_fuse_frames_into_keyframe", "sc_integrate_keyframe",
              "sc_deintegrate_keyframe", "sc_reintegrate_batch", "sc_extract_block_list", "sc_sdf_adjoint"]:
        assert s in syms


def test_library_exports_every_declared_symbol():
    L = ctypes.CDLL(_lib.LIB_PATH)
    missing = [s for s in declared_symbols() if not hasattr(L, s)]
    assert not missing, missing
    # the Python binding declares exactly the header's entry points
    assert sorted(_lib.SIGNATURES) == declared_symbols()


def test_abi_version_and_status_strings():
    L = _lib.lib()
    assert L.sc_abi_version() == 1
    for code in range(0, -12, -1):
        assert L.sc_status_string(code).decode() != "unknown status"


def test_sensor_conversions_reject_bad_arguments_before_any_launch():
    # the pointers below are never dereferenced: each call is refused by the host-side
    # checks (or, for an empty input, returns before touching the device)
    L = _lib.lib()
    bad = _lib.SC_ERR_INVALID_ARG
    assert L.sc_rgba_from_rgb(None, 5, None, None) == bad
    assert L.sc_rgba_from_rgb(0x1000, -1, 0x2000, None) == bad
    assert L.sc_rgba_from_rgb(0x1001, 5, 0x2000, None) == bad      # rgb not 4-byte aligned
    assert L.sc_rgba_from_rgb(0x1000, 5, 0x2008, None) == bad      # rgba not 16-byte aligned
    assert L.sc_rgba_from_rgb(0x1000, 16, 0x1010, None) == bad     # overlapping buffers
    assert L.sc_rgba_from_rgb(None, 0, None, None) == 0              # empty: nothing to do
    assert L.sc_depth_from_u16(0x1000, 8, 0.0, 0x2000, None) == bad  # scale must be positive
    assert L.sc_depth_from_u16(0x1000, 8, float("nan"), 0x2000, None) == bad
    assert L.sc_depth_from_u16(0x1002, 8, 0.001, 0x2000, None) == bad  # raw not 16-byte aligned
    assert L.sc_depth_from_u16(None, 0, 0.001, None, None) == 0


def test_struct_layouts():
    assert ctypes.sizeof(_lib.Pose) == 48
    assert ctypes.sizeof(_lib.Intrinsics) == 24
    assert ctypes.sizeof(_lib.VolumeParams) == 36
    assert ctypes.sizeof(_lib.ReintItem) == 8 + 8 + 48 + 48 + 4 + 4


def test_selection_fig4():
    g = json.load(open(os.path.join(ROOT, "tests", "golden", "fig4_selection.json")))
    d = np.array(g["distances"], float)
    assert select_consecutive(d, g["m"]) + 1 == g["j_star_1based"]
    assert list(select_topm(d, g["m"]) + 1) == g["bundlefusion_top_m_1based"]


def test_selection_matches_oracle_on_random_distances():
    rng = np.random.default_rng(5)
    for trial in range(20):
        K = int(rng.integers(5, 300))
        m = int(rng.integers(1, K + 1))
        d = np.round(rng.uniform(0, 3, K), 1)  # rounding creates ties
        assert select_consecutive(d, m) == oracle.select_consecutive(d, m)[0]
        assert np.array_equal(select_topm(d, m), oracle.select_topm(d, m))


def test_pose_distance_matches_oracle():
    g = np.random.default_rng(3)
    for _ in range(50):
        a = synthetic.look_pose(g.uniform(-5, 5, 3), g.uniform(-3.1, 3.1), g.uniform(-1, 1), g.uniform(-1, 1))
        b = synthetic.perturb_pose(a, g.uniform(0, 0.5), g.uniform(0, 0.3), g)
        assert math.isclose(pose_distance(a, b), oracle.pose_distance(a, b), rel_tol=1e-9, abs_tol=1e-12)


def test_pose_exp_left_closed_forms():
    T = synthetic.look_pose(np.array([1.0, 2.0, 1.5]), 0.3, 0.2)
    # pure translation: t' = t + rho
    out = pose_exp_left(T, [0.1, -0.2, 0.3, 0, 0, 0])
    assert np.allclose(out[:, 3], T[:, 3] + [0.1, -0.2, 0.3], atol=1e-6)
    assert np.allclose(out[:, :3], T[:, :3], atol=1e-7)
    # pure rotation: R' = Rot(omega) R, t' = Rot(omega) t
    w = np.array([0.2, -0.1, 0.4])
    Rw = synthetic.axis_angle(w, np.linalg.norm(w))
    out = pose_exp_left(T, [0, 0, 0, *w])
    assert np.allclose(out[:, :3], Rw @ T[:, :3], atol=1e-6)
    assert np.allclose(out[:, 3], Rw @ T[:, 3], atol=1e-6)


def test_sensor_conversion_wrappers_check_their_tensors():
    # the binding refuses wrong dtypes, shapes and host tensors before calling the library
    import torch
    from paper_1709_03763_b300 import depth_from_u16, rgba_from_rgb
    with pytest.raises(TypeError):
        rgba_from_rgb(torch.zeros((4, 3), dtype=torch.int16))
    with pytest.raises(TypeError):
        rgba_from_rgb(torch.zeros((4, 4), dtype=torch.uint8))
    with pytest.raises(ValueError):
        rgba_from_rgb(torch.zeros((4, 3), dtype=torch.uint8))          # host tensor
    with pytest.raises(TypeError):
        depth_from_u16(torch.zeros(8, dtype=torch.float32), 0.001)
    with pytest.raises(ValueError):
        depth_from_u16(torch.zeros(8, dtype=torch.int16), 0.001)        # host tensor
