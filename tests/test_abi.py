"""The C-ABI library builds, loads without a GPU, exports every entry point
that include/*.h declares, and rejects bad arguments on the host before it
touches the device."""
import ctypes
import glob
import os
import re

import pytest

import paper_2506_23364_gb300 as awo
from paper_2506_23364_gb300 import build as awo_build

ROOT = os.path.abspath(os.path.join(os.path.dirname(__file__), ".."))


@pytest.fixture(scope="module")
def L():
    awo_build.build()
    return awo.lib()


def _declared():
    names = set()
    for hdr in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(hdr).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        names |= set(re.findall(r"\b(awo_\w+)\s*\(", text))
    return names


def test_every_declared_symbol_is_exported(L):
    names = _declared()
    assert {"awo_normals", "awo_release", "awo_simulate", "awo_overlay_lod"} <= names
    for n in sorted(names):
        assert hasattr(L, n), n


def test_struct_layouts():
    assert ctypes.sizeof(awo.Grid) == 12
    assert ctypes.sizeof(awo.SimParams) == 48
    assert awo.SimParams.seed.offset == 32


def test_status_strings_and_version(L):
    assert awo.status_string(0) == "ok"
    assert awo.status_string(1) == "invalid argument"
    assert L.awo_version() >= 10000


def test_workspace_sizes(L):
    assert awo.awo_simulate_workspace_bytes(0) >= 48
    assert awo.awo_simulate_workspace_bytes(1000) >= awo.awo_simulate_workspace_bytes(0) + 16000
    g = awo.grid(8192, 8192, 10.0)
    assert awo.awo_release_workspace_bytes(g) >= 2 * 4 * (8192 * 8192 // 4096)
    assert awo.awo_release_workspace_bytes(awo.grid(0, 5, 1.0)) == 0


@pytest.mark.parametrize("g", [(0, 5, 1.0), (5, 0, 1.0), (70000, 2, 1.0), (65536, 65536, 1.0), (4, 4, 0.0),
                               (4, 4, float("nan")), (4, 4, -1.0)])
def test_bad_grids_rejected_on_host(L, g):
    G = awo.grid(*g)
    fake = ctypes.c_void_p(16)  # never dereferenced: validation fails first
    assert L.awo_normals(fake, G, fake, fake, None, None) == awo.AWO_EINVAL
    assert L.awo_finalize(fake, G, ctypes.c_float(9.81), fake, None) == awo.AWO_EINVAL
    assert L.awo_finalize_lod(fake, fake, G, ctypes.c_float(9.81), 1, fake, None, None, None) == awo.AWO_EINVAL


def test_bad_arguments_rejected_on_host(L):
    G = awo.grid(16, 16, 10.0)
    fake = ctypes.c_void_p(256)
    assert L.awo_normals(None, G, fake, None, None, None) == awo.AWO_EINVAL
    assert L.awo_normals_u16(None, G, ctypes.c_float(0.1), fake, fake, None, None, None) == awo.AWO_EINVAL
    assert L.awo_normals_u16(fake, G, ctypes.c_float(0.1), None, fake, None, None, None) == awo.AWO_EINVAL
    assert L.awo_normals_u16(fake, G, ctypes.c_float(0.0), fake, fake, None, None, None) == awo.AWO_EINVAL
    ws = awo.awo_release_workspace_bytes(G)
    assert L.awo_release(fake, G, 40.0, 30.0, fake, fake, fake, fake, ws, None) == awo.AWO_EINVAL
    assert L.awo_release(fake, G, 30.0, 90.0, fake, fake, fake, fake, ws, None) == awo.AWO_EINVAL
    assert L.awo_release(fake, G, 30.0, 45.0, fake, fake, fake, fake, ws - 1, None) == awo.AWO_ENOMEM
    assert L.awo_release(fake, G, 30.0, 45.0, fake, fake, fake, ctypes.c_void_p(258), ws, None) == awo.AWO_EINVAL
    for kw in (dict(persistence=1.5), dict(randomness=-1.0), dict(mu=-0.1), dict(drag_k=0.2),
               dict(step_scale=0.0), dict(step_scale=2.0), dict(gravity=0.0), dict(flags=2)):
        p = awo.SimParams.make(**kw)
        assert L.awo_simulate(fake, G, fake, None, 4, ctypes.byref(p), fake, fake, None, fake, 64,
                              None) == awo.AWO_EINVAL, kw
    p = awo.SimParams.make()
    assert L.awo_simulate(fake, G, fake, None, 4, ctypes.byref(p), fake, fake, None, fake, 8,
                          None) == awo.AWO_ENOMEM
    assert L.awo_simulate(fake, G, None, None, 4, ctypes.byref(p), fake, fake, None, fake, 64,
                          None) == awo.AWO_EINVAL
    arr = (ctypes.c_void_p * 1)(fake)
    assert L.awo_overlay_lod(fake, fake, G, 0, arr, arr, None) == awo.AWO_EINVAL
    assert L.awo_overlay_lod(fake, fake, G, 17, arr, arr, None) == awo.AWO_EINVAL
    assert L.awo_overlay_lod(fake, fake, G, 2, None, None, None) == awo.AWO_EINVAL
    g98 = ctypes.c_float(9.81)
    assert L.awo_finalize_lod(fake, fake, G, g98, 0, fake, arr, arr, None) == awo.AWO_EINVAL
    assert L.awo_finalize_lod(fake, fake, G, g98, 17, fake, arr, arr, None) == awo.AWO_EINVAL
    assert L.awo_finalize_lod(fake, fake, G, g98, 2, fake, None, None, None) == awo.AWO_EINVAL
    assert L.awo_finalize_lod(fake, None, G, g98, 2, fake, arr, arr, None) == awo.AWO_EINVAL
    assert L.awo_finalize_lod(fake, fake, G, ctypes.c_float(0.0), 2, fake, arr, arr, None) == awo.AWO_EINVAL


def test_batched_structs_and_host_validation(L):
    assert ctypes.sizeof(awo.SimRequest) == 112 and awo.SimRequest.params.offset == 48
    assert ctypes.sizeof(awo.Tuning) == 16
    G = awo.grid(16, 16, 10.0)
    fake = 256
    r = awo.SimRequest(fake, G, fake, None, 4, 0, awo.SimParams.make(), fake, fake)
    arr = (awo.SimRequest * 1)(r)
    ws_need = L.awo_simulate_batched_workspace_bytes(arr, 1)
    assert ws_need >= 4 * 16
    assert L.awo_simulate_batched_workspace_bytes(arr, 0) == 0
    assert L.awo_simulate_batched(arr, 0, None, None, fake, ws_need, None) == awo.AWO_EINVAL
    assert L.awo_simulate_batched(arr, 129, None, None, fake, ws_need, None) == awo.AWO_EINVAL
    assert L.awo_simulate_batched(arr, 1, None, None, fake, ws_need - 1, None) == awo.AWO_ENOMEM
    for t in (awo.Tuning(100, 0, 0, 0), awo.Tuning(128, 16, 0, 0), awo.Tuning(128, 1024, 2, 0)):
        assert L.awo_simulate_batched(arr, 1, ctypes.byref(t), None, fake, ws_need, None) == awo.AWO_EINVAL
    bad = awo.SimRequest(fake, G, fake, None, 4, 0, awo.SimParams.make(persistence=3.0), fake, fake)
    arr2 = (awo.SimRequest * 2)(r, bad)
    assert L.awo_simulate_batched(arr2, 2, None, None, fake, 1 << 20, None) == awo.AWO_EINVAL
    best = awo.Tuning()
    assert L.awo_tune_batched(arr, 0, fake, ws_need, None, ctypes.byref(best), None) == awo.AWO_EINVAL


def test_release_texture_host_side(L):
    """Texture sizes, workspace sizes and argument checks of the release
    texture (no device work: validation fails before any launch)."""
    G = awo.grid(5, 3, 10.0)
    for r, want in ((0, (5, 3)), (1, (10, 6)), (3, (40, 24)), (-1, (3, 2)), (-3, (1, 1))):
        assert awo.awo_release_texture_dims(G, r) == want
    for r in (4, -4):
        with pytest.raises(awo.AwoError):
            awo.awo_release_texture_dims(G, r)
    with pytest.raises(awo.AwoError):
        awo.awo_release_texture_dims(awo.grid(65536, 8192, 1.0), 1)  # 2^31 texels
    g8 = awo.grid(8192, 8192, 10.0)
    assert awo.awo_release_texture_workspace_bytes(g8, 0) == awo.awo_release_workspace_bytes(g8)
    assert awo.awo_release_texture_workspace_bytes(g8, 1) >= 2 * 4 * (4 * 8192 * 8192 // 4096)
    assert awo.awo_release_texture_workspace_bytes(g8, 5) == 0
    fake = ctypes.c_void_p(256)
    G16 = awo.grid(16, 16, 10.0)
    ws = awo.awo_release_texture_workspace_bytes(G16, 2)
    assert L.awo_release_texture(fake, G16, 2, 30.0, 45.0, None, fake, fake, fake, ws, None) == awo.AWO_EINVAL
    assert L.awo_release_texture(fake, G16, 4, 30.0, 45.0, fake, fake, fake, fake, ws, None) == awo.AWO_EINVAL
    assert L.awo_release_texture(fake, G16, 2, 45.0, 30.0, fake, fake, fake, fake, ws, None) == awo.AWO_EINVAL
    assert L.awo_release_texture(fake, G16, 2, 30.0, 45.0, fake, fake, fake, fake, ws - 1, None) == awo.AWO_ENOMEM
    # particle parameters naming a texture out of range
    for r in (4, -4):
        p = awo.SimParams.make(release_log2=r)
        assert L.awo_simulate(fake, G16, fake, None, 4, ctypes.byref(p), fake, fake, None, fake, 1 << 20,
                              None) == awo.AWO_EINVAL
    # soft mode takes DEM cells only
    p = awo.SimParams.make(release_log2=1)
    assert L.awo_soft_forward(fake, G16, fake, None, 4, fake, ctypes.byref(p), ctypes.c_float(1.0), fake, None,
                              fake, 1 << 20, None) == awo.AWO_EINVAL
    assert ctypes.sizeof(awo.SimParams) == 48 and awo.SimParams.release_log2.offset == 44


def test_selftest_and_gather_path_host_validation(L):
    fake = ctypes.c_void_p(256)
    assert L.awo_selftest_rcp_sqrt(0, 1 << 32, None, None) == awo.AWO_EINVAL
    assert L.awo_selftest_rcp_sqrt(0, 1 << 32, ctypes.c_void_p(260), None) == awo.AWO_EINVAL  # misaligned
    assert L.awo_selftest_rcp_sqrt(1, 1 << 32, fake, None) == awo.AWO_EINVAL  # past 2^32
    assert L.awo_selftest_visit_cell(0, 1 << 32, None, None) == awo.AWO_EINVAL
    assert L.awo_selftest_visit_cell(5, 1 << 32, fake, None) == awo.AWO_EINVAL
    assert L.awo_selftest_div_rn(None, 4, 0, fake, None) == awo.AWO_EINVAL
    assert L.awo_selftest_div_rn(fake, 0, 0, fake, None) == awo.AWO_EINVAL  # no divisors
    assert L.awo_selftest_div_rn(ctypes.c_void_p(258), 4, 0, fake, None) == awo.AWO_EINVAL  # misaligned
    assert L.awo_selftest_div_rn(fake, 4, 0, ctypes.c_void_p(260), None) == awo.AWO_EINVAL  # misaligned
    assert L.awo_simulate_time_kernel(fake, None) == awo.AWO_EINVAL  # one event only
    assert L.awo_simulate_time_kernel(None, fake) == awo.AWO_EINVAL
    assert L.awo_simulate_time_kernel(None, None) == awo.AWO_OK  # withdraws (nothing recorded)
    assert L.awo_probe_philox(None, 4, 0, 0, fake, None) == awo.AWO_EINVAL
    assert L.awo_probe_philox(fake, 4, 0, 0, None, None) == awo.AWO_EINVAL
    assert L.awo_probe_philox(fake, -1, 0, 1, fake, None) == awo.AWO_EINVAL
    assert L.awo_probe_philox(ctypes.c_void_p(264), 4, 0, 0, fake, None) == awo.AWO_EINVAL  # misaligned
    assert L.awo_probe_philox(fake, 4, 0, 0, ctypes.c_void_p(264), None) == awo.AWO_EINVAL
    assert L.awo_probe_philox(fake, 0, 0, 0, fake, None) == awo.AWO_OK  # nothing to draw
    t = ctypes.c_int32(7)
    assert L.awo_dem_gather_path(None, awo.grid(16, 16, 10.0), None, ctypes.byref(t)) == awo.AWO_EINVAL
    assert L.awo_dem_gather_path(fake, awo.grid(0, 16, 10.0), None, ctypes.byref(t)) == awo.AWO_EINVAL
    assert L.awo_dem_gather_path(fake, awo.grid(16, 16, 10.0), None, None) == awo.AWO_EINVAL
