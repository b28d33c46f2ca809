"""Synchronous argument errors of the C-ABI boundary: a call with a bad
argument returns GS_ERR_INVALID_ARG before anything is launched and leaves a
message for gs_last_error.  Every call here fails its argument check before
any device work, so no GPU is needed; the pointers are never dereferenced."""
from ctypes import byref, c_float, c_int64, c_size_t, c_void_p

import pytest

from paper_2403_01444_gb300 import build, gs3

FAKE = c_void_p(0x10000)   # a 16-byte aligned address no call below reaches


@pytest.fixture(scope="module")
def L():
    build.build()
    return gs3.lib()


def _fails(L, status, *words):
    assert status == gs3.GS_ERR_INVALID_ARG
    msg = L.gs_last_error().decode()
    for w in words:
        assert w in msg, msg


def _gauss(n=10, deg=1):
    return gs3.GsGaussians(FAKE, FAKE, FAKE, FAKE, FAKE, n, deg)


def _proj():
    return gs3.GsProjected(FAKE, FAKE, FAKE, FAKE, FAKE, FAKE)


def test_projection_rejects_bad_arguments(L):
    g, out = _gauss(), _proj()
    _fails(L, L.gs_project(None, FAKE, 1, 64, 48, byref(out), None, None), "gs_project", "null")
    _fails(L, L.gs_project(byref(g), FAKE, 0, 64, 48, byref(out), None, None), "V must be")
    _fails(L, L.gs_project(byref(g), FAKE, 65, 64, 48, byref(out), None, None), "V must be")   # GS_MAX_VIEWS + 1
    _fails(L, L.gs_project(byref(g), FAKE, 1, 0, 48, byref(out), None, None), "image size")
    _fails(L, L.gs_project(byref(_gauss(deg=4)), FAKE, 1, 64, 48, byref(out), None, None), "sh_deg")
    _fails(L, L.gs_project(byref(_gauss(n=-1)), FAKE, 1, 64, 48, byref(out), None, None), "n out of range")
    misaligned = gs3.GsGaussians(FAKE, c_void_p(0x10004), FAKE, FAKE, FAKE, 10, 1)
    _fails(L, L.gs_project(byref(misaligned), FAKE, 1, 64, 48, byref(out), None, None), "aligned")


def test_binning_and_compositing_reject_bad_arguments(L):
    p = _proj()
    # bins outside 1..64 tiles
    _fails(L, L.gs_bin_sort(byref(p), c_int64(10), 1, 64, 48, 0, c_int64(100), FAKE, FAKE, None,
                            FAKE, FAKE, FAKE, c_size_t(1 << 20), None), "bin")
    _fails(L, L.gs_raster_fwd(byref(p), c_int64(10), 1, 64, 48, 65, None, FAKE, FAKE, FAKE, FAKE,
                              FAKE, None, None, None), "bin")
    # views outside 1..GS_MAX_VIEWS, image too large
    _fails(L, L.gs_raster_fwd(byref(p), c_int64(10), 0, 64, 48, 1, None, FAKE, FAKE, FAKE, FAKE,
                              FAKE, None, None, None), "bad n or V")
    _fails(L, L.gs_raster_fwd(byref(p), c_int64(10), 1, 20000, 48, 1, None, FAKE, FAKE, FAKE, FAKE,
                              FAKE, None, None, None), "image size")


def test_compositing_rejects_bad_tile_lists(L):
    p = _proj()
    for lists, words in ((gs3.GsTileLists(FAKE, FAKE, 0), "cap"), (gs3.GsTileLists(None, FAKE, 16), "rec"),
                         (gs3.GsTileLists(c_void_p(0x10004), FAKE, 16), "misaligned")):
        _fails(L, L.gs_raster_fwd(byref(p), c_int64(10), 1, 64, 48, 1, None, FAKE, FAKE, FAKE, FAKE,
                                  FAKE, None, byref(lists), None), words)
        _fails(L, L.gs_raster_bwd(byref(p), c_int64(10), 1, 64, 48, 1, None, FAKE, FAKE, FAKE, FAKE,
                                  FAKE, FAKE, None, None, byref(lists), None), words)


def test_binning_rejects_wrapping_entry_counts(L):
    """n is bounded before n * V is formed: n = 2^62 Gaussians in 4 views would
    wrap the 64-bit product to 0 and pass a check made on the product."""
    p = _proj()
    n = c_int64(1 << 62)
    L.gs_bin_sort_workspace_size.restype = c_size_t
    assert L.gs_bin_sort_workspace_size(n, 4, 64, 48, c_int64(100)) == 0
    assert L.gs_bin_sort_workspace_size(c_int64(1000), 4, 64, 48, c_int64(100)) > 0
    _fails(L, L.gs_bin_sort(byref(p), n, 4, 64, 48, 1, c_int64(100), FAKE, FAKE, None,
                            FAKE, FAKE, FAKE, c_size_t(1 << 20), None), "32 bits")
    _fails(L, L.gs_bin_sort_noalloc(byref(p), n, 4, 64, 48, 1, c_int64(100), FAKE, FAKE, None,
                                    FAKE, FAKE, None), "built-in limit")
    _fails(L, L.gs_bin_sort_noalloc(byref(p), c_int64(32769), 4, 64, 48, 1, c_int64(100), FAKE, FAKE,
                                    None, FAKE, FAKE, None), "built-in limit")


def test_loss_rejects_bad_shapes_and_small_workspaces(L):
    L.gs_loss_workspace_size.restype = c_size_t
    need = L.gs_loss_workspace_size(3, 48, 64)
    assert need > 0
    _fails(L, L.gs_loss_l1_dssim(FAKE, FAKE, 0, 48, 64, c_float(0.2), FAKE, FAKE, None, FAKE,
                                 c_size_t(need), None), "bad shape")
    _fails(L, L.gs_loss_l1_dssim(FAKE, FAKE, 3, 48, 64, c_float(0.2), FAKE, FAKE, None, FAKE,
                                 c_size_t(need - 1), None), "workspace too small")
    _fails(L, L.gs_loss_l1_dssim(FAKE, FAKE, 3, 48, 64, c_float(0.2), FAKE, FAKE, None,
                                 c_void_p(0x10010), c_size_t(need), None), "256-byte aligned")


def test_cache_and_optimiser_reject_bad_arguments(L):
    bad_grid = gs3.hashgrid()
    bad_grid.levels = 0
    _fails(L, L.ntc_encode_fwd(FAKE, c_int64(10), byref(bad_grid), FAKE, gs3.GS_F16, FAKE,
                               gs3.GS_F32, None, None), "invalid hash grid")
    good = gs3.hashgrid()
    _fails(L, L.ntc_encode_fwd(FAKE, c_int64(10), byref(good), FAKE, gs3.GS_BF16, FAKE, gs3.GS_F32,
                               None, None), "table dtype")
    _fails(L, L.adam_step(FAKE, FAKE, FAKE, FAKE, c_int64(16), None, FAKE, None, gs3.GS_NONE, None),
           "adam_step")
    _fails(L, L.gs_sh_rotate(FAKE, FAKE, FAKE, c_int64(10), 4, FAKE, None), "sh_deg")
    # empty inputs are valid and do nothing (no device work either)
    assert L.gs_sh_rotate(FAKE, FAKE, FAKE, c_int64(0), 3, FAKE, None) == gs3.GS_OK
    assert L.ntc_encode_fwd(None, c_int64(0), byref(good), None, gs3.GS_F16, None, gs3.GS_F32,
                            None, None) == gs3.GS_OK
    L.ntc_spatial_order_workspace_size.restype = c_size_t
    assert L.ntc_spatial_order_workspace_size(c_int64(-1)) == 0
    need = L.ntc_spatial_order_workspace_size(c_int64(1000))
    assert need > 0
    _fails(L, L.ntc_spatial_order(FAKE, c_int64(1000), byref(good), FAKE, FAKE, c_size_t(need - 1), None),
           "workspace too small")
    _fails(L, L.ntc_spatial_order(FAKE, c_int64(1000), byref(bad_grid), FAKE, FAKE, c_size_t(need), None),
           "invalid hash grid")
    # the reverse over a list of active rows: the count goes with its list
    _fails(L, L.ntc_encode_bwd(FAKE, c_int64(10), byref(good), FAKE, FAKE, None, FAKE, None),
           "a count needs its row list")
    _fails(L, L.ntc_active_rows(FAKE, c_int64(-1), FAKE, FAKE, None), "n out of range")
    _fails(L, L.ntc_active_rows(FAKE, c_int64(10), FAKE, None, None), "null count")
    _fails(L, L.ntc_active_rows(None, c_int64(10), FAKE, FAKE, None), "null argument")
    mlp = gs3.GsMlp(gs3.GS_MLP_BF16, FAKE, FAKE)
    _fails(L, L.ntc_mlp_bwd(FAKE, gs3.GS_BF16, c_int64(10), byref(mlp), FAKE, None, FAKE, FAKE, FAKE, None, None),
           "rows and d_rows go together")
