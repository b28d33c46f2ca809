"""The C-ABI library builds for sm_103a, loads, and exports every entry point
include/gs3.h declares (no compute call: this runs without a GPU)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "gs3.h")).read()
    return sorted(set(re.findall(r"^GS_API [^(]*?\b([a-z_0-9]+)\(", src, flags=re.M)))


def test_header_declares_the_boundary():
    names = _declared()
    for want in ("gs_project", "gs_project_bwd", "gs_bin_sort", "gs_raster_fwd", "gs_raster_bwd",
                 "gs_loss_l1_dssim", "ntc_encode_fwd", "ntc_encode_bwd", "ntc_spatial_order",
                 "ntc_spatial_order_workspace_size", "ntc_mlp_fwd",
                 "ntc_mlp_bwd", "ntc_apply", "ntc_apply_bwd", "adam_step"):
        assert want in names


def test_library_exports_every_declared_symbol():
    from paper_2403_01444_gb300 import build
    path = build.build()
    lib = ctypes.CDLL(path)
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing
    # host-only entry points are callable without a device
    lib.gs_bin_sort_workspace_size.restype = ctypes.c_size_t
    lib.gs_bin_sort_workspace_size.argtypes = [ctypes.c_int64, ctypes.c_int, ctypes.c_int,
                                               ctypes.c_int, ctypes.c_int64]
    assert lib.gs_bin_sort_workspace_size(1000, 4, 64, 48, 10000) > 0
    from paper_2403_01444_gb300 import gs3
    import oracle
    g = gs3.hashgrid()
    assert gs3.ntc_hashgrid_entries(g) == oracle.Grid().n_entries == 1647607
    assert gs3.lib().gs_version() >= 1
