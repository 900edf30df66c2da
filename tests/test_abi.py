"""Host-side checks of the C-ABI library (no GPU needed): it builds, loads, exports
every entry point include/nurbs.h declares, and its planner validates
descriptors and sizes the workspace without touching the device."""
import ctypes
import os
import re

import numpy as np
import pytest

from paper_2104_14547_gb300 import _lib, batch, synth

HEADER = os.path.join(os.path.dirname(os.path.dirname(__file__)), "include", "nurbs.h")


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(nurbs_[a-z_0-9]+)\s*\(", src)))


def test_library_exports_every_declared_symbol():
    lib = _lib.load()
    names = declared_functions()
    assert len(names) >= 15
    for name in names:
        assert hasattr(lib, name), name
    assert set(names) == set(_lib.SIGNATURES)


def _plan(kind, descs, cfg=None):
    lib = _lib.load()
    h = ctypes.c_void_p()
    d = np.ascontiguousarray(descs, dtype=batch.DESC_DTYPE)
    st = lib.nurbs_plan_create(kind, d.ctypes.data_as(ctypes.POINTER(_lib.Desc)), len(d),
                               ctypes.byref(cfg) if cfg else None, ctypes.byref(h))
    return st, h


def test_planner_tiles_and_points():
    surfs, _ = synth.bicubic_batch(0, batch=3, net=12, grid=40)
    pk = batch.pack_surfaces(surfs)
    st, h = _plan(_lib.KIND_SURFACE, pk.descs)
    assert st == 0
    lib = _lib.load()
    assert lib.nurbs_plan_points(h) == 3 * 40 * 40
    assert lib.nurbs_plan_tiles(h) >= 3
    assert lib.nurbs_plan_workspace_size(h) > 256
    # binding needs a real, aligned workspace: rejected before any CUDA call
    assert lib.nurbs_plan_bind(h, None, 0, None) == 6
    assert lib.nurbs_eval_surface(h, None, None, None, None, None) == 1
    lib.nurbs_plan_destroy(h)


def test_planner_rejects_bad_descriptors():
    s = synth.single_bicubic(0)
    pk = batch.pack_surfaces([s])
    d = pk.descs.copy()
    d["p"] = 0
    assert _plan(_lib.KIND_SURFACE, d)[0] == 3          # degree
    d = pk.descs.copy()
    d["p"] = 6
    assert _plan(_lib.KIND_SURFACE, d)[0] == 3
    d = pk.descs.copy()
    d["n1"] = 3                                          # fewer than p+1 control points
    assert _plan(_lib.KIND_SURFACE, d)[0] == 3
    d = pk.descs.copy()
    d["nu"] = -1
    assert _plan(_lib.KIND_SURFACE, d)[0] == 1
    assert _plan(7, pk.descs)[0] == 1                    # kind
    for bad in (-1.0, float("nan"), float("inf")):        # an item's own loss scale
        d = pk.descs.copy()
        d["grad_scale"] = bad
        assert _plan(_lib.KIND_SURFACE, d)[0] == 1
    d = pk.descs.copy()
    d["grad_scale"] = 1e-4
    assert _plan(_lib.KIND_SURFACE, d)[0] == 0
    cfg = _lib.TileCfg(0, 9, 0, 0)                       # more warps than the kernels allow
    assert _plan(_lib.KIND_SURFACE, pk.descs, cfg)[0] == 1
    cfg = _lib.TileCfg(0, 8, 0, -1)                      # negative CTA cap
    assert _plan(_lib.KIND_SURFACE, pk.descs, cfg)[0] == 1


def test_curve_plan_and_empty_items():
    rng = np.random.default_rng(0)
    cs = [synth.curve(rng, 3, 20, n) for n in (0, 1, 300, 1025)]
    pk = batch.pack_curves(cs)
    st, h = _plan(_lib.KIND_CURVE, pk.descs)
    assert st == 0
    lib = _lib.load()
    assert lib.nurbs_plan_points(h) == 0 + 1 + 300 + 1025
    # a curve plan refuses the surface entry point
    assert lib.nurbs_plan_tiles(h) >= 4
    lib.nurbs_plan_destroy(h)


def test_status_strings():
    lib = _lib.load()
    for k in range(10):
        assert lib.nurbs_status_string(k).decode()


def test_knot_sigma_setter_validates():
    s = synth.single_bicubic(0)
    pk = batch.pack_surfaces([s])
    st, h = _plan(_lib.KIND_SURFACE, pk.descs)
    assert st == 0
    lib = _lib.load()
    assert lib.nurbs_plan_set_knot_sigma(h, 0.0) == 0
    assert lib.nurbs_plan_set_knot_sigma(h, 1e-3) == 0
    assert lib.nurbs_plan_set_knot_sigma(h, -1e-3) == 1
    assert lib.nurbs_plan_set_knot_sigma(h, float("nan")) == 1
    assert lib.nurbs_plan_set_knot_sigma(h, float("inf")) == 1
    assert lib.nurbs_plan_set_knot_sigma(None, 1e-3) == 1
    lib.nurbs_plan_destroy(h)


def test_grad_homogeneous_setter_validates():
    s = synth.single_bicubic(0)
    pk = batch.pack_surfaces([s])
    st, h = _plan(_lib.KIND_SURFACE, pk.descs)
    assert st == 0
    lib = _lib.load()
    assert lib.nurbs_plan_set_grad_homogeneous(h, 1) == 0
    assert lib.nurbs_plan_set_grad_homogeneous(h, 0) == 0
    assert lib.nurbs_plan_set_grad_homogeneous(h, 2) == 1
    assert lib.nurbs_plan_set_grad_homogeneous(h, -1) == 1
    assert lib.nurbs_plan_set_grad_homogeneous(None, 1) == 1
    lib.nurbs_plan_destroy(h)


def test_occupancy_query_validates_arguments():
    # argument errors are found before any device query
    s = synth.single_bicubic(0)
    pk = batch.pack_surfaces([s])
    st, h = _plan(_lib.KIND_SURFACE, pk.descs)
    assert st == 0
    lib = _lib.load()
    occ = ctypes.c_int32(0)
    assert lib.nurbs_plan_occupancy(None, 4, ctypes.byref(occ), None) == 1
    assert lib.nurbs_plan_occupancy(h, 6, ctypes.byref(occ), None) == 1
    assert lib.nurbs_plan_occupancy(h, -1, ctypes.byref(occ), None) == 1
    assert lib.nurbs_plan_occupancy(h, 4, None, None) == 1
    lib.nurbs_plan_destroy(h)


@pytest.mark.parametrize("warps,rows", [(8, 0), (8, 128), (4, 32), (2, 7), (1, 0), (6, 50)])
def test_planner_tile_count_follows_the_tiling_rule(warps, rows):
    # a surface is cut into column tiles of at most 32 * warps samples (equal widths,
    # rounded up to whole warps) and row tiles of `rows` samples (default: 16 rows per
    # row group of warps); a curve on the curve kernels is one tile; longer curves are
    # single-row surfaces
    rng = np.random.default_rng(5)
    shapes = [(40, 40), (1, 1), (0, 10), (10, 0), (129, 300), (513, 257), (64, 1000)]
    surfs = [synth.surface(rng, 3, 2, 6, 7, nu, nv) for nu, nv in shapes]
    pk = batch.pack_surfaces(surfs)
    st, h = _plan(_lib.KIND_SURFACE, pk.descs, _lib.TileCfg(rows, warps, 0, 0))
    assert st == 0
    want = 0
    for nu, nv in shapes:
        nct = max(1, -(-nv // (32 * warps)))
        width = -(-(-(-nv // nct)) // 32) * 32 if nv > 0 else 32
        groups = max(1, warps // max(1, min(warps, width // 32)))
        R = rows if rows > 0 else 16 * groups
        want += max(1, -(-nu // R)) * nct
    lib = _lib.load()
    assert lib.nurbs_plan_tiles(h) == want
    lib.nurbs_plan_destroy(h)
    curves = [synth.curve(rng, 3, n1, ns, knots="uniform") for n1, ns in ((20, 100), (256, 7), (257, 700), (400, 0))]
    ck = batch.pack_curves(curves)
    st, h = _plan(_lib.KIND_CURVE, ck.descs, _lib.TileCfg(rows, warps, 0, 0))
    assert st == 0
    want = 2 + sum(max(1, -(-ns // (32 * warps))) for ns in (700, 0))
    assert lib.nurbs_plan_tiles(h) == want
    lib.nurbs_plan_destroy(h)


def test_build_compiles_every_tile_kernel_once():
    # k_tiles.cu is compiled once per (u degree, variant) pair; every other .cu once
    jobs = _lib._jobs()
    tiles = sorted(tuple(x for x in extra) for src, _, extra in jobs if src.endswith("k_tiles.cu"))
    assert tiles == sorted((f"-DNURBS_P={p}", f"-DNURBS_V={v}") for p in range(6) for v in range(6))
    objs = [o for _, o, _ in jobs]
    assert len(objs) == len(set(objs))
    others = {os.path.basename(src) for src, _, extra in jobs if not extra}
    cu = {f for f in os.listdir(os.path.dirname(jobs[0][0])) if f.endswith(".cu")} - {"k_tiles.cu"}
    assert others == cu
