"""Build and load ``libnurbs`` (the C-ABI declared in include/nurbs.h).

The library is compiled in-tree with nvcc for sm_103a into
``paper_2104_14547_gb300/_build/libnurbs.so`` and loaded with ctypes.  There is no
fallback: if the library cannot be built or loaded, every entry point raises.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import tempfile
import threading
import time

_PKG = os.path.dirname(os.path.abspath(__file__))
_ROOT = os.path.dirname(_PKG)
_CSRC = os.path.join(_PKG, "csrc")
_BUILD = os.path.join(_PKG, "_build")
SO_PATH = os.path.join(_BUILD, "libnurbs.so")
HEADER = os.path.join(_ROOT, "include", "nurbs.h")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "--expt-relaxed-constexpr"]

_lock = threading.Lock()
_lib = None


def _nvcc() -> str:
    home = os.environ.get("CUDA_HOME", "/usr/local/cuda")
    cand = os.path.join(home, "bin", "nvcc")
    return cand if os.path.exists(cand) else "nvcc"


def _jobs():
    """(source, object, extra flags) per translation unit: k_tiles.cu once per
    (u degree, variant) pair, every other .cu once."""
    jobs = []
    for f in sorted(os.listdir(_CSRC)):
        if not f.endswith(".cu"):
            continue
        src = os.path.join(_CSRC, f)
        if f == "k_tiles.cu":
            for p in range(6):
                for v in range(6):
                    jobs.append((src, os.path.join(_BUILD, f"k_tiles_p{p}_v{v}.o"),
                                 [f"-DNURBS_P={p}", f"-DNURBS_V={v}"]))
        else:
            jobs.append((src, os.path.join(_BUILD, f[:-3] + ".o"), []))
    return jobs


def _deps():
    return [os.path.join(_CSRC, f) for f in os.listdir(_CSRC)] + [HEADER]


def build(force: bool = False, verbose: bool = False) -> str:
    """Compile every .cu under csrc/ (in parallel) and link libnurbs.so."""
    os.makedirs(_BUILD, exist_ok=True)
    newest = max(os.path.getmtime(p) for p in _deps())
    if not force and os.path.exists(SO_PATH) and os.path.getmtime(SO_PATH) >= newest:
        return SO_PATH
    nvcc = _nvcc()
    # at most one nvcc per core, the tile kernels (the longest jobs) first
    jobs = sorted(_jobs(), key=lambda j: "k_tiles" not in j[0])
    objs = [o for _, o, _ in jobs]
    pending = list(jobs)
    running, errors = [], []
    ncpu = max(1, os.cpu_count() or 1)
    while pending or running:
        while pending and len(running) < ncpu:
            src, obj, extra = pending.pop(0)
            cmd = [nvcc, *ARCH, *NVCC_FLAGS, *extra, "-c", src, "-o", obj]
            log = tempfile.TemporaryFile()
            running.append((cmd, log, subprocess.Popen(cmd, stdout=log, stderr=subprocess.STDOUT)))
        done = [r for r in running if r[2].poll() is not None]
        if not done:
            time.sleep(0.05)
            continue
        for r in done:
            running.remove(r)
            cmd, log, p = r
            log.seek(0)
            out = log.read()
            log.close()
            if verbose and out:
                print(out.decode(errors="replace"))
            if p.returncode != 0:
                errors.append(" ".join(cmd) + "\n" + out.decode(errors="replace"))
    if errors:
        raise RuntimeError("libnurbs build failed:\n" + "\n".join(errors))
    cudalib = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "lib64")
    tmp = SO_PATH + f".tmp{os.getpid()}"
    subprocess.check_call([nvcc, *ARCH, "-shared", "-cudart", "shared", "-o", tmp, *objs,
                           "-Xlinker", f"-rpath,{cudalib}"])
    os.replace(tmp, SO_PATH)
    return SO_PATH


class NurbsError(RuntimeError):
    def __init__(self, status: int, what: str):
        self.status = status
        super().__init__(f"{what}: {status_string(status)} (status {status})")


# ----------------------------------------------------------------- ctypes types
class Desc(ctypes.Structure):
    _fields_ = [("p", ctypes.c_int32), ("q", ctypes.c_int32), ("n1", ctypes.c_int32), ("m1", ctypes.c_int32),
                ("nu", ctypes.c_int32), ("nv", ctypes.c_int32), ("adam_step", ctypes.c_int32),
                ("grad_scale", ctypes.c_float), ("knot_u", ctypes.c_int64), ("knot_v", ctypes.c_int64),
                ("ctrl", ctypes.c_int64), ("param_u", ctypes.c_int64), ("param_v", ctypes.c_int64),
                ("pts", ctypes.c_int64)]


class TileCfg(ctypes.Structure):
    _fields_ = [("rows", ctypes.c_int32), ("warps", ctypes.c_int32), ("ctas_per_sm", ctypes.c_int32),
                ("max_ctas", ctypes.c_int32)]


class Adam(ctypes.Structure):
    _fields_ = [("lr", ctypes.c_float), ("beta1", ctypes.c_float), ("beta2", ctypes.c_float), ("eps", ctypes.c_float)]


KIND_SURFACE, KIND_CURVE = 0, 1
ERR_SIZE = 8   # NURBS_ERR_SIZE: an item or tile shape exceeds a kernel limit

# every function the header declares, with its ctypes signature
_vp, _f, _i32, _i64, _sz = ctypes.c_void_p, ctypes.c_float, ctypes.c_int32, ctypes.c_int64, ctypes.c_size_t
SIGNATURES = {
    "nurbs_plan_create": (_i32, [_i32, ctypes.POINTER(Desc), _i32, ctypes.POINTER(TileCfg), ctypes.POINTER(_vp)]),
    "nurbs_plan_workspace_size": (_sz, [_vp]),
    "nurbs_plan_points": (_i64, [_vp]),
    "nurbs_plan_tiles": (_i32, [_vp]),
    "nurbs_plan_ctas": (_i32, [_vp]),
    "nurbs_plan_occupancy": (_i32, [_vp, _i32, ctypes.POINTER(_i32), ctypes.POINTER(_i32)]),
    "nurbs_plan_set_knot_sigma": (_i32, [_vp, _f]),
    "nurbs_plan_set_grad_homogeneous": (_i32, [_vp, _i32]),
    "nurbs_plan_bind": (_i32, [_vp, _vp, _sz, _vp]),
    "nurbs_plan_destroy": (None, [_vp]),
    "nurbs_plan_get_error": (_i32, [_vp, _vp, ctypes.POINTER(ctypes.c_uint32)]),
    "nurbs_eval_surface": (_i32, [_vp, _vp, _vp, _vp, _vp, _vp]),
    "nurbs_eval_curve": (_i32, [_vp, _vp, _vp, _vp, _vp, _vp]),
    "nurbs_eval_surface_derivs": (_i32, [_vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp]),
    "nurbs_eval_curve_derivs": (_i32, [_vp, _vp, _vp, _vp, _vp, _vp, _vp]),
    "nurbs_backward": (_i32, [_vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp]),
    "nurbs_mse_fwd_bwd": (_i32, [_vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _f, _vp]),
    "nurbs_mse_fwd_bwd_noalloc": (_i32, [_vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _f, _vp]),
    "nurbs_noalloc_get_error": (_i32, [_vp, ctypes.POINTER(ctypes.c_uint32)]),
    "nurbs_fit_step": (_i32, [_vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp, ctypes.POINTER(Adam), _i32, _f, _vp, _vp, _vp]),
    "nurbs_chamfer": (_i32, [_i32, _vp, _vp, _i32, _i32, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp,
                             _i64, _i64, _vp]),
    "nurbs_status_string": (ctypes.c_char_p, [_i32]),
    "nurbs_last_cuda_error": (_i32, []),
}


def load(build_if_missing: bool = True):
    """Load libnurbs (building it first if needed).  Raises if that fails."""
    global _lib
    with _lock:
        if _lib is None:
            if build_if_missing:
                build()
            if not os.path.exists(SO_PATH):
                raise RuntimeError(f"libnurbs not built: {SO_PATH} is missing")
            lib = ctypes.CDLL(SO_PATH)
            for name, (res, args) in SIGNATURES.items():
                fn = getattr(lib, name)
                fn.restype = res
                fn.argtypes = args
            _lib = lib
    return _lib


def status_string(status: int) -> str:
    try:
        return load(build_if_missing=False).nurbs_status_string(status).decode()
    except Exception:  # pragma: no cover - library not loadable
        return "unknown"


def check(status: int, what: str) -> None:
    if status != 0:
        if status == 7:
            raise NurbsError(status, f"{what} (cuda error {load().nurbs_last_cuda_error()})")
        raise NurbsError(status, what)
