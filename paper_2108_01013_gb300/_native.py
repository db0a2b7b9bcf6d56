"""Build and load libdss.so (the C ABI of include/dss.h) through ctypes.

The library is compiled in-tree for sm_103a with nvcc.  Nothing here computes
anything: it declares the C structs and function signatures and marshals
pointers.  Importing the package never falls back to another implementation:
a missing or unloadable library raises.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from concurrent.futures import ThreadPoolExecutor
from ctypes import POINTER, Structure, c_char_p, c_double, c_int, c_int32, c_int64, c_size_t, c_void_p

_HERE = os.path.dirname(os.path.abspath(__file__))
_CSRC = os.path.join(_HERE, "csrc")
_BUILD = os.path.join(_HERE, "_build")
LIB_PATH = os.path.join(_BUILD, "libdss.so")
INCLUDE = os.path.join(os.path.dirname(_HERE), "include")
SOURCES = ["dss_sort.cu", "dss_neighbour.cu", "dss_force.cu", "dss_api.cu", "dss_noalloc.cu",
           "dss_adjoint.cu", "dss_analysis.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xptxas", "-v"]


def _nvcc() -> str:
    cand = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "bin", "nvcc")
    return cand if os.path.exists(cand) else "nvcc"


def _deps():
    files = [os.path.join(_CSRC, f) for f in os.listdir(_CSRC) if f.endswith((".cu", ".cuh"))]
    files.append(os.path.join(INCLUDE, "dss.h"))
    return files


def build(force: bool = False, verbose: bool = False) -> str:
    """Compile every translation unit in parallel and link libdss.so."""
    os.makedirs(_BUILD, exist_ok=True)
    if not force and os.path.exists(LIB_PATH):
        t = os.path.getmtime(LIB_PATH)
        if all(os.path.getmtime(f) <= t for f in _deps()):
            return LIB_PATH
    nvcc = _nvcc()
    objs = []

    def compile_one(src):
        obj = os.path.join(_BUILD, src.replace(".cu", ".o"))
        cmd = [nvcc, *ARCH, *NVCC_FLAGS, "-I", INCLUDE, "-c", os.path.join(_CSRC, src), "-o", obj]
        res = subprocess.run(cmd, capture_output=True, text=True)
        if res.returncode != 0:
            raise RuntimeError("nvcc failed for %s:\n%s" % (src, res.stderr))
        return obj, res.stderr

    with ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        for obj, log in ex.map(compile_one, SOURCES):
            objs.append(obj)
            if verbose:
                print(log)
    tmp = LIB_PATH + ".tmp%d" % os.getpid()
    cmd = [nvcc, *ARCH, "-shared", "-o", tmp, *objs, "-lcudart"]
    res = subprocess.run(cmd, capture_output=True, text=True)
    if res.returncode != 0:
        raise RuntimeError("nvcc link failed:\n" + res.stderr)
    os.replace(tmp, LIB_PATH)
    return LIB_PATH


class Params(Structure):
    """Mirror of ``dss_params``."""
    _fields_ = [("kn", c_double), ("kt", c_double), ("gamma_n", c_double), ("mu", c_double),
                ("eta0", c_double), ("rho", c_double), ("delta_lub", c_double),
                ("lub_eps", c_double), ("a0", c_double), ("lub_cutoff_mode", c_int32),
                ("precision", c_int32), ("shear_rate", c_double), ("dt", c_double),
                ("cell_size", c_double), ("capacity_M", c_int32), ("pair_capacity", c_int32),
                ("lub_taper", c_double), ("cell_mode", c_int32), ("reserved_", c_int32),
                ("f_er", c_double), ("lambda_d", c_double), ("hamaker", c_double),
                ("vdw_eps", c_double), ("wave_amp", c_double), ("k_r", c_double),
                ("wave_n", c_int32), ("reserved2_", c_int32)]


class Counters(Structure):
    """Mirror of ``dss_counters``."""
    _fields_ = [("steps_done", c_int64), ("nstep", c_int64), ("npairs", c_int64),
                ("ncontacts", c_int64), ("max_row", c_int64), ("band_checks", c_int64),
                ("M", c_int32), ("pad_", c_int32), ("ncell", c_int64 * 3)]


FP64, MIXED = 0, 1
PROF_KERNELS = 7
BATCH_MIN_N = 256
ERRORS = {0: "DSS_OK", -1: "DSS_ERR_ARG", -2: "DSS_ERR_BOX", -3: "DSS_ERR_CAPACITY",
          -4: "DSS_ERR_NONFINITE", -5: "DSS_ERR_UNSTABLE", -6: "DSS_ERR_CUDA",
          -7: "DSS_ERR_TIMEOUT", -8: "DSS_ERR_STATE", -9: "DSS_ERR_INTERNAL",
          -10: "DSS_ERR_SCRATCH_LIMIT", -11: "DSS_ERR_NOMEM"}

# every symbol include/dss.h declares, with (restype, argtypes)
_dp, _ip, _lp, _vp = POINTER(c_double), POINTER(c_int32), POINTER(c_int64), c_void_p
SIGNATURES = {
    "dss_capacity_estimate": (c_int32, [c_double, c_double, c_double]),
    "dss_create": (c_int, [POINTER(c_void_p), POINTER(Params), c_int64, _dp, c_void_p]),
    "dss_batch_create": (c_int, [POINTER(c_void_p), POINTER(Params), c_int32, _lp, _dp, _dp, _dp,
                                 c_void_p]),
    "dss_batch_size": (c_int32, [c_void_p]),
    "dss_batch_stress": (c_int, [c_void_p, _vp, _vp, _lp, c_int]),
    "dss_save": (c_int, [c_void_p, _vp, POINTER(c_size_t)]),
    "dss_load": (c_int, [c_void_p, _vp, c_size_t]),
    "dss_autotune": (c_int, [c_void_p, c_int32, c_int32, _dp, _dp, _dp]),
    "dss_autotune_kernels": (c_int, [c_void_p, c_int32, _dp, _ip]),
    "dss_selftest_bounded_wait": (c_int, [c_void_p]),
    "dss_selftest_conversions": (c_int, [_vp, c_int64, c_double, _vp, _vp, _vp, _vp, _vp, _vp, _vp,
                                         c_void_p]),
    "dss_rheology": (c_int, [c_void_p, c_int, _vp]),
    "dss_get_images": (c_int, [c_void_p, _vp]),
    "dss_dispersion_mark": (c_int, [c_void_p]),
    "dss_dispersion": (c_int, [c_void_p, _vp]),
    "dss_contact_clusters": (c_int, [c_void_p, _vp, _lp]),
    "dss_phi_profile": (c_int, [c_void_p, c_int32, c_double, _vp]),
    "dss_adjoint": (c_int, [c_void_p, c_int64, c_int32, _vp, c_int32, _dp, _dp, _vp, _vp, _vp, _vp, _vp]),
    "dss_set_state": (c_int, [c_void_p, _vp, _vp, _vp, _vp, _vp, _vp, _vp, c_int64]),
    "dss_get_state": (c_int, [c_void_p, _vp, _vp, _vp, _vp, _vp]),
    "dss_set_history": (c_int, [c_void_p, c_int64, _vp, _vp]),
    "dss_get_history": (c_int, [c_void_p, _vp, _vp, c_int64, _lp]),
    "dss_set_history_rolling": (c_int, [c_void_p, c_int64, _vp, _vp, _vp]),
    "dss_get_history_rolling": (c_int, [c_void_p, _vp, _vp, _vp, c_int64, _lp]),
    "dss_neighbour_build": (c_int, [c_void_p]),
    "dss_get_pairs": (c_int, [c_void_p, _vp, c_int64, _lp]),
    "dss_force_eval": (c_int, [c_void_p, _vp, _vp]),
    "dss_step": (c_int, [c_void_p, c_int64]),
    "dss_stress": (c_int, [c_void_p, _dp]),
    "dss_get_counters": (c_int, [c_void_p, POINTER(Counters)]),
    "dss_load_state": (c_int, [c_void_p, _vp, _vp, _vp, _vp, _vp]),
    "dss_step_io": (c_int, [c_void_p, POINTER(c_void_p), c_int64, POINTER(c_void_p), _vp]),
    "dss_set_profiling": (c_int, [c_void_p, c_int]),
    "dss_get_profile": (c_int, [c_void_p, _dp, _lp]),
    "dss_profile_name": (c_char_p, [c_int]),
    "dss_last_step_ms": (c_int, [c_void_p, _dp]),
    "dss_device_bytes": (c_int64, [c_void_p]),
    "dss_destroy": (None, [c_void_p]),
    "dss_strerror": (c_char_p, [c_int]),
    "dss_pairs_noalloc": (c_int, [_vp, _vp, _vp, c_int64, _dp, POINTER(Params), c_double, c_int64,
                                  _vp, c_int64, _lp, c_void_p]),
}

_lib = None


def load(path: str | None = None):
    """Load libdss.so and declare its signatures (raises when missing)."""
    global _lib
    if _lib is None:
        p = path or LIB_PATH
        if not os.path.exists(p):
            raise RuntimeError("libdss.so is not built: run __graft_entry__.build() "
                               "(or paper_2108_01013_gb300.build())")
        lib = ctypes.CDLL(p)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
    return _lib


class DssError(RuntimeError):
    def __init__(self, code: int, where: str):
        self.code = code
        msg = load().dss_strerror(code).decode()
        super().__init__("%s: %s (%s)" % (where, ERRORS.get(code, code), msg))


def check(code: int, where: str) -> None:
    if code != 0:
        raise DssError(code, where)
