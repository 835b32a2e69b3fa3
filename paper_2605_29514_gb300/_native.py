"""Build and load the native library (libstn.so, sm_103a) and declare its C ABI
(include/stn.h) for ctypes.  Argument marshalling only: every step of the
simulation runs in the library's kernels."""

import ctypes
import os
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(ROOT, "_build")
LIB = os.path.join(PKG, "libstn.so")
SOURCES = ["engine_f32.cu", "engine_f64.cu", "engine.cu", "engine_noalloc.cu", "peaks.cu", "tc_gemm.cu",
           "program.cpp", "api.cpp"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC = os.environ.get("NVCC", "/usr/local/cuda/bin/nvcc")


def _compile(src):
    obj = os.path.join(BUILD, os.path.splitext(src)[0] + ".o")
    cmd = [NVCC, *ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-I", INCLUDE,
           "-c", os.path.join(CSRC, src), "-o", obj]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed for {src}:\n{r.stderr}")
    return obj


def build(force=False):
    """Compile the CUDA sources for sm_103a and link libstn.so in the package."""
    srcs = [os.path.join(CSRC, s) for s in SOURCES] + [os.path.join(INCLUDE, "stn.h")]
    srcs += [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".h", ".cuh"))]
    if not force and os.path.exists(LIB):
        newest = max(os.path.getmtime(s) for s in srcs)
        if os.path.getmtime(LIB) >= newest:
            return LIB
    os.makedirs(BUILD, exist_ok=True)
    with ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        objs = list(ex.map(_compile, SOURCES))
    tmp = LIB + ".tmp"
    cmd = [NVCC, *ARCH, "-shared", "-o", tmp, *objs, "-lcudart"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stderr}")
    os.replace(tmp, LIB)
    return LIB


class Config(ctypes.Structure):
    _fields_ = [
        ("distance", ctypes.c_int32),
        ("rounds", ctypes.c_int32),
        ("pair_rule", ctypes.c_int32),
        ("chi_cap", ctypes.c_int32),
        ("p", ctypes.c_double),
        ("p1_scale", ctypes.c_double),
        ("p2_scale", ctypes.c_double),
        ("pR_scale", ctypes.c_double),
        ("pM_scale", ctypes.c_double),
        ("svd_cutoff", ctypes.c_double),
        ("degeneracy_tol", ctypes.c_double),
        ("precision", ctypes.c_int32),
        ("seed", ctypes.c_uint64),
        ("memory_basis", ctypes.c_int32),
        ("n_pairs", ctypes.c_int32),
        ("cnot_schedule", ctypes.c_void_p),
        ("pairs", ctypes.c_void_p),
        ("pair_pauli", ctypes.c_void_p),
        ("pair_layer_mask", ctypes.c_void_p),
        ("arena_cap_bytes", ctypes.c_int64),
        ("gemm_units", ctypes.c_int32),
    ]


class ShotStats(ctypes.Structure):
    _fields_ = [
        ("max_chi", ctypes.c_int32),
        ("near_draws", ctypes.c_int32),
        ("discarded", ctypes.c_double),
        ("logp", ctypes.c_double),
    ]


EXPORTS = [
    # name, restype, argtypes
    ("stn_create", ctypes.c_int, [ctypes.POINTER(Config), ctypes.c_int64, ctypes.c_void_p,
                                  ctypes.POINTER(ctypes.c_void_p)]),
    ("stn_destroy", None, [ctypes.c_void_p]),
    ("stn_layout", ctypes.c_int32, [ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p]),
    ("stn_last_error", ctypes.c_char_p, [ctypes.c_void_p]),
    ("stn_num_qubits", ctypes.c_int32, [ctypes.c_void_p]),
    ("stn_num_pairs", ctypes.c_int32, [ctypes.c_void_p]),
    ("stn_num_meas", ctypes.c_int32, [ctypes.c_void_p]),
    ("stn_num_events", ctypes.c_int32, [ctypes.c_void_p]),
    ("stn_num_ops", ctypes.c_int32, [ctypes.c_void_p]),
    ("stn_get_program", ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    ("stn_compile_program", ctypes.c_int, [ctypes.POINTER(Config), ctypes.c_void_p, ctypes.c_void_p,
                                           ctypes.c_void_p]),
    ("stn_begin_batch", ctypes.c_int, [ctypes.c_void_p, ctypes.c_int64, ctypes.c_uint64]),
    ("stn_apply_round", ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p]),
    ("stn_apply_round_device", ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p]),
    ("stn_num_steps", ctypes.c_int32, [ctypes.c_void_p]),
    ("stn_apply_step_device", ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p]),
    ("stn_sync", ctypes.c_int, [ctypes.c_void_p]),
    ("stn_capture_batch", ctypes.c_int, [ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p]),
    ("stn_launch_captured", ctypes.c_int, [ctypes.c_void_p, ctypes.c_uint64]),
    ("stn_read_records", ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                        ctypes.c_void_p]),
    ("stn_device_records", ctypes.c_void_p, [ctypes.c_void_p]),
    ("stn_num_detectors", ctypes.c_int32, [ctypes.c_void_p]),
    ("stn_read_detectors", ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    ("stn_compile_detectors", ctypes.c_int, [ctypes.POINTER(Config), ctypes.c_void_p, ctypes.c_void_p,
                                             ctypes.c_void_p]),
    ("stn_algorithmic_flops", ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_double)]),
    ("stn_profile_counters", ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p]),
    ("stn_read_tableau", ctypes.c_int, [ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p,
                                        ctypes.c_void_p, ctypes.c_void_p]),
    ("stn_read_bonds", ctypes.c_int, [ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p]),
    ("stn_read_site", ctypes.c_int, [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_void_p]),
    ("stn_logical_expectation", ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p]),
    ("stn_schmidt_values", ctypes.c_int, [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_void_p,
                                          ctypes.POINTER(ctypes.c_int32)]),
    ("stn_sample_shots", ctypes.c_int, [ctypes.c_void_p, ctypes.c_int64, ctypes.c_uint64,
                                        ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                        ctypes.c_void_p]),
    ("stn_logprob_grad", ctypes.c_int, [ctypes.c_void_p, ctypes.c_uint64, ctypes.c_int64, ctypes.c_void_p,
                                        ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    ("stn_dense_qr_q", ctypes.c_int, [ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, ctypes.c_void_p,
                                      ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    ("stn_dense_qr", ctypes.c_int, [ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, ctypes.c_void_p,
                                    ctypes.c_void_p]),
    ("stn_dense_svd", ctypes.c_int, [ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, ctypes.c_void_p,
                                     ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p]),
    ("stn_dense_svd_noalloc", ctypes.c_int, [ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, ctypes.c_void_p,
                                             ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    ("stn_dense_gemm_tc", ctypes.c_int, [ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, ctypes.c_void_p,
                                         ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    ("stn_dense_cgemm", ctypes.c_int, [ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                                       ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                                       ctypes.POINTER(ctypes.c_double), ctypes.c_void_p, ctypes.c_int32,
                                       ctypes.c_void_p, ctypes.c_int32, ctypes.POINTER(ctypes.c_double),
                                       ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p]),
    ("stn_peak_probe", ctypes.c_int, [ctypes.c_int32, ctypes.c_int64, ctypes.POINTER(ctypes.c_double),
                                      ctypes.c_void_p]),
    ("stn_philox_uniforms", ctypes.c_int, [ctypes.c_uint64, ctypes.c_uint64, ctypes.c_int64,
                                           ctypes.c_uint32, ctypes.c_int32, ctypes.c_void_p,
                                           ctypes.c_void_p]),
]

_lib = None


def load():
    """Load libstn.so; raises if it has not been built (no fallback exists)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB):
        raise RuntimeError(f"{LIB} is missing: run paper_2605_29514_gb300.build() first")
    lib = ctypes.CDLL(LIB)
    for name, res, args in EXPORTS:
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


if __name__ == "__main__":
    print(build(force="--force" in sys.argv))
