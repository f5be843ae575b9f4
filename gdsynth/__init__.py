"""Seeded synthetic EM-like stacks, shared by the CUDA solver's tests and
benchmark and by the CPU oracle's tests.

This module only draws inputs.  It holds none of the gradient-domain method's
arithmetic and imports neither the solver package nor the oracle.

Recipe (one stack = one ``(geom_seed, photo_seed, noise_seed)`` triple):

* Voronoi mosaic per slice; seeds uniform in the slice and drifting smoothly in
  z (linear drift |v| <= 0.3 px/slice plus a sinusoidal wobble of amplitude
  <= 2 px and period ~U(20,60) slices).  Cell interiors ~N(160,15), membranes
  (pixels within 1 px of the bisector of the two nearest seeds) ~N(50,10),
  both drawn once per cell.
* Per slice: gain ~U(0.8,1.2), offset ~U(-20,20), a linear ramp running from
  -a to +a across the slice with a ~U(-15,15) along a direction ~U(0, 2 pi).
* Per pixel noise ~N(0, sigma), sigma = 3 by default.
* Clip to [0,255], round half to even, store as uint8.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "synth.c")
_LIB_PATH = os.path.join(_HERE, "libgdsynth.so")
_lock = threading.Lock()
_lib = None

#: cell density of the 1024x1024 / 2000-cell workload, in px^2 per cell
PX2_PER_CELL = 1024.0 * 1024.0 / 2000.0


def build(force: bool = False) -> str:
    """Compile ``synth.c`` into ``libgdsynth.so`` next to it (gcc, OpenMP)."""
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + ".tmp%d" % os.getpid()
        cmd = ["gcc", "-O2", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off", "-std=c11",
               _SRC, "-o", tmp, "-lm"]
        subprocess.check_call(cmd)
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


_CU_SRC = os.path.join(_HERE, "synth_cuda.cu")
_CU_LIB_PATH = os.path.join(_HERE, "libgdsynth_cuda.so")
_cu_lib = None


def build_cuda(force: bool = False) -> str:
    """Compile ``synth_cuda.cu`` (the same generator on the GPU) into
    ``libgdsynth_cuda.so`` (nvcc, sm_103a)."""
    deps = [_CU_SRC, _SRC]
    if force or not os.path.exists(_CU_LIB_PATH) or any(
            os.path.getmtime(_CU_LIB_PATH) < os.path.getmtime(d) for d in deps):
        nvcc = os.environ.get("NVCC") or "nvcc"
        if not os.path.exists(nvcc) and os.path.exists("/usr/local/cuda/bin/nvcc"):
            nvcc = "/usr/local/cuda/bin/nvcc"
        tmp = _CU_LIB_PATH + ".tmp%d" % os.getpid()
        cmd = [nvcc, "-O2", "-std=c++17", "-fmad=false", "-gencode", "arch=compute_103a,code=sm_103a",
               "-Xcompiler", "-fPIC", "-shared", "-I", _HERE, _CU_SRC, "-o", tmp]
        subprocess.check_call(cmd)
        os.replace(tmp, _CU_LIB_PATH)
    return _CU_LIB_PATH


def _load_cuda():
    global _cu_lib
    with _lock:
        if _cu_lib is None:
            build_cuda()
            lib = ctypes.CDLL(_CU_LIB_PATH)
            lib.gds_em_window_cuda.restype = ctypes.c_int
            lib.gds_em_window_cuda.argtypes = [
                ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                ctypes.c_uint64, ctypes.c_uint64, ctypes.c_uint64, ctypes.c_double,
                ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                ctypes.c_void_p]
            _cu_lib = lib
    return _cu_lib


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB_PATH)
            lib.gds_em_window.restype = ctypes.c_int
            lib.gds_em_window.argtypes = [
                ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                ctypes.c_uint64, ctypes.c_uint64, ctypes.c_uint64, ctypes.c_double,
                ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int]
            _lib = lib
    return _lib


def default_cells(nx: int, ny: int) -> int:
    """Cell count at the workloads' density (40 on 64^2, 2000 on 1024^2)."""
    if (nx, ny) == (64, 64):
        return 40
    return max(2, int(round(nx * ny / PX2_PER_CELL)))


def em_stack(nx: int, ny: int, nz: int, seed: int = 0, ncells: int | None = None,
             photo_seed: int | None = None, noise_seed: int | None = None,
             noise_sigma: float = 3.0, window=None) -> np.ndarray:
    """uint8 array ``[nz][ny][nx]`` (x fastest) of the synthetic stack.

    ``window = (x0, y0, z0, wx, wy, wz)`` returns only that window of the
    ``nx x ny x nz`` stack (identical to slicing the full stack).
    """
    lib = _load()
    if ncells is None:
        ncells = default_cells(nx, ny)
    if photo_seed is None:
        photo_seed = seed * 2 + 1
    if noise_seed is None:
        noise_seed = seed * 2 + 2
    if window is None:
        window = (0, 0, 0, nx, ny, nz)
    x0, y0, z0, wx, wy, wz = (int(v) for v in window)
    out = np.empty((wz, wy, wx), dtype=np.uint8)
    rc = lib.gds_em_window(out.ctypes.data, nx, ny, nz, int(ncells),
                           int(seed) & (2**64 - 1), int(photo_seed) & (2**64 - 1),
                           int(noise_seed) & (2**64 - 1), float(noise_sigma),
                           x0, y0, z0, wx, wy, wz)
    if rc != 0:
        raise ValueError("gds_em_window failed with status %d" % rc)
    return out


def em_stack_cuda(nx: int, ny: int, nz: int, seed: int = 0, ncells: int | None = None,
                  photo_seed: int | None = None, noise_seed: int | None = None,
                  noise_sigma: float = 3.0, window=None, out=None):
    """The stack of :func:`em_stack` drawn on the GPU: a torch uint8 CUDA
    tensor ``[nz][ny][nx]`` (or the window), written into ``out`` if given."""
    import torch
    lib = _load_cuda()
    if ncells is None:
        ncells = default_cells(nx, ny)
    if photo_seed is None:
        photo_seed = seed * 2 + 1
    if noise_seed is None:
        noise_seed = seed * 2 + 2
    if window is None:
        window = (0, 0, 0, nx, ny, nz)
    x0, y0, z0, wx, wy, wz = (int(v) for v in window)
    if out is None:
        out = torch.empty((wz, wy, wx), dtype=torch.uint8, device="cuda")
    assert out.is_cuda and out.dtype == torch.uint8 and out.numel() == wx * wy * wz
    stream = torch.cuda.current_stream().cuda_stream
    rc = lib.gds_em_window_cuda(ctypes.c_void_p(out.data_ptr()), nx, ny, nz, int(ncells),
                                int(seed) & (2**64 - 1), int(photo_seed) & (2**64 - 1),
                                int(noise_seed) & (2**64 - 1), float(noise_sigma),
                                x0, y0, z0, wx, wy, wz, ctypes.c_void_p(stream) if stream else None)
    if rc != 0:
        raise ValueError("gds_em_window_cuda failed with status %d" % rc)
    return out


def sp_pair(n: int, seed: int):
    """(I0, I1) for one square 2D slice of side ``n``: I0 is a noisy slice; I1
    is the same mosaic with a fresh gain/offset/ramp draw and no noise,
    standing in for an anisotropic-diffusion output."""
    i0 = em_stack(n, n, 1, seed=seed)[0]
    i1 = em_stack(n, n, 1, seed=seed, photo_seed=seed * 2 + 7, noise_sigma=0.0)[0]
    return i0, i1


# ---------------------------------------------------------------------------
# batches of independent slices of different sizes
# ---------------------------------------------------------------------------
def batch_sides(n: int, lo: int = 256, hi: int = 4096, seed: int = 0) -> list:
    """``n`` integer slice sides, log-uniform in ``[lo, hi]``."""
    rng = np.random.default_rng(seed)
    u = rng.uniform(np.log(lo), np.log(hi + 1.0), n)
    return [int(v) for v in np.clip(np.floor(np.exp(u)), lo, hi)]


def batch_alphas(n: int, lo: float = 0.001, hi: float = 0.1, seed: int = 0) -> list:
    """``n`` screening weights, uniform in ``[lo, hi)``."""
    rng = np.random.default_rng(seed + 7919)
    return [float(v) for v in rng.uniform(lo, hi, n)]


def batch_slices(nx, ny, seed: int = 0):
    """(I0, I1) lists of float32 ``[ny_s][nx_s]`` slices.  Every slice is a
    crop, at a seeded offset, of one synthetic EM slice as large as the
    largest (so a batch costs one slice's generation); I1 is the crop with a
    fresh per-slice gain ~U(0.85, 1.15), offset ~U(-15, 15) and a linear ramp
    of amplitude ~U(-10, 10) across the slice, standing in for the output of
    a previous step."""
    W, H = max(nx), max(ny)
    master = em_stack(W, H, 1, seed=seed, ncells=default_cells(W, H))[0].astype(np.float32)
    rng = np.random.default_rng(seed + 104729)
    I0s, I1s = [], []
    for a, b in zip(nx, ny):
        x0 = int(rng.integers(0, W - a + 1))
        y0 = int(rng.integers(0, H - b + 1))
        i0 = np.ascontiguousarray(master[y0:y0 + b, x0:x0 + a])
        g, o, r = rng.uniform(0.85, 1.15), rng.uniform(-15, 15), rng.uniform(-10, 10)
        ramp = np.linspace(-r, r, a, dtype=np.float32)[None, :] if a > 1 else np.zeros((1, 1), np.float32)
        i1 = np.clip(g * i0 + o + ramp, 0.0, 255.0).astype(np.float32)
        I0s.append(i0)
        I1s.append(np.ascontiguousarray(i1))
    return I0s, I1s


def pack(slices) -> np.ndarray:
    """Concatenates 2D slices (x fastest) into one float32 array."""
    return np.ascontiguousarray(np.concatenate([np.asarray(s, np.float32).ravel() for s in slices]))


def unpack(flat, nx, ny) -> list:
    """Splits a packed array into ``[ny_s][nx_s]`` slices (views)."""
    out, o = [], 0
    for a, b in zip(nx, ny):
        out.append(np.asarray(flat[o:o + a * b]).reshape(b, a))
        o += a * b
    return out
