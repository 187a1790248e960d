"""Python binding of libamriso (include/amriso.h): argument marshalling only.

Every step of the method runs in the library's CUDA kernels; PyTorch only
provides device memory (tensors) and the CUDA stream. Importing this module
on a machine where the compiled library is missing raises immediately: there
is no CPU fallback.

    import torch
    from paper_2004_08475_b300 import amriso
    ctx = amriso.AmrContext()                       # device 0, torch's stream
    ctx.upload(xyz, level, scalar)                  # int32 [N,3], uint8 [N], fp32 [N]
    ctx.build_locator()                             # Sec. 3.2
    n_dual = ctx.dual_cells()                       # Sec. 4
    tris = ctx.iso(iso)                             # Sec. 5: fp32 [T,3,3]
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import numpy as np
import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libamriso.so")

OK = 0
ERR_INVALID_ARG = -1
ERR_UNALIGNED = -2
ERR_RANGE = -3
ERR_NONFINITE = -4
ERR_DUPLICATE = -5
ERR_OVERLAP = -6
ERR_STATE = -7
ERR_OOM = -8
ERR_CAPACITY = -9
ERR_TIMEOUT = -10
ERR_CUDA = -11

DEVICE_PTRS = 0
HOST_PTRS = 1
COPY = 2


class _IsoJob(ctypes.Structure):
    _fields_ = [("ctx", ctypes.c_void_p), ("n_iso", ctypes.c_int)]


class AmrError(RuntimeError):
    def __init__(self, code: int, what: str):
        super().__init__(f"{what}: {strerror(code)} ({code})")
        self.code = code


class _LocatorOpts(ctypes.Structure):
    _fields_ = [("log2_brick", ctypes.c_int), ("load_factor", ctypes.c_float),
                ("block_size", ctypes.c_int), ("check_overlap", ctypes.c_int),
                ("partitioned", ctypes.c_int)]


class _Info(ctypes.Structure):
    _fields_ = [("n_cells", ctypes.c_int64), ("n_bricks", ctypes.c_int64),
                ("n_slots", ctypes.c_int64), ("n_dual", ctypes.c_int64),
                ("n_levels", ctypes.c_int32), ("log2_brick", ctypes.c_int32),
                ("device_bytes", ctypes.c_int64), ("placement", ctypes.c_int32), ("reserved", ctypes.c_int32)]


ABI_VERSION = 11   # AMR_ABI_VERSION of include/amriso.h


def _load() -> ctypes.CDLL:
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"libamriso.so not built ({LIB_PATH}); run "
                          "`python -m paper_2004_08475_b300.build` (nvcc, sm_103a)")
    lib = ctypes.CDLL(LIB_PATH)
    P, I, I64, F = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_float
    sig = {
        "amr_create": (I, [ctypes.POINTER(P), I, P]),
        "amr_destroy": (None, [P]),
        "amr_set_stream": (I, [P, P]),
        "amr_upload": (I, [P, P, P, P, I64, I]),
        "amr_build_locator": (I, [P, ctypes.POINTER(_LocatorOpts)]),
        "amr_dual_cells": (I, [P, ctypes.POINTER(I64)]),
        "amr_dual_cells_owned": (I, [P, ctypes.c_int32, ctypes.c_int32, ctypes.POINTER(I64)]),
        "amr_get_duals": (I, [P, P, I64, I]),
        "amr_dual_cells_iso": (I, [P, F, P, I64, ctypes.POINTER(I64), ctypes.POINTER(I64), I]),
        "amr_iso": (I, [P, F, P, I64, ctypes.POINTER(I64), I]),
        "amr_iso_tagged": (I, [P, F, P, P, I64, ctypes.POINTER(I64), I]),
        "amr_iso_indexed": (I, [P, F, P, I64, P, I64, P, ctypes.POINTER(I64), ctypes.POINTER(I64), I]),
        "amr_interpolate": (I, [P, F, P, P, I64, P, I]),
        "amr_dual_shapes": (I, [P, P, P, I]),
        "amr_iso_cases": (I, [P, F, P, P, I]),
        "amr_iso_batch": (I, [P, P, I, P, I64, P, I]),
        "amr_iso_batch_async": (I, [P, P, I, P, I64, P]),
        "amr_iso_multi_workspace": (I64, [P, I]),
        "amr_iso_multi_async": (I, [P, I, P, P, I64, P, P, I64, P]),
        "amr_sync": (I, [P]),
        "amr_trim": (I, [P]),
        "amr_strerror": (ctypes.c_char_p, [I]),
        "amr_mc_table": (I, [P, P]),
        "amr_get_info": (I, [P, ctypes.POINTER(_Info)]),
        "amr_enable_timing": (I, [P, I]),
        "amr_kernel_times": (I, [P, P, P, I]),
        "amr_kernel_name": (ctypes.c_char_p, [I]),
        "amr_extract_noalloc": (I, [P, P, P, I64, F, P, I64, ctypes.POINTER(I64), P]),
        "amr_abi_version": (I, []),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    if lib.amr_abi_version() != ABI_VERSION:   # structs above must match the library's
        raise ImportError(f"libamriso.so has ABI {lib.amr_abi_version()}, this binding {ABI_VERSION}: "
                          "rebuild it (`python -m paper_2004_08475_b300.build`)")
    return lib


_lib = _load()

# Every symbol the header declares (checked by the tests).
EXPORTS = ("amr_create", "amr_destroy", "amr_set_stream", "amr_upload", "amr_build_locator",
           "amr_dual_cells", "amr_get_duals", "amr_iso", "amr_iso_cases", "amr_iso_batch",
           "amr_sync", "amr_strerror", "amr_mc_table", "amr_get_info", "amr_enable_timing",
           "amr_kernel_times", "amr_kernel_name", "amr_extract_noalloc", "amr_iso_batch_async",
           "amr_dual_cells_iso", "amr_trim", "amr_abi_version", "amr_iso_indexed",
           "amr_interpolate", "amr_dual_shapes", "amr_iso_tagged", "amr_iso_multi_workspace",
           "amr_iso_multi_async", "amr_dual_cells_owned")


def lib() -> ctypes.CDLL:
    return _lib


def strerror(code: int) -> str:
    return _lib.amr_strerror(int(code)).decode()


def _check(rc: int, what: str):
    if rc != OK:
        raise AmrError(rc, what)


def mc_table():
    """(count[256] u8, edges[256][15] u8) - the kernels' MC table (host only)."""
    count = np.zeros(256, dtype=np.uint8)
    edges = np.zeros((256, 15), dtype=np.uint8)
    _check(_lib.amr_mc_table(count.ctypes.data, edges.ctypes.data), "amr_mc_table")
    return count, edges


def _ptr(t) -> int:
    if t is None:
        return 0
    if isinstance(t, np.ndarray):
        return t.ctypes.data
    return t.data_ptr()


def _jobs(contexts, n_isos):
    arr = (_IsoJob * len(contexts))()
    for j, (c, k) in enumerate(zip(contexts, n_isos)):
        arr[j].ctx = c._h
        arr[j].n_iso = int(k)
    return arr


def iso_multi_workspace(contexts, n_isos) -> int:
    """Device bytes amr_iso_multi_async needs for these (context, iso count)
    jobs."""
    r = _lib.amr_iso_multi_workspace(_jobs(contexts, n_isos), len(contexts))
    if r < 0:
        _check(int(r), "amr_iso_multi_workspace")
    return int(r)


def iso_multi_async(contexts, n_isos, d_isos: torch.Tensor, out: torch.Tensor, d_offsets: torch.Tensor,
                    workspace: torch.Tensor, stream: torch.cuda.Stream | None = None):
    """Enqueue one batch over several data sets: job j = contexts[j] at its
    n_isos[j] iso-values (consecutive in d_isos); segment q of the batch is
    out[d_offsets[q]:d_offsets[q+1]]. Neither synchronises nor allocates."""
    assert d_isos.is_cuda and d_isos.dtype == torch.float32 and d_offsets.dtype == torch.int64
    assert d_offsets.numel() >= sum(n_isos) + 1 and out.is_cuda and workspace.is_cuda
    st = stream if stream is not None else torch.cuda.current_stream()
    _check(_lib.amr_iso_multi_async(_jobs(contexts, n_isos), len(contexts), _ptr(d_isos), _ptr(out),
                                    int(out.shape[0]), _ptr(d_offsets), _ptr(workspace),
                                    int(workspace.numel() * workspace.element_size()),
                                    ctypes.c_void_p(st.cuda_stream)), "amr_iso_multi_async")


@dataclass
class Info:
    n_cells: int
    n_bricks: int
    n_slots: int
    n_dual: int
    n_levels: int
    log2_brick: int
    device_bytes: int
    placement: int = 0   # 0 direct scatter, 1 binned


class AmrContext:
    """One data set on one GPU and everything derived from it."""

    def __init__(self, device: int = 0, stream: torch.cuda.Stream | None = None):
        if not torch.cuda.is_available():
            raise RuntimeError("AmrContext needs a CUDA device")
        self.device = torch.device("cuda", device)
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        h = ctypes.c_void_p()
        _check(_lib.amr_create(ctypes.byref(h), int(device), ctypes.c_void_p(self.stream.cuda_stream)),
               "amr_create")
        self._h = h
        self._keep = None
        self.n_dual = -1

    def close(self):
        if getattr(self, "_h", None):
            _lib.amr_destroy(self._h)
            self._h = None
        self._keep = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_stream(self, stream: torch.cuda.Stream):
        self.stream = stream
        _check(_lib.amr_set_stream(self._h, ctypes.c_void_p(stream.cuda_stream)), "amr_set_stream")

    # -- hot path ----------------------------------------------------------
    def upload(self, xyz, level, scalar, copy: bool = False):
        """xyz int32 [N,3], level uint8 [N], scalar fp32 [N]; all on the GPU
        (borrowed: this object keeps them alive until the next upload or
        close, since interpolate reads xyz and scalar; copy=True copies) or
        all on the host (copied inside the call)."""
        xyz = xyz.contiguous()
        level = level.contiguous()
        scalar = scalar.contiguous()
        assert xyz.dtype == torch.int32 and level.dtype == torch.uint8 and scalar.dtype == torch.float32
        n = scalar.shape[0]
        assert xyz.shape == (n, 3) and level.shape == (n,)
        on_dev = xyz.is_cuda
        assert level.is_cuda == on_dev and scalar.is_cuda == on_dev
        flags = (COPY if copy else DEVICE_PTRS) if on_dev else HOST_PTRS
        self._keep = (xyz, level, scalar)
        _check(_lib.amr_upload(self._h, _ptr(xyz), _ptr(level), _ptr(scalar), int(n), flags),
               "amr_upload")
        self.n_dual = -1

    def build_locator(self, log2_brick: int = 3, load_factor: float = 0.5, block_size: int = 256,
                      check_overlap: bool = False, partitioned: int = 0):
        """partitioned: 1 places the cells by the binned passes (split by
        slot range, then each window of slots written whole), -1 by a direct
        scatter, 0 binned from 2^20 cells on (binned falls back to the direct
        scatter when the brick table outgrows the cell codes)."""
        o = _LocatorOpts(int(log2_brick), float(load_factor), int(block_size), int(check_overlap),
                         int(partitioned))
        rc = _lib.amr_build_locator(self._h, ctypes.byref(o))
        _check(rc, "amr_build_locator")

    def dual_cells(self, owned_x: tuple | None = None) -> int:
        """Dual cells (kept resident); owned_x = (x_begin, x_end) keeps only
        those whose owning cell's lower corner x lies in [x_begin, x_end)."""
        n = ctypes.c_int64(0)
        if owned_x is None:
            _check(_lib.amr_dual_cells(self._h, ctypes.byref(n)), "amr_dual_cells")
        else:
            _check(_lib.amr_dual_cells_owned(self._h, int(owned_x[0]), int(owned_x[1]), ctypes.byref(n)),
                   "amr_dual_cells_owned")
        self.n_dual = n.value
        return n.value

    def dual_cells_iso(self, iso: float, out: torch.Tensor):
        """Dual cells (kept resident) and the triangles at `iso` in one pass.
        Returns (n_dual, n_tris); n_tris may exceed out.shape[0], in which case
        the triangle output is partial (the dual list is complete)."""
        nd = ctypes.c_int64(0)
        nt = ctypes.c_int64(0)
        flags = HOST_PTRS if not out.is_cuda else DEVICE_PTRS
        rc = _lib.amr_dual_cells_iso(self._h, ctypes.c_float(iso), _ptr(out), int(out.shape[0]),
                                     ctypes.byref(nd), ctypes.byref(nt), flags)
        if rc not in (OK, ERR_CAPACITY):
            _check(rc, "amr_dual_cells_iso")
        self.n_dual = nd.value
        return nd.value, nt.value

    def get_duals(self, out: torch.Tensor | None = None) -> torch.Tensor:
        """Resident dual cells as input cell IDs, int32 [D, 8]."""
        nd = self.n_dual
        if out is None:
            out = torch.empty((max(nd, 0), 8), dtype=torch.int32, device=self.device)
        flags = DEVICE_PTRS if out.is_cuda else HOST_PTRS
        _check(_lib.amr_get_duals(self._h, _ptr(out), int(out.shape[0]), flags), "amr_get_duals")
        return out[:nd]

    def iso(self, iso: float, out: torch.Tensor | None = None, host: bool = False):
        """Fat triangles fp32 [T,3,3] at `iso`. Grows `out` when too small."""
        n = ctypes.c_int64(0)
        if out is None:
            cap = max(1024, self.n_dual // 4)
            out = self._tri_buffer(cap, host)
        cap = out.shape[0]
        flags = HOST_PTRS if not out.is_cuda else DEVICE_PTRS
        rc = _lib.amr_iso(self._h, ctypes.c_float(iso), _ptr(out), int(cap), ctypes.byref(n), flags)
        if rc == ERR_CAPACITY:
            out = self._tri_buffer(n.value, not out.is_cuda)
            rc = _lib.amr_iso(self._h, ctypes.c_float(iso), _ptr(out), int(out.shape[0]),
                              ctypes.byref(n), flags)
        _check(rc, "amr_iso")
        return out[:n.value]

    def iso_tagged(self, iso: float, host: bool = False):
        """(tris fp32 [T,3,3], tri_dual int64 [T]): the triangles of `iso`,
        each with the index of its dual cell in get_duals order."""
        n = ctypes.c_int64(0)
        flags = HOST_PTRS if host else DEVICE_PTRS
        cap = max(1024, self.n_dual // 4)
        for _ in range(2):
            tris = self._tri_buffer(cap, host)
            tags = torch.empty(cap, dtype=torch.int64, device="cpu" if host else self.device)
            if host:
                tags = tags.pin_memory()
            rc = _lib.amr_iso_tagged(self._h, ctypes.c_float(iso), _ptr(tris), _ptr(tags), int(cap),
                                     ctypes.byref(n), flags)
            if rc != ERR_CAPACITY:
                break
            cap = n.value
        _check(rc, "amr_iso_tagged")
        return tris[:n.value], tags[:n.value]

    def iso_indexed(self, iso: float, host: bool = False, with_keys: bool = True):
        """Indexed face set at `iso`: (vtx [V,3] f32, tri [T,3] i32, keys [V,2]
        i32 input-cell indices or None), on the device or in host memory."""
        nv, nt = ctypes.c_int64(0), ctypes.c_int64(0)
        flags = HOST_PTRS if host else DEVICE_PTRS
        dev = "cpu" if host else self.device
        vcap = max(1024, self.n_dual // 4)
        tcap = vcap
        for _ in range(2):
            vtx = torch.empty((vcap, 3), dtype=torch.float32, device=dev)
            tri = torch.empty((tcap, 3), dtype=torch.int32, device=dev)
            keys = torch.empty((vcap, 2), dtype=torch.int32, device=dev) if with_keys else None
            if host:
                vtx, tri = vtx.pin_memory(), tri.pin_memory()
                keys = keys.pin_memory() if keys is not None else None
            rc = _lib.amr_iso_indexed(self._h, ctypes.c_float(iso), _ptr(vtx), vcap, _ptr(tri), tcap,
                                      _ptr(keys) if keys is not None else None, ctypes.byref(nv),
                                      ctypes.byref(nt), flags)
            if rc != ERR_CAPACITY:
                break
            vcap, tcap = max(vcap, nv.value), max(tcap, nt.value)
        _check(rc, "amr_iso_indexed")
        return vtx[:nv.value], tri[:nt.value], (keys[:nv.value] if keys is not None else None)

    def interpolate(self, iso: float, attr: torch.Tensor, vkeys: torch.Tensor) -> torch.Tensor:
        """Per-vertex values of the per-cell field `attr` [n] f32 at the
        vertices `vkeys` [V,2] (from iso_indexed) of the surface at `iso`;
        on the device of `attr`."""
        host = not attr.is_cuda
        attr = attr.contiguous().to(torch.float32)
        vkeys = vkeys.contiguous().to(torch.int32)
        if host:
            attr, vkeys = attr.pin_memory(), vkeys.pin_memory()
        out = torch.empty(vkeys.shape[0], dtype=torch.float32, device=attr.device)
        if host:
            out = out.pin_memory()
        _check(_lib.amr_interpolate(self._h, ctypes.c_float(iso), _ptr(attr), _ptr(vkeys), int(vkeys.shape[0]),
                                    _ptr(out), HOST_PTRS if host else DEVICE_PTRS), "amr_interpolate")
        return out

    def dual_shapes(self):
        """Per resident dual the number of distinct cells among its 8
        vertices (u8 [n_dual] on the device) and the histogram over 0..8."""
        counts = torch.empty(max(self.n_dual, 0), dtype=torch.uint8, device=self.device)
        hist = np.zeros(9, dtype=np.int64)
        _check(_lib.amr_dual_shapes(self._h, _ptr(counts), hist.ctypes.data, DEVICE_PTRS), "amr_dual_shapes")
        return counts, hist

    def iso_count(self, iso: float, out: torch.Tensor) -> int:
        """amr_iso into a preallocated buffer; returns the exact count (may
        exceed out.shape[0], in which case the output is partial)."""
        n = ctypes.c_int64(0)
        flags = HOST_PTRS if not out.is_cuda else DEVICE_PTRS
        rc = _lib.amr_iso(self._h, ctypes.c_float(iso), _ptr(out), int(out.shape[0]), ctypes.byref(n),
                          flags)
        if rc not in (OK, ERR_CAPACITY):
            _check(rc, "amr_iso")
        return n.value

    def iso_cases(self, iso: float):
        """Per-dual (case index u8 [D], kept triangles u8 [D]) in get_duals order."""
        nd = self.n_dual
        cases = torch.empty(max(nd, 1), dtype=torch.uint8, device=self.device)
        ntri = torch.empty(max(nd, 1), dtype=torch.uint8, device=self.device)
        _check(_lib.amr_iso_cases(self._h, ctypes.c_float(iso), _ptr(cases), _ptr(ntri), DEVICE_PTRS),
               "amr_iso_cases")
        return cases[:nd], ntri[:nd]

    def iso_batch(self, isos, out: torch.Tensor | None = None):
        """Triangles of several iso-values in one launch: (tris [sum T,3,3],
        offsets int64 [n_iso+1])."""
        isos = np.ascontiguousarray(np.asarray(isos, dtype=np.float32).reshape(-1))
        k = isos.shape[0]
        offs = np.zeros(k + 1, dtype=np.int64)
        if out is None:
            out = torch.empty((0, 3, 3), dtype=torch.float32, device=self.device)
        flags = DEVICE_PTRS if out.is_cuda else HOST_PTRS
        rc = _lib.amr_iso_batch(self._h, isos.ctypes.data, k, _ptr(out) if out.numel() else None,
                                int(out.shape[0]), offs.ctypes.data, flags)
        if rc == ERR_CAPACITY:
            out = self._tri_buffer(int(offs[-1]), not out.is_cuda)
            rc = _lib.amr_iso_batch(self._h, isos.ctypes.data, k, _ptr(out), int(out.shape[0]),
                                    offs.ctypes.data, flags)
        _check(rc, "amr_iso_batch")
        return out[:int(offs[-1])], torch.from_numpy(offs)

    def iso_batch_async(self, d_isos: torch.Tensor, out: torch.Tensor, d_offsets: torch.Tensor):
        """Enqueue a batched extraction (iso-values and offsets on the device);
        no host synchronisation, so it can be captured in a CUDA graph."""
        assert d_isos.is_cuda and d_isos.dtype == torch.float32 and d_offsets.dtype == torch.int64
        assert d_offsets.numel() >= d_isos.numel() + 1 and out.is_cuda
        _check(_lib.amr_iso_batch_async(self._h, _ptr(d_isos), int(d_isos.numel()), _ptr(out),
                                        int(out.shape[0]), _ptr(d_offsets)), "amr_iso_batch_async")

    def sync(self):
        _check(_lib.amr_sync(self._h), "amr_sync")

    def trim(self):
        """Free the scratch workspace (binned-placement and host-delivery
        staging); the locator and dual cells stay resident."""
        _check(_lib.amr_trim(self._h), "amr_trim")

    # -- introspection -----------------------------------------------------
    def info(self) -> Info:
        i = _Info()
        _check(_lib.amr_get_info(self._h, ctypes.byref(i)), "amr_get_info")
        return Info(i.n_cells, i.n_bricks, i.n_slots, i.n_dual, i.n_levels, i.log2_brick,
                    i.device_bytes, i.placement)

    def enable_timing(self, on: bool = True):
        _check(_lib.amr_enable_timing(self._h, int(on)), "amr_enable_timing")

    def kernel_times(self):
        """{kernel name: (total ms, launches)} since the previous call."""
        cap = 64
        ms = (ctypes.c_double * cap)()
        cnt = (ctypes.c_int64 * cap)()
        k = _lib.amr_kernel_times(self._h, ms, cnt, cap)
        if k < 0:
            _check(k, "amr_kernel_times")
        return {_lib.amr_kernel_name(i).decode(): (ms[i], cnt[i]) for i in range(min(k, cap))}

    def _tri_buffer(self, n, host=False):
        if host:
            return torch.empty((int(n), 3, 3), dtype=torch.float32).pin_memory()
        return torch.empty((int(n), 3, 3), dtype=torch.float32, device=self.device)
