"""Thin Python binding of libgfh (the C ABI declared in include/gfh.h).

Only argument marshalling lives here: every step of the method runs in the library's CUDA kernels
or its host planner.  torch tensors are accepted as device buffers (their data pointers are passed
to the library) and torch streams as the stream; there is no CPU fallback, and importing this
module fails loudly when the library has not been built.
"""
from __future__ import annotations

import ctypes
import dataclasses
import pathlib

import numpy as np

_PKG = pathlib.Path(__file__).resolve().parent
_LIB_PATH = _PKG / "libgfh.so"

GFH_OK = 0
GFH_ERR_ARG = -1
GFH_ERR_SIZE = -2
GFH_ERR_CUDA = -3
GFH_ERR_INPUT = -4
GFH_ERR_TIMEOUT = -5
GFH_ERR_NOMEM = -6

EXPORTED = [
    "gfh_create", "gfh_destroy", "gfh_set_stream", "gfh_check", "gfh_strerror",
    "gfh_grid_make", "gfh_grid_tables", "gfh_grid_columns",
    "gfh_peaks_from_power", "gfh_peakmap", "gfh_peakmap_async",
    "gfh_plan_create", "gfh_plan_destroy", "gfh_plan_execute", "gfh_plan_autotune",
    "gfh_hough", "gfh_select", "gfh_peaks_from_power_static",
]
STATIC_SCRATCH_BYTES = 8 << 20


class GfhError(RuntimeError):
    def __init__(self, code: int, where: str):
        super().__init__(f"{where}: {strerror(code)} ({code})")
        self.code = code


class GridC(ctypes.Structure):
    _fields_ = [
        ("n", ctypes.c_double), ("df", ctypes.c_double),
        ("bin_lo", ctypes.c_int32), ("bin_hi", ctypes.c_int32),
        ("n_fft", ctypes.c_int32), ("n_k", ctypes.c_int32),
        ("t_first", ctypes.c_double), ("t_hop", ctypes.c_double), ("t_obs", ctypes.c_double),
        ("k_min", ctypes.c_double), ("dk", ctypes.c_double), ("f_max", ctypes.c_double),
        ("ana_lo", ctypes.c_double), ("ana_hi", ctypes.c_double), ("band_hz", ctypes.c_double),
        ("list", ctypes.c_int32), ("n_bands", ctypes.c_int32),
        ("dx0", ctypes.c_double), ("x0_min", ctypes.c_double),
        ("n_x0", ctypes.c_int64), ("ld_x0", ctypes.c_int64),
    ]


class CandidateC(ctypes.Structure):
    _fields_ = [
        ("band", ctypes.c_int32), ("row", ctypes.c_int32), ("col", ctypes.c_int64),
        ("count", ctypes.c_int32), ("reserved", ctypes.c_int32),
        ("cr", ctypes.c_double), ("x0", ctypes.c_double), ("k", ctypes.c_double),
        ("f0", ctypes.c_double), ("fdot0", ctypes.c_double),
    ]


class MapStatsC(ctypes.Structure):
    _fields_ = [("sum", ctypes.c_int64), ("sum_sq", ctypes.c_int64), ("cells", ctypes.c_int64)]


class PeaksC(ctypes.Structure):
    _fields_ = [("fft_idx", ctypes.c_void_p), ("bin", ctypes.c_void_p),
                ("offsets", ctypes.c_void_p), ("n_lists", ctypes.c_int32)]


class TileConfigC(ctypes.Structure):
    _fields_ = [("rows", ctypes.c_int32), ("cols", ctypes.c_int32),
                ("threads", ctypes.c_int32), ("reserved", ctypes.c_int32)]


CANDIDATE_BYTES = ctypes.sizeof(CandidateC)   # 64
STATS_BYTES = ctypes.sizeof(MapStatsC)        # 24
CANDIDATE_DTYPE = np.dtype([("band", "<i4"), ("row", "<i4"), ("col", "<i8"), ("count", "<i4"),
                            ("reserved", "<i4"), ("cr", "<f8"), ("x0", "<f8"), ("k", "<f8"),
                            ("f0", "<f8"), ("fdot0", "<f8")])
STATS_DTYPE = np.dtype([("sum", "<i8"), ("sum_sq", "<i8"), ("cells", "<i8")])

_lib = None


def lib() -> ctypes.CDLL:
    """The loaded libgfh; raises if it has not been built (no fallback exists)."""
    global _lib
    if _lib is None:
        if not _LIB_PATH.exists():
            raise RuntimeError(f"{_LIB_PATH} is missing: build it with "
                               "`python -m paper_1810_09784_gb300.build`")
        L = ctypes.CDLL(str(_LIB_PATH))
        vp, i32, i64, dbl = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_double
        P = ctypes.POINTER
        sig = {
            "gfh_create": [P(vp), ctypes.c_int, vp],
            "gfh_destroy": [vp],
            "gfh_set_stream": [vp, vp],
            "gfh_check": [vp],
            "gfh_grid_make": [P(GridC)],
            "gfh_grid_tables": [P(GridC), vp, vp, vp],
            "gfh_grid_columns": [P(GridC), vp, vp, vp],
            "gfh_peaks_from_power": [vp, vp, i64, i32, i32, i32, dbl, vp, vp, i64, P(i64)],
            "gfh_peakmap": [vp, vp, i64, dbl, dbl, i32, i32, dbl, vp, vp, i64, P(i64)],
            "gfh_peakmap_async": [vp, vp, i64, dbl, dbl, i32, i32, dbl, vp, vp, i64, vp],
            "gfh_plan_create": [vp, i32, P(GridC), P(vp), P(vp), vp, P(TileConfigC), P(vp)],
            "gfh_plan_destroy": [vp],
            "gfh_plan_execute": [vp, P(PeaksC)],
            "gfh_plan_autotune": [vp, P(PeaksC), i32, P(TileConfigC), P(ctypes.c_float)],
            "gfh_hough": [vp, vp, vp, i64, P(GridC), vp, vp, vp],
            "gfh_select": [vp, vp, P(GridC), vp, vp],
            "gfh_peaks_from_power_static": [vp, vp, i64, i32, i32, i32, dbl, vp, vp, i64, vp],
        }
        for name, args in sig.items():
            fn = getattr(L, name)
            fn.argtypes = args
            fn.restype = ctypes.c_int
        L.gfh_strerror.argtypes = [ctypes.c_int]
        L.gfh_strerror.restype = ctypes.c_char_p
        _lib = L
    return _lib


def strerror(code: int) -> str:
    return lib().gfh_strerror(code).decode()


def _ok(code: int, where: str) -> None:
    if code != GFH_OK:
        raise GfhError(code, where)


def _ptr(t) -> int | None:
    """Device (or host) address of a torch tensor / numpy array, None for None."""
    if t is None:
        return None
    if hasattr(t, "data_ptr"):
        return t.data_ptr()
    return t.ctypes.data


# ---- grids (host-side planning) ----------------------------------------------------------------

@dataclasses.dataclass
class Grid:
    """Python mirror of gfh_grid (request fields; derived fields after make())."""

    n: float
    df: float
    bin_lo: int
    bin_hi: int
    n_fft: int
    t_first: float
    t_hop: float
    t_obs: float
    n_k: int
    k_min: float = 0.0
    dk: float = 0.0
    f_max: float = 0.0
    ana_lo: float = 0.0
    ana_hi: float = 0.0
    band_hz: float = 1.0
    list: int = 0
    n_bands: int = 0
    dx0: float = 0.0
    x0_min: float = 0.0
    n_x0: int = 0
    ld_x0: int = 0

    def to_c(self) -> GridC:
        return GridC(**{f.name: getattr(self, f.name) for f in dataclasses.fields(self)})

    @classmethod
    def from_c(cls, c: GridC) -> "Grid":
        return cls(**{name: getattr(c, name) for name, _ in GridC._fields_})


def grid_make(g: Grid) -> Grid:
    c = g.to_c()
    _ok(lib().gfh_grid_make(ctypes.byref(c)), "gfh_grid_make")
    return Grid.from_c(c)


def grid_tables(g: Grid):
    """(U, B, S) int64 numpy arrays of the grid's fixed-point tables."""
    c = g.to_c()
    J = g.bin_hi - g.bin_lo + 1
    U = np.empty(J + 1, np.int64)
    B = np.empty(g.n_fft, np.int64)
    S = np.empty(g.n_fft, np.int64)
    _ok(lib().gfh_grid_tables(ctypes.byref(c), U.ctypes.data, B.ctypes.data, S.ctypes.data),
        "gfh_grid_tables")
    return U, B, S


def grid_columns(g: Grid):
    """(band int32, f0, f0^n) per column m < n_x0."""
    c = g.to_c()
    band = np.empty(g.n_x0, np.int32)
    f0 = np.empty(g.n_x0, np.float64)
    f0n = np.empty(g.n_x0, np.float64)
    _ok(lib().gfh_grid_columns(ctypes.byref(c), band.ctypes.data, f0.ctypes.data, f0n.ctypes.data),
        "gfh_grid_columns")
    return band, f0, f0n


# ---- GPU entry points -------------------------------------------------------------------------

class Context:
    """gfh_create / gfh_destroy; `stream` is a torch.cuda.Stream, a raw handle or None."""

    def __init__(self, device: int = 0, stream=None):
        self._h = ctypes.c_void_p()
        _ok(lib().gfh_create(ctypes.byref(self._h), device, _stream_handle(stream)), "gfh_create")
        self.device = device

    @property
    def handle(self):
        return self._h

    def set_stream(self, stream) -> None:
        _ok(lib().gfh_set_stream(self._h, _stream_handle(stream)), "gfh_set_stream")

    def check(self) -> int:
        """gfh_check: GFH_OK or GFH_ERR_INPUT (does not raise)."""
        return lib().gfh_check(self._h)

    def close(self) -> None:
        if self._h:
            lib().gfh_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ---- peakmap (Sec. III)
    def peaks_from_power(self, power, bin_lo: int, bin_hi: int, theta: float, fft_out, bin_out):
        """power: float32 device tensor [n_fft][ld]; returns the number of peaks."""
        n = ctypes.c_int64()
        rc = lib().gfh_peaks_from_power(self._h, _ptr(power), power.stride(0), power.shape[0],
                                        bin_lo, bin_hi, theta, _ptr(fft_out), _ptr(bin_out),
                                        fft_out.numel(), ctypes.byref(n))
        _ok(rc, "gfh_peaks_from_power")
        return n.value

    def peakmap(self, series, fs: float, t_fft: float, bin_lo: int, bin_hi: int, theta: float,
                fft_out, bin_out) -> int:
        n = ctypes.c_int64()
        rc = lib().gfh_peakmap(self._h, _ptr(series), series.numel(), fs, t_fft, bin_lo, bin_hi,
                               theta, _ptr(fft_out), _ptr(bin_out), fft_out.numel(),
                               ctypes.byref(n))
        _ok(rc, "gfh_peakmap")
        return n.value

    def peakmap_async(self, series, fs: float, t_fft: float, bin_lo: int, bin_hi: int,
                      theta: float, fft_out, bin_out, n_out) -> None:
        """gfh_peakmap_async: no host synchronisation; min(total, capacity) goes to the device
        int64 `n_out` (a one-element view such as offsets[1:2])."""
        rc = lib().gfh_peakmap_async(self._h, _ptr(series), series.numel(), fs, t_fft, bin_lo,
                                     bin_hi, theta, _ptr(fft_out), _ptr(bin_out),
                                     fft_out.numel(), _ptr(n_out))
        _ok(rc, "gfh_peakmap_async")

    # ---- Hough map + candidates (Sec. IV)
    def hough(self, fft_idx, bins, n_peaks: int, g: Grid, out_map, cands=None, stats=None) -> None:
        c = g.to_c()
        rc = lib().gfh_hough(self._h, _ptr(fft_idx), _ptr(bins), n_peaks, ctypes.byref(c),
                             _ptr(out_map), _ptr(cands), _ptr(stats))
        _ok(rc, "gfh_hough")

    def select(self, hmap, g: Grid, cands, stats=None) -> None:
        c = g.to_c()
        _ok(lib().gfh_select(self._h, _ptr(hmap), ctypes.byref(c), _ptr(cands), _ptr(stats)),
            "gfh_select")


def _stream_handle(stream):
    if stream is None:
        return None
    if hasattr(stream, "cuda_stream"):
        return ctypes.c_void_p(stream.cuda_stream)
    return ctypes.c_void_p(int(stream))


class Plan:
    """gfh_plan_create / gfh_plan_execute / gfh_plan_destroy over several grids."""

    def __init__(self, ctx: Context, grids, maps, cands=None, stats=None, tile=None):
        n = len(grids)
        self._grids_c = (GridC * n)(*[g.to_c() for g in grids])
        self._maps = (ctypes.c_void_p * n)(*[_ptr(m) for m in maps])
        self._cands = (ctypes.c_void_p * n)(*[_ptr(c) for c in cands]) if cands is not None else None
        self._tile = TileConfigC(*(tuple(tile) + (0,) * (4 - len(tile)))) if tile is not None else None
        self._h = ctypes.c_void_p()
        self.ctx = ctx
        rc = lib().gfh_plan_create(ctx.handle, n, self._grids_c, self._maps, self._cands,
                                   _ptr(stats), ctypes.byref(self._tile) if self._tile else None,
                                   ctypes.byref(self._h))
        _ok(rc, "gfh_plan_create")

    def execute(self, fft_idx, bins, offsets, n_lists: int) -> None:
        pk = PeaksC(_ptr(fft_idx), _ptr(bins), _ptr(offsets), n_lists)
        _ok(lib().gfh_plan_execute(self._h, ctypes.byref(pk)), "gfh_plan_execute")

    def autotune(self, fft_idx, bins, offsets, n_lists: int, reps: int = 3):
        """gfh_plan_autotune: returns ((rows, cols, threads), ms per execute) of the chosen shape."""
        pk = PeaksC(_ptr(fft_idx), _ptr(bins), _ptr(offsets), n_lists)
        best = TileConfigC()
        ms = ctypes.c_float()
        _ok(lib().gfh_plan_autotune(self._h, ctypes.byref(pk), reps, ctypes.byref(best),
                                    ctypes.byref(ms)), "gfh_plan_autotune")
        return (best.rows, best.cols, best.threads), ms.value

    def close(self) -> None:
        if self._h:
            lib().gfh_plan_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def candidates_to_numpy(cands_tensor) -> np.ndarray:
    """Device candidate buffer (uint8 tensor of n_bands * 64 bytes) -> structured numpy array."""
    return np.frombuffer(cands_tensor.cpu().numpy().tobytes(), dtype=CANDIDATE_DTYPE)


def peaks_from_power_static(stream, power, bin_lo: int, bin_hi: int, theta: float, fft_out,
                            bin_out, n_out) -> None:
    """gfh_peaks_from_power_static: peak selection without any device allocation, for callers
    whose device memory belongs to another allocator.  Asynchronous on `stream`; the peak count
    goes to the device int64 tensor `n_out`."""
    rc = lib().gfh_peaks_from_power_static(_stream_handle(stream), _ptr(power), power.stride(0),
                                           power.shape[0], bin_lo, bin_hi, theta, _ptr(fft_out),
                                           _ptr(bin_out), fft_out.numel(), _ptr(n_out))
    _ok(rc, "gfh_peaks_from_power_static")
