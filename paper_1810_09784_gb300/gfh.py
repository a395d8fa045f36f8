"""Thin Python binding of libgfh (the C ABI declared in include/gfh.h).

Only argument marshalling lives here: every step of the method runs in the library's CUDA kernels
or its host planner.  torch tensors are accepted as device buffers (their data pointers are passed
to the library) and torch streams as the stream; there is no CPU fallback, and importing this
module fails loudly when the library has not been built.
"""
from __future__ import annotations

import atexit
import ctypes
import dataclasses
import pathlib
import weakref

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
    "gfh_autotune_cache_size", "gfh_autotune_cache_clear", "gfh_hough", "gfh_select", "gfh_peaks_from_power_static",
    "gfh_plan_set_coarse", "gfh_plan_execute_tiles",
    "gfh_synth_peaks", "gfh_synth_images", "gfh_peaks_to_images",
    "gfh_cnn_create", "gfh_cnn_destroy", "gfh_cnn_param_count", "gfh_cnn_get_params",
    "gfh_cnn_set_params", "gfh_cnn_forward", "gfh_cnn_gradients", "gfh_cnn_train_step",
    "gfh_propose_tiles", "gfh_conv3x3", "gfh_select_squares", "gfh_coincide",
    "gfh_n_grid", "gfh_k_segments", "gfh_wait_check",
    "gfh_heterodyne", "gfh_peakmap_complex", "gfh_project_peaks", "gfh_tfft_portions",
    "gfh_heterodyne_band_peaks", "gfh_cnn_get_state", "gfh_cnn_set_state",
    "gfh_cnn_read_tensor", "gfh_line_scores", "gfh_probe_smem_atomics", "gfh_device_sms",
]
# gfh_cnn_read_tensor selectors
CNN_ACT, CNN_DACT, CNN_WBF16 = 0, 10, 20
CNN_POOLED, CNN_LOGITS, CNN_DLOGITS, CNN_LOSS = 30, 31, 32, 33
_ACT_SHAPE = {1: (256, 32), 2: (128, 32), 3: (128, 64), 4: (64, 64), 5: (64, 64)}
N_CLASSES = 4097        # 64 x 64 coarse tiles + no signal
IMG = 256
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
                ("threads", ctypes.c_int32), ("form", ctypes.c_int32)]


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
        u32, u64 = ctypes.c_uint32, ctypes.c_uint64
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
            "gfh_autotune_cache_size": [],
            "gfh_autotune_cache_clear": [],
            "gfh_hough": [vp, vp, vp, i64, P(GridC), vp, vp, vp],
            "gfh_select": [vp, vp, P(GridC), vp, vp],
            "gfh_peaks_from_power_static": [vp, vp, i64, i32, i32, i32, dbl, vp, vp, i64, vp],
            "gfh_plan_set_coarse": [vp, i32, i32, i32],
            "gfh_plan_execute_tiles": [vp, P(PeaksC), vp, i32, vp],
            "gfh_synth_peaks": [vp, u64, i64, i32, i32, i32, u32, u32, vp, vp, vp, i64, P(i64)],
            "gfh_synth_images": [vp, u64, i64, i32, i32, i32, i32, u32, vp, vp, vp, vp],
            "gfh_peaks_to_images": [vp, P(PeaksC), i32, i32, i32, vp, vp],
            "gfh_cnn_create": [vp, i32, u64, P(vp)],
            "gfh_cnn_destroy": [vp],
            "gfh_cnn_get_params": [vp, vp, vp],
            "gfh_cnn_set_params": [vp, vp],
            "gfh_cnn_forward": [vp, vp, i32, vp],
            "gfh_cnn_gradients": [vp, vp, vp, i32, P(ctypes.c_float)],
            "gfh_cnn_train_step": [vp, vp, vp, i32, ctypes.c_float, ctypes.c_float,
                                   P(ctypes.c_float)],
            "gfh_propose_tiles": [vp, vp, i32, vp, i32, ctypes.c_float, vp, vp, vp],
            "gfh_conv3x3": [vp, i32, i32, i32, i32, i32, i32, vp, vp, vp, vp, vp, vp, vp],
            "gfh_select_squares": [vp, vp, P(GridC), i32, i32, i32, vp, vp],
            "gfh_coincide": [vp, vp, i32, vp, i32, dbl, dbl, dbl, vp, vp],
            "gfh_n_grid": [dbl, dbl, dbl, dbl, dbl, dbl, dbl, i32, vp, P(i32)],
            "gfh_wait_check": [vp, i64],
            "gfh_k_segments": [dbl, dbl, dbl, dbl, dbl, dbl, dbl, i32, i32, vp, P(i32)],
            "gfh_heterodyne": [vp, vp, i64, dbl, dbl, dbl, dbl, dbl, vp],
            "gfh_peakmap_complex": [vp, vp, i64, dbl, dbl, i32, i32, dbl, vp, vp, i64, P(i64)],
            "gfh_project_peaks": [vp, vp, vp, i64, dbl, dbl, dbl, dbl, i32, i32, vp],
            "gfh_tfft_portions": [dbl, dbl, dbl, dbl, dbl, i32, i32, vp, P(i32)],
            "gfh_heterodyne_band_peaks": [vp, vp, i64, dbl, dbl, dbl, dbl, dbl, dbl, i32, i32, dbl,
                                          vp, vp, i64, P(i64)],
            "gfh_cnn_get_state": [vp, vp, vp, vp, P(i64)],
            "gfh_cnn_set_state": [vp, vp, vp, vp, i64],
            "gfh_cnn_read_tensor": [vp, i32, i32, vp, i64],
            "gfh_line_scores": [vp, vp, i32, i32, i32, ctypes.c_float, ctypes.c_float,
                                ctypes.c_float, vp, vp],
            "gfh_probe_smem_atomics": [vp, i32, i32, i32, i32, vp, vp],
            "gfh_device_sms": [vp, P(i32)],
        }
        for name, args in sig.items():
            fn = getattr(L, name)
            fn.argtypes = args
            fn.restype = ctypes.c_int
        L.gfh_cnn_param_count.argtypes = [vp]
        L.gfh_cnn_param_count.restype = i64
        L.gfh_strerror.argtypes = [ctypes.c_int]
        L.gfh_strerror.restype = ctypes.c_char_p
        L.gfh_autotune_cache_clear.restype = None
        _lib = L
    return _lib


def strerror(code: int) -> str:
    return lib().gfh_strerror(code).decode()


def autotune_cache_size() -> int:
    """gfh_autotune_cache_size: plan signatures whose tuned tile shape this process keeps."""
    return int(lib().gfh_autotune_cache_size())


def autotune_cache_clear() -> None:
    """gfh_autotune_cache_clear: forget every tuned shape (the next autotune times them all)."""
    lib().gfh_autotune_cache_clear()


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


def n_grid(n_lo: float, n_hi: float, df: float, f_min: float, f_max: float, fdot_hi: float,
           t_obs: float, cap: int = 100000) -> np.ndarray:
    """gfh_n_grid: braking indices of Eq. dn_powlaws (Sec. VI.A)."""
    out = np.empty(cap, np.float64)
    n = ctypes.c_int32()
    _ok(lib().gfh_n_grid(n_lo, n_hi, df, f_min, f_max, fdot_hi, t_obs, cap, out.ctypes.data,
                         ctypes.byref(n)), "gfh_n_grid")
    return out[: n.value].copy()


K_SEGMENT_DTYPE = np.dtype([("k_min", "<f8"), ("dk", "<f8"), ("n_k", "<i4"), ("reserved", "<i4")])


def k_segments(n: float, df: float, f_min: float, f_max: float, fdot_lo: float, fdot_hi: float,
               growth: float = 1.0, max_rows: int = 1 << 30, cap: int = 1 << 20) -> np.ndarray:
    """gfh_k_segments: the Eq. dkeqn k grid (Sec. VI.B) as uniform segments."""
    out = np.zeros(cap, K_SEGMENT_DTYPE)
    cnt = ctypes.c_int32()
    _ok(lib().gfh_k_segments(n, df, f_min, f_max, fdot_lo, fdot_hi, growth, max_rows, cap,
                             out.ctypes.data, ctypes.byref(cnt)), "gfh_k_segments")
    return out[: cnt.value].copy()


PORTION_DTYPE = np.dtype([("level", "<i4"), ("reserved", "<i4"), ("t_begin", "<f8"),
                          ("t_end", "<f8"), ("t_fft", "<f8")])


def tfft_portions(n: float, f_hi: float, fdot_hi: float, t_fft0: float, t_obs: float,
                  max_levels: int, cap: int = 64) -> np.ndarray:
    """gfh_tfft_portions: the Sec. VI.D time portions and their FFT lengths."""
    out = np.zeros(cap, PORTION_DTYPE)
    cnt = ctypes.c_int32()
    _ok(lib().gfh_tfft_portions(n, f_hi, fdot_hi, t_fft0, t_obs, max_levels, cap,
                                out.ctypes.data, ctypes.byref(cnt)), "gfh_tfft_portions")
    return out[: cnt.value].copy()


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

_LIVE_CONTEXTS = weakref.WeakSet()


@atexit.register
def _close_live_contexts() -> None:
    """Contexts (and their plans and networks) still open at exit are destroyed while the CUDA
    runtime and the caller's streams are still alive, not in whatever order the interpreter's
    teardown collects them."""
    for c in list(_LIVE_CONTEXTS):
        try:
            c.close()
        except Exception:
            pass


class Context:
    """gfh_create / gfh_destroy; `stream` is a torch.cuda.Stream, a raw handle or None.  The
    context keeps a reference to the stream object, so the stream outlives it."""

    def __init__(self, device: int = 0, stream=None):
        self._h = ctypes.c_void_p()
        _ok(lib().gfh_create(ctypes.byref(self._h), device, _stream_handle(stream)), "gfh_create")
        self.device = device
        self._stream = stream
        self._children = weakref.WeakSet()     # plans and networks: destroyed before the context
        _LIVE_CONTEXTS.add(self)

    def _adopt(self, child) -> None:
        self._children.add(child)

    @property
    def handle(self):
        return self._h

    def set_stream(self, stream) -> None:
        _ok(lib().gfh_set_stream(self._h, _stream_handle(stream)), "gfh_set_stream")
        self._stream = stream

    def check(self) -> int:
        """gfh_check: GFH_OK or GFH_ERR_INPUT (does not raise)."""
        return lib().gfh_check(self._h)

    def close(self) -> None:
        if self._h:
            for c in list(self._children):
                c.close()
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

    # ---- follow-up of a candidate (Sec. V)
    def heterodyne(self, series, fs: float, t_start: float, f0: float, k: float, n: float,
                   out) -> None:
        """gfh_heterodyne: out (complex64, as many samples as series) = series corrected by the
        spin-down phase of (f0, k, n)."""
        if out.numel() * out.element_size() < 8 * series.numel():
            raise ValueError("output smaller than the series")
        _ok(lib().gfh_heterodyne(self._h, _ptr(series), series.numel(), fs, t_start, f0, k, n,
                                 _ptr(out)), "gfh_heterodyne")

    def peakmap_complex(self, z, fs: float, t_fft: float, bin_lo: int, bin_hi: int, theta: float,
                        fft_out, bin_out) -> int:
        """gfh_peakmap_complex on a complex64 series z; returns the number of peaks."""
        n = ctypes.c_int64()
        n_samples = z.numel() * z.element_size() // 8
        rc = lib().gfh_peakmap_complex(self._h, _ptr(z), n_samples, fs, t_fft, bin_lo, bin_hi,
                                       theta, _ptr(fft_out), _ptr(bin_out), fft_out.numel(),
                                       ctypes.byref(n))
        _ok(rc, "gfh_peakmap_complex")
        return n.value

    def heterodyne_band_peaks(self, series, fs: float, t_start: float, f0: float, k: float,
                              n: float, t_fft: float, bin_lo: int, bin_hi: int, theta: float,
                              fft_out, bin_out) -> int:
        """gfh_heterodyne_band_peaks: the peaks of the series corrected by (f0, k, n), computed
        from the series in one pass; returns the number of peaks."""
        cnt = ctypes.c_int64()
        rc = lib().gfh_heterodyne_band_peaks(self._h, _ptr(series), series.numel(), fs, t_start,
                                             f0, k, n, t_fft, bin_lo, bin_hi, theta,
                                             _ptr(fft_out), _ptr(bin_out), fft_out.numel(),
                                             ctypes.byref(cnt))
        _ok(rc, "gfh_heterodyne_band_peaks")
        return cnt.value

    def project_peaks(self, fft_idx, bins, n_peaks: int, t_first: float, t_hop: float, df: float,
                      fdot: float, bin_lo: int, bin_hi: int, counts) -> None:
        """gfh_project_peaks: counts (int32, bin_hi - bin_lo + 1) of the bin-shifted peaks."""
        _ok(lib().gfh_project_peaks(self._h, _ptr(fft_idx), _ptr(bins), n_peaks, t_first, t_hop,
                                    df, fdot, bin_lo, bin_hi, _ptr(counts)), "gfh_project_peaks")

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

    def sms(self) -> int:
        """The SM count of the context's device."""
        n = ctypes.c_int32()
        _ok(lib().gfh_device_sms(self.handle, ctypes.byref(n)), "gfh_device_sms")
        return n.value

    def probe_smem_atomics(self, mode: int, blocks: int, threads: int, iters: int, cycles,
                           sink) -> None:
        """gfh_probe_smem_atomics: shared-memory atomicAdd throughput kernel (caller times it)."""
        _ok(lib().gfh_probe_smem_atomics(self.handle, mode, blocks, threads, iters, _ptr(cycles),
                                         _ptr(sink)), "gfh_probe_smem_atomics")

    def wait_check(self, cycles: int) -> None:
        """gfh_wait_check: a bounded device wait that runs out (the next check() reports it)."""
        _ok(lib().gfh_wait_check(self._h, cycles), "gfh_wait_check")

    def select_squares(self, hmap, g: Grid, n_sx: int, n_sk: int, out, min_dk: int = 3,
                       stats=None) -> None:
        """gfh_select_squares: two candidates per square into out (uint8 tensor of
        2 n_sx n_sk x 64 bytes)."""
        gc = g.to_c()
        _ok(lib().gfh_select_squares(self._h, _ptr(hmap), ctypes.byref(gc), n_sx, n_sk, min_dk,
                                     _ptr(out), _ptr(stats)), "gfh_select_squares")

    def coincide(self, a, na: int, b, nb: int, dx0: float, dk: float, radius: float, match,
                 dist) -> None:
        """gfh_coincide: nearest candidate of b for each candidate of a (device buffers)."""
        _ok(lib().gfh_coincide(self._h, _ptr(a), na, _ptr(b), nb, dx0, dk, radius, _ptr(match),
                               _ptr(dist)), "gfh_coincide")

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
        ctx._adopt(self)

    def execute(self, fft_idx, bins, offsets, n_lists: int) -> None:
        pk = PeaksC(_ptr(fft_idx), _ptr(bins), _ptr(offsets), n_lists)
        _ok(lib().gfh_plan_execute(self._h, ctypes.byref(pk)), "gfh_plan_execute")

    def autotune(self, fft_idx, bins, offsets, n_lists: int, reps: int = 3):
        """gfh_plan_autotune: returns ((rows, cols, threads, form), ms per execute) of the chosen
        shape."""
        pk = PeaksC(_ptr(fft_idx), _ptr(bins), _ptr(offsets), n_lists)
        best = TileConfigC()
        ms = ctypes.c_float()
        _ok(lib().gfh_plan_autotune(self._h, ctypes.byref(pk), reps, ctypes.byref(best),
                                    ctypes.byref(ms)), "gfh_plan_autotune")
        return (best.rows, best.cols, best.threads, best.form), ms.value

    def set_coarse(self, coarse_k: int, coarse_x: int, max_sel: int) -> None:
        _ok(lib().gfh_plan_set_coarse(self._h, coarse_k, coarse_x, max_sel), "gfh_plan_set_coarse")

    def execute_tiles(self, fft_idx, bins, offsets, n_lists: int, coarse, n_sel: int,
                      full=None) -> None:
        """Exact Hough on the coarse tiles listed in the int32 device tensor coarse [maps][n_sel];
        maps flagged in the int32 device tensor `full` are searched in full."""
        pk = PeaksC(_ptr(fft_idx), _ptr(bins), _ptr(offsets), n_lists)
        _ok(lib().gfh_plan_execute_tiles(self._h, ctypes.byref(pk), _ptr(coarse), n_sel,
                                         _ptr(full)), "gfh_plan_execute_tiles")

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
    whose device memory belongs to another allocator.  Asynchronous on `stream`, which must belong
    to the current device; the total peak count goes to the device int64 tensor `n_out` and may
    exceed fft_out.numel() (then only the first fft_out.numel() peaks, in (bin, FFT) order, are
    written)."""
    rc = lib().gfh_peaks_from_power_static(_stream_handle(stream), _ptr(power), power.stride(0),
                                           power.shape[0], bin_lo, bin_hi, theta, _ptr(fft_out),
                                           _ptr(bin_out), fft_out.numel(), _ptr(n_out))
    _ok(rc, "gfh_peaks_from_power_static")


# ---- statistical peakmaps, images, the proposal network ------------------------------------------

def synth_peaks(ctx: Context, seed: int, sample: int, n_fft: int, bin_lo: int, bin_hi: int,
                p_noise24: int, p_track24: int, track, fft_out, bin_out) -> int:
    """gfh_synth_peaks: the peak list of one sample of the statistical model; returns its length."""
    n = ctypes.c_int64()
    rc = lib().gfh_synth_peaks(ctx.handle, seed, sample, n_fft, bin_lo, bin_hi, p_noise24,
                               p_track24, _ptr(track), _ptr(fft_out), _ptr(bin_out),
                               fft_out.numel(), ctypes.byref(n))
    _ok(rc, "gfh_synth_peaks")
    return n.value


def synth_images(ctx: Context, seed: int, sample0: int, n_fft: int, bin_lo: int, bin_hi: int,
                 p_noise24: int, p_track24, tracks, nplane, images) -> None:
    """gfh_synth_images into the bf16 tensor images [B][256][256][2]."""
    rc = lib().gfh_synth_images(ctx.handle, seed, sample0, images.shape[0], n_fft, bin_lo, bin_hi,
                                p_noise24, _ptr(p_track24), _ptr(tracks), _ptr(nplane),
                                _ptr(images))
    _ok(rc, "gfh_synth_images")


def peaks_to_images(ctx: Context, fft_idx, bins, offsets, n_lists: int, n_fft: int, bin_lo: int,
                    bin_hi: int, nplane, images) -> None:
    """gfh_peaks_to_images: image l from peak list l (device offsets [n_lists + 1])."""
    pk = PeaksC(_ptr(fft_idx), _ptr(bins), _ptr(offsets), n_lists)
    rc = lib().gfh_peaks_to_images(ctx.handle, ctypes.byref(pk), n_fft, bin_lo, bin_hi,
                                   _ptr(nplane), _ptr(images))
    _ok(rc, "gfh_peaks_to_images")


def propose_tiles(ctx: Context, logits, gain, k: int, top, resid, tau: float = -1.0,
                  full=None) -> None:
    """gfh_propose_tiles: the best coarse tiles per map (cut at resid <= tau when tau >= 0), the
    probability left outside them, and the maps that need the full search."""
    rc = lib().gfh_propose_tiles(ctx.handle, _ptr(logits), logits.shape[0], _ptr(gain), k, tau,
                                 _ptr(top), _ptr(resid), _ptr(full))
    _ok(rc, "gfh_propose_tiles")


def line_scores(ctx: Context, images, n_k: int, n_bins: int, beta: float, det_a: float,
                det_c: float, logits, scores=None) -> None:
    """gfh_line_scores: the non-learned proposer's straight-line sums and their logits."""
    rc = lib().gfh_line_scores(ctx.handle, _ptr(images), images.shape[0], n_k, n_bins, beta,
                               det_a, det_c, _ptr(scores), _ptr(logits))
    _ok(rc, "gfh_line_scores")


def conv3x3(ctx: Context, mode: int, cin: int, cout: int, stride: int, batch: int, h: int,
            inp=None, w=None, bias=None, out=None, dout=None, res=None, db=None) -> None:
    """gfh_conv3x3: one 3x3 layer alone (0 forward, 1 input gradient, 2 weight gradient)."""
    rc = lib().gfh_conv3x3(ctx.handle, mode, cin, cout, stride, batch, h, _ptr(inp), _ptr(w),
                           _ptr(bias), _ptr(out), _ptr(dout), _ptr(res), _ptr(db))
    _ok(rc, "gfh_conv3x3")


class Cnn:
    """The proposal network (gfh_cnn_*): device-resident fp32 master weights, bf16 copies."""

    def __init__(self, ctx: Context, max_batch: int, seed: int):
        self.ctx = ctx
        self._h = ctypes.c_void_p()
        _ok(lib().gfh_cnn_create(ctx.handle, max_batch, seed, ctypes.byref(self._h)),
            "gfh_cnn_create")
        ctx._adopt(self)
        self.n_params = int(lib().gfh_cnn_param_count(self._h))

    def params(self) -> np.ndarray:
        out = np.empty(self.n_params, np.float32)
        _ok(lib().gfh_cnn_get_params(self._h, out.ctypes.data, None), "gfh_cnn_get_params")
        return out

    def grads(self) -> np.ndarray:
        out = np.empty(self.n_params, np.float32)
        _ok(lib().gfh_cnn_get_params(self._h, None, out.ctypes.data), "gfh_cnn_get_params")
        return out

    def set_params(self, params: np.ndarray) -> None:
        a = np.ascontiguousarray(params, dtype=np.float32)
        assert a.size == self.n_params
        _ok(lib().gfh_cnn_set_params(self._h, a.ctypes.data), "gfh_cnn_set_params")

    def state(self) -> dict:
        """Training state for a checkpoint: parameters, AdamW moments, step count."""
        p, m, v = (np.empty(self.n_params, np.float32) for _ in range(3))
        step = ctypes.c_int64()
        _ok(lib().gfh_cnn_get_state(self._h, p.ctypes.data, m.ctypes.data, v.ctypes.data,
                                    ctypes.byref(step)), "gfh_cnn_get_state")
        return {"params": p, "m": m, "v": v, "step": int(step.value)}

    def set_state(self, st: dict) -> None:
        p, m, v = (np.ascontiguousarray(st[k], dtype=np.float32) for k in ("params", "m", "v"))
        assert p.size == m.size == v.size == self.n_params
        _ok(lib().gfh_cnn_set_state(self._h, p.ctypes.data, m.ctypes.data, v.ctypes.data,
                                    int(st["step"])), "gfh_cnn_set_state")

    def read_tensor(self, which: int, batch: int) -> np.ndarray:
        """An internal tensor of the last pass (gfh_cnn_read_tensor): bf16 ones as uint16 bits."""
        if CNN_ACT < which <= CNN_ACT + 5 or CNN_DACT < which <= CNN_DACT + 5:
            h, c = _ACT_SHAPE[which % 10]
            out = np.empty((batch, h, h, c), np.uint16)
        elif CNN_WBF16 <= which < CNN_WBF16 + 5:
            l = which - CNN_WBF16
            out = np.empty(((32, 32, 64, 64, 64)[l], 3, 3, (2, 32, 32, 64, 64)[l]), np.uint16)
        elif which == CNN_POOLED:
            out = np.empty((batch, 64, 64), np.float32)
        elif which in (CNN_LOGITS, CNN_DLOGITS):
            out = np.empty((batch, N_CLASSES), np.float32)
        else:
            out = np.empty(batch, np.float32)
        _ok(lib().gfh_cnn_read_tensor(self._h, which, batch, out.ctypes.data, out.nbytes),
            "gfh_cnn_read_tensor")
        return out

    def forward(self, images, logits=None) -> None:
        _ok(lib().gfh_cnn_forward(self._h, _ptr(images), images.shape[0], _ptr(logits)),
            "gfh_cnn_forward")

    def gradients(self, images, labels) -> float:
        loss = ctypes.c_float()
        _ok(lib().gfh_cnn_gradients(self._h, _ptr(images), _ptr(labels), images.shape[0],
                                    ctypes.byref(loss)), "gfh_cnn_gradients")
        return loss.value

    def train_step(self, images, labels, lr: float, weight_decay: float = 0.0,
                   want_loss: bool = True):
        loss = ctypes.c_float()
        _ok(lib().gfh_cnn_train_step(self._h, _ptr(images), _ptr(labels), images.shape[0], lr,
                                     weight_decay, ctypes.byref(loss) if want_loss else None),
            "gfh_cnn_train_step")
        return loss.value if want_loss else None

    def close(self) -> None:
        if self._h:
            lib().gfh_cnn_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
