"""The learned tile proposer around the exact Hough: data, training and evaluation.

The paper names machine learning as future work (Sec. VIII).  Here a small convolutional network
looks at a coarse image of a peakmap and ranks the coarse (x0, k) tiles of its Hough map (Sec. IV),
so that the exact Hough runs on the best 32 of 64 x 64 tiles only.  Candidates always come from
exact counts; a map whose proposal leaves more than `tau` probability outside the chosen tiles is
searched in full instead (the exact Hough is the fallback and the reference for recall).

Workload: maps shaped like the small plain search (1024 Hz sampling, 1800 s, T_FFT 2 s, 1799 FFTs,
band 100-400 Hz, 500 k rows), one braking index per map from n = 2.0, 2.1, ..., 7.0 (sample s has
index s mod 51), half of them with one power-law injection (Sec. II Eq. powlaws) of spectral SNR
uniform in [2, 8], f0 uniform over the band, k on a uniformly drawn row of the map's k grid.
Peakmaps (spec.peakmaps = "series", the default) come from the method's own chain: a seeded
white-noise strain series with the sample's injection (synth), then the library's peakmap
(short FFTs, equaliser, threshold 2.5, local maximum; Sec. III).  The alternative "statistical"
model draws each cell independently on the GPU (a noise peak with the probability p0 of an
equalised exponential spectrum above 2.5 that is a local maximum; the track's cell with the
probability that a signal of that SNR exceeds 2.5); it serves the kernel tests.

Labels: class d * 64 + xt, xt = floor((f0 - ana_lo) / (ana_hi - ana_lo) * 64) and drift class
d = floor(r (f0 / f_max)^n * 64 / K) (a track on k row r drifts r x0 columns over the observation,
one column spanning (f / f_max)^n bins), or 4096 without a signal.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

from . import gfh, synth

N_GRID = tuple(round(2.0 + 0.1 * i, 10) for i in range(51))
TILES = 64
NULL_CLASS = TILES * TILES
THETA = 2.5


@dataclasses.dataclass(frozen=True)
class ProposerSpec:
    fs: float = 1024.0
    t_obs: float = 1800.0
    t_fft: float = 2.0
    bin_lo: int = 200
    bin_hi: int = 799
    n_k: int = 500
    ana_lo: float = 100.0
    ana_hi: float = 400.0
    p_noise: float = 0.0755         # strict local maximum of an exp(1) spectrum above 2.5
    snr_lo: float = 2.0
    snr_hi: float = 8.0
    p_signal: float = 0.5
    seed: int = 20181023
    peakmaps: str = "series"        # "series" (series -> gfh_peakmap) or "statistical"

    @property
    def n_fft(self) -> int:
        N = int(round(self.fs * self.t_fft))
        return (int(round(self.fs * self.t_obs)) - N) // (N // 2) + 1

    @property
    def df(self) -> float:
        return 1.0 / self.t_fft

    @property
    def p_noise24(self) -> int:
        return int(round(self.p_noise * 2 ** 24))

    def grid_fields(self, n: float, list_idx: int = 0) -> dict:
        return dict(n=n, df=self.df, bin_lo=self.bin_lo, bin_hi=self.bin_hi, n_fft=self.n_fft,
                    t_first=self.t_fft / 2, t_hop=self.t_fft / 2, t_obs=self.t_obs, n_k=self.n_k,
                    k_min=0.0, dk=0.0, f_max=0.0, ana_lo=self.ana_lo, ana_hi=self.ana_hi,
                    band_hz=1.0, list=list_idx)


def track_probability(snr) -> np.ndarray:
    """P(|X|^2 / E|noise|^2 > 2.5) for a bin holding a signal of power `snr` noise units: half a
    non-central chi-square of 2 degrees of freedom and non-centrality 2 snr."""
    import scipy.stats
    return scipy.stats.ncx2.sf(2 * THETA, 2, 2 * np.asarray(snr, np.float64))


_GRIDS: dict = {}


def grid_of(spec: ProposerSpec, n: float) -> gfh.Grid:
    key = (spec, n)
    if key not in _GRIDS:
        _GRIDS[key] = gfh.grid_make(gfh.Grid(**spec.grid_fields(n)))
    return _GRIDS[key]


@dataclasses.dataclass
class Samples:
    index: np.ndarray       # sample ids
    n: np.ndarray
    signal: np.ndarray      # bool
    f0: np.ndarray
    row: np.ndarray         # k row of the injection (-1 without)
    k: np.ndarray
    snr: np.ndarray
    p_track24: np.ndarray   # uint32
    tracks: np.ndarray      # [B][n_fft] int32 bin per FFT or -1
    labels: np.ndarray      # int32 class
    col: np.ndarray         # x0 column of the injection (-1 without)
    nplane: np.ndarray      # float32
    gain: np.ndarray        # [B][64][2] float32 (ga, gb)
    phase0: np.ndarray      # initial phase of the injection [rad]


def draw(spec: ProposerSpec, index) -> Samples:
    """Parameters, tracks and labels of samples `index` (deterministic functions of the ids)."""
    s = np.asarray(index, np.int64)
    u = [synth.hashed_uniform(spec.seed, s.astype(np.uint64), 2, slot) for slot in range(5)]
    n = np.array([N_GRID[i % len(N_GRID)] for i in s])
    signal = u[0] < spec.p_signal
    f_top = spec.bin_hi * spec.df
    f0 = spec.ana_lo + u[1] * (f_top - spec.ana_lo)
    row = np.minimum((u[2] * spec.n_k).astype(np.int64), spec.n_k - 1)
    snr = spec.snr_lo + u[3] * (spec.snr_hi - spec.snr_lo)
    p24 = np.where(signal, np.round(track_probability(snr) * 2 ** 24), 0).astype(np.uint32)
    B = s.size
    tracks = np.full((B, spec.n_fft), -1, np.int32)
    labels = np.full(B, NULL_CLASS, np.int32)
    col = np.full(B, -1, np.int64)
    k = np.zeros(B)
    gain = np.zeros((B, TILES, 2), np.float32)
    xt_w = (spec.ana_hi - spec.ana_lo) / TILES
    fa = spec.ana_lo + xt_w * np.arange(TILES)
    for b in range(B):
        g = grid_of(spec, float(n[b]))
        f_max = g.f_max
        gain[b, :, 0] = (f_max / fa) ** n[b]
        gain[b, :, 1] = (f_max / (fa + xt_w)) ** n[b]
        if not signal[b]:
            row[b] = -1
            continue
        k[b] = g.k_min + row[b] * g.dk
        tr = synth.powerlaw_track(float(f0[b]), float(k[b]), float(n[b]), spec.df, spec.n_fft,
                                  spec.t_fft / 2, spec.t_fft / 2)
        tr[(tr < spec.bin_lo) | (tr > spec.bin_hi)] = -1
        tracks[b] = tr
        xt = min(TILES - 1, int((f0[b] - spec.ana_lo) / (spec.ana_hi - spec.ana_lo) * TILES))
        d = min(TILES - 1, int(row[b] * (f0[b] / f_max) ** n[b] * TILES / spec.n_k))
        labels[b] = d * TILES + xt
        col[b] = int(math.floor((f0[b] ** (1.0 - n[b]) - g.x0_min) / g.dx0))
    return Samples(s, n, signal, f0, row, k, snr, p24, tracks, labels, col,
                   ((n - 2.0) / 5.0).astype(np.float32), gain, 2.0 * math.pi * u[4])


def injection_of(spec: ProposerSpec, smp: Samples, b: int):
    """The power-law signal of sample b of a draw (None without one): amplitude for its spectral
    SNR with spec.fs * spec.t_fft samples per FFT."""
    if not smp.signal[b]:
        return None
    N = int(round(spec.fs * spec.t_fft))
    return synth.Injection(f0=float(smp.f0[b]), k=float(smp.k[b]), n=float(smp.n[b]),
                           amp=synth.amplitude_for_snr(float(smp.snr[b]), 1.0, N),
                           phase0=float(smp.phase0[b]))


def series_seed(spec: ProposerSpec, sample: int) -> int:
    """Seed of the noise of sample `sample`'s strain series."""
    return int(synth.sample_key(spec.seed, np.uint64(sample), 3))


class PeakSource:
    """Peak lists of up to max_maps samples on the device, sample i of a draw -> list i, compacted
    so that list i is [offsets[i], offsets[i + 1]).  Series peakmaps: each sample's strain series is
    drawn on the device and searched by gfh_peakmap_async into its own slot; statistical ones come
    from gfh_synth_peaks.  One host synchronisation per load (the list lengths)."""

    def __init__(self, ctx: gfh.Context, spec: ProposerSpec, max_maps: int):
        import torch
        self.torch, self.ctx, self.spec = torch, ctx, spec
        nb = spec.bin_hi - spec.bin_lo + 1
        self.cap = int(spec.n_fft * nb * 0.12) + 4096
        self.fft = torch.empty(max_maps * self.cap, dtype=torch.int32, device="cuda")
        self.bin = torch.empty(max_maps * self.cap, dtype=torch.int32, device="cuda")
        self.cnt = torch.zeros(max_maps, dtype=torch.int64, device="cuda")
        self.offsets = torch.zeros(max_maps + 1, dtype=torch.int64, device="cuda")
        self.max_maps = max_maps
        self.x = None
        if spec.peakmaps == "series":
            self.x = torch.empty(int(round(spec.fs * spec.t_obs)), dtype=torch.float32, device="cuda")

    def load(self, smp: Samples) -> None:
        torch, ctx, spec = self.torch, self.ctx, self.spec
        B = smp.index.size
        assert B <= self.max_maps
        if spec.peakmaps == "series":
            for i in range(B):
                inj = injection_of(spec, smp, i)
                synth.strain_series_device(self.x, spec.fs, series_seed(spec, int(smp.index[i])),
                                           () if inj is None else (inj,))
                o = i * self.cap
                ctx.peakmap_async(self.x, spec.fs, spec.t_fft, spec.bin_lo, spec.bin_hi, THETA,
                                  self.fft[o:o + self.cap], self.bin[o:o + self.cap],
                                  self.cnt[i:i + 1])
            counts = self.cnt[:B].cpu().numpy()
            if ctx.check() != gfh.GFH_OK:
                raise RuntimeError("peakmap capacity or input check failed")
        else:
            tracks = torch.from_numpy(smp.tracks).cuda()
            counts = np.zeros(B, np.int64)
            for i in range(B):
                o = i * self.cap
                counts[i] = gfh.synth_peaks(ctx, spec.seed, int(smp.index[i]), spec.n_fft,
                                            spec.bin_lo, spec.bin_hi, spec.p_noise24,
                                            int(smp.p_track24[i]), tracks[i],
                                            self.fft[o:o + self.cap], self.bin[o:o + self.cap])
        offs = np.concatenate([[0], np.cumsum(counts)]).astype(np.int64)
        self.fft_c = torch.cat([self.fft[i * self.cap:i * self.cap + int(counts[i])] for i in range(B)])
        self.bin_c = torch.cat([self.bin[i * self.cap:i * self.cap + int(counts[i])] for i in range(B)])
        self.offsets[:B + 1].copy_(torch.from_numpy(offs))
        self.counts = counts.astype(np.int64)
        self.offs_host = [int(v) for v in offs]
        self.n_lists = B


class DeviceBatch:
    """Device buffers of one batch: images, labels, tracks, per-sample scalars."""

    def __init__(self, spec: ProposerSpec, batch: int, device="cuda"):
        import torch
        self.torch = torch
        self.images = torch.empty((batch, 256, 256, 2), dtype=torch.bfloat16, device=device)
        self.labels = torch.empty(batch, dtype=torch.int32, device=device)
        self.tracks = torch.empty((batch, spec.n_fft), dtype=torch.int32, device=device)
        self.p24 = torch.empty(batch, dtype=torch.int32, device=device)
        self.nplane = torch.empty(batch, dtype=torch.float32, device=device)
        self.gain = torch.empty((batch, TILES, 2), dtype=torch.float32, device=device)
        self.logits = torch.empty((batch, gfh.N_CLASSES), dtype=torch.float32, device=device)

    def load(self, ctx: gfh.Context, spec: ProposerSpec, smp: Samples) -> int:
        """Uploads a draw and renders its images on the GPU (series peakmaps: through gfh_peakmap
        and gfh_peaks_to_images; statistical ones: gfh_synth_images); returns the batch size."""
        torch = self.torch
        B = smp.index.size
        self.labels[:B].copy_(torch.from_numpy(smp.labels))
        self.tracks[:B].copy_(torch.from_numpy(smp.tracks))
        self.p24[:B].copy_(torch.from_numpy(smp.p_track24.view(np.int32)))
        self.nplane[:B].copy_(torch.from_numpy(smp.nplane))
        self.gain[:B].copy_(torch.from_numpy(smp.gain))
        if spec.peakmaps == "series":
            if getattr(self, "source", None) is None:
                self.source = PeakSource(ctx, spec, self.images.shape[0])
            src = self.source
            src.load(smp)
            gfh.peaks_to_images(ctx, src.fft_c, src.bin_c, src.offsets, B, spec.n_fft,
                                spec.bin_lo, spec.bin_hi, self.nplane[:B], self.images[:B])
        else:
            assert np.all(np.diff(smp.index) == 1), "the statistical images take consecutive samples"
            gfh.synth_images(ctx, spec.seed, int(smp.index[0]), spec.n_fft, spec.bin_lo,
                             spec.bin_hi, spec.p_noise24, self.p24[:B], self.tracks[:B],
                             self.nplane[:B], self.images[:B])
        return B


class ImageCache:
    """Images and labels of samples [first, first + count) rendered once and kept on the device
    (256 KB per image), so that several training passes draw each series and peakmap only once."""

    def __init__(self, ctx: gfh.Context, spec: ProposerSpec, first: int, count: int,
                 chunk: int = 256, log=None):
        import torch
        self.first, self.count = first, count
        self.images = torch.empty((count, 256, 256, 2), dtype=torch.bfloat16, device="cuda")
        self.labels = torch.empty(count, dtype=torch.int32, device="cuda")
        buf = DeviceBatch(spec, chunk)
        for c0 in range(0, count, chunk):
            B = min(chunk, count - c0)
            buf.load(ctx, spec, draw(spec, np.arange(first + c0, first + c0 + B)))
            self.images[c0:c0 + B].copy_(buf.images[:B])
            self.labels[c0:c0 + B].copy_(buf.labels[:B])
            if log and (c0 // chunk) % 50 == 0:
                log(f"images {c0 + B}/{count}")

    def batch(self, s0: int, B: int):
        o = s0 - self.first
        assert 0 <= o and o + B <= self.count
        return self.images[o:o + B], self.labels[o:o + B]


def save_checkpoint(path, state: dict, meta: dict) -> None:
    """Writes a training state (gfh.Cnn.state(): parameters, AdamW moments, step count) and a
    JSON-serialisable description (schedule position, tau, data recipe) to one .npz file."""
    import json
    np.savez(path, params=np.asarray(state["params"], np.float32),
             m=np.asarray(state["m"], np.float32), v=np.asarray(state["v"], np.float32),
             step=np.int64(state["step"]), meta=np.frombuffer(json.dumps(meta).encode(), np.uint8))


def load_checkpoint(path) -> tuple:
    """(state, meta) written by save_checkpoint."""
    import json
    with np.load(path) as z:
        state = {"params": z["params"].copy(), "m": z["m"].copy(), "v": z["v"].copy(),
                 "step": int(z["step"])}
        meta = json.loads(bytes(z["meta"]).decode())
    return state, meta


def train(ctx: gfh.Context, net: gfh.Cnn, spec: ProposerSpec, first: int, count: int,
          batch: int = 256, lr: float = 2e-3, weight_decay: float = 1e-4, log=None,
          cache: ImageCache | None = None, start_step: int = 0) -> list:
    """AdamW over samples [first, first + count) in order, cosine learning-rate decay, from step
    `start_step` of the pass on (a resumed pass); images from `cache` when given, else rendered per
    batch; returns the loss of every step taken."""
    buf = None if cache is not None else DeviceBatch(spec, batch)
    steps = (count + batch - 1) // batch
    losses = []
    for st in range(start_step, steps):
        s0 = first + st * batch
        B = min(batch, first + count - s0)
        if cache is not None:
            images, labels = cache.batch(s0, B)
        else:
            buf.load(ctx, spec, draw(spec, np.arange(s0, s0 + B)))
            images, labels = buf.images[:B], buf.labels[:B]
        lr_t = lr * 0.5 * (1.0 + math.cos(math.pi * st / steps))
        loss = net.train_step(images, labels, lr_t, weight_decay)
        losses.append(loss)
        if log and (st % 50 == 0 or st == steps - 1):
            log(f"step {st}/{steps} loss {loss:.4f} lr {lr_t:.2e}")
    return losses


# ---- evaluation against the full exact Hough ---------------------------------------------------------

class HoughBank:
    """One batched plan over the 51 braking indices (map b reads peak list b, coarse tiles 64 x 64)
    with its maps and candidate buffers."""

    def __init__(self, ctx: gfh.Context, spec: ProposerSpec, max_sel: int = 256, tile=None):
        import torch
        self.torch = torch
        self.spec = spec
        self.ctx = ctx
        self.grids = [gfh.grid_make(gfh.Grid(**spec.grid_fields(n, i))) for i, n in enumerate(N_GRID)]
        self.maps = [torch.empty((g.n_k, g.ld_x0), dtype=torch.int32, device="cuda") for g in self.grids]
        self.cands = [torch.empty(g.n_bands * 64, dtype=torch.uint8, device="cuda") for g in self.grids]
        self.plan = gfh.Plan(ctx, self.grids, self.maps, self.cands, tile=tile)
        self.plan.set_coarse(TILES, TILES, max_sel)
        self.max_sel = max_sel
        self.source = PeakSource(ctx, spec, len(N_GRID))
        self.counts = np.zeros(len(N_GRID), np.int64)

    def load_peaks(self, smp: Samples) -> None:
        """Peak lists of the 51 samples smp (sample i -> list i), made on the GPU."""
        src = self.source
        src.load(smp)
        self.fft_c, self.bin_c, self.offsets = src.fft_c, src.bin_c, src.offsets
        self.counts, self.offs_host = src.counts, src.offs_host

    def updates(self) -> int:
        """Hough updates of the full search of the loaded lists: peaks x k rows per map."""
        return int(sum(self.counts[i] * g.n_k for i, g in enumerate(self.grids)))

    def autotune(self, reps: int = 2):
        """Tile shape of the plan timed on the loaded peak lists (the coarse tiles follow it)."""
        return self.plan.autotune(self.fft_c, self.bin_c, self.offsets, len(N_GRID), reps)

    def full(self) -> None:
        self.plan.execute(self.fft_c, self.bin_c, self.offsets, len(N_GRID))

    def pruned(self, coarse, n_sel: int, full_flags=None) -> None:
        self.plan.execute_tiles(self.fft_c, self.bin_c, self.offsets, len(N_GRID), coarse, n_sel,
                                full_flags)

    def candidates(self) -> list:
        return [gfh.candidates_to_numpy(c) for c in self.cands]


def detected(cands: np.ndarray, col: int, row: int, radius: float = 3.0) -> bool:
    """A candidate within distance `radius` (x0 columns, k rows) of the injection (Sec. IV)."""
    ok = cands["count"] >= 0
    d2 = (cands["col"][ok] - col) ** 2 + (cands["row"][ok] - row) ** 2
    return bool(np.any(d2 <= radius * radius))


class PrunedSearch:
    """The proposer-guided search of the bank's loaded peak lists, all on the device without a
    host round trip: images from the peak lists, the network, the proposals (at most n_sel tiles,
    cut where the probability left outside is at most tau), and one exact-Hough launch over the
    proposed coarse tiles of every map and all tiles of the maps whose proposal cannot reach tau."""

    def __init__(self, ctx: gfh.Context, net: gfh.Cnn, bank: HoughBank, tau: float,
                 n_sel: int = 32):
        import torch
        spec = bank.spec
        nl = len(N_GRID)
        assert n_sel <= bank.max_sel
        self.ctx, self.net, self.bank, self.tau, self.n_sel = ctx, net, bank, tau, n_sel
        smp = draw(spec, np.arange(nl))            # gains and n planes depend on the map slot only
        self.gain = torch.from_numpy(smp.gain).cuda()
        self.nplane = torch.from_numpy(smp.nplane).cuda()
        self.images = torch.empty((nl, 256, 256, 2), dtype=torch.bfloat16, device="cuda")
        self.logits = torch.empty((nl, gfh.N_CLASSES), dtype=torch.float32, device="cuda")
        self.top = torch.empty((nl, n_sel), dtype=torch.int32, device="cuda")
        self.resid = torch.empty(nl, dtype=torch.float32, device="cuda")
        self.full = torch.empty(nl, dtype=torch.int32, device="cuda")

    def propose(self) -> None:
        spec, bank = self.bank.spec, self.bank
        gfh.peaks_to_images(self.ctx, bank.fft_c, bank.bin_c, bank.offsets, len(N_GRID),
                            spec.n_fft, spec.bin_lo, spec.bin_hi, self.nplane, self.images)
        self.net.forward(self.images, self.logits)
        gfh.propose_tiles(self.ctx, self.logits, self.gain, self.n_sel, self.top, self.resid,
                          self.tau, self.full)

    def run(self) -> None:
        self.propose()
        self.bank.pruned(self.top, self.n_sel, self.full)


def evaluate(ctx: gfh.Context, net: gfh.Cnn, spec: ProposerSpec, first: int, count: int,
             bank: HoughBank, tau: float, n_sel: int = 32, log=None) -> dict:
    """Per-map records of the pruned search (PrunedSearch) against the full exact Hough on samples
    [first, first + count), in batches of 51 maps (first and count multiples of 51, so that
    sample s lands on the bank's map s mod 51)."""
    nl = len(N_GRID)
    # sample s has braking index N_GRID[s % 51] = the grid of map s % 51 of the bank
    assert first % nl == 0 and count % nl == 0, "evaluate whole batches of 51 maps"
    search = PrunedSearch(ctx, net, bank, tau, n_sel)
    rec = {k: [] for k in ("signal", "resid", "full", "tiles", "det_full", "det_pruned", "agree",
                           "truth_in_top", "f0", "n", "row")}
    for b0 in range(first, first + count, nl):
        smp = draw(spec, np.arange(b0, b0 + nl))
        bank.load_peaks(smp)
        bank.full()
        full = bank.candidates()
        search.run()
        pr = bank.candidates()
        r = search.resid.cpu().numpy()
        fl = search.full.cpu().numpy()
        tp = search.top.cpu().numpy()
        for i in range(nl):
            rec["signal"].append(bool(smp.signal[i]))
            rec["resid"].append(float(r[i]))
            rec["full"].append(bool(fl[i]))
            rec["tiles"].append(4096 if fl[i] else int((tp[i] >= 0).sum()))
            rec["f0"].append(float(smp.f0[i]))
            rec["n"].append(float(smp.n[i]))
            rec["row"].append(int(smp.row[i]))
            if not smp.signal[i]:
                for k in ("det_full", "det_pruned", "agree", "truth_in_top"):
                    rec[k].append(False)
                continue
            kt = int(smp.row[i]) * TILES // spec.n_k
            xt = min(TILES - 1, int((smp.f0[i] - spec.ana_lo) / (spec.ana_hi - spec.ana_lo) * TILES))
            rec["truth_in_top"].append(bool(fl[i]) or kt * TILES + xt in set(tp[i].tolist()))
            cf, cp = full[i], pr[i]
            rec["det_full"].append(detected(cf, int(smp.col[i]), int(smp.row[i])))
            rec["det_pruned"].append(detected(cp, int(smp.col[i]), int(smp.row[i])))
            band = int(math.floor(smp.f0[i] - spec.ana_lo))
            rec["agree"].append(bool(0 <= band < cf.size and cp["count"][band] == cf["count"][band]))
        if log and ((b0 - first) // nl) % 20 == 0:
            log(f"eval {b0 + nl - first}/{count}")
    return {k: np.array(v) for k, v in rec.items()}


def summarize(rec: dict) -> dict:
    """Recall (detections of the full search that the pruned search keeps), agreement of the
    injection band's top count, fallback (full-search) rates, tiles searched per map."""
    sig = rec["signal"]
    det_full = rec["det_full"] & sig
    kept = det_full & rec["det_pruned"]
    return dict(maps=int(sig.size), injected=int(sig.sum()),
                det_full=int(det_full.sum()), det_kept=int(kept.sum()),
                recall=float(kept.sum() / max(1, det_full.sum())),
                agreement=float((rec["agree"] & sig).sum() / max(1, sig.sum())),
                fallback_frac=float(rec["full"].mean()),
                fallback_injected=float(rec["full"][sig].mean()) if sig.any() else 0.0,
                fallback_noise=float(rec["full"][~sig].mean()) if (~sig).any() else 0.0,
                mean_tiles_pruned=float(rec["tiles"][~rec["full"]].mean()) if (~rec["full"]).any() else 0.0,
                truth_in_top=float(rec["truth_in_top"][sig].mean()) if sig.any() else 0.0)


def choose_tau(ctx: gfh.Context, net: gfh.Cnn, spec: ProposerSpec, first: int, count: int,
               bank: HoughBank, n_sel: int, target: float = 0.995,
               taus=(0.3, 0.2, 0.15, 0.1, 0.075, 0.05, 0.03, 0.02, 0.01, 0.005)) -> tuple:
    """The largest tau whose recall on the validation samples reaches `target`."""
    for tau in taus:
        sm = summarize(evaluate(ctx, net, spec, first, count, bank, tau, n_sel))
        if sm["recall"] >= target:
            return tau, sm
    return 0.0, summarize(evaluate(ctx, net, spec, first, count, bank, 0.0, n_sel))


def train_default(ctx: gfh.Context, net: gfh.Cnn, spec: ProposerSpec, epochs: int = 3,
                  n_train: int = 100000, batch: int = 256, lr: float = 2e-3, log=None,
                  checkpoint=None, resume=None, cache: ImageCache | None = None) -> list:
    """The training schedule of the proposer: `epochs` passes over samples [0, n_train), each a
    cosine decay from lr / 2^epoch.  Series images are rendered once (ImageCache).  `checkpoint`:
    a path written after every pass (state and schedule position); `resume`: a (state, meta) pair
    from load_checkpoint to continue from."""
    e0, st0 = 0, 0
    if resume is not None:
        state, meta = resume
        net.set_state(state)
        e0, st0 = int(meta["epoch"]), int(meta["step_in_epoch"])
    if cache is None and spec.peakmaps == "series" and e0 < epochs:
        cache = ImageCache(ctx, spec, 0, n_train, log=log)
    losses = []
    for e in range(e0, epochs):
        losses += train(ctx, net, spec, 0, n_train, batch=batch, lr=lr * 0.5 ** e, log=log,
                        cache=cache, start_step=st0 if e == e0 else 0)
        if checkpoint is not None:
            save_checkpoint(checkpoint, net.state(),
                            {"epoch": e + 1, "step_in_epoch": 0, "epochs": epochs,
                             "n_train": n_train, "batch": batch, "lr": lr,
                             "peakmaps": spec.peakmaps})
    return losses


# ---- the non-learned proposer ------------------------------------------------------------------

class LineHeuristic:
    """Stand-in for the network in PrunedSearch: gfh_line_scores ranks each class by the peak
    counts along its straight mid-drift line in the image (no learning): class logits beta z, and
    p(no signal) = 1 / (1 + exp(det_a (zmax - det_b))) from the largest standardised line sum.
    beta, det_a and det_b are its only numbers, fitted by calibrate_heuristic."""

    def __init__(self, ctx: gfh.Context, spec: ProposerSpec, beta: float = 1.0,
                 det_a: float = 1.0, det_b: float = 6.0):
        self.ctx, self.spec = ctx, spec
        self.beta, self.det_a, self.det_b = beta, det_a, det_b

    def forward(self, images, logits, scores=None) -> None:
        spec = self.spec
        gfh.line_scores(self.ctx, images, spec.n_k, spec.bin_hi - spec.bin_lo + 1, self.beta,
                        self.det_a, self.det_a * self.det_b, logits, scores)


def calibrate_heuristic(ctx: gfh.Context, spec: ProposerSpec, first: int, count: int,
                        betas=(0.5, 1.0, 2.0, 3.0, 4.0, 6.0, 8.0, 12.0),
                        slopes=(0.25, 0.5, 1.0, 2.0, 4.0),
                        thresholds=tuple(np.linspace(2.0, 14.0, 49))) -> LineHeuristic:
    """The (beta, det_a, det_b) of least mean cross-entropy of the line-sum logits against the
    labels of samples [first, first + count): a three-number fit, as a temperature and a detection
    threshold would be."""
    import torch
    h = LineHeuristic(ctx, spec)
    buf = DeviceBatch(spec, 256)
    zs, labels = [], []
    scores = torch.empty((256, TILES * TILES), dtype=torch.float32, device="cuda")
    logits = torch.empty((256, gfh.N_CLASSES), dtype=torch.float32, device="cuda")
    for c0 in range(first, first + count, 256):
        B = min(256, first + count - c0)
        smp = draw(spec, np.arange(c0, c0 + B))
        buf.load(ctx, spec, smp)
        h.forward(buf.images[:B], logits[:B], scores[:B])
        sc = scores[:B].double().cpu().numpy()
        sd = sc.std(axis=1, keepdims=True)
        zs.append((sc - sc.mean(axis=1, keepdims=True)) / np.where(sd > 0, sd, 1.0))
        labels.append(smp.labels)
    z = np.concatenate(zs)
    y = np.concatenate(labels).astype(np.int64)
    sig = y < NULL_CLASS
    zmax = z.max(axis=1)
    zy = z[np.arange(y.size), np.minimum(y, NULL_CLASS - 1)]
    best = None
    for beta in betas:
        bz = beta * z
        m = bz.max(axis=1)
        lse = m + np.log(np.exp(bz - m[:, None]).sum(axis=1))
        for a in slopes:
            for b in thresholds:
                u = a * (b - zmax)                       # no-signal logit minus LSE
                sp = np.logaddexp(0.0, u)
                nll = np.where(sig, lse + sp - beta * zy, np.logaddexp(0.0, -u))
                ce = float(nll.mean())
                if best is None or ce < best[0]:
                    best = (ce, beta, a, float(b))
    h.beta, h.det_a, h.det_b = best[1], best[2], best[3]
    h.cross_entropy = best[0]
    return h


# ---- command line: train a checkpoint, or evaluate one -------------------------------------------

DEFAULT_CHECKPOINT = "weights/proposer_series.npz"
VALIDATION_FIRST, HELD_OUT_FIRST = 200022, 100011


def checkpoint_path(name: str = DEFAULT_CHECKPOINT):
    import pathlib
    return pathlib.Path(__file__).resolve().parent / name


def _main(argv=None) -> None:
    import argparse
    import json
    import time

    import torch
    ap = argparse.ArgumentParser(description="Train (or evaluate) the tile proposer on the GPU.")
    ap.add_argument("cmd", choices=["train", "eval"])
    ap.add_argument("--out", default=str(checkpoint_path()))
    ap.add_argument("--epochs", type=int, default=3)
    ap.add_argument("--n-train", type=int, default=100000)
    ap.add_argument("--val-maps", type=int, default=51 * 40)
    ap.add_argument("--eval-maps", type=int, default=51 * 196)
    ap.add_argument("--resume", default=None)
    args = ap.parse_args(argv)
    log = lambda m: print(m, flush=True)
    stream = torch.cuda.Stream()
    ctx = gfh.Context(0, stream)
    spec = ProposerSpec()
    meta = {}
    with torch.cuda.stream(stream):
        net = gfh.Cnn(ctx, 256, seed=1)
        if args.cmd == "train":
            t0 = time.perf_counter()
            resume = load_checkpoint(args.resume) if args.resume else None
            losses = train_default(ctx, net, spec, epochs=args.epochs, n_train=args.n_train,
                                   log=log, checkpoint=args.out + ".partial.npz", resume=resume)
            torch.cuda.synchronize()
            meta.update(train_s=round(time.perf_counter() - t0, 1),
                        final_loss=float(np.mean(losses[-20:])) if losses else None)
        else:
            st, meta = load_checkpoint(args.out)
            net.set_state(st)
        bank = HoughBank(ctx, spec, max_sel=256)
        bank.load_peaks(draw(spec, np.arange(VALIDATION_FIRST, VALIDATION_FIRST + 51)))
        bank.autotune()
        heur = calibrate_heuristic(ctx, spec, 0, 4096)
        meta["heuristic"] = {"beta": heur.beta, "det_a": heur.det_a, "det_b": heur.det_b,
                             "cross_entropy": heur.cross_entropy, "calibration_maps": 4096}
        for cap in (32, 256):
            for name, scorer in (("network", net), ("heuristic", heur)):
                tau, val = choose_tau(ctx, scorer, spec, VALIDATION_FIRST, args.val_maps, bank, cap)
                summ = summarize(evaluate(ctx, scorer, spec, HELD_OUT_FIRST, args.eval_maps, bank,
                                          tau, cap))
                meta.setdefault("tau", {}).setdefault(name, {})[str(cap)] = tau
                meta.setdefault("validation", {}).setdefault(name, {})[str(cap)] = val
                meta.setdefault("held_out", {}).setdefault(name, {})[str(cap)] = summ
                log(f"{name} <= {cap} tiles: tau {tau} held-out {json.dumps(summ)}")
        meta.update(epoch=args.epochs, step_in_epoch=0, epochs=args.epochs, n_train=args.n_train,
                    peakmaps=spec.peakmaps, validation_first=VALIDATION_FIRST,
                    held_out_first=HELD_OUT_FIRST, eval_maps=args.eval_maps)
        save_checkpoint(args.out, net.state(), meta)
        log(f"wrote {args.out}")
    net.close()
    bank.plan.close()
    ctx.close()


if __name__ == "__main__":
    _main()
