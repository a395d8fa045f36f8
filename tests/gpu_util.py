"""Helpers shared by the GPU parity tests: device buffers and oracle comparisons."""
import dataclasses

import numpy as np

from oracle import gfh_oracle as O


def oracle_grid(fields):
    keep = {f.name for f in dataclasses.fields(O.Grid)}
    return O.make_grid(O.Grid(**{k: v for k, v in fields.items() if k in keep}))


def alloc_outputs(torch, g):
    hmap = torch.full((g.n_k, g.ld_x0), -7, dtype=torch.int32, device="cuda")
    cands = torch.zeros(g.n_bands * 64, dtype=torch.uint8, device="cuda")
    stats = torch.zeros(24, dtype=torch.uint8, device="cuda")
    return hmap, cands, stats


def to_dev(torch, a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def read_cands(gfh, t):
    return gfh.candidates_to_numpy(t)


def read_stats(gfh, t):
    return np.frombuffer(t.cpu().numpy().tobytes(), dtype=gfh.STATS_DTYPE)


def assert_candidates_equal(gpu, ocands, n_bands):
    """Integer fields bit-exact; floating fields exactly equal (same IEEE operations)."""
    by_band = {c["band"]: c for c in ocands}
    assert len(gpu) == n_bands
    for rec in gpu:
        b = int(rec["band"])
        if b not in by_band:
            assert rec["count"] == -1, b
            continue
        c = by_band[b]
        assert (int(rec["count"]), int(rec["row"]), int(rec["col"])) == (c["count"], c["row"], c["col"]), b
        for name in ("cr", "x0", "k", "f0", "fdot0"):
            assert float(rec[name]) == c[name], (b, name, float(rec[name]), c[name])
