"""A whole search step (asynchronous peakmap + plan execute) captured in a CUDA graph and replayed
gives the same peaks, maps and candidates as the direct calls; overflow is reported, not faulted."""
import numpy as np
import pytest

from paper_1810_09784_gb300 import workloads

from gpu_util import read_cands

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def test_graph_replay_matches_direct_calls(built_lib):
    gfh = built_lib
    spec, pm, fields = workloads.plain_small()
    x = torch.from_numpy(spec.series()).cuda()
    side = torch.cuda.Stream()
    ctx = gfh.Context(0, side)
    g = gfh.grid_make(gfh.Grid(**fields[0]))
    cap = 200_000
    fo = torch.zeros(cap, dtype=torch.int32, device="cuda")
    bo = torch.zeros(cap, dtype=torch.int32, device="cuda")
    off = torch.zeros(2, dtype=torch.int64, device="cuda")
    hmap = torch.zeros((g.n_k, g.ld_x0), dtype=torch.int32, device="cuda")
    cands = torch.zeros(g.n_bands * gfh.CANDIDATE_BYTES, dtype=torch.uint8, device="cuda")
    plan = gfh.Plan(ctx, [g], [hmap], [cands])
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        # direct calls (also builds the cuFFT plan and the scratch before the capture)
        n = ctx.peakmap(x, spec.fs, spec.t_fft, pm["bin_lo"], pm["bin_hi"], 2.5, fo, bo)
        off[1] = n
        plan.execute(fo, bo, off, 1)
    torch.cuda.synchronize()
    ref_peaks = (fo[:n].clone(), bo[:n].clone())
    ref_map = hmap.clone()
    ref_c = read_cands(gfh, cands)
    fo.zero_(); bo.zero_(); hmap.zero_(); cands.zero_(); off.zero_()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=side):
        ctx.peakmap_async(x, spec.fs, spec.t_fft, pm["bin_lo"], pm["bin_hi"], 2.5, fo, bo, off[1:2])
        plan.execute(fo, bo, off, 1)
    for _ in range(2):
        hmap.fill_(-1)
        graph.replay()
    torch.cuda.synchronize()
    assert ctx.check() == gfh.GFH_OK
    assert int(off[1].item()) == n
    assert torch.equal(fo[:n], ref_peaks[0]) and torch.equal(bo[:n], ref_peaks[1])
    assert torch.equal(hmap, ref_map)
    assert np.array_equal(read_cands(gfh, cands), ref_c)
    plan.close()
    ctx.close()


def test_async_capacity_overflow_is_flagged(built_lib, gpu_ctx):
    gfh = built_lib
    spec, pm, _ = workloads.plain_small()
    x = torch.from_numpy(spec.series()).cuda()
    fo = torch.zeros(1000, dtype=torch.int32, device="cuda")
    bo = torch.zeros(1000, dtype=torch.int32, device="cuda")
    n = torch.zeros(1, dtype=torch.int64, device="cuda")
    gpu_ctx.peakmap_async(x, spec.fs, spec.t_fft, pm["bin_lo"], pm["bin_hi"], 2.5, fo, bo, n)
    assert gpu_ctx.check() == gfh.GFH_ERR_SIZE
    assert int(n.item()) == 1000
    assert gpu_ctx.check() == gfh.GFH_OK
