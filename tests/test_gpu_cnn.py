"""The proposal network's kernels against the CPU oracle: the counter-based peakmap generator and the
images (bit-exact), each 3x3 layer's forward, input-gradient and weight-gradient kernel (within the
fp32-accumulation and bf16-rounding bound derived below), every stage of the whole network's
forward and backward pass element by element on the GPU's own stage inputs,
one AdamW step, determinism and checkpoint resume, and the tile proposals."""
import math

import numpy as np
import pytest

from oracle import cnn_oracle as C
from paper_1810_09784_gb300 import proposer as PR
from paper_1810_09784_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

U32 = 2.0 ** -24          # fp32 unit roundoff


def bf16_tensor(bits: np.ndarray):
    return torch.from_numpy(np.ascontiguousarray(bits).view(np.int16)).cuda().view(torch.bfloat16)


def tensor_bits(t) -> np.ndarray:
    return t.view(torch.int16).cpu().numpy().view(np.uint16)


def rand_bf16(rng, shape, scale=1.0, relu=False):
    v = rng.standard_normal(shape) * scale
    if relu:
        v = np.maximum(v, 0.0)
    return C.bf16_bits(v)


def ulp_bf16(v):
    v = np.maximum(np.abs(v), 2.0 ** -126)
    return 2.0 ** (np.floor(np.log2(v)) - 7)


def assert_bf16_close(gpu, exact, err):
    """gpu = bf16(a) with |a - exact| <= err: |gpu - exact| <= half an ulp of |exact| + err + err."""
    bound = 0.5 * ulp_bf16(np.abs(exact) + err) + err
    bad = np.abs(gpu - exact) > bound
    assert not bad.any(), (int(bad.sum()), np.argwhere(bad)[:3], gpu[bad][:3], exact[bad][:3])


# ---- generator and images ------------------------------------------------------------------------------

@pytest.mark.parametrize("case", [(300, 40, 339, 0.05, 0, None), (1799, 200, 799, 0.0755, 1 << 23, 450)])
def test_synth_peaks_bit_exact(built_lib, gpu_ctx, case):
    gfh = built_lib
    n_fft, lo, hi, p, pt, tb = case
    track = np.full(n_fft, -1, np.int32)
    if tb is not None:
        track[:] = tb - (np.arange(n_fft) // 7)
    p24 = int(p * 2 ** 24)
    cap = n_fft * (hi - lo + 1)
    fo = torch.empty(cap, dtype=torch.int32, device="cuda")
    bo = torch.empty(cap, dtype=torch.int32, device="cuda")
    n = gfh.synth_peaks(gpu_ctx, 99, 12, n_fft, lo, hi, p24, pt, torch.from_numpy(track).cuda(), fo, bo)
    rf, rb = synth.hashed_peaklist(99, 12, n_fft, lo, hi, p24, pt, track)
    assert n == rf.size
    assert np.array_equal(fo[:n].cpu().numpy().astype(np.uint32), rf)
    assert np.array_equal(bo[:n].cpu().numpy().astype(np.uint32), rb)


def test_images_bit_exact(built_lib, gpu_ctx):
    """gfh_synth_images (cells drawn in the kernel) and gfh_peaks_to_images (from peak lists, one
    launch for all lists) both equal the oracle's binning of the generator's peak list."""
    gfh = built_lib
    spec = PR.ProposerSpec(peakmaps="statistical")
    smp = PR.draw(spec, np.arange(40, 46))
    buf = PR.DeviceBatch(spec, 6)
    buf.load(gpu_ctx, spec, smp)
    img2 = torch.zeros((6, 256, 256, 2), dtype=torch.bfloat16, device="cuda")
    got = tensor_bits(buf.images)
    lists = []
    for b in range(6):
        rf, rb = synth.hashed_peaklist(spec.seed, int(smp.index[b]), spec.n_fft, spec.bin_lo,
                                       spec.bin_hi, spec.p_noise24, int(smp.p_track24[b]),
                                       smp.tracks[b])
        ref = C.image_bits(C.image_counts(rf, rb, spec.n_fft, spec.bin_lo, spec.bin_hi),
                           float(smp.nplane[b]))
        assert np.array_equal(got[b], ref), b
        lists.append((rf, rb))
    fi = torch.from_numpy(np.concatenate([l[0] for l in lists]).view(np.int32)).cuda()
    bj = torch.from_numpy(np.concatenate([l[1] for l in lists]).view(np.int32)).cuda()
    off = torch.from_numpy(np.cumsum([0] + [l[0].size for l in lists]).astype(np.int64)).cuda()
    gfh.peaks_to_images(gpu_ctx, fi, bj, off, 6, spec.n_fft, spec.bin_lo, spec.bin_hi,
                        buf.nplane[:6], img2)
    torch.cuda.synchronize()
    assert np.array_equal(tensor_bits(img2), got)


# ---- single layers ---------------------------------------------------------------------------------

LAYERS = [(32, 32, 2), (32, 64, 1), (64, 64, 2), (64, 64, 1)]
ALL_LAYERS = [(2, 32, 1)] + LAYERS          # the first layer has no input gradient


@pytest.mark.parametrize("cin,cout,S", ALL_LAYERS)
def test_conv_forward(built_lib, gpu_ctx, cin, cout, S):
    """relu(conv + bias) rounded to bf16: the fp32 sum of K = 9 cin + 1 terms is within
    K u sum|terms| of the exact one (u = 2^-24), then one bf16 rounding."""
    gfh = built_lib
    rng = np.random.default_rng(cin + cout + S)
    B, H = 2, 48
    xb = rand_bf16(rng, (B, H, H, cin), relu=True)
    wb = rand_bf16(rng, (cout, 3, 3, cin), scale=math.sqrt(2.0 / (9 * cin)))
    bias = rng.uniform(-0.1, 0.1, cout).astype(np.float32)
    out = torch.empty((B, H // S, H // S, cout), dtype=torch.bfloat16, device="cuda")
    gfh.conv3x3(gpu_ctx, 0, cin, cout, S, B, H, inp=bf16_tensor(xb), w=bf16_tensor(wb),
                bias=torch.from_numpy(bias).cuda(), res=out)
    torch.cuda.synchronize()
    x, W = C.bf16_value(xb), C.bf16_value(wb)
    exact = np.maximum(C.conv3x3(x, W, S) + bias.astype(np.float64), 0.0)
    err = (9 * cin + 1) * U32 * (C.conv3x3(np.abs(x), np.abs(W), S) + np.abs(bias))
    assert_bf16_close(C.bf16_value(tensor_bits(out)), exact, err)


@pytest.mark.parametrize("cin,cout,S", LAYERS)
def test_conv_input_gradient(built_lib, gpu_ctx, cin, cout, S):
    gfh = built_lib
    rng = np.random.default_rng(100 + cin + cout + S)
    B, H = 2, 48
    Ho = H // S
    gb = rand_bf16(rng, (B, Ho, Ho, cout), scale=0.01)
    ob = rand_bf16(rng, (B, Ho, Ho, cout), relu=True)      # layer output: ReLU mask
    wb = rand_bf16(rng, (cout, 3, 3, cin), scale=math.sqrt(2.0 / (9 * cin)))
    din = torch.empty((B, H, H, cin), dtype=torch.bfloat16, device="cuda")
    gfh.conv3x3(gpu_ctx, 1, cin, cout, S, B, H, w=bf16_tensor(wb), out=bf16_tensor(ob),
                dout=bf16_tensor(gb), res=din)
    torch.cuda.synchronize()
    G = C.bf16_value(gb) * (C.bf16_value(ob) > 0)
    W = C.bf16_value(wb)
    exact = C.conv3x3_input_grad(G, W, S, H)
    err = 9 * cout * U32 * C.conv3x3_input_grad(np.abs(G), np.abs(W), S, H)
    assert_bf16_close(C.bf16_value(tensor_bits(din)), exact, err)


@pytest.mark.parametrize("cin,cout,S", ALL_LAYERS)
def test_conv_weight_gradient(built_lib, gpu_ctx, cin, cout, S):
    """fp32 sums over M = B (H/S)^2 pixels (per-chunk sums in tensor memory or registers, then the
    chunks added in order): at most M + 1024 rounded additions on any path, so within
    (M + 1024) u sum|terms| of the exact sum; bias gradient likewise.  Run twice: the result is
    the same bit for bit (no atomics)."""
    gfh = built_lib
    rng = np.random.default_rng(200 + cin + cout + S)
    B = 3
    H = 64 * S                              # the tensor-core kernel takes output sides of 64k
    Ho = H // S
    xb = rand_bf16(rng, (B, H, H, cin), relu=True)
    gb = rand_bf16(rng, (B, Ho, Ho, cout), scale=0.01)
    ob = rand_bf16(rng, (B, Ho, Ho, cout), relu=True)
    dw = torch.zeros((cout, 3, 3, cin), dtype=torch.float32, device="cuda")
    db = torch.zeros(cout, dtype=torch.float32, device="cuda")
    gfh.conv3x3(gpu_ctx, 2, cin, cout, S, B, H, inp=bf16_tensor(xb), out=bf16_tensor(ob),
                dout=bf16_tensor(gb), res=dw, db=db)
    torch.cuda.synchronize()
    G = C.bf16_value(gb) * (C.bf16_value(ob) > 0)
    x = C.bf16_value(xb)
    M = B * Ho * Ho
    exact = C.conv3x3_weight_grad(G, x, S)
    err = (M + 1024) * U32 * C.conv3x3_weight_grad(np.abs(G), np.abs(x), S)
    got_w, got_b = dw.cpu().numpy(), db.cpu().numpy()
    assert np.all(np.abs(got_w - exact) <= err + 1e-30)
    eb = G.sum(axis=(0, 1, 2))
    errb = (M + 8192) * U32 * np.abs(G).sum(axis=(0, 1, 2))
    assert np.all(np.abs(got_b - eb) <= errb + 1e-30)
    dw.zero_()
    db.zero_()
    gfh.conv3x3(gpu_ctx, 2, cin, cout, S, B, H, inp=bf16_tensor(xb), out=bf16_tensor(ob),
                dout=bf16_tensor(gb), res=dw, db=db)
    torch.cuda.synchronize()
    assert np.array_equal(dw.cpu().numpy(), got_w) and np.array_equal(db.cpu().numpy(), got_b)


# ---- the whole network -------------------------------------------------------------------------

def _batch(gpu_ctx, idx):
    spec = PR.ProposerSpec()
    smp = PR.draw(spec, np.asarray(idx))
    buf = PR.DeviceBatch(spec, len(idx))
    buf.load(gpu_ctx, spec, smp)
    return smp, buf


def _signal_and_noise_ids(n_each):
    spec = PR.ProposerSpec()
    smp = PR.draw(spec, np.arange(0, 60))
    return (list(smp.index[smp.signal][:n_each]) + list(smp.index[~smp.signal][:n_each]))


def _softmax_ce_bound(lg, labels, B):
    """Element-wise bound of the fp32 softmax cross-entropy kernel against the exact one on the
    same logits.  The sum of the 4097 exponentials takes at most 25 rounded additions on any path
    (16 per thread, 8 tree levels) of terms each within 2 ulp (expf) and u |l - max| (the rounded
    argument); logf adds 1 ulp and the final add half an ulp of lse.  p = expf(l - lse) adds the
    rounding of its argument and 2 ulp; (p - onehot) / B one more rounding (B is a power of two)."""
    l = lg.astype(np.float64)
    mx = l.max(axis=1, keepdims=True)
    S = np.exp(l - mx).sum(axis=1, keepdims=True)
    lse = mx + np.log(S)
    ulp32 = lambda v: np.spacing(np.abs(v).astype(np.float32)).astype(np.float64)
    d_lse = (25 + 4) * U32 + U32 * np.abs(l - mx).max(axis=1, keepdims=True) + 2 * ulp32(np.log(S)) + ulp32(lse)
    p = np.exp(l - lse)
    eps_p = d_lse + U32 * np.abs(l - lse) + 4 * U32
    onehot = np.zeros_like(l)
    onehot[np.arange(B), labels] = 1.0
    dl_err = (p * eps_p * 1.01 + U32 * np.abs(p - onehot)) / B + 1e-30
    loss_err = (d_lse[:, 0] + U32 * np.abs(lse[:, 0] - l[np.arange(B), labels])) * 1.01
    return dl_err, loss_err


def test_network_stages_elementwise(built_lib, gpu_ctx):
    """Every kernel of one forward and backward pass against the oracle's definition of its stage,
    evaluated on the GPU's own stored inputs of that stage, element by element.  Bounds: a sum of K
    fp32-rounded terms is within K u sum|terms| of the exact sum (u = 2^-24), and a stored bf16
    tensor adds one rounding (assert_bf16_close)."""
    gfh = built_lib
    B = 4
    net = gfh.Cnn(gpu_ctx, B, seed=3)
    smp, buf = _batch(gpu_ctx, _signal_and_noise_ids(2))
    labels = smp.labels.astype(np.int64)
    loss = net.gradients(buf.images, buf.labels)
    P = C.unpack(net.params().astype(np.float64))
    GW = C.unpack(net.grads().astype(np.float64))
    acts = [C.bf16_value(tensor_bits(buf.images))]
    for l in range(1, 6):
        acts.append(C.bf16_value(net.read_tensor(gfh.CNN_ACT + l, B)))
    # forward: five 3x3 layers on the bf16 weight copies
    Wb = []
    for l in range(5):
        W = C.bf16_value(net.read_tensor(gfh.CNN_WBF16 + l, B))
        assert np.array_equal(W, C.bf16(P[f"W{l + 1}"])), l          # RNE copies of the fp32 weights
        Wb.append(W)
        b = P[f"b{l + 1}"]
        S = C.STRIDE[l]
        exact = np.maximum(C.conv3x3(acts[l], W, S) + b, 0.0)
        err = (9 * C.CIN[l] + 1) * U32 * (C.conv3x3(np.abs(acts[l]), np.abs(W), S) + np.abs(b))
        assert_bf16_close(acts[l + 1], exact, err)
    # mean over time: 64 fp32 additions, times 1/64 (exact)
    pooled = net.read_tensor(gfh.CNN_POOLED, B).astype(np.float64)
    assert np.all(np.abs(pooled - C.pool(acts[5])) <= 64 * U32 * C.pool(np.abs(acts[5])))
    # head on the fp32 weights: 3 x 64 products and their sums per logit, plus the bias
    lg = net.read_tensor(gfh.CNN_LOGITS, B)
    exact = C.head(pooled, P["WH"], P["bH"], P["bnull"][0])
    err = 4 * 64 * U32 * C.head(np.abs(pooled), np.abs(P["WH"]), np.abs(P["bH"]), abs(P["bnull"][0]))
    assert np.all(np.abs(lg - exact) <= err + 1e-30)
    assert np.all(lg[:, -1] == np.float32(P["bnull"][0]))
    # softmax cross-entropy on the GPU's logits
    dl = net.read_tensor(gfh.CNN_DLOGITS, B).astype(np.float64)
    lo = net.read_tensor(gfh.CNN_LOSS, B).astype(np.float64)
    lx, dlx = C.softmax_ce(lg.astype(np.float64), labels)
    dl_err, loss_err = _softmax_ce_bound(lg, labels, B)
    assert np.all(np.abs(dl - dlx) <= dl_err)
    assert np.all(np.abs(lo - lx) <= loss_err)
    assert math.isclose(loss, float(lo.mean()), rel_tol=1e-6)
    # head gradients: B x 64 products per weight in one fp32 sum
    gWH, gbH, gbn, dpool = C.head_grads(dl, pooled, P["WH"])
    aWH, abH, abn, adpool = C.head_grads(np.abs(dl), np.abs(pooled), np.abs(P["WH"]))
    K = 2 * B * 64
    assert np.all(np.abs(GW["WH"] - gWH) <= K * U32 * aWH + 1e-30)
    assert np.all(np.abs(GW["bH"] - gbH) <= K * U32 * abH + 1e-30)
    assert np.all(np.abs(GW["bnull"] - gbn) <= K * U32 * abn + 1e-30)
    # gradient in layer 5's pre-activation: 3 x 64 terms, / 64, one bf16 rounding, the same on
    # every row, stored masked by the ReLU (activation 5 > 0)
    da = C.bf16_value(net.read_tensor(gfh.CNN_DACT + 5, B))
    m5 = acts[5] > 0
    assert_bf16_close(da, C.pool_grad(dpool, 64) * m5, 2 * 192 * U32 * C.pool_grad(adpool, 64) * m5)
    # backward through the five layers on the GPU's stored gradients
    for l in range(4, -1, -1):
        S = C.STRIDE[l]
        G = C.bf16_value(net.read_tensor(gfh.CNN_DACT + l + 1, B)) * (acts[l + 1] > 0)
        M = G.shape[0] * G.shape[1] * G.shape[2]
        exact = C.conv3x3_weight_grad(G, acts[l], S)
        err = (M + 1024) * U32 * C.conv3x3_weight_grad(np.abs(G), np.abs(acts[l]), S)
        assert np.all(np.abs(GW[f"W{l + 1}"] - exact) <= err + 1e-30), l
        eb = G.sum(axis=(0, 1, 2))
        errb = (M + 8192) * U32 * np.abs(G).sum(axis=(0, 1, 2))
        assert np.all(np.abs(GW[f"b{l + 1}"] - eb) <= errb + 1e-30), l
        if l > 0:      # stored masked by the ReLU of activation l
            din = C.bf16_value(net.read_tensor(gfh.CNN_DACT + l, B))
            H = acts[l].shape[1]
            ml = acts[l] > 0
            exact = C.conv3x3_input_grad(G, Wb[l], S, H) * ml
            err = 9 * C.COUT[l] * U32 * C.conv3x3_input_grad(np.abs(G), np.abs(Wb[l]), S, H) * ml
            assert_bf16_close(din, exact, err)
    net.close()


def test_network_agrees_with_the_whole_oracle(built_lib, gpu_ctx):
    """The whole pass once more against the oracle run end to end with the kernels' bf16 storage
    points (its own fp64 arithmetic between them): the loss and the logits agree closely; this
    checks the wiring of the stages (which tensor feeds which), not their rounding."""
    gfh = built_lib
    net = gfh.Cnn(gpu_ctx, 4, seed=3)
    smp, buf = _batch(gpu_ctx, _signal_and_noise_ids(2))
    loss = net.gradients(buf.images, buf.labels)
    cache = C.forward(net.params().astype(np.float64), C.bf16_value(tensor_bits(buf.images)))
    lo, _ = C.backward(cache, smp.labels.astype(np.int64))
    lg = net.read_tensor(gfh.CNN_LOGITS, 4)
    assert np.abs(lg - cache["logits"]).max() <= 2e-2 * np.abs(cache["logits"]).max()
    assert math.isclose(loss, lo, rel_tol=1e-2)
    net.close()


def test_training_is_deterministic_and_resumes_bit_identically(built_lib, gpu_ctx, tmp_path):
    """Six AdamW steps without a stop, and three steps, a checkpoint written to disk, a fresh
    network loaded from it and three more steps: the parameters and both moments are equal bit
    for bit (the gradients reduce in a fixed order), and so is a second uninterrupted run."""
    gfh = built_lib
    spec = PR.ProposerSpec()
    batches = [PR.draw(spec, np.arange(300 + 8 * i, 308 + 8 * i)) for i in range(6)]
    buf = PR.DeviceBatch(spec, 8)
    lrs = [2e-3 * (0.5 + 0.5 * math.cos(math.pi * i / 6)) for i in range(6)]

    def steps(net, rng_):
        for i in rng_:
            buf.load(gpu_ctx, spec, batches[i])
            net.train_step(buf.images, buf.labels, lrs[i], 1e-4, want_loss=False)

    a = gfh.Cnn(gpu_ctx, 8, seed=7)
    steps(a, range(6))
    sa = a.state()
    b = gfh.Cnn(gpu_ctx, 8, seed=7)
    steps(b, range(3))
    path = tmp_path / "ck.npz"
    PR.save_checkpoint(path, b.state(), {"epoch": 0, "step_in_epoch": 3})
    b.close()
    c = gfh.Cnn(gpu_ctx, 8, seed=99)
    st, meta = PR.load_checkpoint(path)
    assert meta["step_in_epoch"] == 3 and st["step"] == 3
    c.set_state(st)
    steps(c, range(3, 6))
    sc = c.state()
    assert sc["step"] == sa["step"] == 6
    for k in ("params", "m", "v"):
        assert np.array_equal(sa[k], sc[k]), k
    d = gfh.Cnn(gpu_ctx, 8, seed=7)
    steps(d, range(6))
    assert np.array_equal(d.state()["params"], sa["params"])
    for n in (a, c, d):
        n.close()


def test_adamw_step(built_lib, gpu_ctx):
    """One AdamW step on the GPU's own gradient equals the fp64 formula within fp32 rounding."""
    gfh = built_lib
    net = gfh.Cnn(gpu_ctx, 2, seed=4)
    _, buf = _batch(gpu_ctx, [7, 8])
    p0 = net.params().astype(np.float64)
    lr, wd = 1e-3, 1e-2
    net.train_step(buf.images, buf.labels, lr, wd)
    p1 = net.params().astype(np.float64)
    g = net.grads().astype(np.float64)
    ref, _, _ = C.adamw(p0, g, np.zeros_like(p0), np.zeros_like(p0), 1, lr, wd)
    assert np.all(np.abs(p1 - ref) <= 8 * U32 * (np.abs(p0) + lr) + 1e-12)
    net.close()


def test_proposals(built_lib, gpu_ctx):
    """Ranked tiles, the cut at tau and the full-search flags against the oracle (ranks compared up
    to fp32 near-ties of the scores)."""
    gfh = built_lib
    spec = PR.ProposerSpec()
    smp = PR.draw(spec, np.arange(100, 108))
    rng = np.random.default_rng(9)
    logits = (rng.standard_normal((8, gfh.N_CLASSES)) * 3).astype(np.float32)
    logits[3, 4096] = 40.0                                     # confident "no signal"
    logits[5, 64 * 2 + 40] = 25.0                              # one confident class
    lt = torch.from_numpy(logits).cuda()
    gain = torch.from_numpy(smp.gain).cuda()
    for k, tau in ((32, -1.0), (256, 0.05), (32, 0.5)):
        top = torch.empty((8, k), dtype=torch.int32, device="cuda")
        resid = torch.empty(8, dtype=torch.float32, device="cuda")
        full = torch.empty(8, dtype=torch.int32, device="cuda")
        gfh.propose_tiles(gpu_ctx, lt, gain, k, top, resid, tau, full)
        torch.cuda.synchronize()
        tp, rs, fl = top.cpu().numpy(), resid.cpu().numpy(), full.cpu().numpy()
        for b in range(8):
            sc, pnull = C.tile_scores(logits[b].astype(np.float64), smp.gain[b].astype(np.float64))
            otop, ores, ofull = C.propose(logits[b].astype(np.float64), smp.gain[b].astype(np.float64), k, tau)
            kept = tp[b][tp[b] >= 0]
            okept = otop[otop >= 0]
            srt = np.sort(sc)[::-1]
            assert len(set(kept.tolist())) == kept.size
            # the same prefix length unless the cut falls within fp32 rounding of the leftover
            if abs(kept.size - okept.size) > 0:
                assert tau >= 0 and abs(ores - tau) < 1e-4, (k, tau, b, kept.size, okept.size)
            n = min(kept.size, okept.size)
            assert np.all(sc[kept[:n]] >= srt[n - 1] - 1e-6 * srt[0])
            assert abs(rs[b] - max(0.0, 1 - pnull - sc[kept].sum())) <= 1e-4
            assert bool(fl[b]) == ofull or abs(ores - tau) < 1e-4
        if tau < 0:
            assert rs[3] < 1e-3 and np.all(fl == 0)


def test_proposal_selection_equals_full_ranking(built_lib, gpu_ctx):
    """For k <= 512 the tiles are found by a radix selection of the k best keys and a sort of those
    alone; k = 4096 sorts every tile.  The selected tiles are the full ranking's first k, in the
    same order, ties included (equal scores go to the lower tile id)."""
    gfh = built_lib
    spec = PR.ProposerSpec()
    smp = PR.draw(spec, np.arange(200, 208))
    rng = np.random.default_rng(11)
    logits = (rng.standard_normal((8, gfh.N_CLASSES)) * 3).astype(np.float32)
    logits[2] = 0.0                                    # equal logits: many equal scores
    logits[4, : 2048] = -np.inf                        # half the classes without probability
    logits[6, 64 * 7 + 3] = 30.0                       # one confident class
    lt = torch.from_numpy(logits).cuda()
    gain = torch.from_numpy(smp.gain).cuda()

    def ranked(k):
        top = torch.empty((8, k), dtype=torch.int32, device="cuda")
        resid = torch.empty(8, dtype=torch.float32, device="cuda")
        gfh.propose_tiles(gpu_ctx, lt, gain, k, top, resid, -1.0, None)
        torch.cuda.synchronize()
        return top.cpu().numpy()

    full = ranked(4096)
    assert np.all(np.sort(full, axis=1) == np.arange(4096))
    for k in (1, 32, 256, 300, 512):
        assert np.array_equal(ranked(k), full[:, :k]), k


def test_bounded_wait_reports_timeout_and_context_survives(built_lib, gpu_ctx):
    """A device wait that nothing ends gives up after its limit and raises the timeout status;
    the context then works normally (the same network forward as before, no fault)."""
    gfh = built_lib
    assert gpu_ctx.check() == gfh.GFH_OK
    gpu_ctx.wait_check(2_000_000)                 # ~1 ms at the maximum SM clock
    assert gpu_ctx.check() == gfh.GFH_ERR_TIMEOUT
    assert gpu_ctx.check() == gfh.GFH_OK          # cleared
    net = gfh.Cnn(gpu_ctx, 2, seed=5)
    _, buf = _batch(gpu_ctx, [1, 2])
    net.forward(buf.images, buf.logits)
    torch.cuda.synchronize()
    assert gpu_ctx.check() == gfh.GFH_OK
    assert torch.isfinite(buf.logits).all()
    net.close()
