"""CPU oracle of the learned tile proposer (the network, its gradients, its inputs and proposals).

TEST INFRASTRUCTURE ONLY.  Only the test-suite, the smoke check of the build entry module and the
benchmark's CPU-baseline / reference leg may import or call this module.  The library never imports
it and it imports nothing from the library.  Plain fp64 numpy throughout.

The paper leaves machine learning to future work (Sec. VIII); the proposer is a search aid that
ranks coarse (x0, k) tiles of a Hough map so that the exact Hough of Sec. IV runs on the best ones.
What is written here is the plain definition of each step:

  image      pixel (tb, fb) of a peakmap of N FFTs and nb bins counts the peaks with FFT i in
             [tb N/256, (tb+1) N/256) and bin offset in [fb nb/256, (fb+1) nb/256);
             channel 0 = bf16(float32(log(1 + count))), channel 1 = bf16(float32(nplane))
  conv3x3    out[b, y, x, o] = bias[o] + sum_{dy, dx, c} in[b, yS + dy - 1, xS + dx - 1, c] W[o, dy, dx, c]
             (zero outside the image), followed by ReLU; its input gradient and weight gradient are
             the adjoints of that linear map
  pool       mean over the 64 rows of the last activation (time axis); its adjoint spreads
             d pooled / 64 over those rows
  head       logits[b, kt * F + f] = bh[kt] + sum_{d, c} WH[kt, d, c] pooled[b, f + d - 1, c], and
             one no-signal logit = bnull
  loss       mean softmax cross-entropy
  head grads the adjoints of the head (a linear map) in its weights, biases and input
  AdamW      m = b1 m + (1-b1) g; v = b2 v + (1-b2) g^2; w -= lr (m/c1 / (sqrt(v/c2) + eps) + wd w)
  lines      the non-learned proposer: per class the pixel sum along the straight line of its
             mid drift from each of the x0 tile's start columns, the best start kept; class logits
             beta times the standardised sums z, and a no-signal probability that falls
             logistically with the largest z
  proposal   p = softmax(logits); class (d, xt) spreads p evenly over k tiles
             [floor(d gb), max(lo, ceil((d+1) ga) - 1)] (clamped to 63); tiles ranked by score, ties
             to the lower id; the first n leave resid_n = max(0, 1 - p_null - their sum); with
             tau >= 0 the list stops at the first n with resid_n <= tau

`forward(..., mirror=True)` rounds the tensors the kernels store in bf16 (activations, activation
gradients, the bf16 weight copies) at the same points, in fp64 otherwise; with
mirror=False everything is exact fp64 (for finite differences).
"""
from __future__ import annotations

import math

import numpy as np

TILES = 64
CIN = (2, 32, 32, 64, 64)
COUT = (32, 32, 64, 64, 64)
STRIDE = (1, 2, 1, 2, 1)


# ---- number formats --------------------------------------------------------------------------------

def to_f32(x) -> np.ndarray:
    return np.asarray(x, dtype=np.float64).astype(np.float32).astype(np.float64)


def bf16_bits(x) -> np.ndarray:
    """bfloat16 bit patterns of float32(x), round to nearest even (finite inputs)."""
    u = np.asarray(x, dtype=np.float64).astype(np.float32).view(np.uint32).astype(np.uint64)
    r = (u + np.uint64(0x7FFF) + ((u >> np.uint64(16)) & np.uint64(1))) >> np.uint64(16)
    return r.astype(np.uint16)


def bf16_value(bits) -> np.ndarray:
    return (np.asarray(bits, dtype=np.uint32) << np.uint32(16)).view(np.float32).astype(np.float64)


def bf16(x) -> np.ndarray:
    """float64 -> float32 -> bfloat16 -> float64 (the kernels round fp32 accumulators to bf16)."""
    return bf16_value(bf16_bits(x))


# ---- parameter layout ----------------------------------------------------------------------------

def layout(f_pos: int = 64):
    """Offsets of the flat fp32 parameter vector: W1, b1, ..., W5, b5, WH, bH, bnull."""
    off, o = {}, 0
    for l in range(5):
        off[f"W{l + 1}"] = (o, (COUT[l], 3, 3, CIN[l])); o += COUT[l] * 9 * CIN[l]
        off[f"b{l + 1}"] = (o, (COUT[l],)); o += COUT[l]
    off["WH"] = (o, (TILES, 3, 64)); o += TILES * 3 * 64
    off["bH"] = (o, (TILES,)); o += TILES
    off["bnull"] = (o, (1,)); o += 1
    return off, o


def unpack(params: np.ndarray) -> dict:
    off, total = layout()
    assert params.size == total
    return {k: np.asarray(params[o:o + int(np.prod(sh))], np.float64).reshape(sh)
            for k, (o, sh) in off.items()}


def pack(parts: dict) -> np.ndarray:
    off, total = layout()
    out = np.zeros(total, np.float64)
    for k, (o, sh) in off.items():
        out[o:o + int(np.prod(sh))] = np.asarray(parts[k]).reshape(-1)
    return out


# ---- image ---------------------------------------------------------------------------------------

def image_counts(fft_idx, bins, n_fft: int, bin_lo: int, bin_hi: int, img: int = 256) -> np.ndarray:
    """Peak count per pixel [img t][img f], by the pixel ranges of the module docstring."""
    nb = bin_hi - bin_lo + 1
    counts = np.zeros((img, img), np.int64)
    t_edges = np.array([tb * n_fft // img for tb in range(img + 1)])
    f_edges = np.array([fb * nb // img for fb in range(img + 1)])
    fi = np.asarray(fft_idx, np.int64)
    jl = np.asarray(bins, np.int64) - bin_lo
    keep = (jl >= 0) & (jl < nb) & (fi < n_fft)
    tb = np.searchsorted(t_edges, fi[keep], side="right") - 1
    fb = np.searchsorted(f_edges, jl[keep], side="right") - 1
    np.add.at(counts, (tb, fb), 1)
    return counts


def image_bits(counts: np.ndarray, nplane: float) -> np.ndarray:
    """bf16 bit patterns [img][img][2] of the network input."""
    out = np.empty(counts.shape + (2,), np.uint16)
    out[..., 0] = bf16_bits(np.log1p(counts.astype(np.float64)))
    out[..., 1] = bf16_bits(np.float32(nplane))
    return out


# ---- layers ----------------------------------------------------------------------------------------

def conv3x3(x: np.ndarray, W: np.ndarray, S: int) -> np.ndarray:
    """Linear part of a 3x3 layer with zero padding 1 and stride S: [B, H/S, H/S, Cout]."""
    B, H, _, _ = x.shape
    Ho = H // S
    xp = np.pad(x, ((0, 0), (1, 1), (1, 1), (0, 0)))
    out = np.zeros((B, Ho, Ho, W.shape[0]))
    for dy in range(3):
        for dx in range(3):
            patch = xp[:, dy:dy + S * Ho:S, dx:dx + S * Ho:S, :]
            out += np.einsum("bhwc,oc->bhwo", patch, W[:, dy, dx, :])
    return out


def conv3x3_input_grad(G: np.ndarray, W: np.ndarray, S: int, H: int) -> np.ndarray:
    """Adjoint of conv3x3 in its input: [B, H, H, Cin] from G [B, H/S, H/S, Cout]."""
    B, Ho, _, _ = G.shape
    gp = np.zeros((B, H + 2, H + 2, W.shape[3]))
    for dy in range(3):
        for dx in range(3):
            gp[:, dy:dy + S * Ho:S, dx:dx + S * Ho:S, :] += np.einsum("bhwo,oc->bhwc", G, W[:, dy, dx, :])
    return gp[:, 1:H + 1, 1:H + 1, :]


def conv3x3_weight_grad(G: np.ndarray, x: np.ndarray, S: int) -> np.ndarray:
    """Adjoint of conv3x3 in its weights: [Cout, 3, 3, Cin]."""
    B, H, _, C = x.shape
    Ho = H // S
    xp = np.pad(x, ((0, 0), (1, 1), (1, 1), (0, 0)))
    dW = np.zeros((G.shape[3], 3, 3, C))
    for dy in range(3):
        for dx in range(3):
            patch = xp[:, dy:dy + S * Ho:S, dx:dx + S * Ho:S, :]
            dW[:, dy, dx, :] = np.einsum("bhwo,bhwc->oc", G, patch)
    return dW


def head(pooled: np.ndarray, WH: np.ndarray, bH: np.ndarray, bnull: float) -> np.ndarray:
    """logits [B, TILES * F + 1] from pooled [B, F, 64]."""
    B, F, _ = pooled.shape
    pp = np.pad(pooled, ((0, 0), (1, 1), (0, 0)))
    out = np.zeros((B, TILES, F))
    for d in range(3):
        out += np.einsum("kc,bfc->bkf", WH[:, d, :], pp[:, d:d + F, :])
    out += bH[None, :, None]
    return np.concatenate([out.reshape(B, TILES * F), np.full((B, 1), float(bnull))], axis=1)


def pool(a5: np.ndarray) -> np.ndarray:
    """Mean over the time axis of the last activation [B, T, F, C] -> [B, F, C]."""
    return a5.mean(axis=1)


def pool_grad(dpooled: np.ndarray, T: int) -> np.ndarray:
    """Adjoint of pool: every time row of [B, T, F, C] receives dpooled / T."""
    return np.repeat((dpooled / T)[:, None, :, :], T, axis=1)


def head_grads(dl: np.ndarray, pooled: np.ndarray, WH: np.ndarray):
    """Adjoint of head in its parameters and its input, from d(loss)/d logits [B, TILES * F + 1]:
    (dWH [TILES, 3, 64], dbH [TILES], dbnull [1], dpooled [B, F, 64])."""
    B, F, _ = pooled.shape
    dt = dl[:, :TILES * F].reshape(B, TILES, F)
    pp = np.pad(pooled, ((0, 0), (1, 1), (0, 0)))
    dWH = np.stack([np.einsum("bkf,bfc->kc", dt, pp[:, d:d + F, :]) for d in range(3)], axis=1)
    dbH = dt.sum(axis=(0, 2))
    dbnull = np.array([dl[:, TILES * F].sum()])
    dpp = np.zeros((B, F + 2, 64))
    for d in range(3):                       # tap d of logit f reads pooled row f + d - 1
        dpp[:, d:d + F, :] += np.einsum("bkf,kc->bfc", dt, WH[:, d, :])
    return dWH, dbH, dbnull, dpp[:, 1:F + 1, :]


def softmax_ce(logits: np.ndarray, labels: np.ndarray):
    """Per-sample losses and d(mean loss)/d logits."""
    B = logits.shape[0]
    m = logits.max(axis=1, keepdims=True)
    lse = m[:, 0] + np.log(np.exp(logits - m).sum(axis=1))
    p = np.exp(logits - lse[:, None])
    loss = lse - logits[np.arange(B), labels]
    d = p.copy()
    d[np.arange(B), labels] -= 1.0
    return loss, d / B


# ---- the network ---------------------------------------------------------------------------------

def forward(params: np.ndarray, images: np.ndarray, mirror: bool = True) -> dict:
    """images: [B, H, H, 2] values (already bf16 when mirroring the kernels)."""
    P = unpack(params)
    rnd = bf16 if mirror else (lambda v: v)
    acts = [np.asarray(images, np.float64)]
    for l in range(5):
        W = P[f"W{l + 1}"]
        if mirror:
            W = bf16(W)                                 # the layers run on bf16 weight copies
        pre = conv3x3(acts[-1], W, STRIDE[l]) + P[f"b{l + 1}"]
        acts.append(rnd(np.maximum(pre, 0.0)))
    pooled = pool(acts[5])
    logits = head(pooled, P["WH"], P["bH"], P["bnull"][0])
    return {"P": P, "acts": acts, "pooled": pooled, "logits": logits, "mirror": mirror}


def backward(cache: dict, labels: np.ndarray):
    """(mean loss, flat gradient) of the mean cross-entropy."""
    P, acts, pooled, mirror = cache["P"], cache["acts"], cache["pooled"], cache["mirror"]
    rnd = bf16 if mirror else (lambda v: v)
    loss, dl = softmax_ce(cache["logits"], labels)
    g = {}
    g["WH"], g["bH"], g["bnull"], dpool = head_grads(dl, pooled, P["WH"])
    da = rnd(pool_grad(dpool, acts[5].shape[1]))
    for l in range(4, -1, -1):
        G = da * (acts[l + 1] > 0)
        g[f"W{l + 1}"] = conv3x3_weight_grad(G, acts[l], STRIDE[l])
        g[f"b{l + 1}"] = G.sum(axis=(0, 1, 2))
        if l > 0:
            W = bf16(P[f"W{l + 1}"]) if mirror else P[f"W{l + 1}"]
            da = rnd(conv3x3_input_grad(G, W, STRIDE[l], acts[l].shape[1]))
    return float(loss.mean()), pack(g)


def adamw(w, g, m, v, step: int, lr: float, wd: float, b1=0.9, b2=0.999, eps=1e-8):
    """One AdamW step (decoupled weight decay), bias-corrected; returns (w, m, v)."""
    m = b1 * m + (1 - b1) * g
    v = b2 * v + (1 - b2) * g * g
    c1 = 1 - b1 ** step
    c2 = 1 - b2 ** step
    w = w - lr * ((m / c1) / (np.sqrt(v / c2) + eps) + wd * w)
    return w, m, v


# ---- the non-learned proposer -------------------------------------------------------------------

def line_scores(ch0: np.ndarray, K: int, nb: int) -> np.ndarray:
    """Straight-line sums of one image's channel 0 values [256 t][256 f] per class d * 64 + xt: a
    track starting in image columns 4 xt .. 4 xt + 3 at t0 and drifting (d + 1/2) K / 64 bins over
    the observation sits, in time bin tb (centre (tb + 1/2) / 256 of the observation),
    (d + 1/2) (K / 64) (256 / nb) (tb + 1/2) / 256 columns left of its start, rounded to nearest
    (halves up); the score is the best of the four start columns; columns left of 0 add nothing."""
    img = np.asarray(ch0, np.float64)
    out = np.zeros(TILES * TILES)
    tb = np.arange(256)
    for d in range(TILES):
        off = ((2 * d + 1) * (2 * tb + 1) * K + 128 * nb) // (256 * nb)
        for xt in range(TILES):
            best = None
            for c0 in range(4 * xt, 4 * xt + 4):
                c = c0 - off
                s = float(img[tb[c >= 0], c[c >= 0]].sum())
                best = s if best is None else max(best, s)
            out[d * TILES + xt] = best
    return out


def heuristic_logits(scores: np.ndarray, beta: float, det_a: float, det_c: float) -> np.ndarray:
    """z = (score - mean) / std over the 4096 scores (population std; 0 if constant); class logits
    beta z; no-signal logit log(sum exp(beta z)) + det_c - det_a max(z), which makes
    p(no signal) = 1 / (1 + exp(det_a max(z) - det_c))."""
    s = np.asarray(scores, np.float64)
    sd = s.std()
    z = (s - s.mean()) / sd if sd > 0 else np.zeros_like(s)
    lz = beta * z
    m = lz.max()
    lse = m + math.log(np.exp(lz - m).sum())
    return np.concatenate([lz, [lse + det_c - det_a * z.max()]])


# ---- proposals ---------------------------------------------------------------------------------

def tile_scores(logits: np.ndarray, gain: np.ndarray):
    """(scores [4096] of coarse tiles kt * 64 + xt, p_null) of one map."""
    l = np.asarray(logits, np.float64)
    m = l.max()
    p = np.exp(l - m)
    p /= p.sum()
    sc = np.zeros((TILES, TILES))
    pd = p[:TILES * TILES].reshape(TILES, TILES)        # [d][xt]
    for xt in range(TILES):
        ga, gb = gain[xt]
        for d in range(TILES):
            lo = min(TILES - 1, math.floor(d * gb))
            hi = min(TILES - 1, max(lo, math.ceil((d + 1) * ga) - 1))
            sc[lo:hi + 1, xt] += pd[d, xt] / (hi - lo + 1)
    return sc.reshape(-1), p[TILES * TILES]


def propose(logits: np.ndarray, gain: np.ndarray, k: int, tau: float = -1.0):
    """(tiles, resid, full): the ranked tiles (cut at the first n with resid_n <= tau when
    tau >= 0, padded with -1 to k), resid of the kept list, and whether even k tiles leave more
    than tau."""
    sc, pnull = tile_scores(logits, gain)
    order = sorted(range(sc.size), key=lambda c: (-sc[c], c))[:k]
    cum, n, res = 0.0, k, 1.0
    for q in range(k):
        cum += max(sc[order[q]], 0.0)
        res = max(0.0, 1.0 - pnull - cum)
        if tau >= 0 and res <= tau:
            n = q + 1
            break
    tiles = np.array(order[:n] + [-1] * (k - n))
    return tiles, res, bool(tau >= 0 and res > tau)
