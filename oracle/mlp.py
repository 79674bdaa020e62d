"""Local density MLP and global colour MLP (oracle, FP64).  Test infrastructure only.

Paper basis: Sec. 4.1 - the NGP features of a sample go into a local density
network that outputs the density and a "density embedding"; the embedding is
the input of a colour network shared across the NeRFs of the scene (after
NeRF-XL).  The paper gives no sizes; the workloads fix them:

* density MLP: in = L*F -> 64 -> 64 -> G, ReLU on hidden layers, no biases
  (tiny-cuda-nn style), linear output g (G = 16, or G = 4 without a colour net);
* sigma = exp(g_0); its gradient is taken as exp(clamp(g_0, -15, 15))
  (the truncated exponential of Mueller et al. 2022);
* colour MLP: G -> 64 -> 64 -> 3 on the whole embedding g, ReLU hidden,
  sigmoid output (no view direction: the synthetic scenes are Lambertian);
  the view-direction variant feeds [g | SH_16(d)] (viewdir.py), G + 16 inputs;
* without a colour net (G = 4) rgb = sigmoid(g_1..3).

Weights are row-major W[out][in]; a layer computes y = W x.
"""
import numpy as np


def relu(x):
    return np.maximum(x, 0.0)


def sigmoid(x):
    return 1.0 / (1.0 + np.exp(-x))


def forward(feat, geo, col, sh=None):
    """feat (S, in) float64; geo = [W1, W2, W3]; col = [V1, V2, V3] or None;
    sh (S, 16) view-direction encoding appended to the colour input, or None.
    Returns sigma (S,), rgb (S, 3) and the activations needed by backward."""
    acts = {"x0": feat}
    h = feat
    pre = []
    for li, W in enumerate(geo):
        z = h @ W.T
        pre.append(z)
        h = relu(z) if li < len(geo) - 1 else z
        acts["geo%d" % li] = h
    g = h
    sigma = np.exp(g[:, 0])
    acts["geo_pre"] = pre
    acts["g"] = g
    if col is None:
        rgb = sigmoid(g[:, 1:4])
        acts["col_pre"] = None
    else:
        h = g if sh is None else np.concatenate([g, sh], 1)
        acts["col_in"] = h
        cpre = []
        for li, V in enumerate(col):
            z = h @ V.T
            cpre.append(z)
            h = relu(z) if li < len(col) - 1 else z
            acts["col%d" % li] = h
        rgb = sigmoid(h)
        acts["col_pre"] = cpre
    acts["rgb"] = rgb
    return sigma, rgb, acts


def backward(dsigma, drgb, geo, col, acts):
    """Gradients of sum(dsigma * sigma + drgb . rgb) w.r.t. the weights and the
    input features.  Returns (dgeo list, dcol list or None, dfeat)."""
    g = acts["g"]
    rgb = acts["rgb"]
    dz_out = drgb * rgb * (1.0 - rgb)          # through the sigmoid
    dg = np.zeros_like(g)
    dg[:, 0] = dsigma * np.exp(np.clip(g[:, 0], -15.0, 15.0))
    dcol = None
    if col is None:
        dg[:, 1:4] += dz_out
    else:
        cpre = acts["col_pre"]
        ins = [acts.get("col_in", g)] + [relu(z) for z in cpre[:-1]]
        dcol = [None] * len(col)
        dz = dz_out
        for li in range(len(col) - 1, -1, -1):
            dcol[li] = dz.T @ ins[li]
            dh = dz @ col[li]
            if li > 0:
                dz = dh * (cpre[li - 1] > 0)
            else:
                dg += dh[:, :g.shape[1]]  # the direction part of the input has no parameters behind it
    pre = acts["geo_pre"]
    ins = [acts["x0"]] + [relu(z) for z in pre[:-1]]
    dgeo = [None] * len(geo)
    dz = dg
    dfeat = None
    for li in range(len(geo) - 1, -1, -1):
        dgeo[li] = dz.T @ ins[li]
        dh = dz @ geo[li]
        if li > 0:
            dz = dh * (pre[li - 1] > 0)
        else:
            dfeat = dh
    return dgeo, dcol, dfeat
