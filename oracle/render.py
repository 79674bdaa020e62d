"""Front-to-back volume rendering, colour loss and their backward (oracle, FP64).
Test infrastructure only.

Paper basis: Sec. 4.5 - the samples of all segments of a ray are rendered
with the unchanged NeRF rendering equation (Eq. 3 of Mildenhall et al. 2020),
which weights each sample by the spacing delta between samples; Sec. 4.4 /
Sec. 4.6 - the loss is the standard NeRF colour consistency loss, shared with
I-NGP.

For the samples i = 0..K-1 of one ray, in order along the ray:
    tau_i   = sigma_i * delta_i
    T_i     = exp(-sum_{j<i} tau_j)            (transmittance)
    alpha_i = 1 - exp(-tau_i)
    w_i     = T_i * alpha_i
    C = sum_i w_i c_i,  depth = sum_i w_i t_i,  opacity = sum_i w_i,
    T_final = exp(-sum_i tau_i).
Readings: black background (nothing added for 1 - opacity); depth measured
along the ray from its top point; loss = mean squared error over the colour
channels of the accepted rays (the paper's L2 colour loss; I-NGP also has a
Huber option, not used here).

Backward for an upstream gradient g = dLoss/dC (3-vector per ray):
    dLoss/dc_i     = w_i g
    dLoss/dsigma_i = delta_i [ T_{i+1} (g . c_i) - sum_{j>i} w_j (g . c_j) ]
with T_{i+1} = T_i exp(-tau_i).
"""
import numpy as np


def composite(sigma, rgb, t, dt, ray_off):
    """Returns per-ray rgb (B, 3), depth (B,), opacity (B,), T_final (B,) and
    per-sample weights w (S,)."""
    B = len(ray_off) - 1
    out_rgb = np.zeros((B, 3))
    depth = np.zeros(B)
    opac = np.zeros(B)
    t_fin = np.ones(B)
    w_all = np.zeros(len(sigma))
    for r in range(B):
        a, b = int(ray_off[r]), int(ray_off[r + 1])
        if b == a:
            continue
        tau = sigma[a:b] * dt[a:b]
        T = np.exp(-(np.cumsum(tau) - tau))
        w = T * (1.0 - np.exp(-tau))
        w_all[a:b] = w
        out_rgb[r] = w @ rgb[a:b]
        depth[r] = w @ t[a:b]
        opac[r] = w.sum()
        t_fin[r] = np.exp(-tau.sum())
    return out_rgb, depth, opac, t_fin, w_all


def mse_loss(pred_rgb, gt_rgb, ray_ok):
    """Mean of (C - C_gt)^2 over the 3 channels of the accepted rays, and its
    gradient with respect to C (zero on rejected rays)."""
    m = np.asarray(ray_ok).astype(bool)
    n = int(m.sum())
    diff = np.where(m[:, None], pred_rgb - gt_rgb, 0.0)
    if n == 0:
        return 0.0, np.zeros_like(pred_rgb)
    loss = float((diff ** 2).sum() / (3.0 * n))
    return loss, 2.0 * diff / (3.0 * n)


def composite_backward(g_rgb, sigma, rgb, t, dt, ray_off):
    """dLoss/dsigma (S,) and dLoss/drgb (S, 3) for per-ray colour gradients g_rgb (B, 3)."""
    S = len(sigma)
    dsigma = np.zeros(S)
    drgb = np.zeros((S, 3))
    B = len(ray_off) - 1
    for r in range(B):
        a, b = int(ray_off[r]), int(ray_off[r + 1])
        if b == a:
            continue
        tau = sigma[a:b] * dt[a:b]
        T = np.exp(-(np.cumsum(tau) - tau))
        T_next = np.exp(-np.cumsum(tau))
        w = T * (1.0 - np.exp(-tau))
        gc = rgb[a:b] @ g_rgb[r]                    # g . c_i
        wgc = w * gc
        after = wgc[::-1].cumsum()[::-1] - wgc       # sum_{j>i} w_j (g . c_j)
        dsigma[a:b] = dt[a:b] * (T_next * gc - after)
        drgb[a:b] = w[:, None] * g_rgb[r][None, :]
    return dsigma, drgb
