"""Adam update (oracle, FP64).  Test infrastructure only.

Paper basis: Sec. 4.1 - the NGP features and density network of each NeRF
have their own optimiser, the shared colour network has a separate one, and
training continues without resetting them when the window moves (Sec. 4.4);
Sec. 4.6 - the optimisation strategy is I-NGP's.

Restated from Kingma & Ba (2015) with I-NGP's hyper-parameters (reading):
lr = 1e-2, beta1 = 0.9, beta2 = 0.99, eps = 1e-15, L2 weight decay 1e-6 on
MLP weights only (added to the gradient), constant learning rate.  Step
count t starts at 1 on the first update and is kept per optimiser.

    g' = g + lambda w
    m  = beta1 m + (1 - beta1) g'
    v  = beta2 v + (1 - beta2) g'^2
    w  = w - lr * (m / (1 - beta1^t)) / (sqrt(v / (1 - beta2^t)) + eps)
"""
import numpy as np

LR = 1e-2
BETA1 = 0.9
BETA2 = 0.99
EPS = 1e-15
L2_MLP = 1e-6


def step(w, g, m, v, t, lr=LR, beta1=BETA1, beta2=BETA2, eps=EPS, l2=0.0):
    """One Adam update at step count t (>= 1).  Returns new (w, m, v)."""
    g = g + l2 * w
    m = beta1 * m + (1.0 - beta1) * g
    v = beta2 * v + (1.0 - beta2) * g * g
    mhat = m / (1.0 - beta1 ** t)
    vhat = v / (1.0 - beta2 ** t)
    return w - lr * mhat / (np.sqrt(vhat) + eps), m, v
