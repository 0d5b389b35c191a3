"""FP64 oracle of the training step around the rasterizer (Sec. 5.1, Algorithm 1): the loss
L = (1 - lambda) L1 + lambda (1 - SSIM) with its gradient, and the Adam update of the
activated parameters.

TEST INFRASTRUCTURE ONLY: only tests/, the smoke check and the CPU legs of bench.py use this
module; it shares no code with the CUDA path and the product path never calls it.

Readings (the paper names the loss but not its constants): SSIM of Wang et al. 2004 with an
11x11 Gaussian window of sigma 1.5 (normalised), C1 = 0.01^2, C2 = 0.03^2, zero padding outside
the image ("same" size), per channel, averaged over all pixels and channels; D-SSIM = 1 - SSIM;
L1 = mean |x - y| with derivative sign(x - y) (0 at x = y); Adam of Kingma & Ba with bias
correction, eps added to the square root; opacity = sigmoid(raw), scale = exp(raw)."""
from __future__ import annotations

import numpy as np

C1 = 0.01 ** 2
C2 = 0.03 ** 2
SIGMA = 1.5
HALF = 5


def window() -> np.ndarray:
    """Normalised 1-D Gaussian window (11 taps); the 2-D window is its outer product."""
    k = np.arange(-HALF, HALF + 1, dtype=np.float64)
    g = np.exp(-(k * k) / (2.0 * SIGMA * SIGMA))
    return g / g.sum()


def window_sum(img: np.ndarray) -> np.ndarray:
    """out[y, x] = sum_{i, j} w[i] w[j] img[y + i - 5, x + j - 5], zero outside the image:
    the 121 offsets summed one by one."""
    w = window()
    H, W = img.shape
    pad = np.zeros((H + 2 * HALF, W + 2 * HALF))
    pad[HALF:HALF + H, HALF:HALF + W] = img
    out = np.zeros((H, W))
    for i in range(2 * HALF + 1):
        for j in range(2 * HALF + 1):
            out += w[i] * w[j] * pad[i:i + H, j:j + W]
    return out


def ssim_terms(x: np.ndarray, y: np.ndarray):
    """Per-pixel SSIM of one channel and the partial derivatives of S with respect to the
    window moments mx, Exx, Exy (the coefficient maps of the gradient)."""
    mx, my = window_sum(x), window_sum(y)
    exx, eyy, exy = window_sum(x * x), window_sum(y * y), window_sum(x * y)
    a1 = 2 * mx * my + C1
    a2 = 2 * (exy - mx * my) + C2
    b1 = mx * mx + my * my + C1
    b2 = (exx - mx * mx) + (eyy - my * my) + C2
    s = a1 * a2 / (b1 * b2)
    # S = a1 a2 / (b1 b2): partial derivatives through a1, a2, b1, b2
    ds_dmx = (2 * my * a2 - 2 * my * a1) / (b1 * b2) - s * (2 * mx / b1 - 2 * mx / b2)
    ds_dexx = -s / b2
    ds_dexy = 2 * a1 / (b1 * b2)
    return s, ds_dmx, ds_dexx, ds_dexy


def ssim_map(img: np.ndarray, target: np.ndarray) -> np.ndarray:
    """[3, H, W] per-pixel SSIM."""
    return np.stack([ssim_terms(np.asarray(img[c], np.float64), np.asarray(target[c], np.float64))[0]
                     for c in range(img.shape[0])])


def loss(img, target, lam: float = 0.2):
    """(L, L1, mean SSIM, dL/dimg) for planar [3, H, W] images."""
    x = np.asarray(img, np.float64)
    y = np.asarray(target, np.float64)
    n = x.size
    l1 = np.abs(x - y).sum() / n
    grad = np.empty_like(x)
    ssim_total = 0.0
    for c in range(x.shape[0]):
        s, a, b, cc = ssim_terms(x[c], y[c])
        ssim_total += s.sum()
        # d(sum_p S(p))/dx(q) = sum_p w(p - q) [a(p) + 2 x(q) b(p) + y(q) c(p)]; w is symmetric
        dssim = window_sum(a) + 2 * x[c] * window_sum(b) + y[c] * window_sum(cc)
        grad[c] = (1 - lam) * np.sign(x[c] - y[c]) / n - lam * dssim / n
    ssim = ssim_total / n
    return (1 - lam) * l1 + lam * (1 - ssim), l1, ssim, grad


def activate(raw, activation: str):
    raw = np.asarray(raw, np.float64)
    if activation == "exp":
        return np.exp(raw)
    if activation == "sigmoid":
        return 1.0 / (1.0 + np.exp(-raw))
    return raw.copy()


def adam_step(param, grad_act, m, v, lr, step, activation="none", b1=0.9, b2=0.999, eps=1e-15):
    """One Adam step of a raw parameter tensor whose loss gradient is given with respect to
    its activated value.  Returns (param, m, v, activated)."""
    p = np.asarray(param, np.float64)
    act = activate(p, activation)
    g = np.asarray(grad_act, np.float64)
    if activation == "exp":
        g = g * act
    elif activation == "sigmoid":
        g = g * act * (1 - act)
    m = b1 * np.asarray(m, np.float64) + (1 - b1) * g
    v = b2 * np.asarray(v, np.float64) + (1 - b2) * g * g
    mhat = m / (1 - b1 ** step)
    vhat = v / (1 - b2 ** step)
    p = p - lr * mhat / (np.sqrt(vhat) + eps)
    return p, m, v, activate(p, activation)


def position_lr(step: int, lr_init: float, lr_final: float, max_steps: int) -> float:
    """Exponential decay of the position learning rate (Sec. 5.1): log-linear from lr_init at
    step 0 to lr_final at max_steps, constant after."""
    t = min(max(step / max(max_steps, 1), 0.0), 1.0)
    return float(np.exp((1 - t) * np.log(lr_init) + t * np.log(lr_final)))
