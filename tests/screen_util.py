"""Seeded screen-space splats for the binning tests: screen mean (u, v), fp32 depth, an
elliptical footprint Sigma' with its conic's Cholesky factor, opacity, the alpha level tau
and the 3-sigma radius, as the preprocess stage would hand them to the binning stage."""
from __future__ import annotations

import numpy as np

ALPHA_MIN = 1.0 / 255.0


def random_splats(seed, n, W, H, rmax, culled=0.1, ties=0.1, huge=0, faint=0.05):
    rng = np.random.default_rng(seed)
    uv = np.stack([rng.uniform(-40, W + 40, n), rng.uniform(-40, H + 40, n)], 1).astype(np.float32)
    depth = rng.uniform(0.2, 30, n).astype(np.float32)
    if n:
        depth[rng.random(n) < ties] = depth[0]                       # exact depth ties
        depth[rng.random(n) < ties / 2] = np.nextafter(depth[0], np.float32(1e9))
    # Sigma' = R diag(s1^2, s2^2) R^T, axis lengths up to rmax / 3, some needle-thin
    s1 = rng.uniform(0.3, max(rmax / 3.0, 0.4), n)
    s2 = s1 * np.where(rng.random(n) < 0.3, rng.uniform(0.02, 0.2, n), rng.uniform(0.2, 1.0, n))
    if huge and n:
        idx = rng.choice(n, huge, replace=False)
        s1[idx] = 1700.0
        s2[idx] = rng.uniform(50.0, 1700.0, huge)
    th = rng.uniform(0, np.pi, n)
    c, s = np.cos(th), np.sin(th)
    a = c * c * s1 ** 2 + s * s * s2 ** 2
    b = c * s * (s1 ** 2 - s2 ** 2)
    d = s * s * s1 ** 2 + c * c * s2 ** 2
    det = a * d - b * b
    conic = np.stack([d / det, -b / det, a / det], 1)                 # Q = Sigma'^-1
    l11 = np.sqrt(conic[:, 0])
    l21 = conic[:, 1] / l11
    l22 = np.sqrt(conic[:, 2] - l21 ** 2)
    chol = np.stack([l11, l21, l22], 1).astype(np.float32)
    opac = rng.uniform(0.02, 1.0, n)
    faint_mask = rng.random(n) < faint
    opac[faint_mask] = rng.uniform(0.0005, ALPHA_MIN * 0.999, int(faint_mask.sum()))   # never visible
    tau = (2.0 * np.log(opac / ALPHA_MIN)).astype(np.float32)
    lam = 0.5 * (a + d) + np.sqrt(0.25 * (a - d) ** 2 + b * b)
    radius = np.ceil(3.0 * np.sqrt(lam)).astype(np.int32)
    radius[rng.random(n) < culled] = 0
    return dict(uv=uv, depth=depth, chol=chol, tau=tau, radius=radius, conic=conic, opacity=opac)
