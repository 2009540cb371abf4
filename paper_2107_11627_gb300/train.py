"""Training the P2S network (Sec. 3.3) on the basis dictionary.

The paper re-uses the 50,000 dictionary PSFs (Sec. 3.2) to train the network:
the input is a PSF's higher-order Zernike vector, the target its basis
coefficients found by projecting the PSF onto the learned basis, and the loss
the l2 distance between predicted and target coefficients.  Here:

  pairs    alpha_4..36 of each dictionary draw (radians, no normalisation) and
           beta* = H h, h the centred unit-sum PSF (H has orthonormal rows, so
           this is the least-squares projection);
  network  dims[0] = 33 -> ... -> dims[-1] = K, ReLU after every layer but the
           last (the reading the simulator uses);
  fit      Adam on the mean squared error of beta, seeded, on the host or a
           GPU through PyTorch (this is an offline step, not the per-frame path).

Reported: the coefficient MSE, and the PSF error ||H^T beta - h|| / ||h|| of
the network on held-out draws beside the projection floor ||H^T beta* - h|| / ||h||
(the part no network can remove: the basis truncation).
"""
from __future__ import annotations

import os

import numpy as np

from . import basis

_CACHE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "_build")


def training_pairs(Hb: np.ndarray, n_dict: int, taps: int, seed: int = 2021, dr0_range=(0.5, 6.0)):
    """(alpha_4..36 [n, 33], beta* [n, K], psf [n, T]) of the dictionary draws."""
    D, alpha = basis.psf_dictionary(n_dict, taps, seed=seed, dr0_range=dr0_range, with_alpha=True)
    return alpha[:, 2:], D @ Hb.T, D


def psf_errors(Hb: np.ndarray, beta: np.ndarray, psf: np.ndarray) -> np.ndarray:
    """Per-sample ||H^T beta - h|| / ||h||."""
    r = beta @ Hb - psf
    return np.linalg.norm(r, axis=1) / np.linalg.norm(psf, axis=1)


def train_p2s(Hb: np.ndarray, dims, n_dict: int = 50_000, taps: int = 33, epochs: int = 80, batch: int = 256,
              lr: float = 1e-3, val_frac: float = 0.1, seed: int = 7, device: str = "cpu", cache: bool = True,
              scale_inputs: bool = False):
    """Fit the network; returns (layers [(W [out, in], b [out]) float64], report dict).

    scale_inputs: the fit sees alpha divided by each mode's standard deviation over the
    training draws; the scale is folded into the first layer afterwards (W1 <- W1 / sigma),
    so the returned network still takes raw alpha, exactly."""
    import torch

    tag = (f"p2s_{'-'.join(map(str, dims))}_N{n_dict}_T{taps}_E{epochs}_B{batch}_S{seed}_L{lr}_X{int(scale_inputs)}_"
           f"{abs(hash(Hb.tobytes())) % 10**8}")
    path = os.path.join(_CACHE, tag + ".npz")
    if cache and os.path.exists(path):
        z = np.load(path, allow_pickle=True)
        layers = [(z[f"W{i}"], z[f"b{i}"]) for i in range(len(dims) - 1)]
        return layers, z["report"].item()
    a, beta_t, psf = training_pairs(Hb, n_dict, taps)
    rng = np.random.default_rng(seed)
    perm = rng.permutation(len(a))
    n_val = max(1, int(val_frac * len(a)))
    val, tr = perm[:n_val], perm[n_val:]
    sigma = a[tr].std(axis=0) if scale_inputs else np.ones(a.shape[1])
    sigma = np.where(sigma > 0, sigma, 1.0)
    a_s = a / sigma
    torch.manual_seed(seed)
    mods = []
    for i in range(len(dims) - 1):
        mods.append(torch.nn.Linear(dims[i], dims[i + 1]))
        if i + 2 < len(dims):
            mods.append(torch.nn.ReLU())
    net = torch.nn.Sequential(*mods).to(device=device, dtype=torch.float32)
    opt = torch.optim.Adam(net.parameters(), lr=lr)
    sched = torch.optim.lr_scheduler.CosineAnnealingLR(opt, T_max=epochs)
    xa = torch.tensor(a_s[tr], dtype=torch.float32, device=device)
    ya = torch.tensor(beta_t[tr], dtype=torch.float32, device=device)
    xv = torch.tensor(a_s[val], dtype=torch.float32, device=device)
    yv = torch.tensor(beta_t[val], dtype=torch.float32, device=device)
    g = torch.Generator(device="cpu").manual_seed(seed)
    history = []
    for ep in range(epochs):
        order = torch.randperm(len(xa), generator=g).to(device)
        net.train()
        for s0 in range(0, len(xa), batch):
            idx = order[s0:s0 + batch]
            loss = torch.mean((net(xa[idx]) - ya[idx]) ** 2)
            opt.zero_grad()
            loss.backward()
            opt.step()
        sched.step()
        with torch.no_grad():
            history.append(float(torch.mean((net(xv) - yv) ** 2)))
    layers = []
    for m in net:
        if isinstance(m, torch.nn.Linear):
            layers.append((m.weight.detach().cpu().double().numpy(), m.bias.detach().cpu().double().numpy()))
    layers[0] = (layers[0][0] / sigma[None, :], layers[0][1])  # raw alpha in
    with torch.no_grad():
        pred = net(xv).cpu().double().numpy()
    e_net = psf_errors(Hb, pred, psf[val])
    e_proj = psf_errors(Hb, beta_t[val], psf[val])
    report = {"val_beta_mse": history[-1], "val_beta_mse_first_epoch": history[0],
              "val_beta_mse_zero_predictor": float(np.mean(beta_t[val] ** 2)),
              "psf_rel_err_network_median": float(np.median(e_net)),
              "psf_rel_err_projection_median": float(np.median(e_proj)),
              "n_train": int(len(tr)), "n_val": int(n_val), "epochs": epochs}
    if cache:
        os.makedirs(_CACHE, exist_ok=True)
        np.savez(path, report=np.array(report, dtype=object),
                 **{f"W{i}": W for i, (W, _) in enumerate(layers)}, **{f"b{i}": b for i, (_, b) in enumerate(layers)})
    return layers, report


def network_psfs(Hb: np.ndarray, layers, alpha_hi: np.ndarray) -> np.ndarray:
    """[n, T] PSFs H^T beta(alpha) of the network (ReLU after every layer but the last)."""
    h = np.asarray(alpha_hi, dtype=np.float64)
    for i, (W, b) in enumerate(layers):
        h = h @ W.T + b
        if i + 1 < len(layers):
            h = np.maximum(h, 0.0)
    return h @ Hb


def _width(psf: np.ndarray) -> float:
    """RMS radius (pixels) of a PSF about its centroid."""
    n = psf.shape[0]
    yy, xx = np.meshgrid(np.arange(n, dtype=np.float64), np.arange(n, dtype=np.float64), indexing="ij")
    m = psf.sum()
    cy, cx = (psf * yy).sum() / m, (psf * xx).sum() / m
    return float(np.sqrt((psf * ((yy - cy) ** 2 + (xx - cx) ** 2)).sum() / m))


def exposure_psfs(Hb: np.ndarray, layers, taps: int, d_over_r0: float, n: int = 2000, seed: int = 5,
                  margin: int = 8, kappa: float = -4.0 / np.pi):
    """Short- and long-exposure PSFs (Sec. 4.1, Evaluation 2) of the network against the
    pupil-FFT PSFs it stands in for, over n draws at one turbulence strength.

    SE: the mean of the centred PSFs (tilts left out), network H^T beta(alpha) against the
    Eq. 2 PSF of the same alpha.  LE: the mean of the same PSFs each shifted by its tilt
    displacement d = kappa (alpha_3, alpha_2) pixels (the simulator's warp), placed
    bilinearly on a grid `margin` pixels wider on each side.  Returns the PSFs and, per
    exposure, the relative L2 distance network vs pupil FFT and both RMS widths."""
    D, alpha = basis.psf_dictionary(n, taps, seed=seed, dr0_range=(d_over_r0, d_over_r0), with_alpha=True)
    P = network_psfs(Hb, layers, alpha[:, 2:])
    out = {}
    se_x, se_n = D.mean(axis=0).reshape(taps, taps), P.mean(axis=0).reshape(taps, taps)
    G = taps + 2 * margin
    le_x, le_n = np.zeros((G, G)), np.zeros((G, G))
    dy, dx = kappa * alpha[:, 1], kappa * alpha[:, 0]
    for i in range(n):
        iy, ix = int(np.floor(dy[i])), int(np.floor(dx[i]))
        fy, fx = dy[i] - iy, dx[i] - ix
        for src, dst in ((D[i], le_x), (P[i], le_n)):
            p = src.reshape(taps, taps)
            for oy, wy in ((0, 1 - fy), (1, fy)):
                for ox, wx in ((0, 1 - fx), (1, fx)):
                    y0, x0 = margin + iy + oy, margin + ix + ox
                    if 0 <= y0 and y0 + taps <= G and 0 <= x0 and x0 + taps <= G:
                        dst[y0:y0 + taps, x0:x0 + taps] += wy * wx * p
    le_x /= n
    le_n /= n
    for name, a, b in (("se", se_x, se_n), ("le", le_x, le_n)):
        out[name] = {"rel_l2": float(np.linalg.norm(b - a) / np.linalg.norm(a)), "width_psf": _width(a),
                     "width_network": _width(b), "psf": a, "network": b}
    return out
