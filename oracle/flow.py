"""FP64 CPU oracle of the rational-quadratic-spline coupling flow -- TEST INFRASTRUCTURE ONLY.

Only tests/ and the CPU-baseline leg of bench.py use it; it shares no code with the CUDA flow.

The flow is the learned proposal that replaces or refines the VEGAS grid (the paper's
neural importance sampling, Sec. 3.2.2, with rational-quadratic spline transformations after
Durkan et al. 2019; its single-bin case is the paper's RQF, Sec. 2.3).  Written in plain
PyTorch CPU ops in float64; gradients come from torch.autograd.

  coupling layer l: the dims with mask_l == 0 (A) condition an MLP
      A -> Linear(H) -> SiLU -> Linear(H) -> SiLU -> Linear(n_B (3K+1))
  whose outputs per transformed dim are K width logits, K height logits, K+1 derivative
  pre-activations; widths/heights = m + (1 - K m) softmax(.), derivatives = m + softplus(.).
  The dims with mask_l == 1 (B) go through the monotone spline F on [0, 1].

The GEMM operands are rounded to bfloat16 before the FP64 products when `bf16=True`, as in the
GPU kernels (bfloat16 operands, wide accumulation).
"""
from __future__ import annotations

import math

import torch

MIN_W = 1e-3
MIN_H = 1e-3
MIN_D = 1e-3


def masks(d, n_layers):
    """Transformed dims of each layer: up to 16 dims, bit (l mod nbits) of the dim index, flipped
    every nbits layers; above 16 dims, the group j mod 3 == l mod 3 (at most 8 transformed and 16
    conditioning dims per layer for d <= 24)."""
    if d > 16:
        return [[j for j in range(d) if j % 3 == l % 3] for l in range(n_layers)]
    nb = max(1, math.ceil(math.log2(d)))
    out = []
    for l in range(n_layers):
        b, flip = l % nb, (l // nb) % 2
        out.append([j for j in range(d) if ((j >> b) & 1) != flip])
    return out


def bf16(t):
    return t.to(torch.bfloat16).to(torch.float64)


def silu(x):
    return x * torch.sigmoid(x)


def spline_params(raw, K):
    """raw [..., 3K+1] -> widths, heights [..., K], derivatives [..., K+1]."""
    w = MIN_W + (1 - K * MIN_W) * torch.softmax(raw[..., :K], dim=-1)
    h = MIN_H + (1 - K * MIN_H) * torch.softmax(raw[..., K:2 * K], dim=-1)
    dv = MIN_D + torch.nn.functional.softplus(raw[..., 2 * K:])
    return w, h, dv


def rq_forward(x, w, h, dv):
    """Monotone rational-quadratic spline on [0,1] (Durkan et al. 2019, Eq. for the bin k):
    y = y_k + h_k [s xi^2 + d_k xi (1-xi)] / [s + (d_{k+1} + d_k - 2s) xi (1-xi)],  s = h_k / w_k,
    dy/dx = s^2 [d_{k+1} xi^2 + 2 s xi (1-xi) + d_k (1-xi)^2] / [..]^2.  Returns y, dy/dx."""
    K = w.shape[-1]
    xk = torch.cumsum(w, dim=-1) - w          # left knots
    yk = torch.cumsum(h, dim=-1) - h
    # bin of x: the last knot <= x (x in [0,1])
    k = torch.clamp((x.unsqueeze(-1) >= xk).sum(dim=-1) - 1, 0, K - 1)
    g = lambda t: torch.gather(t, -1, k.unsqueeze(-1)).squeeze(-1)
    x0, wk, y0, hk = g(xk), g(w), g(yk), g(h)
    d0 = torch.gather(dv, -1, k.unsqueeze(-1)).squeeze(-1)
    d1 = torch.gather(dv, -1, (k + 1).unsqueeze(-1)).squeeze(-1)
    xi = (x - x0) / wk
    s = hk / wk
    om = xi * (1 - xi)
    den = s + (d1 + d0 - 2 * s) * om
    y = y0 + hk * (s * xi * xi + d0 * om) / den
    dydx = s * s * (d1 * xi * xi + 2 * s * om + d0 * (1 - xi) ** 2) / (den * den)
    return y, dydx


def rq_inverse(y, w, h, dv):
    """Inverse of rq_forward: the root of the quadratic in xi (numerically stable form)."""
    K = w.shape[-1]
    xk = torch.cumsum(w, dim=-1) - w
    yk = torch.cumsum(h, dim=-1) - h
    k = torch.clamp((y.unsqueeze(-1) >= yk).sum(dim=-1) - 1, 0, K - 1)
    g = lambda t: torch.gather(t, -1, k.unsqueeze(-1)).squeeze(-1)
    x0, wk, y0, hk = g(xk), g(w), g(yk), g(h)
    d0 = torch.gather(dv, -1, k.unsqueeze(-1)).squeeze(-1)
    d1 = torch.gather(dv, -1, (k + 1).unsqueeze(-1)).squeeze(-1)
    s = hk / wk
    dy = y - y0
    a = hk * (s - d0) + dy * (d1 + d0 - 2 * s)
    b = hk * d0 - dy * (d1 + d0 - 2 * s)
    c = -s * dy
    xi = 2 * c / (-b - torch.sqrt(b * b - 4 * a * c))
    return x0 + xi * wk


class Flow:
    """Parameters: list of per-layer dicts {W1 [H, A], b1 [H], W2 [H, H], b2, W3 [P, H], b3 [P]}
    (float64), with P = n_B (3K+1)."""

    def __init__(self, d, n_layers=6, bins=16, hidden=128):
        self.d, self.L, self.K, self.H = d, n_layers, bins, hidden
        self.masks = masks(d, n_layers)
        self.params = None

    def cond_dims(self, l):
        return [j for j in range(self.d) if j not in self.masks[l]]

    def mlp(self, l, xa, bf=True):
        p = self.params[l]
        c = bf16 if bf else (lambda t: t)
        z1 = c(xa) @ c(p["W1"]).T + p["b1"]
        z2 = c(silu(z1)) @ c(p["W2"]).T + p["b2"]
        return c(silu(z2)) @ c(p["W3"]).T + p["b3"]

    def forward(self, z, bf=True):
        """z [B, d] in (0,1) -> r [B, d], log |dr/dz| [B]."""
        x = z.clone()
        logdet = torch.zeros(z.shape[0], dtype=torch.float64)
        for l in range(self.L):
            tb, ta = self.masks[l], self.cond_dims(l)
            raw = self.mlp(l, x[:, ta], bf).reshape(z.shape[0], len(tb), 3 * self.K + 1)
            w, h, dv = spline_params(raw, self.K)
            y, dydx = rq_forward(x[:, tb], w, h, dv)
            x = x.clone()
            x[:, tb] = y
            logdet = logdet + torch.log(dydx).sum(dim=1)
        return x, logdet

    def inverse(self, r, bf=True):
        """r [B, d] -> z [B, d], log g(r) = log |dz/dr| [B]."""
        x = r.clone()
        logq = torch.zeros(r.shape[0], dtype=torch.float64)
        for l in reversed(range(self.L)):
            tb, ta = self.masks[l], self.cond_dims(l)
            raw = self.mlp(l, x[:, ta], bf).reshape(r.shape[0], len(tb), 3 * self.K + 1)
            w, h, dv = spline_params(raw, self.K)
            xb = rq_inverse(x[:, tb], w, h, dv)
            _, dydx = rq_forward(xb, w, h, dv)
            x = x.clone()
            x[:, tb] = xb
            logq = logq - torch.log(dydx).sum(dim=1)
        return x, logq

    def loss(self, r, w, bf=True):
        """Importance-weighted forward KL: -sum_b (w_b / sum w) log g(r_b)."""
        _, logq = self.inverse(r, bf)
        return -(w / w.sum() * logq).sum()

    def loss_and_grads(self, r, w, bf=True):
        for p in self.params:
            for t in p.values():
                t.requires_grad_(True)
                t.grad = None
        L = self.loss(r, w, bf)
        L.backward()
        grads = [{k: t.grad.detach().clone() for k, t in p.items()} for p in self.params]
        for p in self.params:
            for t in p.values():
                t.requires_grad_(False)
        return float(L.detach()), grads
