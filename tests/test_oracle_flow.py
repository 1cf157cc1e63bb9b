"""Pins of the flow oracle (oracle/flow.py): the single-bin spline is the paper's RQF
(Sec. 2.3, Eqs. mass_measure_rqs and r_to_y_inverse) and coincides with the RamboOnDiet map
G_diet at k = 1 for c = 2; inverse(forward) is the identity; the log-determinant matches a
finite-difference Jacobian determinant; autograd gradients match finite differences; a zero
last layer gives the identity flow."""
import math

import numpy as np
import pytest
import torch

from oracle import flow as F

torch.set_default_dtype(torch.float64)


def rqf_paper(y, c):
    return (y * y + c * y * (1 - y)) / (1 + (c - 2) * y * (1 - y))


def g_rqf_paper(y, c):
    return (2 * y * (1 - y) + c * (1 - y) ** 2) / (1 + (c - 2) * y * (1 - y)) ** 2


def rqf_inverse_paper(rp, c):
    b = c - (c - 2) * rp
    return 2 * rp / (b + torch.sqrt(b * b + 4 * rp * (1 - b)))


@pytest.mark.parametrize("c", [0.5, 2.0, 2.712001, 3.662872])
def test_single_bin_is_the_papers_rqf(c):
    x = torch.linspace(1e-6, 1 - 1e-6, 1001)
    one = torch.ones(x.shape[0], 1)
    dv = torch.tensor([c, 0.0]).expand(x.shape[0], 2)
    y, dydx = F.rq_forward(x, one, one, dv)
    assert torch.allclose(y, rqf_paper(x, c), rtol=0, atol=1e-15)
    assert torch.allclose(dydx, g_rqf_paper(x, c), rtol=1e-13, atol=0)
    xi = F.rq_inverse(y, one, one, dv)
    assert torch.allclose(xi, x, atol=1e-12)
    assert torch.allclose(rqf_inverse_paper(y, c), x, atol=1e-12)
    if c == 2.0:
        assert torch.allclose(y, 2 * x - x * x, atol=1e-15)  # G_diet(x, k=1)


def random_flow(d=6, layers=4, bins=8, hidden=16, seed=0, scale=0.5):
    g = torch.Generator().manual_seed(seed)
    fl = F.Flow(d, layers, bins, hidden)
    fl.params = []
    for l in range(layers):
        a, b = len(fl.cond_dims(l)), len(fl.masks[l])
        P = b * (3 * bins + 1)
        fl.params.append({"W1": torch.randn(hidden, a, generator=g) * scale, "b1": torch.randn(hidden, generator=g) * 0.1,
                          "W2": torch.randn(hidden, hidden, generator=g) * scale / 4, "b2": torch.randn(hidden, generator=g) * 0.1,
                          "W3": torch.randn(P, hidden, generator=g) * scale, "b3": torch.randn(P, generator=g) * 0.5})
    return fl


def test_masks_cover_every_dimension():
    for d in (2, 5, 10, 13):
        m = F.masks(d, 6)
        assert all(len(t) > 0 and len(t) < d for t in m)
        assert set().union(*map(set, m)) == set(range(d))


def test_inverse_of_forward_and_unit_cube():
    fl = random_flow()
    z = torch.rand(500, 6, generator=torch.Generator().manual_seed(1)) * 0.999 + 0.0005
    r, ld = fl.forward(z, bf=False)
    assert float(r.min()) > 0 and float(r.max()) < 1
    zb, lq = fl.inverse(r, bf=False)
    assert torch.allclose(zb, z, atol=1e-10)
    assert torch.allclose(lq, -ld, atol=1e-9)


def test_logdet_against_finite_differences():
    fl = random_flow(d=4, layers=3, bins=6, hidden=8)
    z0 = torch.tensor([[0.21, 0.47, 0.73, 0.35]])
    _, ld = fl.forward(z0, bf=False)
    h = 1e-6
    J = torch.zeros(4, 4)
    for j in range(4):
        e = torch.zeros(1, 4)
        e[0, j] = h
        rp, _ = fl.forward(z0 + e, bf=False)
        rm, _ = fl.forward(z0 - e, bf=False)
        J[:, j] = (rp - rm)[0] / (2 * h)
    assert abs(math.log(abs(float(torch.det(J)))) - float(ld[0])) < 1e-7


def test_autograd_gradient_against_finite_differences():
    fl = random_flow(d=4, layers=3, bins=6, hidden=8, seed=3)
    g = torch.Generator().manual_seed(4)
    r = torch.rand(64, 4, generator=g) * 0.98 + 0.01
    w = torch.rand(64, generator=g) + 0.1
    L, grads = fl.loss_and_grads(r, w, bf=False)
    rng = np.random.default_rng(5)
    for l in range(3):
        for name in ("W1", "b2", "W3", "b3"):
            t = fl.params[l][name]
            idx = tuple(int(rng.integers(0, s)) for s in t.shape)
            old = float(t[idx])
            eps = 1e-6
            t[idx] = old + eps
            lp = float(fl.loss(r, w, bf=False))
            t[idx] = old - eps
            lm = float(fl.loss(r, w, bf=False))
            t[idx] = old
            fd = (lp - lm) / (2 * eps)
            an = float(grads[l][name][idx])
            assert abs(fd - an) <= 1e-6 * max(1.0, abs(an)), (l, name, fd, an)


def test_zero_last_layer_is_identity():
    fl = random_flow(d=5, layers=4, bins=16, hidden=16)
    for p in fl.params:
        p["W3"].zero_()
        K = 16
        b = torch.zeros_like(p["b3"]).reshape(-1, 3 * K + 1)
        b[:, 2 * K:] = math.log(math.expm1(1.0 - F.MIN_D))  # derivative 1 at every knot
        p["b3"] = b.reshape(-1)
    z = torch.rand(200, 5, generator=torch.Generator().manual_seed(2))
    r, ld = fl.forward(z, bf=False)
    assert torch.allclose(r, z, atol=1e-14) and torch.allclose(ld, torch.zeros(200), atol=1e-12)
