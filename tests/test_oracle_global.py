"""Pins of the oracle's global multichannel weights (Eq. channel_densities and Eq.
multi-channel-standard; oracle.global_weights):
  - one channel: w = f g_1^-1 = f J_1 is the channel's own forward weight (round trip r -> p -> r);
  - a duplicated channel leaves the density unchanged (g = g_A for any alpha split) and doubles
    the SDE integrand, so w doubles exactly;
  - the global estimate sum_i alpha_i <w>_i and the SDE estimate sum_i <w_i> are two unbiased
    estimates of the same integral (Eq. multi-channel-standard vs the SDE decomposition).
"""
import numpy as np

import oracle as O
from paper_2602_06895_gb300 import workloads as W


def test_single_channel_is_the_forward_weight():
    # momenta in the partonic frame: the round trip is then well conditioned (in the lab frame a
    # beam boost of sqrt(x1/x2) up to ~1e6 costs up to that factor in the recovered r)
    ch = dict(W.ww_hadronic(vegas_dims=0), partonic=True)
    out = O.generate(ch, 11, 0, 4000)
    keep = out["w"] > 0
    w, J, P, _ = O.global_weights([ch], [1.0], out["mom"][keep], out["x"][keep])
    rel = np.abs(w / out["w"][keep] - 1.0)
    assert np.median(rel) < 1e-13 and np.quantile(rel, 0.99) < 1e-10 and rel.max() < 1e-7, \
        (np.median(rel), np.quantile(rel, 0.99), rel.max())


def test_single_channel_lab_frame():
    ch = W.ww_hadronic(vegas_dims=0)
    out = O.generate(ch, 11, 0, 4000)
    keep = out["w"] > 0
    w, *_ = O.global_weights([ch], [1.0], out["mom"][keep], out["x"][keep])
    rel = np.abs(w / out["w"][keep] - 1.0)
    assert np.median(rel) < 1e-11 and np.quantile(rel, 0.99) < 1e-4, (np.median(rel), np.quantile(rel, 0.99))


def test_duplicated_channel():
    ch = W.ww_hadronic(vegas_dims=0)
    out = O.generate(ch, 12, 0, 500)
    keep = out["w"] > 0
    w1, *_ = O.global_weights([ch], [1.0], out["mom"][keep], out["x"][keep])
    w2, *_ = O.global_weights([ch, ch], [0.3, 0.7], out["mom"][keep], out["x"][keep])
    assert np.allclose(w2, 2.0 * w1, rtol=1e-14, atol=0)


def test_global_and_sde_estimate_the_same_integral():
    chans = W.multichannel_2to5()
    M = len(chans)
    n = 20_000
    alphas = np.full(M, 1.0 / M)
    sde_means, sde_vars, glob_means, glob_vars = [], [], [], []
    for i, ch in enumerate(chans):
        out = O.generate(ch, 100 + i, 0, n, channels=chans, chan=i)
        sde_means.append(out["w"].mean())
        sde_vars.append(out["w"].var() / n)
        keep = out["w"] > 0  # events the cut removes carry no weight in either estimate
        wg = np.zeros(n)
        wg[keep], *_ = O.global_weights(chans, alphas, out["mom"][keep], out["x"][keep])
        glob_means.append(wg.mean())
        glob_vars.append(wg.var() / n)
    I_sde = sum(sde_means)
    s_sde = np.sqrt(sum(sde_vars))
    I_glob = float(np.dot(alphas, glob_means))
    s_glob = np.sqrt(float(np.dot(alphas ** 2, glob_vars)))
    assert abs(I_glob - I_sde) <= 5 * np.hypot(s_sde, s_glob), (I_glob, I_sde, s_glob, s_sde)
    assert s_glob < 0.2 * I_glob and s_sde < 0.2 * I_sde  # the comparison has power
