"""Oracle pins for the local (SDE) multichannel weights (Sec. 2.1,
Eq. multi-channel-mg): the channel's own propagator product from its sampled
invariants equals the one recomputed from momenta (the masks are right),
alpha lies in [0,1], and sum_c I_c does not depend on the choice of alpha."""
import math

import numpy as np

from paper_2602_06895_gb300 import workloads as W


def test_own_channel_weight_matches_momenta(oracle_mod):
    chans = W.multichannel_2to5()
    for i, ch in enumerate(chans):
        d = oracle_mod.dims(ch)
        assert d == 13
        r = W.uniform_r(200 + i, 20_000, d)
        o = oracle_mod.forward(ch, r, channels=chans, chan=i, aux=True)
        a = o["aux"]
        rel = np.abs(a[:, oracle_mod.AUX["p_own"]] / a[:, oracle_mod.AUX["p_own_momenta"]] - 1.0)
        assert np.median(rel) < 1e-12 and np.percentile(rel, 99.9) < 1e-6, ch["name"]
        assert np.all((o["alpha"] >= 0) & (o["alpha"] <= 1))


def test_sum_of_channels_independent_of_alpha(oracle_mod):
    chans = W.multichannel_2to5()
    uni = []
    for ch in chans:
        c = dict(ch)
        c["integrand"] = "pdf_sde_uniform"
        uni.append(c)
    tot = {}
    for name, cs in (("sde", chans), ("uniform", uni)):
        mean, var = 0.0, 0.0
        for i, ch in enumerate(cs):
            r = W.uniform_r(300 + i, 200_000, 13)
            w = oracle_mod.forward(ch, r, channels=chans, chan=i)["w"]
            mean += w.mean()
            var += w.var() / w.size
        tot[name] = (mean, math.sqrt(var))
    (a, ea), (b, eb) = tot["sde"], tot["uniform"]
    assert abs(a - b) < 4.5 * math.sqrt(ea ** 2 + eb ** 2), (a, ea, b, eb)
    assert ea / a < 0.05
