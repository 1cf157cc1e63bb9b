"""Oracle of event unweighting -- TEST INFRASTRUCTURE ONLY (tests/, the CPU-baseline and
reference legs of bench.py).  Plain numpy in float64; shares no code with the CUDA path.

Unweighting and file output (Sec. "Unweighting and file output", event-generation workflow):
events are accepted against a maximum weight that is estimated allowing a user-defined amount
of over-weight events relative to the total cross section (0.1% in the validation runs of the
results section).  Reading used here (the paper gives no formula):

  w_max(eps) = the smallest t >= 0 with  sum_b max(0, w_b - t) <= eps * sum_b w_b,

i.e. the part of the cross section carried above w_max by over-weight events is at most eps.
The excess is continuous and decreasing in t, so with the weights sorted in decreasing order
(w_(1) >= w_(2) >= ...) and s_k = w_(1) + ... + w_(k), w_max = (s_k - eps S) / k for the first k
with (s_k - eps S) / k >= w_(k+1)  (w_(n+1) = 0), clipped at 0.

Event b is accepted iff  u_b * w_max < w_b  with u_b the first uniform of the event's random
point in stream UNWEIGHT_STREAM (the generator's Philox point definition: counter (event lo,
event hi, stream, 0), key (seed lo, seed hi), top 52 bits of words (1,0), (k + 1/2) 2^-52), and
keeps the weight max(w_b, w_max): E[accepted weight] = min(1, w/w_max) max(w, w_max) = w.
"""
from __future__ import annotations

import numpy as np

import oracle as O

UNWEIGHT_STREAM = 0x556E7700  # "Unw\0"


def excess(w, t):
    """sum_b max(0, w_b - t), the over-weight part of the cross section at threshold t."""
    w = np.asarray(w, dtype=np.float64)
    return float(np.sum(np.maximum(w - t, 0.0)))


def max_weight(w, eps):
    """w_max(eps) from the sorted weights (closed form on the segment holding the root)."""
    w = np.asarray(w, dtype=np.float64)
    if w.size == 0:
        return 0.0
    if np.any(w < 0) or not np.all(np.isfinite(w)):
        raise ValueError("weights must be finite and non-negative")
    S = float(np.sum(w))
    if S == 0.0:
        return 0.0
    target = eps * S
    ws = np.sort(w)[::-1]
    s = np.cumsum(ws)
    k = np.arange(1, ws.size + 1, dtype=np.float64)
    t = (s - target) / k
    lower = np.append(ws[1:], 0.0)
    first = int(np.argmax(t >= lower))
    return max(float(t[first]), 0.0)


def uniforms(seed, ev0, n):
    """u_b for events ev0 .. ev0 + n - 1."""
    return O.random(seed, UNWEIGHT_STREAM, ev0, n, 1)[:, 0]


def accept(w, w_max, seed, ev0=0):
    """(indices of accepted events in increasing order, their weights max(w, w_max))."""
    w = np.asarray(w, dtype=np.float64)
    u = uniforms(seed, ev0, w.size)
    keep = u * w_max < w
    idx = np.nonzero(keep)[0]
    return idx, np.maximum(w[idx], w_max)
