"""GPU parity of the rational-quadratic-spline coupling flow (the learned proposal, Sec. 3.2.2)
against the FP64 flow oracle (oracle/flow.py), through the C ABI.

Tolerances (the GPU runs the MLP GEMMs with bfloat16 operands and FP32 accumulation, and the
splines in FP32; the oracle rounds the same GEMM operands to bfloat16 and computes in FP64):
  z, masks      bit-exact (Philox bits, integer layout)
  r, z (inv.)   |d| <= 2e-3 for every event, mean |d| <= 1e-4: an FP32 pre-activation that
                lies within its FP32 error of a bfloat16 rounding boundary rounds the other
                way in one of the two (a 2^-8 relative step of one activation, a few per
                event at H = 128), moving the spline parameters by ~1e-3 relative; the FP32
                spline itself contributes ~1e-6
  log-det       |d| <= 2e-2 per event, mean |d| <= 1e-3 (the same flips, through log F')
  gradients     relative L2 error per parameter tensor <= 5e-2 (the backward GEMMs also round
                their adjoints to bfloat16: ~2^-9 relative per term, averaged over the batch)
  loss          relative 1e-3
"""
import math

import numpy as np
import pytest

import oracle as O
from oracle import flow as OF
from paper_2602_06895_gb300 import ps
from paper_2602_06895_gb300 import workloads as W

pytestmark = pytest.mark.gpu

D, L, K, H = 10, 6, 16, 128


@pytest.fixture(scope="module")
def torch_cuda():
    import torch

    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2602_06895_gb300 import build

    build.build()
    return torch


def random_params(fl, seed, scale=0.15):
    """Random logical parameters of a GPU flow, and the same in the oracle's per-layer form."""
    import torch

    g = np.random.default_rng(seed)
    masks = [fl.mask(l) for l in range(fl.n_layers)]
    layout, n = ps.flow_param_layout(fl.dims, fl.n_layers, fl.bins, fl.hidden, masks)
    assert n == fl.n_params
    p = np.zeros(n, dtype=np.float32)
    for lay in layout:
        na = lay["W1"][1][1]
        for name, (o, shape) in lay.items():
            size = int(np.prod(shape))
            if name == "W1":
                v = g.uniform(-1, 1, size) / math.sqrt(na)
            elif name == "W2":
                v = g.uniform(-1, 1, size) / math.sqrt(fl.hidden)
            elif name == "W3":
                v = g.normal(0, scale, size)
            elif name == "b3":
                v = g.normal(0, 0.3, size)
            else:
                v = g.normal(0, 0.1, size)
            p[o:o + size] = v
    orc = OF.Flow(fl.dims, fl.n_layers, fl.bins, fl.hidden)
    orc.params = [{k: torch.from_numpy(p[o:o + int(np.prod(s))].astype(np.float64)).reshape(s)
                   for k, (o, s) in lay.items()} for lay in layout]
    return p, orc, layout


def sample(torch, fl, B, seed, offset=0):
    r = torch.empty((fl.dims, B), dtype=torch.float64, device="cuda")
    z = torch.empty_like(r)
    ld = torch.empty(B, dtype=torch.float64, device="cuda")
    fl.sample(B, seed, r, ld, z, event_offset=offset)
    torch.cuda.synchronize()
    return r, ld, z


def test_masks_match_oracle(torch_cuda):
    for d in (2, 5, 10, 16, 17, 22, 24):
        fl = ps.Flow(d, 6, 4, 32, max_batch=64)
        assert [fl.mask(l) for l in range(6)] == OF.masks(d, 6)


def test_z_is_philox(torch_cuda):
    torch = torch_cuda
    fl = ps.Flow(D, L, K, H, max_batch=4096)
    B, seed, off = 1000, 0x1234_5678_9ABC, 77
    _, _, z = sample(torch, fl, B, seed, off)
    z = z.cpu().numpy()
    for b in (0, 1, 499, 999):
        ev = off + b
        for j in range(0, D, 2):
            words = O.philox([ev & 0xFFFFFFFF, ev >> 32, 0x466C6F77, j // 2], [seed & 0xFFFFFFFF, seed >> 32])
            assert z[j, b] == ((words[0] >> 9) + 0.5) * 2.0 ** -23
            assert z[j + 1, b] == ((words[1] >> 9) + 0.5) * 2.0 ** -23


def test_new_flow_is_identity(torch_cuda):
    torch = torch_cuda
    fl = ps.Flow(D, L, K, H, max_batch=8192)
    r, ld, z = sample(torch, fl, 5000, 3)
    assert torch.max(torch.abs(r - z)).item() < 2e-6
    assert torch.max(torch.abs(ld)).item() < 1e-4


@pytest.mark.parametrize("B", [1, 4099])
def test_forward_matches_oracle(torch_cuda, B):
    torch = torch_cuda
    fl = ps.Flow(D, L, K, H, max_batch=4160)
    p, orc, _ = random_params(fl, 11)
    fl.set_params(p)
    assert np.array_equal(fl.get_params(), p)
    r, ld, z = sample(torch, fl, B, 5)
    r_o, ld_o = orc.forward(z.T.cpu(), bf=True)
    dr = np.abs(r.T.cpu().numpy() - r_o.numpy())
    dl = np.abs(ld.cpu().numpy() - ld_o.numpy())
    assert np.all(np.isfinite(r.cpu().numpy())) and np.all(np.isfinite(ld.cpu().numpy()))
    assert dr.max() <= 2e-3 and dr.mean() <= 1e-4, (dr.max(), dr.mean())
    assert dl.max() <= 2e-2 and dl.mean() <= 1e-3, (dl.max(), dl.mean())
    # the parameters move the points: the test is not passing on an identity map
    if B > 1:
        assert np.abs(r_o.numpy() - z.T.cpu().numpy()).mean() > 1e-2


def test_sample_in_chunks_matches_one_call(torch_cuda):
    torch = torch_cuda
    big = ps.Flow(D, L, K, H, max_batch=4096)
    small = ps.Flow(D, L, K, H, max_batch=1000)
    p, _, _ = random_params(big, 12)
    big.set_params(p)
    small.set_params(p)
    r1, l1, _ = sample(torch, big, 3001, 9)
    r2, l2, _ = sample(torch, small, 3001, 9)
    assert torch.equal(r1, r2) and torch.equal(l1, l2)


def test_generate_across_its_internal_chunks(torch_cuda):
    """A generate call longer than the fused path's internal chunk (2^22 events) equals two calls
    split at an arbitrary event, with the second call's event offset: points, log-det and z."""
    torch = torch_cuda
    fl = ps.Flow(D, L, K, H, max_batch=4096)
    p, _, _ = random_params(fl, 15)
    fl.set_params(p)
    n, n1 = (1 << 22) + 4099, 1_234_567
    r = torch.empty((D, n), dtype=torch.float64, device="cuda")
    ld = torch.empty(n, dtype=torch.float64, device="cuda")
    z = torch.empty_like(r)
    fl.generate(n, 21, r, ld, z, event_offset=5)
    parts = []
    for lo, hi in ((0, n1), (n1, n)):
        rp = torch.empty((D, hi - lo), dtype=torch.float64, device="cuda")
        lp = torch.empty(hi - lo, dtype=torch.float64, device="cuda")
        zp = torch.empty_like(rp)
        fl.generate(hi - lo, 21, rp, lp, zp, event_offset=5 + lo)
        parts.append((rp, lp, zp))
    torch.cuda.synchronize()
    assert torch.equal(r, torch.cat([parts[0][0], parts[1][0]], dim=1))
    assert torch.equal(ld, torch.cat([parts[0][1], parts[1][1]]))
    assert torch.equal(z, torch.cat([parts[0][2], parts[1][2]], dim=1))
    assert fl.status() == 0


def test_inverse_matches_oracle_and_round_trips(torch_cuda):
    torch = torch_cuda
    fl = ps.Flow(D, L, K, H, max_batch=4096)
    p, orc, _ = random_params(fl, 13)
    fl.set_params(p)
    B = 3000
    r, ld, z = sample(torch, fl, B, 21)
    zb = torch.empty_like(r)
    lq = torch.empty(B, dtype=torch.float64, device="cuda")
    fl.inverse(r, zb, lq)
    torch.cuda.synchronize()
    assert fl.status() == 0
    z_o, lq_o = orc.inverse(r.T.cpu(), bf=True)
    dz = np.abs(zb.T.cpu().numpy() - z_o.numpy())
    assert dz.max() <= 2e-3 and dz.mean() <= 1e-4, (dz.max(), dz.mean())
    dl = np.abs(lq.cpu().numpy() - lq_o.numpy())
    assert dl.max() <= 2e-2 and dl.mean() <= 1e-3, (dl.max(), dl.mean())
    # round trip on the device: same activations rounding on both sides except near knots
    rt = np.abs(zb.cpu().numpy() - z.cpu().numpy())
    assert np.median(rt) <= 1e-5 and rt.max() <= 2e-3, (np.median(rt), rt.max())
    assert np.abs(lq.cpu().numpy() + ld.cpu().numpy()).mean() <= 1e-3


@pytest.mark.parametrize("flags", [0, 2], ids=["tcgen05_forward", "layer_by_layer_forward"])
def test_gradients_match_oracle(torch_cuda, flags):
    """The training gradients against the oracle's autograd, with the training forward on the
    tcgen05 layer kernel (the default) and layer by layer (test flag)."""
    torch = torch_cuda
    fl = ps.Flow(D, L, K, H, max_batch=4096)
    p, orc, layout = random_params(fl, 14)
    fl.set_params(p)
    fl.set_debug(flags)
    B = 3000
    r, ld, z = sample(torch, fl, B, 31)
    # a correlated test integrand on the unit cube as the phase-space weight
    x = r.T
    w_map = (torch.exp(-((x[:, 0] - x[:, 1]) ** 2) / 0.02) * (1.0 + 4.0 * x[:, 2] * x[:, 3]) + 0.05).contiguous()
    loss, g = fl.gradients(w_map)
    w = (w_map * torch.exp(ld)).cpu()
    loss_o, grads_o = orc.loss_and_grads(r.T.cpu(), w, bf=True)
    assert abs(loss - loss_o) <= 1e-3 * max(1.0, abs(loss_o)), (loss, loss_o)
    worst = 0.0
    for l, lay in enumerate(layout):
        for name, (o, shape) in lay.items():
            ref = grads_o[l][name].numpy().ravel()
            got = g[o:o + ref.size].astype(np.float64)
            nrm = np.linalg.norm(ref)
            if nrm == 0:
                assert np.all(got == 0)
                continue
            err = np.linalg.norm(got - ref) / nrm
            worst = max(worst, err)
            assert err <= 5e-2, (l, name, err)
    assert worst > 0


def test_training_beats_the_vegas_grid(torch_cuda):
    """C2's integrand: the flow trained on the method's own weights (map in explicit-input
    mode after the flow) lowers the weight variance of the adapted VEGAS grid it refines, and
    both estimate the same integral."""
    torch = torch_cuda
    ch = W.ww_hadronic()
    prog = ps.program_for([ch])
    d = W.n_random_dims(ch)
    prog.vegas_training(True)
    out, ws = prog.alloc([200_000], 6)
    for it in range(6):
        prog.generate([200_000], 900 + it, out, ws)
        prog.vegas_adapt(0, alpha=1.5)
    prog.vegas_training(False)
    torch.cuda.synchronize()

    def rel_var(w):
        w = w.double()
        return (w.pow(2).mean() / w.mean() ** 2 - 1.0).item(), w.mean().item()

    n_eval = 1 << 18
    out_v, ws_v = prog.alloc([n_eval], 6)
    prog.generate([n_eval], 12345, out_v, ws_v)
    torch.cuda.synchronize()
    var_vegas, mean_vegas = rel_var(out_v["weight"])

    B = 1 << 14
    fl = ps.Flow(d, L, K, H, max_batch=B, init_seed=4)
    r = torch.empty((d, B), dtype=torch.float64, device="cuda")
    ld = torch.empty(B, dtype=torch.float64, device="cuda")
    out_f, ws_f = prog.alloc([B], 6)
    for step in range(400):
        fl.sample(B, 77, r, ld, event_offset=step * B)
        prog.map(0, r, out_f, ws_f)
        fl.train_step(out_f["weight"], 1e-3)
    torch.cuda.synchronize()
    loss, sw = fl.loss()
    assert math.isfinite(loss) and sw > 0

    fl_eval = fl  # inference in chunks of max_batch
    r = torch.empty((d, n_eval), dtype=torch.float64, device="cuda")
    ld = torch.empty(n_eval, dtype=torch.float64, device="cuda")
    fl_eval.generate(n_eval, 999, r, ld)
    out_e, ws_e = prog.alloc([n_eval], 6)
    prog.map(0, r, out_e, ws_e)
    w = torch.empty(n_eval, dtype=torch.float64, device="cuda")
    fl_eval.weights(out_e["weight"], ld, w)
    torch.cuda.synchronize()
    var_flow, mean_flow = rel_var(w)
    print(f"relative variance: VEGAS {var_vegas:.4g}, flow refining it {var_flow:.4g}")
    # unbiased: the two estimates agree within 5 combined standard errors
    se = math.sqrt((var_vegas * mean_vegas ** 2 + var_flow * mean_flow ** 2) / n_eval)
    assert abs(mean_flow - mean_vegas) <= 5 * se, (mean_flow, mean_vegas, se)
    assert var_flow < var_vegas, (var_flow, var_vegas)


@pytest.mark.parametrize("B", [1, 4099, 300_001])
def test_fused_generate_matches_layer_by_layer_and_oracle(torch_cuda, B):
    """ps_flow_generate (one fused kernel per layer) against ps_flow_sample (GEMM / spline
    kernels per layer) on the same draws, and against the oracle on a sample of events."""
    torch = torch_cuda
    fl = ps.Flow(D, L, K, H, max_batch=4160)
    p, orc, _ = random_params(fl, 15)
    fl.set_params(p)
    r = torch.empty((D, B), dtype=torch.float64, device="cuda")
    ld = torch.empty(B, dtype=torch.float64, device="cuda")
    z = torch.empty_like(r)
    fl.generate(B, 8, r, ld, z, event_offset=3)
    r2 = torch.empty_like(r)
    ld2 = torch.empty_like(ld)
    z2 = torch.empty_like(r)
    fl.set_debug(2)  # the training forward layer by layer: GEMM, gather and spline kernels
    fl.sample(B, 8, r2, ld2, z2, event_offset=3)
    fl.set_debug(0)
    r3 = torch.empty_like(r)
    ld3 = torch.empty_like(ld)
    fl.sample(B, 8, r3, ld3, event_offset=3)  # the training forward on the tcgen05 layer kernel
    torch.cuda.synchronize()
    assert torch.equal(z, z2)
    # the tcgen05 training forward and the fused sampling kernel evaluate the same arithmetic
    assert torch.max(torch.abs(r - r3)).item() <= 1e-6 and torch.max(torch.abs(ld - ld3)).item() <= 1e-5
    assert torch.max(torch.abs(r - r2)).item() <= 1e-5, torch.max(torch.abs(r - r2)).item()
    assert torch.max(torch.abs(ld - ld2)).item() <= 1e-3
    idx = torch.arange(0, B, max(1, B // 4096), device="cuda")
    r_o, ld_o = orc.forward(z[:, idx].T.cpu(), bf=True)
    dr = np.abs(r[:, idx].T.cpu().numpy() - r_o.numpy())
    dl = np.abs(ld[idx].cpu().numpy() - ld_o.numpy())
    assert dr.max() <= 2e-3 and dr.mean() <= 1e-4, (dr.max(), dr.mean())
    assert dl.max() <= 2e-2 and dl.mean() <= 1e-3, (dl.max(), dl.mean())
    assert fl.status() == 0


def test_warp_mma_fused_path(torch_cuda):
    """12 bins: the fused layer with warp-level MMAs (the tcgen05 form takes 16 bins), generate and
    inverse against the oracle."""
    torch = torch_cuda
    fl = ps.Flow(D, L, 12, H, max_batch=2048)
    p, orc, _ = random_params(fl, 17)
    fl.set_params(p)
    B = 4099
    r = torch.empty((D, B), dtype=torch.float64, device="cuda")
    ld = torch.empty(B, dtype=torch.float64, device="cuda")
    z = torch.empty_like(r)
    fl.generate(B, 10, r, ld, z)
    zb = torch.empty_like(r)
    lq = torch.empty_like(ld)
    fl.inverse(r, zb, lq)
    torch.cuda.synchronize()
    r_o, ld_o = orc.forward(z.T.cpu(), bf=True)
    dr = np.abs(r.T.cpu().numpy() - r_o.numpy())
    assert dr.max() <= 2e-3 and dr.mean() <= 1e-4, (dr.max(), dr.mean())
    assert np.abs(ld.cpu().numpy() - ld_o.numpy()).max() <= 2e-2
    z_o, lq_o = orc.inverse(r.T.cpu(), bf=True)
    assert np.abs(zb.T.cpu().numpy() - z_o.numpy()).max() <= 2e-3
    assert np.abs(lq.cpu().numpy() - lq_o.numpy()).max() <= 2e-2


def test_layer_by_layer_inverse_and_generate_fallback(torch_cuda):
    """A flow outside the fused kernel's shape (hidden 64) inverts and generates layer by layer."""
    torch = torch_cuda
    fl = ps.Flow(D, 4, 8, 64, max_batch=2048)
    p, orc, _ = random_params(fl, 16)
    fl.set_params(p)
    B = 3000
    r = torch.empty((D, B), dtype=torch.float64, device="cuda")
    ld = torch.empty(B, dtype=torch.float64, device="cuda")
    z = torch.empty_like(r)
    fl.generate(B, 9, r, ld, z)
    zb = torch.empty_like(r)
    lq = torch.empty_like(ld)
    fl.inverse(r, zb, lq)
    torch.cuda.synchronize()
    r_o, ld_o = orc.forward(z.T.cpu(), bf=True)
    assert np.abs(r.T.cpu().numpy() - r_o.numpy()).max() <= 2e-3
    z_o, lq_o = orc.inverse(r.T.cpu(), bf=True)
    assert np.abs(zb.T.cpu().numpy() - z_o.numpy()).max() <= 2e-3
    assert np.abs(lq.cpu().numpy() - lq_o.numpy()).max() <= 2e-2


def test_bounded_waits_report_timeouts_and_recover(torch_cuda):
    """A completion signal that never arrives (the test flag withholds it) and a 4-poll bound make
    a tcgen05 completion wait run out: the kernel counts the timeout in the status word, drains
    its MMAs and frees its TMEM, and the next run with the defaults is correct again (no device
    fault, no hang)."""
    torch = torch_cuda
    fl = ps.Flow(D, L, K, H, max_batch=1024)
    p, orc, _ = random_params(fl, 18)
    fl.set_params(p)
    B = 20_000
    r = torch.empty((D, B), dtype=torch.float64, device="cuda")
    ld = torch.empty(B, dtype=torch.float64, device="cuda")
    z = torch.empty_like(r)
    assert fl.status() == 0
    fl.set_wait_limit(4)
    fl.set_debug(1)
    fl.generate(B, 12, r, ld, z)
    assert fl.status() > 0
    fl.set_debug(0)
    fl.set_wait_limit(0)
    fl.generate(B, 12, r, ld, z)
    assert fl.status() == 0
    r_o, ld_o = orc.forward(z[:, :3000].T.cpu(), bf=True)
    dr = np.abs(r[:, :3000].T.cpu().numpy() - r_o.numpy())
    assert dr.max() <= 2e-3 and dr.mean() <= 1e-4, (dr.max(), dr.mean())


def test_22_dims_fused_inverse_and_gradients(torch_cuda):
    """d = 22 (the 2->8 channels: six massless and two massive particles): three interleaved
    coupling groups, at most 8 transformed dims per layer, so the fused tensor-core layer runs;
    fused generate against the layer-by-layer path and the oracle, the inverse, and the
    gradients of the training loss."""
    torch = torch_cuda
    d, B = 22, 3001
    fl = ps.Flow(d, L, K, H, max_batch=4096)
    assert [fl.mask(l) for l in range(L)] == OF.masks(d, L)
    assert max(len(fl.mask(l)) for l in range(L)) <= 8
    p, orc, layout = random_params(fl, 16)
    fl.set_params(p)
    r = torch.empty((d, B), dtype=torch.float64, device="cuda")
    ld = torch.empty(B, dtype=torch.float64, device="cuda")
    z = torch.empty_like(r)
    fl.generate(B, 41, r, ld, z)
    r2, ld2, z2 = torch.empty_like(r), torch.empty_like(ld), torch.empty_like(r)
    fl.sample(B, 41, r2, ld2, z2)
    torch.cuda.synchronize()
    assert torch.equal(z, z2)
    assert torch.max(torch.abs(r - r2)).item() <= 1e-5
    assert torch.max(torch.abs(ld - ld2)).item() <= 1e-3
    r_o, ld_o = orc.forward(z.T.cpu(), bf=True)
    dr = np.abs(r.T.cpu().numpy() - r_o.numpy())
    dl = np.abs(ld.cpu().numpy() - ld_o.numpy())
    assert dr.max() <= 2e-3 and dr.mean() <= 1e-4, (dr.max(), dr.mean())
    assert dl.max() <= 2e-2 and dl.mean() <= 1e-3, (dl.max(), dl.mean())
    assert np.abs(r_o.numpy() - z.T.cpu().numpy()).mean() > 1e-2
    zb = torch.empty_like(r)
    lq = torch.empty(B, dtype=torch.float64, device="cuda")
    fl.inverse(r, zb, lq)
    torch.cuda.synchronize()
    z_o, lq_o = orc.inverse(r.T.cpu(), bf=True)
    dz = np.abs(zb.T.cpu().numpy() - z_o.numpy())
    assert dz.max() <= 2e-3 and dz.mean() <= 1e-4, (dz.max(), dz.mean())
    x = r.T
    w_map = (torch.exp(-((x[:, 0] - x[:, 13]) ** 2) / 0.02) * (1.0 + 4.0 * x[:, 2] * x[:, 21]) + 0.05).contiguous()
    fl.sample(B, 41, r2, ld2, z2)  # the training batch is the last sampled one
    loss, g = fl.gradients(w_map)
    w = (w_map * torch.exp(ld2)).cpu()
    loss_o, grads_o = orc.loss_and_grads(r2.T.cpu(), w, bf=True)
    assert abs(loss - loss_o) <= 1e-3 * max(1.0, abs(loss_o)), (loss, loss_o)
    for l, lay in enumerate(layout):
        for name, (o, shape) in lay.items():
            ref = grads_o[l][name].numpy().ravel()
            got = g[o:o + ref.size].astype(np.float64)
            nrm = np.linalg.norm(ref)
            if nrm == 0:
                assert np.all(got == 0)
                continue
            assert np.linalg.norm(got - ref) / nrm <= 5e-2, (l, name)
    assert fl.status() == 0
