"""Why no FP8 form meets the reduced-precision gate with these networks.

The FP8 forms round every convolution's inputs and weights to E4M3 (three
mantissa bits).  This CPU study emulates that rounding in float64 with
torch.float8_e4m3fn on the scale workload's U-Net and real histograms, and
measures KL(P_oracle || P) against the FP64 oracle for finer scalings than
the library's per-tensor ones: weights per output channel, activations per
input channel, and E4M3 confined to the inner layers.  Every E4M3 variant
stays above the 1e-3 gate, while BF16 rounding (eight mantissa bits) meets
it by an order of magnitude: the error comes from E4M3's mantissa, not from
its scaling.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import oracle as O  # noqa: E402
from paper_2010_01775_gb300 import synth  # noqa: E402

F = torch.nn.functional


def _q_tensor(t):
    s = t.abs().max() / 448.0
    s = s if s > 0 else torch.tensor(1.0, dtype=torch.float64)
    return (t / s).to(torch.float8_e4m3fn).to(torch.float64) * s


def _q_out_channel(w):
    s = w.abs().amax(dim=(1, 2, 3), keepdim=True) / 448.0
    s = torch.where(s > 0, s, torch.ones_like(s))
    return (w / s).to(torch.float8_e4m3fn).to(torch.float64) * s


def _q_in_channel(t):
    s = t.abs().amax(dim=(0, 2, 3), keepdim=True) / 448.0
    s = torch.where(s > 0, s, torch.ones_like(s))
    return (t / s).to(torch.float8_e4m3fn).to(torch.float64) * s


def _bf16(t):
    return t.to(torch.bfloat16).to(torch.float64)


def _unet_P(x, net, qa, qw, layers):
    Ls = net["layers"]

    def c(h, i):
        cout, cin, k, st, a, w, b = Ls[i]
        wt = torch.from_numpy(w.astype(np.float64)).permute(0, 3, 1, 2)
        if i in layers:
            h, wt = qa(h), qw(wt)
        h = F.conv2d(h, wt, torch.from_numpy(b.astype(np.float64)), stride=st, padding=k // 2)
        return F.elu(h) if a == O.ACT_ELU else (F.softplus(h) if a == O.ACT_SOFTPLUS else h)

    up = lambda h: F.interpolate(h, scale_factor=2, mode="nearest")
    t = torch.from_numpy(x).permute(0, 3, 1, 2)
    e0 = c(c(t, 0), 1)
    e1 = c(c(e0, 2), 3)
    e2 = c(c(e1, 4), 5)
    e3 = c(c(e2, 6), 7)
    d2 = c(c(torch.cat([up(e3), e2], 1), 8), 9)
    d1 = c(c(torch.cat([up(d2), e1], 1), 10), 11)
    d0 = c(c(torch.cat([up(d1), e0], 1), 12), 13)
    return O.normalise(c(d0, 14)[:, 0].numpy())[0].reshape(x.shape[0], -1)


def test_e4m3_misses_the_gate_at_any_scaling():
    ph = synth.photons(200_000, 16, 31)
    g = O.build_grid(ph, [0, 0, 0], [1, 1, 1], 8, 0, 2000)
    act, _ = O.active_leaves(g)
    cnt = (g["leaf_end"].astype(np.int64) - g["leaf_begin"])[act]
    pick = act[np.argsort(cnt)[np.linspace(0, act.size - 1, 6).astype(np.int64)]]
    x = O.assemble_inputs(O.hist_for_active(O.splat(ph, g, 100_000, 64, 64), pick))
    net = O.parse_net(synth.net_blob(synth.ARCH_UNET4, (32, 64, 128, 256), 1234))
    ref = O.normalise(O.cnn_forward(x, net))[0].reshape(len(pick), -1)

    def kl(P):
        out = [float(np.sum(p[p > 0] * np.log(p[p > 0] / np.maximum(q[p > 0], 1e-300)))) for p, q in zip(ref, P)]
        return float(np.mean(out))

    every, inner = set(range(14)), set(range(3, 12))
    got = {
        "bf16": kl(_unet_P(x, net, _bf16, _bf16, every)),
        "e4m3 per tensor": kl(_unet_P(x, net, _q_tensor, _q_tensor, every)),
        "e4m3 weights per output channel, activations per input channel":
            kl(_unet_P(x, net, _q_in_channel, _q_out_channel, every)),
        "e4m3 per channel, layers 3-11 only": kl(_unet_P(x, net, _q_in_channel, _q_out_channel, inner)),
    }
    print(got)
    assert got["bf16"] < 1e-3 / 5
    for k, v in got.items():
        if k != "bf16":
            assert v > 2e-3, (k, v)
