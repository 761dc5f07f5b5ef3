"""The paper-style reconstruction network (Sec. 5.1 as read here: partial
convolutions with mask updates, ELU, residual links, a dilated bottleneck,
at most 64 channels) through the C ABI against the FP64 oracle, on real
histograms with empty bins.

Gate: the FP32 U-Net gate of tests/test_gpu_parity.py (per bin 1e-5 P +
1e-7 max P, per leaf L1 1e-5) widened to 3e-5 P + 1e-6 max P and L1 3e-5.
The accumulation error per layer is the same (blocked FP32 sums over
K <= 9 x 128 terms); partial-convolution rescaling by up to 9 scales value
and error alike; but each of the six residual sums can cancel (ELU's
negative branch against a positive residual), which magnifies the relative
error of that sum by |a| + |b| over |a + b|, and the head's softplus turns
an absolute pre-activation error e into a relative output error of about
e in its exponential tail, so bins far below the leaf's maximum get the
absolute floor.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import oracle as O  # noqa: E402
from paper_2010_01775_gb300 import pg, synth  # noqa: E402

pytestmark = pytest.mark.gpu

LO = [0.0, 0.0, 0.0]
HI = [1.0, 1.0, 1.0]


@pytest.fixture(scope="module")
def ctx():
    import __graft_entry__
    __graft_entry__.build()
    torch.cuda.set_device(0)
    c = pg.Context()
    yield c
    c.destroy()


def _case(ctx, n, H, W, widths, seed, check=12):
    ph = synth.photons(n, 8, seed)
    d = torch.from_numpy(ph).cuda()
    g = pg.pg_build_grid(ctx, d, n, LO, HI, 4, 0, 800)
    h = pg.pg_splat_photons(ctx, g, d, n, n // 2, H, W)
    blob = synth.net_blob(synth.ARCH_PAPER, widths, seed + 1)
    net = pg.pg_net_load(ctx, blob)
    y = pg.export_map(pg.pg_reconstruct(ctx, h, net, pg.PG_FP32)).astype(np.float64)
    ref = O.build_grid(ph, LO, HI, 4, 0, 800)
    act, _ = O.active_leaves(ref)
    hr = O.hist_for_active(O.splat(ph, ref, n // 2, H, W), act)
    idx = np.linspace(0, act.size - 1, min(check, act.size)).astype(np.int64)
    hsub = {k: (v[idx] if isinstance(v, np.ndarray) else v) for k, v in hr.items()}
    x = O.assemble_inputs(hsub)
    yr = O.cnn_forward(x, O.parse_net(blob))
    return y[idx], yr, x


@pytest.mark.parametrize("n,H,W,widths,seed", [(60_000, 32, 32, (32, 64), 81), (40_000, 64, 64, (32, 64), 82),
                                               (30_000, 16, 32, (16, 32), 83)])
def test_paper_net_fp32(ctx, n, H, W, widths, seed):
    y, yr, x = _case(ctx, n, H, W, widths, seed)
    # The inputs have empty bins, so the masks matter.
    assert (x[..., 4] == 0).mean() > 0.2
    P, Pr = y.reshape(len(y), -1), yr.reshape(len(yr), -1)
    P, Pr = P / P.sum(axis=1, keepdims=True), Pr / Pr.sum(axis=1, keepdims=True)
    for a in range(P.shape[0]):
        tol = 3e-5 * Pr[a] + 1e-6 * Pr[a].max()
        assert np.all(np.abs(P[a] - Pr[a]) <= tol), (a, np.max(np.abs(P[a] - Pr[a]) - tol))
        assert np.abs(P[a] - Pr[a]).sum() <= 3e-5
    big = yr > 1e-3 * yr.max(axis=(1, 2), keepdims=True)
    assert np.max(np.abs(y[big] - yr[big]) / yr[big]) <= 3e-4


def test_paper_net_rejects_small_maps_and_fp8(ctx):
    ph = synth.photons(5000, 2, 84)
    d = torch.from_numpy(ph).cuda()
    g = pg.pg_build_grid(ctx, d, 5000, LO, HI, 3, 0, 500)
    h = pg.pg_splat_photons(ctx, g, d, 5000, 2500, 4, 8)
    net = pg.pg_net_load(ctx, synth.net_blob(synth.ARCH_PAPER, (16, 32), 85))
    with pytest.raises(pg.PgError) as e:
        pg.pg_reconstruct(ctx, h, net, pg.PG_FP32)
    assert e.value.status == 9


def _kl(P, Pr):
    out = []
    for a in range(P.shape[0]):
        p, q = Pr[a].ravel(), np.maximum(P[a].ravel(), 1e-30)
        nz = p > 0
        out.append(float(np.sum(p[nz] * np.log(p[nz] / q[nz]))))
    return np.array(out)


@pytest.mark.parametrize("n,H,W,widths,seed", [(60_000, 32, 32, (32, 64), 91), (40_000, 64, 64, (32, 64), 92)])
def test_paper_net_bf16_kl(ctx, n, H, W, widths, seed):
    """The tensor-core BF16 form within the reduced-precision gate (KL <= 1e-3)."""
    ph = synth.photons(n, 8, seed)
    d = torch.from_numpy(ph).cuda()
    g = pg.pg_build_grid(ctx, d, n, LO, HI, 4, 0, 800)
    h = pg.pg_splat_photons(ctx, g, d, n, n // 2, H, W)
    blob = synth.net_blob(synth.ARCH_PAPER, widths, seed + 1)
    net = pg.pg_net_load(ctx, blob)
    P = pg.export_tables(pg.pg_build_cdf(ctx, pg.pg_reconstruct(ctx, h, net, pg.PG_BF16)))["P"]
    P32 = pg.export_tables(pg.pg_build_cdf(ctx, pg.pg_reconstruct(ctx, h, net, pg.PG_FP32)))["P"]
    ref = O.build_grid(ph, LO, HI, 4, 0, 800)
    act, _ = O.active_leaves(ref)
    hr = O.hist_for_active(O.splat(ph, ref, n // 2, H, W), act)
    idx = np.linspace(0, act.size - 1, min(8, act.size)).astype(np.int64)
    hsub = {k: (v[idx] if isinstance(v, np.ndarray) else v) for k, v in hr.items()}
    Pr, _ = O.normalise(O.cnn_forward(O.assemble_inputs(hsub), O.parse_net(blob)))
    kl = _kl(P[idx].astype(np.float64), Pr)
    assert kl.mean() <= 1e-3, kl
    # Every leaf: BF16 against the FP32 form of the same kernels.
    kl_all = _kl(P.astype(np.float64), P32.astype(np.float64))
    assert np.median(kl_all) <= 1e-3 and np.isfinite(kl_all).all()
    # Autotuned launch shapes (other operand modes sum K in another order, so
    # BF16 activations may round differently) stay within the same gate.
    pg.pg_autotune(ctx, h, net, pg.PG_BF16)
    Pt = pg.export_tables(pg.pg_build_cdf(ctx, pg.pg_reconstruct(ctx, h, net, pg.PG_BF16)))["P"]
    kl_t = _kl(Pt.astype(np.float64), P32.astype(np.float64))
    assert np.median(kl_t) <= 1e-3 and _kl(Pt[idx].astype(np.float64), Pr).mean() <= 1e-3
