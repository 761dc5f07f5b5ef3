"""The seeded input generators follow the stated recipe (blobs on the walls
of the room, vMF directions, lognormal power, uniform queries, He-normal
weights).  Every parity test and the bench draw their inputs here, so the
recipe is pinned by closed forms and exact properties, not by re-running the
generator."""
import math

import numpy as np
import pytest

from paper_2010_01775_gb300 import synth

stats = pytest.importorskip("scipy.stats")


@pytest.fixture(scope="module")
def ph():
    return synth.photons(200_000, 24, 901)


def test_photons_are_deterministic_records(ph):
    assert ph.shape == (200_000, 8) and ph.dtype == np.float32
    assert np.array_equal(ph, synth.photons(200_000, 24, 901))
    assert not np.array_equal(ph, synth.photons(200_000, 24, 902))
    assert np.all(ph[:, 7] == 0.0)
    assert synth.photons(0, 4, 1).shape == (0, 8)


def test_photons_lie_on_the_walls(ph):
    """One coordinate is exactly a wall of [0.02, 0.98]^3, the others in [0, 1)."""
    P = ph[:, :3]
    on = (P == np.float32(synth.ROOM_LO)) | (P == np.float32(synth.ROOM_HI))
    assert np.all(on.sum(axis=1) >= 1)
    assert np.all((P >= 0.0) & (P < 1.0))
    n = synth.wall_normals(ph)
    assert np.all(np.abs(np.linalg.norm(n, axis=1) - 1.0) == 0.0)
    # Normals face into the room: towards the centre from the wall.
    assert np.all(np.sum(n * (0.5 - P), axis=1) > 0.0)
    # All six walls are used by 24 blobs (blob b sits on wall b mod 6).
    walls = set()
    for a in range(3):
        walls |= {2 * a} if np.any(P[:, a] == np.float32(synth.ROOM_LO)) else set()
        walls |= {2 * a + 1} if np.any(P[:, a] == np.float32(synth.ROOM_HI)) else set()
    assert walls == set(range(6))


def test_photon_directions_and_power(ph):
    d = ph[:, 3:6].astype(np.float64)
    assert np.max(np.abs(np.linalg.norm(d, axis=1) - 1.0)) < 1e-6
    p = ph[:, 6].astype(np.float64)
    assert np.all(p > 0.0)
    lp = np.log(p)
    n = lp.size
    # lognormal(0, 1): mean 0, variance 1 of log power (5 sigma).
    assert abs(lp.mean()) < 5.0 / math.sqrt(n)
    assert abs(lp.var() - 1.0) < 5.0 * math.sqrt(2.0 / n)
    # Photons are interleaved: the first half is a random subset, so its
    # share of each wall matches the whole set's.
    half = ph[: n // 2, :3]
    for a in range(3):
        f_all = np.mean(ph[:, a] == np.float32(synth.ROOM_LO))
        f_half = np.mean(half[:, a] == np.float32(synth.ROOM_LO))
        assert abs(f_all - f_half) < 5.0 * math.sqrt(f_all * (1 - f_all) / (n // 2)) + 1e-12


@pytest.mark.parametrize("kappa", [5.0, 30.0, 200.0])
def test_vmf_cosine_follows_its_closed_form(kappa):
    """w = mu . d has density kappa e^{kappa w} / (2 sinh kappa) on [-1, 1]:
    its CDF (e^{kappa w} - e^{-kappa}) / (e^kappa - e^{-kappa}) maps the
    samples to U(0, 1), and E[w] = coth(kappa) - 1/kappa.  The azimuth
    around mu is uniform."""
    rng = np.random.Generator(np.random.PCG64(77))
    m = 100_000
    mu = synth._unit(rng.standard_normal(3))
    d = synth._vmf(rng, np.tile(mu, (m, 1)), np.full(m, kappa))
    assert np.max(np.abs(np.linalg.norm(d, axis=1) - 1.0)) < 1e-12
    w = np.clip(d @ mu, -1.0, 1.0)
    F = (np.exp(kappa * (w - 1.0)) - np.exp(-2.0 * kappa)) / (1.0 - np.exp(-2.0 * kappa))
    assert stats.kstest(F, "uniform").pvalue > 1e-4
    mean = 1.0 / math.tanh(kappa) - 1.0 / kappa
    sd = math.sqrt(max(1e-30, np.var(w)) / m)
    assert abs(w.mean() - mean) < 5.0 * sd
    t1, t2 = synth._frame(mu[None, :])
    c1, c2 = d @ t1[0], d @ t2[0]
    r = np.sqrt(np.maximum(1e-300, c1 * c1 + c2 * c2))
    assert abs(np.mean(c1 / r)) < 5.0 / math.sqrt(2 * m) and abs(np.mean(c2 / r)) < 5.0 / math.sqrt(2 * m)


def test_queries_are_uniform():
    q = 200_000
    pos = synth.query_positions(q, 5)
    assert pos.dtype == np.float32 and np.all((pos >= 0.0) & (pos < 1.0))
    # U(0, 1): mean 1/2, variance 1/12 per axis (5 sigma).
    assert np.all(np.abs(pos.mean(axis=0) - 0.5) < 5.0 * math.sqrt(1.0 / 12.0 / q))
    d = synth.query_directions(q, 5).astype(np.float64)
    assert np.max(np.abs(np.linalg.norm(d, axis=1) - 1.0)) < 1e-6
    # Uniform on S^2: each coordinate is U(-1, 1), so mean 0 and E[x^2] = 1/3.
    assert np.all(np.abs(d.mean(axis=0)) < 5.0 * math.sqrt(1.0 / 3.0 / q))
    assert stats.kstest((d[:, 2] + 1.0) / 2.0, "uniform").pvalue > 1e-4
    phi = np.mod(np.arctan2(d[:, 1], d[:, 0]), 2.0 * np.pi) / (2.0 * np.pi)
    assert stats.kstest(phi, "uniform").pvalue > 1e-4


def test_net_blob_layout_and_he_scale():
    """Header, per-layer records and He-normal weights N(0, 2 / fan_in); the
    U-Net 32-64-128-256 has 1,947,457 parameters."""
    import struct
    layers = synth.net_layers(synth.ARCH_UNET4, (32, 64, 128, 256))
    params = sum(co * ci * k * k + co for co, ci, k, _, _ in layers)
    assert params == 1_947_457
    blob = synth.net_blob(synth.ARCH_UNET4, (32, 64, 128, 256), 3)
    hdr = struct.unpack_from("<IIII4IQ", blob, 0)
    assert hdr[0] == synth.NET_MAGIC and hdr[1] == synth.ARCH_UNET4 and hdr[2] == synth.IN_CHANNELS
    assert hdr[3] == len(layers) and hdr[4:8] == (32, 64, 128, 256) and hdr[8] == 3
    off = struct.calcsize("<IIII4IQ")
    for co, ci, k, s, act in layers:
        rec = struct.unpack_from("<6I", blob, off)
        assert rec[:5] == (co, ci, k, s, act) and rec[5] == 0
        off += 24
        w = np.frombuffer(blob, np.float32, co * k * k * ci, off).astype(np.float64)
        off += 4 * w.size
        b = np.frombuffer(blob, np.float32, co, off)
        off += 4 * co
        if w.size >= 20_000:
            var = 2.0 / (k * k * ci)
            assert abs(w.var() / var - 1.0) < 5.0 * math.sqrt(2.0 / w.size)
        assert np.all(np.abs(b) < 0.1)
    assert off == len(blob)
    # The paper-style net marks its dilated bottleneck layers.
    pb = synth.net_blob(synth.ARCH_PAPER, (32, 64), 3)
    off = struct.calcsize("<IIII4IQ")
    dil = []
    for co, ci, k, s, act in synth.net_layers(synth.ARCH_PAPER, (32, 64)):
        dil.append(struct.unpack_from("<6I", pb, off)[5])
        off += 24 + 4 * (co * k * k * ci + co)
    assert dil == [d if d > 1 else 0 for d in synth.net_dilations(synth.ARCH_PAPER)] and off == len(pb)
