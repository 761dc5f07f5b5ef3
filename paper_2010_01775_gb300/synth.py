"""Seeded synthetic inputs for the guiding hot path.

This module holds none of the method's arithmetic: it only draws photon
records, query positions/directions and network weights from seeded NumPy
generators (PCG64).  Both the CUDA path and the CPU oracle consume what it
returns, so it is the one module the two sides share.

The paper's workloads are photons traced through rendered scenes (Sec. 7,
Sec. 8 "training data"), which are not available here.  The stand-in follows
the photon statistics of an indoor scene: photons land on the six walls of a
room, clustered in blobs (lit patches), arrive from a few dominant directions
(von Mises-Fisher lobes around the wall normal; light sources and caustics)
and carry lognormal power.
"""
from __future__ import annotations

import dataclasses
import struct

import numpy as np

ROOM_LO = 0.02
ROOM_HI = 0.98

# Network architectures understood by the weight blob (both sides parse it).
ARCH_TINY3 = 0
ARCH_UNET4 = 1
ARCH_PAPER = 2  # compact masked U-Net with residual links and a dilated bottleneck
ACT_NONE, ACT_ELU, ACT_SOFTPLUS = 0, 1, 2
NET_MAGIC = 0x314E4750  # "PGN1"
IN_CHANNELS = 5


@dataclasses.dataclass(frozen=True)
class Workload:
    """One synthetic workload: photon set, grid, histogram size, net, queries."""

    name: str
    n_photons: int
    n_blobs: int
    max_depth: int
    split_threshold: int
    H: int
    W: int
    arch: int
    widths: tuple
    n_queries: int
    seed: int
    min_depth: int = 0
    frac_bits: int = 32

    @property
    def n_prev(self) -> int:
        # Photon counts double per iteration, so the photons accumulated up to
        # the previous iteration are about half of the current total.
        return self.n_photons // 2


SEED_BASE = 20101775

# Photon-count bounds of the paper's five expert networks (Sec. 8).
EXPERT_BOUNDS = (100, 500, 1000, 5000)

TINY = Workload("tiny: 100k photons, 8 blobs, depth 4, split 1000, 32x32, 3-layer 16-ch CNN, 64k queries",
                100_000, 8, 4, 1000, 32, 32, ARCH_TINY3, (16,), 65_536, SEED_BASE + 0)
SCALE = Workload("scale: 4M photons, 64 blobs, depth 10, split 2000, 64x64, U-Net 32-64-128-256, 8M queries",
                 4_194_304, 64, 10, 2000, 64, 64, ARCH_UNET4, (32, 64, 128, 256), 8_388_608, SEED_BASE + 1)
PRECISION = dataclasses.replace(
    SCALE, name="precision: 4M photons, 64 blobs, depth 10, split 2000, 128x128, U-Net BF16/FP8, 8M queries",
    H=128, W=128, seed=SEED_BASE + 2)

# A reduced copy of the scale workload for profiler captures (same kernels,
# a few GB on the device).
SCALE_SMALL = dataclasses.replace(
    SCALE, name="scale-small: 262k photons, 16 blobs, depth 10, split 2000, 64x64, U-Net, 512k queries",
    n_photons=262_144, n_blobs=16, n_queries=524_288, seed=SEED_BASE + 11)

# A mid-size copy for profiler captures of the memory-bound kernels (query
# arrays and histograms larger than L2, a few GB on the device in BF16).
SCALE_MID = dataclasses.replace(
    SCALE, name="scale-mid: 1M photons, 32 blobs, depth 10, split 2000, 64x64, U-Net, 4M queries",
    n_photons=1_048_576, n_blobs=32, n_queries=4_194_304, seed=SEED_BASE + 12)

WORKLOADS = {"tiny": TINY, "scale": SCALE, "precision": PRECISION, "scale-small": SCALE_SMALL,
             "scale-mid": SCALE_MID}


def _unit(v):
    return v / np.linalg.norm(v, axis=-1, keepdims=True)


def _frame(n):
    """Two unit tangents orthogonal to each row of n (rows unit length)."""
    a = np.where(np.abs(n[:, :1]) < 0.9, np.array([[1.0, 0, 0]]), np.array([[0, 1.0, 0]]))
    t1 = _unit(np.cross(n, a))
    t2 = np.cross(n, t1)
    return t1, t2


def _vmf(rng, mu, kappa):
    """Directions from vMF(mu, kappa) on S^2, rows of mu unit.

    Stable inversion of the vMF cosine (W. Jakob, "Numerically stable sampling
    of the von Mises-Fisher distribution on S^2", 2012):
    w = 1 + log(xi + (1 - xi) exp(-2 kappa)) / kappa.
    """
    m = mu.shape[0]
    xi = rng.random(m)
    w = 1.0 + np.log(xi + (1.0 - xi) * np.exp(-2.0 * kappa)) / kappa
    w = np.clip(w, -1.0, 1.0)
    v = rng.random(m) * 2.0 * np.pi
    t1, t2 = _frame(mu)
    r = np.sqrt(np.maximum(0.0, 1.0 - w * w))[:, None]
    return w[:, None] * mu + r * (np.cos(v)[:, None] * t1 + np.sin(v)[:, None] * t2)


def uniform_sphere(rng, m):
    z = rng.random(m) * 2.0 - 1.0
    phi = rng.random(m) * 2.0 * np.pi
    r = np.sqrt(np.maximum(0.0, 1.0 - z * z))
    return np.stack([r * np.cos(phi), r * np.sin(phi), z], axis=1)


def photons(n: int, n_blobs: int, seed: int) -> np.ndarray:
    """(n, 8) float32 photon records {px,py,pz, dx,dy,dz, power, 0}.

    Blob b sits on wall b mod 6 of the room [0.02, 0.98]^3; its centre is
    uniform in [0.1, 0.9]^2 in-plane, its in-plane sigma U[0.02, 0.1]; points
    are redrawn until they fall inside [0, 1).  Blob weights are
    lognormal(0, 0.5), photon counts multinomial.  Each blob has 3 vMF lobes
    (Dirichlet(1,1,1) weights, mean uniform on the hemisphere around the wall
    normal, kappa log-uniform in [5, 200]); directions may point below the
    wall (the map covers the full sphere).  Power is lognormal(0, 1).
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    out = np.zeros((n, 8), dtype=np.float32)
    if n == 0:
        return out
    wts = rng.lognormal(0.0, 0.5, n_blobs)
    counts = rng.multinomial(n, wts / wts.sum())
    start = 0
    for b in range(n_blobs):
        m = int(counts[b])
        plane = b % 6
        axis = plane // 2
        level = ROOM_LO if plane % 2 == 0 else ROOM_HI
        normal = np.zeros(3)
        normal[axis] = 1.0 if plane % 2 == 0 else -1.0
        centre = rng.uniform(0.1, 0.9, 2)
        sigma = rng.uniform(0.02, 0.1)
        lobe_w = rng.dirichlet([1.0, 1.0, 1.0])
        lobe_mu = []
        for _ in range(3):
            d = uniform_sphere(rng, 1)[0]
            if d @ normal < 0:
                d = -d
            lobe_mu.append(d)
        lobe_mu = np.array(lobe_mu)
        lobe_k = np.exp(rng.uniform(np.log(5.0), np.log(200.0), 3))
        if m == 0:
            continue
        uv = centre + sigma * rng.standard_normal((m, 2))
        bad = np.any((uv < 0.0) | (uv >= 1.0), axis=1)
        while bad.any():
            uv[bad] = centre + sigma * rng.standard_normal((int(bad.sum()), 2))
            bad = np.any((uv < 0.0) | (uv >= 1.0), axis=1)
        pos = np.empty((m, 3))
        others = [a for a in range(3) if a != axis]
        pos[:, axis] = level
        pos[:, others[0]] = uv[:, 0]
        pos[:, others[1]] = uv[:, 1]
        lobe = rng.choice(3, size=m, p=lobe_w)
        dirs = _vmf(rng, lobe_mu[lobe], lobe_k[lobe])
        dirs = _unit(dirs)
        power = rng.lognormal(0.0, 1.0, m)
        out[start:start + m, 0:3] = pos
        out[start:start + m, 3:6] = dirs
        out[start:start + m, 6] = power
        start += m
    # Photons of one blob would otherwise be contiguous; a tracer emits them
    # interleaved, which is what makes "index < n_prev" a random subset.
    perm = rng.permutation(n)
    return np.ascontiguousarray(out[perm])


def query_positions(q: int, seed: int) -> np.ndarray:
    """(q, 3) float32 path-vertex positions, uniform in [0, 1)^3."""
    rng = np.random.Generator(np.random.PCG64(seed ^ 0x5EED))
    return rng.random((q, 3), dtype=np.float32)


def query_directions(q: int, seed: int) -> np.ndarray:
    """(q, 3) float32 unit directions, uniform on the sphere (stand-in for
    BSDF-sampled directions whose guide pdf a renderer needs for MIS)."""
    rng = np.random.Generator(np.random.PCG64(seed ^ 0xD1EC))
    return np.ascontiguousarray(_unit(uniform_sphere(rng, q)).astype(np.float32))


def wall_normals(ph: np.ndarray) -> np.ndarray:
    """(n, 3) float32 unit normals of the walls the photons of `photons()`
    lie on (a photon on the wall at ROOM_LO of axis a faces +e_a, at ROOM_HI
    -e_a): the surface normals at the photon hit points."""
    n = np.zeros((ph.shape[0], 3), np.float32)
    for a in range(3):
        n[ph[:, a] == np.float32(ROOM_LO), a] = 1.0
        n[ph[:, a] == np.float32(ROOM_HI), a] = -1.0
    return n


def vertex_records(q: int, seed: int):
    """Path-vertex records for one-sample MIS: (q, 3) float32 unit normals
    (uniform on the sphere) and (q,) float32 bounce contributions (lognormal,
    sigma 1), the values a renderer would report for each sampled bounce."""
    rng = np.random.Generator(np.random.PCG64(seed ^ 0x3A15))
    n = np.ascontiguousarray(_unit(uniform_sphere(rng, q)).astype(np.float32))
    c = np.ascontiguousarray(rng.lognormal(0.0, 1.0, q).astype(np.float32))
    return n, c


def net_dilations(arch: int) -> list:
    """Tap spacing of every layer (1 except the paper-style bottleneck)."""
    if arch == ARCH_PAPER:
        return [1, 1, 1, 1, 1, 2, 4, 1, 1, 1, 1, 1]
    return [1] * len(net_layers(arch, (1, 1, 1, 1)))


def net_layers(arch: int, widths) -> list:
    """Layer descriptors (cout, cin, k, stride, act) in blob order."""
    if arch == ARCH_TINY3:
        c = widths[0]
        return [(c, IN_CHANNELS, 3, 1, ACT_ELU), (c, c, 3, 1, ACT_ELU), (1, c, 3, 1, ACT_SOFTPLUS)]
    if arch == ARCH_UNET4:
        c0, c1, c2, c3 = widths
        return [
            (c0, IN_CHANNELS, 3, 1, ACT_ELU), (c0, c0, 3, 1, ACT_ELU),
            (c1, c0, 3, 2, ACT_ELU), (c1, c1, 3, 1, ACT_ELU),
            (c2, c1, 3, 2, ACT_ELU), (c2, c2, 3, 1, ACT_ELU),
            (c3, c2, 3, 2, ACT_ELU), (c3, c3, 3, 1, ACT_ELU),
            (c2, c3 + c2, 3, 1, ACT_ELU), (c2, c2, 3, 1, ACT_ELU),
            (c1, c2 + c1, 3, 1, ACT_ELU), (c1, c1, 3, 1, ACT_ELU),
            (c0, c1 + c0, 3, 1, ACT_ELU), (c0, c0, 3, 1, ACT_ELU),
            (1, c0, 1, 1, ACT_SOFTPLUS),
        ]
    if arch == ARCH_PAPER:
        c0, c1 = widths[0], widths[1]
        return [
            (c0, IN_CHANNELS, 3, 1, ACT_ELU), (c0, c0, 3, 1, ACT_ELU),      # level 0 (+ residual)
            (c1, c0, 3, 2, ACT_ELU), (c1, c1, 3, 1, ACT_ELU),               # level 1 (+ residual)
            (c1, c1, 3, 2, ACT_ELU), (c1, c1, 3, 1, ACT_ELU), (c1, c1, 3, 1, ACT_ELU),  # dilated bottleneck
            (c1, 2 * c1, 3, 1, ACT_ELU), (c1, c1, 3, 1, ACT_ELU),           # decoder level 1
            (c0, c1 + c0, 3, 1, ACT_ELU), (c0, c0, 3, 1, ACT_ELU),          # decoder level 0
            (1, c0, 1, 1, ACT_SOFTPLUS),
        ]
    raise ValueError(f"unknown arch {arch}")


def net_blob(arch: int, widths, seed: int) -> bytes:
    """Seeded He-normal weights (N(0, 2/fan_in)), biases N(0, 0.01^2), float32.

    Blob layout (little endian): u32 magic, u32 arch, u32 in_channels,
    u32 n_layers, u32 widths[4], u64 seed; then per layer u32
    {cout, cin, k, stride, act, dilation (0 = 1)} followed by float32
    weights in [cout][k][k][cin] order and float32 bias[cout].
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    layers = net_layers(arch, widths)
    dil = net_dilations(arch)
    w4 = list(widths) + [0] * (4 - len(widths))
    parts = [struct.pack("<IIII4IQ", NET_MAGIC, arch, IN_CHANNELS, len(layers), *w4, seed)]
    for (cout, cin, k, stride, act), d in zip(layers, dil):
        fan_in = k * k * cin
        w = (rng.standard_normal((cout, k, k, cin)) * np.sqrt(2.0 / fan_in)).astype(np.float32)
        b = (rng.standard_normal(cout) * 0.01).astype(np.float32)
        parts.append(struct.pack("<6I", cout, cin, k, stride, act, d if d > 1 else 0))
        parts.append(w.tobytes())
        parts.append(b.tobytes())
    return b"".join(parts)


def workload_inputs(wl: Workload):
    """Photons, query positions, eval directions and weight blob of a workload."""
    ph = photons(wl.n_photons, wl.n_blobs, wl.seed)
    pos = query_positions(wl.n_queries, wl.seed)
    dirs = query_directions(wl.n_queries, wl.seed)
    blob = net_blob(wl.arch, wl.widths, wl.seed + 77)
    return ph, pos, dirs, blob


@dataclasses.dataclass(frozen=True)
class BatchWorkload:
    """Many independent scenes of uneven size processed as one batch."""

    name: str
    n_scenes: int
    n_median: float
    n_sigma: float
    n_min: int
    n_max: int
    max_depth: int
    split_threshold: int
    H: int
    W: int
    arch: int
    widths: tuple
    n_queries: int
    seed: int
    min_depth: int = 0
    frac_bits: int = 32


BATCH64 = BatchWorkload(
    "batch64: 64 scenes, photons per scene lognormal(ln 4e5, 1.5) clipped to [2e4, 8e6], depth 10, split 1000, "
    "64x64, BF16 U-Net 32-64-128-256, 32M queries split by photon count",
    64, 4e5, 1.5, 20_000, 8_000_000, 10, 1000, 64, 64, ARCH_UNET4, (32, 64, 128, 256), 33_554_432, SEED_BASE + 3)
BATCH8 = dataclasses.replace(
    BATCH64, name="batch8: 8 scenes, photons per scene lognormal(ln 1e5, 1.0) clipped to [2e4, 1e6], 2M queries",
    n_scenes=8, n_median=1e5, n_sigma=1.0, n_max=1_000_000, n_queries=2_097_152, seed=SEED_BASE + 13)

BATCH_WORKLOADS = {"batch64": BATCH64, "batch8": BATCH8}


def batch_inputs(bw: BatchWorkload):
    """Scene-grouped photons with offsets, scene-grouped query positions and
    directions with offsets (queries split in proportion to photon counts),
    and the network blob.  Every scene lives in [0, 1)^3."""
    rng = np.random.Generator(np.random.PCG64(bw.seed))
    sizes = np.clip(np.exp(rng.normal(np.log(bw.n_median), bw.n_sigma, bw.n_scenes)), bw.n_min, bw.n_max)
    sizes = sizes.astype(np.int64)
    phs = []
    for s, n in enumerate(sizes):
        blobs = int(np.clip(n // 62_500, 8, 64))
        phs.append(photons(int(n), blobs, bw.seed * 1000 + s))
    begin = np.concatenate([[0], np.cumsum(sizes)]).astype(np.uint32)
    q = np.floor(bw.n_queries * sizes / sizes.sum()).astype(np.int64)
    q[0] += bw.n_queries - q.sum()
    qbegin = np.concatenate([[0], np.cumsum(q)]).astype(np.uint32)
    pos = query_positions(bw.n_queries, bw.seed)
    dirs = query_directions(bw.n_queries, bw.seed)
    blob = net_blob(bw.arch, bw.widths, bw.seed + 77)
    return np.ascontiguousarray(np.concatenate(phs)), begin, pos, dirs, qbegin, blob


@dataclasses.dataclass(frozen=True)
class ServeTrace:
    """A seeded open-loop request trace for the serving loop."""

    name: str
    rate: float  # Poisson arrivals per second
    duration: float  # seconds of arrivals
    n_min: int
    n_max: int
    q_min: int
    q_max: int
    sizes: tuple  # H = W choices
    precisions: tuple  # cycled over requests
    max_depth: int
    split_threshold: int
    seed: int


SERVE = ServeTrace(
    "serve: Poisson 200 req/s, photons log-uniform [1e4, 2e7], queries log-uniform [65536, 16777216], "
    "H=W in {32, 64, 128}, split 2000, depth 10, BF16/FP8 alternating, U-Net 32-64-128-256",
    200.0, 2.0, 10_000, 20_000_000, 65_536, 16_777_216, (32, 64, 128), ("bf16", "fp8"), 10, 2000, SEED_BASE + 4)
SERVE_SMALL = dataclasses.replace(
    SERVE, name="serve-small: Poisson 200 req/s, photons log-uniform [1e3, 1e5], queries log-uniform [1e3, 1e5], "
    "H=W in {16, 32}", n_min=1_000, n_max=100_000, q_min=1_000, q_max=100_000, sizes=(16, 32), duration=0.2,
    seed=SEED_BASE + 14)

SERVE_TRACES = {"serve": SERVE, "serve-small": SERVE_SMALL}


def serve_trace(tr: ServeTrace, rate: float | None = None, duration: float | None = None,
                n_requests: int | None = None):
    """Request descriptors: dicts with arrival (seconds from start), n, q,
    H, W, precision, stream_id, q_offset (offset into a shared query pool of
    q_max entries; a request's photons are the first n of a shared pool).
    Exactly n_requests requests when given, else every arrival before
    `duration`."""
    rate = tr.rate if rate is None else rate
    duration = tr.duration if duration is None else duration
    rng = np.random.Generator(np.random.PCG64(tr.seed))
    out, t = [], 0.0
    while True:
        t += rng.exponential(1.0 / rate)
        if (n_requests is None and t >= duration) or (n_requests is not None and len(out) >= n_requests):
            break
        n = int(np.exp(rng.uniform(np.log(tr.n_min), np.log(tr.n_max))))
        q = int(np.exp(rng.uniform(np.log(tr.q_min), np.log(tr.q_max))))
        s = int(tr.sizes[rng.integers(len(tr.sizes))])
        out.append(dict(arrival=t, n=n, q=q, H=s, W=s, precision=tr.precisions[len(out) % len(tr.precisions)],
                        stream_id=len(out), q_offset=int(rng.integers(0, tr.q_max - q + 1))))
    return out
