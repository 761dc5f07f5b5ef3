"""Plain FP64 CPU oracle of the guiding-distribution hot path (test infrastructure).

TEST INFRASTRUCTURE ONLY: only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / reference leg of ``bench.py`` may import this module.  It
shares no code with the CUDA library (``paper_2010_01775_gb300``) and imports
nothing from it; the two meet only through the seeded inputs of
``paper_2010_01775_gb300.synth``.

The integer-heavy steps (voxel location, grid, binning, splat, convolution
loops, Philox, sampling) are plain C in ``pg_oracle.c``; this module loads it
with ctypes and writes the remaining steps (activations, U-Net wiring,
normalisation, CDFs) as direct NumPy FP64 expressions.  Each function cites the
passage of the paper it follows.

Parity status: every function here is pinned by ``tests/test_oracle_pins.py``
(closed forms, brute force, library routines, invariants) except the CNN
*weights and architecture*, which the paper does not print: the network
definition is this project's reading (architecture in ``net_layers``), so CNN
outputs are pinned only as convolution/activation arithmetic (against
``torch.nn.functional.conv2d`` in float64 and closed-form special cases), not
against any number from the paper.
"""
from __future__ import annotations

import ctypes
import math
import os
import struct
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "pg_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")

ERR_OVERFLOW = 4
ERR_INVALID_INPUT = 8

ARCH_TINY3 = 0
ARCH_UNET4 = 1
ARCH_PAPER = 2
ACT_NONE, ACT_ELU, ACT_SOFTPLUS = 0, 1, 2
NET_MAGIC = 0x314E4750


def build(force: bool = False) -> str:
    """Compile pg_oracle.c with gcc (IEEE, no FMA contraction, no fast math;
    OpenMP for the per-output loops, which does not change any result)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-D_GNU_SOURCE", "-fPIC", "-shared", "-fopenmp",
                               "-ffp-contract=off", "-fno-fast-math", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(build())
        L = _lib
        P = ctypes.c_void_p
        i64, i32, u32, u64 = ctypes.c_int64, ctypes.c_int, ctypes.c_uint32, ctypes.c_uint64
        L.or_morton3.restype = u64
        L.or_morton3.argtypes = [u32, u32, u32, i32]
        L.or_morton_codes.argtypes = [P, i64, i64, P, P, i32, P]
        L.or_build_grid.restype = i64
        L.or_build_grid.argtypes = [P, i64, P, P, i32, i32, u32, P, P, P, i64, P, P, P, P]
        L.or_phi_table.argtypes = [i32, P, P]
        L.or_dir_bins.argtypes = [P, i64, i64, i32, i32, P, P]
        L.or_splat.argtypes = [P, i64, i64, P, i64, P, P, i32, i32, i32, P, P, P, P]
        L.or_assemble_inputs.argtypes = [i64, i64, P, P, P, P, P]
        L.or_conv2d.argtypes = [P, i64, i32, i32, i32, P, P, i32, i32, i32, P]
        L.or_philox4x32_10.argtypes = [P, P, P]
        L.or_sample.argtypes = [P, i64, P, P, i32, P, i64, P, i32, i32, P, P, P, P, u64, u32,
                                P, P, P, P]
        L.or_eval_pdf.argtypes = [P, P, i64, P, P, i32, P, i64, P, i32, i32, P, P, P]
        L.or_conv2d_dilated.argtypes = [P, i64, i32, i32, i32, P, P, i32, i32, i32, i32, P]
        L.or_sample_leaves.argtypes = [P, i64, P, i32, i32, P, P, P, P, u64, u32, P, P, P, P]
        L.or_eval_pdf_leaves.argtypes = [P, P, i64, P, i32, i32, P, P, P]
        L.or_set_threads.restype = i32
        L.or_set_threads.argtypes = [i32]
    return _lib


def set_threads(n: int = 0) -> int:
    """Host threads of the convolution, sampling and evaluation loops (0: all
    cores); returns the count used.  Outputs are identical for every count."""
    return int(lib().or_set_threads(n))


def _p(a: np.ndarray):
    assert a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(ctypes.c_void_p)


def _f32(x):
    return np.ascontiguousarray(np.asarray(x, dtype=np.float32))


# --------------------------------------------------------------------------
# a1-a4: voxel location and the adaptive hierarchical grid (Sec. 7.1,
# Algorithm 1: locating a position's voxel and subdividing voxels).
# --------------------------------------------------------------------------
def morton_codes(pos, lo, hi, D):
    pos = _f32(pos)
    n = pos.shape[0]
    codes = np.zeros(n, np.uint64)
    st = lib().or_morton_codes(_p(pos), pos.shape[1], n, _p(_f32(lo)), _p(_f32(hi)), D, _p(codes))
    return codes, st


def build_grid(photons, lo, hi, D, min_depth, thr):
    """Octree reading of the voxel subdivision rule (split while count > thr and
    depth < D; every child kept).  Returns a dict with per-photon codes, the
    stable sort permutation, leaf_of (per original photon) and the Morton-ordered
    leaf table (start code at full depth, depth, photon range)."""
    ph = _f32(photons)
    n = ph.shape[0]
    codes = np.zeros(n, np.uint64)
    perm = np.zeros(n, np.uint32)
    leaf_of = np.zeros(n, np.uint32)
    cap = max(1024, 8 ** min_depth + 64)
    while True:
        lc = np.zeros(cap, np.uint64)
        ld = np.zeros(cap, np.int32)
        lb = np.zeros(cap, np.uint32)
        le = np.zeros(cap, np.uint32)
        L = lib().or_build_grid(_p(ph), n, _p(_f32(lo)), _p(_f32(hi)), D, min_depth, thr, _p(codes),
                                _p(perm), _p(leaf_of), cap, _p(lc), _p(ld), _p(lb), _p(le))
        if L < 0:
            raise ValueError(f"oracle grid status {-L}")
        if L <= cap:
            break
        cap = int(L)
    return dict(codes=codes, perm=perm, leaf_of=leaf_of, leaf_code=lc[:L].copy(),
                leaf_depth=ld[:L].copy(), leaf_begin=lb[:L].copy(), leaf_end=le[:L].copy(),
                L=int(L), D=D, lo=_f32(lo), hi=_f32(hi), n=n)


def active_leaves(grid):
    """Leaves that received photons get a map (Sec. 7.2: maps are reconstructed
    for voxels that have photons); slot_of_leaf is -1 for the others."""
    cnt = grid["leaf_end"].astype(np.int64) - grid["leaf_begin"].astype(np.int64)
    act = np.nonzero(cnt > 0)[0].astype(np.uint32)
    slot = np.full(grid["L"], -1, np.int32)
    slot[act] = np.arange(act.size, dtype=np.int32)
    return act, slot


# --------------------------------------------------------------------------
# The paper's grid rule (Sec. 7.1 "An initial regular grid" and "Voxel
# subdivision"; Sec. 8: a 100^3 regular grid, local binary trees of depth at
# most 8, V_thr = 0.5): every voxel of a regular R^3 grid holds a binary tree
# whose nodes split at the median photon position along one axis while the
# node has more than M_thr photons or its normal variance exceeds V_thr.
# --------------------------------------------------------------------------
KD_NORMAL_BITS = 20  # normals enter the variance as round_half_even(n * 2^20)


def kd_scale(lo, hi, R):
    """Cells per unit length, fl32(R / (hi - lo)) formed in double."""
    return np.array([np.float32(R / (float(hi[a]) - float(lo[a]))) for a in range(3)], np.float32)


def kd_cells(pos, lo, hi, R):
    """Voxel of each position: per axis q = clamp(floor(fl32(fl32(x - lo) *
    s)), 0, R - 1) (the a1 rule with R cells), cell = qx + R (qy + R qz).
    Returns (cells int64, invalid-input flag)."""
    pos = _f32(pos)
    lo32 = _f32(lo)
    t = (pos - lo32) * kd_scale(lo, hi, R)  # two IEEE FP32 roundings
    bad = ~np.isfinite(pos).all(axis=1)
    q = np.floor(np.where(np.isfinite(t), t, 0.0)).clip(0, R - 1).astype(np.int64)
    q[bad] = 0
    return q[:, 0] + R * (q[:, 1] + R * q[:, 2]), bool(bad.any())


def kd_normal_variance(S, m):
    """V = 1 - |mean normal|^2 from fixed-point sums S (Python ints) of m unit
    normals, in double with this exact operation order."""
    a, b, c = float(S[0]), float(S[1]), float(S[2])
    r = (a * a + b * b) + c * c
    mm = (float(m) * float(m)) * 2.0 ** (2 * KD_NORMAL_BITS)
    return 1.0 - r / mm


def build_kd_grid(photons, normals, lo, hi, R, max_depth, thr, vthr):
    """Regular grid + one binary tree per voxel, built level by level.

    A node of m photons at depth d splits when d < max_depth, m >= 2, its
    photons are not all at one coordinate along the axis of largest spread
    (max - min in FP32, first axis on ties), and m > thr or V > vthr (V = 0
    without normals).  Split value: the floor(m/2)-th smallest coordinate s
    (0-based); the left child holds x < tau with tau = s, or tau = the next
    float above s when no coordinate is below s.  Children keep the photons'
    order (a stable partition).

    Node numbering: nodes 0 .. R^3-1 are the voxels' roots; each level's
    children follow, two per splitting node in the order of their parents.
    Leaves are numbered depth-first (left first) in voxel order, so their
    photon ranges in `perm` ascend.  node_link is the left child's index
    (right = left + 1) for an internal node and ~leaf for a leaf."""
    ph = _f32(photons)
    n = ph.shape[0]
    cells, bad = kd_cells(ph[:, :3], lo, hi, R)
    if bad:
        raise ValueError("non-finite photon position")
    nfx = None
    if normals is not None:
        nfx = np.rint(_f32(normals).astype(np.float64) * 2.0 ** KD_NORMAL_BITS).astype(np.int64)
    perm = np.argsort(cells, kind="stable").astype(np.int64)
    C = R ** 3
    cnt = np.bincount(cells, minlength=C)
    end = np.cumsum(cnt)
    begin = [int(v) for v in end - cnt]
    end = [int(v) for v in end]
    axis = [0] * C
    tau = [0.0] * C
    link = [-1] * C
    depth = [0] * C
    level = list(range(C))
    d = 0
    while level:
        nxt = []
        for v in level:
            b, e = begin[v], end[v]
            m = e - b
            if d >= max_depth or m < 2:
                continue
            idx = perm[b:e]
            P = ph[idx, :3]
            spread = P.max(axis=0) - P.min(axis=0)  # FP32
            a = int(np.argmax(spread))
            if not spread[a] > 0:
                continue
            V = kd_normal_variance(nfx[idx].sum(axis=0).tolist(), m) if nfx is not None else 0.0
            if not (m > thr or V > vthr):
                continue
            x = P[:, a]
            s = np.sort(x)[m // 2]
            t = s if (x < s).any() else np.nextafter(s, np.float32(np.inf))
            left = x < t
            perm[b:e] = np.concatenate([idx[left], idx[~left]])
            nl = int(left.sum())
            child = len(begin)
            axis[v], tau[v], link[v] = a, float(t), child
            begin += [b, b + nl]
            end += [b + nl, e]
            axis += [0, 0]
            tau += [0.0, 0.0]
            link += [-1, -1]
            depth += [d + 1, d + 1]
            nxt += [child, child + 1]
        level = nxt
        d += 1
    # Leaves depth-first, left first, voxel by voxel.
    leaf_cell, leaf_depth, leaf_begin, leaf_end = [], [], [], []
    for c in range(C):
        stack = [c]
        while stack:
            v = stack.pop()
            if link[v] >= 0:
                stack += [link[v] + 1, link[v]]
            else:
                link[v] = ~len(leaf_cell)
                leaf_cell.append(c)
                leaf_depth.append(depth[v])
                leaf_begin.append(begin[v])
                leaf_end.append(end[v])
    L = len(leaf_cell)
    leaf_of = np.zeros(n, np.uint32)
    for l in range(L):
        leaf_of[perm[leaf_begin[l]:leaf_end[l]]] = l
    return dict(kd=True, R=R, lo=_f32(lo), hi=_f32(hi), n=n, cells=cells, perm=perm.astype(np.uint32),
                leaf_of=leaf_of, L=L, leaf_cell=np.array(leaf_cell, np.uint32),
                leaf_depth=np.array(leaf_depth, np.int32), leaf_begin=np.array(leaf_begin, np.uint32),
                leaf_end=np.array(leaf_end, np.uint32), node_axis=np.array(axis, np.uint8),
                node_tau=np.array(tau, np.float32), node_link=np.array(link, np.int32))


def kd_locate(grid, pos):
    """Leaf of each position: its voxel's root, then left when x[axis] < tau."""
    pos = _f32(pos)
    cells, bad = kd_cells(pos, grid["lo"], grid["hi"], grid["R"])
    link, ax, tau = grid["node_link"], grid["node_axis"], grid["node_tau"]
    out = np.zeros(pos.shape[0], np.int64)
    for i in range(pos.shape[0]):
        v = int(cells[i])
        while link[v] >= 0:
            v = int(link[v]) + (0 if pos[i, ax[v]] < tau[v] else 1)
        out[i] = ~int(link[v])
    return out, bad


# --------------------------------------------------------------------------
# Direction bins (Sec. 4, cylindrical map (z, phi)).
# --------------------------------------------------------------------------
def phi_table(W):
    c = np.zeros(W, np.float32)
    s = np.zeros(W, np.float32)
    lib().or_phi_table(W, _p(c), _p(s))
    return c, s


def dir_bins(dirs, H, W):
    d = _f32(dirs)
    n = d.shape[0]
    rows = np.zeros(n, np.int32)
    cols = np.zeros(n, np.int32)
    st = lib().or_dir_bins(_p(d), d.shape[1], n, H, W, _p(rows), _p(cols))
    return rows, cols, st


# --------------------------------------------------------------------------
# a5: photon energy and count maps, Eq. (photon), Sec. 5 input buffers.
# --------------------------------------------------------------------------
def splat(photons, grid, n_prev, H, W, F=32, n_bound=None):
    """n_bound: the photon count of the fixed-point bound (default: this call's)."""
    ph = _f32(photons)
    L, HW = grid["L"], H * W
    pc = np.zeros((L, HW), np.uint64)
    pp = np.zeros((L, HW), np.uint64)
    cc = np.zeros((L, HW), np.uint32)
    cp = np.zeros((L, HW), np.uint32)
    n = ph.shape[0] if n_bound is None else n_bound
    st = lib().or_splat(_p(ph), n, n_prev, _p(grid["perm"]), L, _p(grid["leaf_begin"]),
                        _p(grid["leaf_end"]), H, W, F, _p(pc), _p(cc), _p(pp), _p(cp))
    return dict(pow_cur=pc, cnt_cur=cc, pow_prev=pp, cnt_prev=cp, H=H, W=W, status=st)


def hist_for_active(hist, act):
    return {k: (v[act] if isinstance(v, np.ndarray) else v) for k, v in hist.items()}


# --------------------------------------------------------------------------
# a6-a7: network input and the reconstruction CNN (Sec. 5, Sec. 5.1).
# --------------------------------------------------------------------------
def assemble_inputs(hist):
    """5-channel input [A][H][W][5] (S_t, S_{t-1}, P_t, P_{t-1}, B), FP64."""
    A, HW = hist["pow_cur"].shape
    x = np.zeros((A, HW, 5), np.float64)
    pc = np.ascontiguousarray(hist["pow_cur"])
    pp = np.ascontiguousarray(hist["pow_prev"])
    cc = np.ascontiguousarray(hist["cnt_cur"])
    cp = np.ascontiguousarray(hist["cnt_prev"])
    lib().or_assemble_inputs(A, HW, _p(pc), _p(cc), _p(pp), _p(cp), _p(x))
    return x.reshape(A, hist["H"], hist["W"], 5)


def parse_net(blob: bytes):
    """Layer list [(cout, cin, k, stride, act, w[cout][k][k][cin], b[cout])];
    the per-layer tap spacing (dilation, 1 unless stored) is in "dil"."""
    magic, arch, cin0, nl, w0, w1, w2, w3, seed = struct.unpack_from("<IIII4IQ", blob, 0)
    if magic != NET_MAGIC:
        raise ValueError("bad net blob")
    off = struct.calcsize("<IIII4IQ")
    layers, dil = [], []
    for _ in range(nl):
        cout, cin, k, stride, act, d = struct.unpack_from("<6I", blob, off)
        dil.append(max(1, d))
        off += 24
        w = np.frombuffer(blob, np.float32, cout * k * k * cin, off).reshape(cout, k, k, cin)
        off += 4 * w.size
        b = np.frombuffer(blob, np.float32, cout, off)
        off += 4 * cout
        layers.append((cout, cin, k, stride, act, np.ascontiguousarray(w), np.ascontiguousarray(b)))
    return dict(arch=arch, widths=(w0, w1, w2, w3), layers=layers, dil=dil, seed=seed)


def conv2d(x, w, b, stride, dil=1):
    """One conv layer, 'same' zero padding, channel-last FP64 (plain loops in
    C); dil spreads the taps dil pixels apart (dilated convolution)."""
    x = np.ascontiguousarray(x, np.float64)
    A, Hin, Win, Cin = x.shape
    cout, k, _, cin = w.shape
    assert cin == Cin
    out = np.zeros((A, Hin // stride, Win // stride, cout), np.float64)
    if dil == 1:
        lib().or_conv2d(_p(x), A, Hin, Win, Cin, _p(_f32(w)), _p(_f32(b)), cout, k, stride, _p(out))
    else:
        lib().or_conv2d_dilated(_p(x), A, Hin, Win, Cin, _p(_f32(w)), _p(_f32(b)), cout, k, stride, dil, _p(out))
    return out


def pconv_mask(m, k, stride, dil):
    """Mask update of a partial (masked) convolution (Sec. 5.1, the masked
    convolutions of Liu et al. 2018): for every output pixel the number c of
    valid input pixels under its k x k window (taps dil apart, zero outside
    the map).  Returns (scale, m_out): scale = k^2 / c where c > 0, else 0;
    m_out = c > 0.  m: [A][H][W] of 0/1."""
    ones = np.ones((1, k, k, 1), np.float32)
    c = conv2d(np.asarray(m, np.float64)[..., None], ones, np.zeros(1, np.float32), stride, dil)[..., 0]
    scale = np.where(c > 0, (k * k) / np.maximum(c, 1.0), 0.0)
    return scale, (c > 0).astype(np.float64)


def pconv(x, m, w, b, stride, dil, act, residual=None):
    """Partial convolution: W (x * m) renormalised by k^2 / (valid pixels
    under the window), plus the bias, where any input pixel is valid, else 0;
    then the activation, then the residual link.  The activations are zero
    wherever their mask is, so x * m = x.  Returns (y, m_out)."""
    cout, k, _, cin = w.shape
    scale, m_out = pconv_mask(m, k, stride, dil)
    y = conv2d(x, w, np.zeros(cout, np.float32), stride, dil)
    y = np.where(scale[..., None] > 0, y * scale[..., None] + np.asarray(b, np.float64), 0.0)
    y = _act(y, act)
    if residual is not None:
        y = y + residual
    return y, m_out


def elu(x):
    """ELU with alpha = 1 (the activation of Sec. 5.1 / the network figure)."""
    return np.where(x > 0, x, np.expm1(np.minimum(x, 0.0)))


def softplus(x):
    """log(1 + e^x), evaluated stably as max(x, 0) + log1p(e^-|x|)."""
    return np.maximum(x, 0.0) + np.log1p(np.exp(-np.abs(x)))


def _act(x, act):
    if act == ACT_ELU:
        return elu(x)
    if act == ACT_SOFTPLUS:
        return softplus(x)
    return x


def upsample2(x):
    """Nearest-neighbour x2 upsampling of [A][h][w][C]."""
    return np.repeat(np.repeat(x, 2, axis=1), 2, axis=2)


def cnn_forward(x, net):
    """Reconstructed map y [A][H][W] (softplus output, before normalisation).

    Tiny net: three 3x3 convs (ELU, ELU, softplus).  U-Net: two 3x3 convs per
    level (the first of levels 1-3 with stride 2), decoder levels upsample the
    deeper output (nearest x2), concatenate [upsampled, skip] and apply two
    3x3 convs, then a 1x1 head with softplus."""
    layers = net["layers"]
    if net["arch"] == ARCH_PAPER:
        return cnn_forward_paper(x, net)
    if net["arch"] == ARCH_TINY3:
        h = x
        for cout, cin, k, stride, act, w, b in layers:
            h = _act(conv2d(h, w, b, stride), act)
        return h[..., 0]
    assert net["arch"] == ARCH_UNET4 and len(layers) == 15

    def run(h, i):
        cout, cin, k, stride, act, w, b = layers[i]
        return _act(conv2d(h, w, b, stride), act)

    e0 = run(run(x, 0), 1)
    e1 = run(run(e0, 2), 3)
    e2 = run(run(e1, 4), 5)
    e3 = run(run(e2, 6), 7)
    d2 = run(run(np.concatenate([upsample2(e3), e2], axis=3), 8), 9)
    d1 = run(run(np.concatenate([upsample2(d2), e1], axis=3), 10), 11)
    d0 = run(run(np.concatenate([upsample2(d1), e0], axis=3), 12), 13)
    return run(d0, 14)[..., 0]


def cnn_forward_paper(x, net):
    """The compact masked U-Net of Sec. 5.1 as read here (the paper's layer
    list is in a figure absent from the text): partial convolutions with ELU
    and residual links, two stride-2 levels, a bottleneck of dilated
    convolutions (taps 2 and 4 apart), decoder levels that upsample (nearest
    x2) and concatenate [upsampled, skip], at most 64 channels, and a 1x1
    head with softplus.  The input mask is the B channel (bins with photons);
    a concatenation's mask is the union of its parts' masks."""
    L, dil = net["layers"], net["dil"]
    assert len(L) == 12

    def run(h, m, i, res=None):
        cout, cin, k, stride, act, w, b = L[i]
        return pconv(h, m, w, b, stride, dil[i], act, res)

    m0 = x[..., 4]
    a0, m1 = run(x[..., :5], m0, 0)
    e0, me0 = run(a0, m1, 1, a0)
    a1, m3 = run(e0, me0, 2)
    e1, me1 = run(a1, m3, 3, a1)
    b0, m5 = run(e1, me1, 4)
    b1, m6 = run(b0, m5, 5, b0)
    b2, m7 = run(b1, m6, 6, b1)
    c1 = np.concatenate([upsample2(b2), e1], axis=3)
    d1, md1 = run(c1, np.maximum(upsample2(m7[..., None])[..., 0], me1), 7)
    d1b, md1b = run(d1, md1, 8, d1)
    c0 = np.concatenate([upsample2(d1b), e0], axis=3)
    d0, md0 = run(c0, np.maximum(upsample2(md1b[..., None])[..., 0], me0), 9)
    d0b, _ = run(d0, md0, 10, d0)
    cout, cin, k, stride, act, w, b = L[11]
    return _act(conv2d(d0b, w, b, stride), act)[..., 0]


# Sec. 8 (implementation): five networks, each trained for the voxels whose
# photon count falls in one range, [0,100), [100,500), [500,1000),
# [1000,5000) and [5000, inf).
PAPER_EXPERT_BOUNDS = (100, 500, 1000, 5000)


def expert_of(counts, bounds=PAPER_EXPERT_BOUNDS):
    """Index of the count range each voxel's photon count falls in."""
    counts = np.asarray(counts, np.int64)
    e = np.zeros(counts.shape, np.int64)
    for b in bounds:
        e += counts >= b
    return e


def cnn_forward_experts(x, counts, nets, bounds=PAPER_EXPERT_BOUNDS):
    """Map of every voxel from the network of its photon-count range."""
    e = expert_of(counts, bounds)
    y = None
    for k, net in enumerate(nets):
        sel = np.nonzero(e == k)[0]
        if sel.size == 0:
            continue
        yk = cnn_forward(x[sel], net)
        if y is None:
            y = np.zeros((x.shape[0],) + yk.shape[1:], np.float64)
        y[sel] = yk
    return y


# --------------------------------------------------------------------------
# a8-a9: sampling map and its CDFs (Eq. energy_target; Sec. 7.3: the CDF is a
# cumulative sum over the map pixels, sampled as an environment map is).
# --------------------------------------------------------------------------
def normalise(y):
    """P_k = y_k / sum_k y (FP64).  A map whose sum is zero is invalid."""
    y = np.asarray(y, np.float64)
    A = y.shape[0]
    flat = y.reshape(A, -1)
    tot = flat.sum(axis=1)
    valid = tot > 0
    P = np.zeros_like(flat)
    P[valid] = flat[valid] / tot[valid, None]
    return P.reshape(y.shape), valid.astype(np.uint8)


def build_cdf(P):
    """Marginal CDF over rows and conditional CDF along each row (FP64).

    m_i = sum_j P_ij, Fz[i] = sum_{i'<=i} m_i' / sum m, Fphi[i][j] =
    sum_{j'<=j} P_ij' / m_i (a zero row gets the uniform (j+1)/W)."""
    A, H, W = P.shape
    m = P.sum(axis=2)
    tot = m.sum(axis=1, keepdims=True)
    Fz = np.cumsum(m, axis=1) / np.where(tot > 0, tot, 1.0)
    rowc = np.cumsum(P, axis=2)
    uni = np.broadcast_to((np.arange(W) + 1.0) / W, P.shape)
    Fphi = np.where(m[:, :, None] > 0, rowc / np.where(m > 0, m, 1.0)[:, :, None], uni)
    return Fz, Fphi


def decision_tables(Fz, Fphi):
    """The FP32 tables the sampling decision is taken on (last entry 1)."""
    fz = Fz.astype(np.float32)
    fp = Fphi.astype(np.float32)
    fz[:, -1] = 1.0
    fp[:, :, -1] = 1.0
    return np.ascontiguousarray(fz), np.ascontiguousarray(fp)


def tables_from_map(y):
    P, valid = normalise(y)
    Fz, Fphi = build_cdf(P)
    fz, fp = decision_tables(Fz, Fphi)
    return dict(P=np.ascontiguousarray(P), valid=valid, Fz=Fz, Fphi=Fphi, fz=fz, fphi=fp,
                H=P.shape[1], W=P.shape[2])


# --------------------------------------------------------------------------
# a10-a12: guided sampling and pdf evaluation (Sec. 7.3; Eq. target_mis).
# --------------------------------------------------------------------------
def philox4x32_10(ctr, key):
    ctr = np.ascontiguousarray(np.asarray(ctr, np.uint32))
    key = np.ascontiguousarray(np.asarray(key, np.uint32))
    out = np.zeros(4, np.uint32)
    lib().or_philox4x32_10(_p(ctr), _p(key), _p(out))
    return out


def sample(grid, slot_of_leaf, tables, pos, seed, stream=0):
    pos = _f32(pos)
    q = pos.shape[0]
    dirs = np.zeros((q, 3), np.float64)
    pdf = np.zeros(q, np.float64)
    leaf = np.zeros(q, np.uint32)
    binv = np.zeros(q, np.uint32)
    slot = np.ascontiguousarray(slot_of_leaf, np.int32)
    if grid.get("kd"):
        lq = np.ascontiguousarray(kd_locate(grid, pos)[0], np.int64)
        lib().or_sample_leaves(_p(lq), q, _p(slot), tables["H"], tables["W"], _p(tables["P"]), _p(tables["fz"]),
                               _p(tables["fphi"]), _p(tables["valid"]), seed, stream, _p(dirs), _p(pdf), _p(leaf),
                               _p(binv))
        return dict(dir=dirs, pdf=pdf, leaf=leaf, bin=binv)
    lib().or_sample(_p(pos), q, _p(grid["lo"]), _p(grid["hi"]), grid["D"], _p(grid["leaf_code"]),
                    grid["L"], _p(slot), tables["H"], tables["W"], _p(tables["P"]), _p(tables["fz"]),
                    _p(tables["fphi"]), _p(tables["valid"]), seed, stream, _p(dirs), _p(pdf),
                    _p(leaf), _p(binv))
    return dict(dir=dirs, pdf=pdf, leaf=leaf, bin=binv)


def eval_pdf(grid, slot_of_leaf, tables, pos, dirs):
    pos = _f32(pos)
    d = _f32(dirs)
    q = pos.shape[0]
    pdf = np.zeros(q, np.float64)
    slot = np.ascontiguousarray(slot_of_leaf, np.int32)
    if grid.get("kd"):
        lq = np.ascontiguousarray(kd_locate(grid, pos)[0], np.int64)
        lib().or_eval_pdf_leaves(_p(lq), _p(d), q, _p(slot), tables["H"], tables["W"], _p(tables["P"]),
                                 _p(tables["valid"]), _p(pdf))
        return pdf
    lib().or_eval_pdf(_p(pos), _p(d), q, _p(grid["lo"]), _p(grid["hi"]), grid["D"],
                      _p(grid["leaf_code"]), grid["L"], _p(slot), tables["H"], tables["W"],
                      _p(tables["P"]), _p(tables["valid"]), _p(pdf))
    return pdf


# --------------------------------------------------------------------------
# One-sample MIS of BSDF and guide (Sec. 7.3, Eq. target_mis, mis_alpha,
# mis_coef; Algorithm 1).  The BSDF is a Lambertian stand-in around the
# vertex normal (no renderer is in scope).
# --------------------------------------------------------------------------
def leaf_of_positions(grid, pos):
    """Leaf containing each position (Algorithm 1, voxel location): its
    code under the a1 rule, then the last leaf whose start code is <= it (a
    walk down the voxel's tree for a grid of the paper's form)."""
    if grid.get("kd"):
        leaf, bad = kd_locate(grid, pos)
        return leaf, (ERR_INVALID_INPUT if bad else 0)
    codes, st = morton_codes(pos, grid["lo"], grid["hi"], grid["D"])
    return np.searchsorted(grid["leaf_code"], codes, side="right").astype(np.int64) - 1, st


def mis_accumulate(L, leaf, strategy, contrib):
    """nu_{j,B}, nu_{j,G}: sums of the bounce contributions in voxel j by the
    strategy that sampled them; Q_{j,B}, Q_{j,G}: their counts (FP64)."""
    strategy = np.asarray(strategy).astype(bool)
    c = np.asarray(contrib, np.float64)
    nu_b, nu_g = np.zeros(L), np.zeros(L)
    q_b, q_g = np.zeros(L, np.int64), np.zeros(L, np.int64)
    np.add.at(nu_b, leaf[~strategy], c[~strategy])
    np.add.at(nu_g, leaf[strategy], c[strategy])
    np.add.at(q_b, leaf[~strategy], 1)
    np.add.at(q_g, leaf[strategy], 1)
    return dict(nu_b=nu_b, nu_g=nu_g, q_b=q_b, q_g=q_g)


def mis_alpha(stats, alpha, min_count=50, lo=0.2, hi=0.8):
    """Eq. mis_alpha where both counts reach min_count: the BSDF share of the
    average contributions, clamped to [lo, hi]; other voxels keep alpha."""
    a = np.array(alpha, np.float64)
    nb, ng = stats["q_b"], stats["q_g"]
    ok = (nb >= min_count) & (ng >= min_count) & (nb > 0) & (ng > 0)
    mb = np.where(ok, stats["nu_b"] / np.maximum(nb, 1), 0.0)
    mg = np.where(ok, stats["nu_g"] / np.maximum(ng, 1), 0.0)
    ok &= (mb + mg) > 0
    a[ok] = np.clip(mb[ok] / (mb[ok] + mg[ok]), lo, hi)
    return a


def tangent_frame(n):
    """Orthonormal frame (b1, b2, n) of unit normals (Duff, Burgess,
    Christensen, Hery, Kensler, Liani, Villemin, JCGT 2017)."""
    n = np.asarray(n, np.float64)
    sgn = np.where(n[:, 2] >= 0, 1.0, -1.0)
    a = -1.0 / (sgn + n[:, 2])
    b = n[:, 0] * n[:, 1] * a
    b1 = np.stack([1.0 + sgn * n[:, 0] ** 2 * a, sgn * b, -sgn * n[:, 0]], axis=1)
    b2 = np.stack([b, sgn + n[:, 1] ** 2 * a, -n[:, 1]], axis=1)
    return b1, b2


def cosine_sample(n, v1, v2):
    """Lambertian lobe around n: a uniform disk sample (r = sqrt(v1), angle
    2 pi v2) lifted onto the hemisphere; pdf cos(theta) / pi."""
    b1, b2 = tangent_frame(n)
    r = np.sqrt(v1)
    ph = 2.0 * np.pi * v2
    lz = np.sqrt(np.maximum(0.0, 1.0 - v1))
    return (b1 * (r * np.cos(ph))[:, None] + b2 * (r * np.sin(ph))[:, None] + np.asarray(n, np.float64) * lz[:, None])


def bsdf_pdf(n, d):
    return np.maximum(0.0, np.sum(np.asarray(n, np.float64) * np.asarray(d, np.float64), axis=1)) / np.pi


def mis_uniforms(q, seed, stream):
    """Selection and BSDF uniforms: Philox4x32-10, counter (i, 0, stream, 1)."""
    key = [seed & 0xFFFFFFFF, (seed >> 32) & 0xFFFFFFFF]
    u = np.array([philox4x32_10([i & 0xFFFFFFFF, i >> 32, stream, 1], key) for i in range(q)], np.uint64)
    return (u >> 8).astype(np.float64) * 2.0 ** -24


def mis_sample(grid, slot_of_leaf, tables, alpha_leaf, pos, normals, seed, stream=0):
    """One-sample MIS: BSDF sampling with probability alpha_j (1 where the
    voxel has no valid map), else the guided sample; pdf of the result under
    alpha p_BSDF + (1 - alpha) p_guide."""
    q = len(pos)
    leaf, _ = leaf_of_positions(grid, pos)
    slot = np.asarray(slot_of_leaf)[leaf]
    valid = (slot >= 0) & (np.asarray(tables["valid"])[np.maximum(slot, 0)] > 0)
    a = np.where(valid, np.asarray(alpha_leaf, np.float64)[leaf], 1.0)
    u = mis_uniforms(q, seed, stream)
    use_bsdf = u[:, 0] < a
    g = sample(grid, slot_of_leaf, tables, pos, seed, stream)
    d = np.where(use_bsdf[:, None], cosine_sample(normals, u[:, 1], u[:, 2]), g["dir"])
    pdf = mis_eval(grid, slot_of_leaf, tables, alpha_leaf, pos, normals, d)
    return dict(dir=d, pdf=pdf, strategy=(~use_bsdf).astype(np.uint8), alpha=a)


def mis_eval(grid, slot_of_leaf, tables, alpha_leaf, pos, normals, dirs):
    leaf, _ = leaf_of_positions(grid, pos)
    slot = np.asarray(slot_of_leaf)[leaf]
    valid = (slot >= 0) & (np.asarray(tables["valid"])[np.maximum(slot, 0)] > 0)
    a = np.where(valid, np.asarray(alpha_leaf, np.float64)[leaf], 1.0)
    pg = np.where(valid, eval_pdf(grid, slot_of_leaf, tables, pos, dirs), 0.0)
    return a * bsdf_pdf(normals, dirs) + (1.0 - a) * pg


# --------------------------------------------------------------------------
# Progressive iterations (Sec. 7.1 "Voxel subdivision", Sec. 7.2; Algorithm 1,
# the photon and reconstruction blocks; Sec. 8: M_thr = c sqrt(2^t), c = 500,
# subdivision in the first two iterations).
# --------------------------------------------------------------------------
def split_threshold(t, c=500.0):
    """M_thr of iteration t; photon counts are integers, so a count exceeds
    c sqrt(2^t) exactly when it exceeds its floor."""
    return int(math.floor(c * math.sqrt(2.0 ** t)))


def bin_batch(grid, photons, H, W, F=32, n_bound=None):
    """A batch binned into the fixed leaves of grid: (L, HW) energy and count
    sums (Algorithm 1: locate voxel j and solid angle k, add the power)."""
    ph = _f32(photons)
    leaf, st = leaf_of_positions(grid, ph[:, :3])
    counts = np.bincount(leaf, minlength=grid["L"]).astype(np.int64)
    end = np.cumsum(counts)
    view = dict(grid, perm=np.argsort(leaf, kind="stable").astype(np.uint32),
                leaf_begin=(end - counts).astype(np.uint32), leaf_end=end.astype(np.uint32))
    h = splat(ph, view, 0, H, W, F, n_bound=n_bound)
    h["status"] |= st
    return h


class Progressive:
    """Per-leaf energy and count maps over iterations.  Refining iterations
    (t < refine_iterations) keep their photons and rebuild the grid from all
    of them with threshold M_thr(t); every leaf with photons is then updated,
    its previous planes being the sums over the earlier iterations.  Later
    batches are binned into the fixed leaves: a leaf that receives photons
    first copies its sums into its previous planes, then adds the batch.
    Maps are reconstructed for the updated leaves only; the others keep
    theirs (zero for a leaf never reconstructed).

    grid_rule "octree" refines by the octree rule of build_grid, "kd" by the
    paper's rule (build_kd_grid: R^3 voxels, median splits, normal variance
    threshold vthr; normals per photon, or none).

    Map slots: after a refinement the leaves with photons take slots 0.. in
    leaf order; a leaf that first receives photons later takes the next slot
    (new leaves of one batch in leaf order).  slot_of_leaf / slot_leaf hold
    the map; planes here stay leaf-indexed."""

    def __init__(self, lo, hi, max_depth, min_depth, H, W, max_photons, split_c=500.0, refine_iterations=2, F=32,
                 grid_rule="octree", R=None, vthr=0.5):
        self.lo, self.hi = _f32(lo), _f32(hi)
        self.D, self.min_depth, self.H, self.W, self.F = max_depth, min_depth, H, W, F
        self.c, self.refine, self.max_photons = split_c, refine_iterations, max_photons
        self.rule, self.R, self.vthr = grid_rule, R, vthr
        self.t = 0
        self.status = 0
        self.stored = np.zeros((0, 8), np.float32)
        self.stored_n = None
        self.grid = None
        self.updated = np.zeros(0, np.int64)
        if refine_iterations == 0:
            self._regrid(0, 2 ** 32 - 1)

    def _regrid(self, n_prev, thr):
        if self.rule == "kd":
            self.grid = build_kd_grid(self.stored, self.stored_n, self.lo, self.hi, self.R, self.D, thr, self.vthr)
        else:
            self.grid = build_grid(self.stored, self.lo, self.hi, self.D, self.min_depth, thr)
        h = splat(self.stored, self.grid, n_prev, self.H, self.W, self.F, n_bound=self.max_photons)
        self.status = h["status"]
        self.pow_cur, self.cnt_cur = h["pow_cur"], h["cnt_cur"]
        self.pow_prev, self.cnt_prev = h["pow_prev"], h["cnt_prev"]
        act, slot = active_leaves(self.grid)
        self.updated = act.astype(np.int64)
        self.slot_of_leaf = slot.astype(np.int64)
        self.slot_leaf = list(act.astype(np.int64))
        self.maps = np.zeros((self.grid["L"], self.H, self.W))

    def add_photons(self, photons, normals=None):
        ph = _f32(photons)
        if self.t < self.refine:
            n_prev = self.stored.shape[0]
            self.stored = np.concatenate([self.stored, ph])
            if normals is not None or self.stored_n is not None:
                prev_n = self.stored_n if self.stored_n is not None else np.zeros((n_prev, 3), np.float32)
                new_n = _f32(normals) if normals is not None else np.zeros((ph.shape[0], 3), np.float32)
                self.stored_n = np.concatenate([prev_n, new_n])
            self._regrid(n_prev, split_threshold(self.t, self.c))
            if self.t + 1 == self.refine:
                self.stored = np.zeros((0, 8), np.float32)
                self.stored_n = None
        else:
            b = bin_batch(self.grid, ph, self.H, self.W, self.F, n_bound=self.max_photons)
            self.status = b["status"]
            touched = np.nonzero(b["cnt_cur"].sum(axis=1) > 0)[0]
            self.pow_prev[touched] = self.pow_cur[touched]
            self.cnt_prev[touched] = self.cnt_cur[touched]
            self.pow_cur[touched] += b["pow_cur"][touched]
            self.cnt_cur[touched] += b["cnt_cur"][touched]
            for l in touched:
                if self.slot_of_leaf[l] < 0:
                    self.slot_of_leaf[l] = len(self.slot_leaf)
                    self.slot_leaf.append(int(l))
            self.updated = touched.astype(np.int64)
        self.t += 1

    @property
    def updated_slots(self):
        return self.slot_of_leaf[self.updated]

    def planes(self, leaves):
        return dict(pow_cur=self.pow_cur[leaves], cnt_cur=self.cnt_cur[leaves], pow_prev=self.pow_prev[leaves],
                    cnt_prev=self.cnt_prev[leaves], H=self.H, W=self.W)

    def reconstruct(self, net):
        if self.updated.size:
            self.maps[self.updated] = cnn_forward(assemble_inputs(self.planes(self.updated)), net)
        return tables_from_map(self.maps)


# --------------------------------------------------------------------------
# The whole path, for smoke checks and the CPU baseline.
# --------------------------------------------------------------------------
def run_path(photons, n_prev, lo, hi, D, min_depth, thr, H, W, blob, pos, dirs, seed, F=32,
             max_leaves=None):
    """Grid -> splat -> CNN -> normalise/CDF -> sample + eval.  With
    ``max_leaves`` only the first that many active leaves are reconstructed
    (the others keep no map), to bound the FP64 CNN on large workloads."""
    g = build_grid(photons, lo, hi, D, min_depth, thr)
    act, slot = active_leaves(g)
    if max_leaves is not None and act.size > max_leaves:
        keep = act[:max_leaves]
        slot = np.full(g["L"], -1, np.int32)
        slot[keep] = np.arange(keep.size, dtype=np.int32)
        act = keep
    h = splat(photons, g, n_prev, H, W, F)
    ha = hist_for_active(h, act)
    x = assemble_inputs(ha)
    y = cnn_forward(x, parse_net(blob))
    t = tables_from_map(y)
    s = sample(g, slot, t, pos, seed)
    e = eval_pdf(g, slot, t, pos, dirs)
    return dict(grid=g, act=act, slot=slot, hist=h, x=x, y=y, tables=t, sample=s, eval=e)
