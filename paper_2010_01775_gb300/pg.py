"""Thin ctypes binding of libpg.so (include/pg.h), same names as the C ABI.

Argument marshalling only: every step of the hot path runs in the library's
CUDA kernels.  Array arguments may be torch tensors (device or host), NumPy
arrays (host) or raw integer addresses.  The binding fails loudly when the
library is missing; there is no fallback of any kind.
"""
from __future__ import annotations

import ctypes
import os
import weakref

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "_lib", "libpg.so")

PG_FP32, PG_BF16, PG_FP8_E4M3, PG_FP8_MIXED = 0, 1, 2, 3
PRECISIONS = {"fp32": PG_FP32, "bf16": PG_BF16, "fp8": PG_FP8_E4M3, "fp8mix": PG_FP8_MIXED}

PG_INFO_N_PHOTONS, PG_INFO_N_LEAVES, PG_INFO_N_ACTIVE, PG_INFO_H, PG_INFO_W, PG_INFO_BYTES, PG_INFO_MAX_DEPTH = range(1, 8)
PG_INFO_N_SCENES, PG_INFO_SCENE_LEVELS = 8, 9
PG_INFO_ITERATION, PG_INFO_N_UPDATED, PG_INFO_KD_NODES = 10, 11, 12
PG_GRID_CODES, PG_GRID_PERM, PG_GRID_LEAF_OF, PG_GRID_LEAF_CODE, PG_GRID_LEAF_DEPTH = 100, 101, 102, 103, 104
PG_GRID_LEAF_BEGIN, PG_GRID_LEAF_END, PG_GRID_ACTIVE, PG_GRID_SLOT_OF_LEAF = 105, 106, 107, 108
PG_GRID_SCENE_LEAF_BEGIN = 109
PG_GRID_KD_AXIS, PG_GRID_KD_TAU, PG_GRID_KD_LINK = 110, 111, 112
PG_HIST_POW_CUR, PG_HIST_CNT_CUR, PG_HIST_POW_PREV, PG_HIST_CNT_PREV = 200, 201, 202, 203
PG_MAP_Y = 300
PG_TAB_P, PG_TAB_CDF_PHI, PG_TAB_CDF_Z, PG_TAB_VALID = 400, 401, 402, 403
PG_MIS_NU_B, PG_MIS_NU_G, PG_MIS_Q_B, PG_MIS_Q_G, PG_MIS_ALPHA = 500, 501, 502, 503, 504
PG_PROGRESS_UPDATED = 600

STATUS = {0: "PG_OK", 1: "PG_ERR_INVALID_ARG", 2: "PG_ERR_NOT_DEVICE_PTR", 3: "PG_ERR_OOM",
          4: "PG_ERR_OVERFLOW", 5: "PG_ERR_NOT_POW2", 6: "PG_ERR_TIMEOUT", 7: "PG_ERR_CUDA",
          8: "PG_ERR_INVALID_INPUT", 9: "PG_ERR_UNSUPPORTED"}

EXPORTED = ["pg_create", "pg_destroy", "pg_set_stream", "pg_sync", "pg_bytes_in_use", "pg_build_grid",
            "pg_splat_photons", "pg_net_load", "pg_reconstruct", "pg_map_import", "pg_build_cdf",
            "pg_sample_dirs", "pg_eval_pdf", "pg_info", "pg_export", "pg_free", "pg_status_string",
            "pg_sort_photons_noalloc", "pg_autotune", "pg_build_grid_batched", "pg_splat_photons_batched",
            "pg_sample_dirs_batched", "pg_eval_pdf_batched", "pg_budget_create", "pg_budget_destroy",
            "pg_ctx_attach_budget", "pg_budget_charge", "pg_budget_release", "pg_budget_wait", "pg_budget_query",
            "pg_launch_count", "pg_net_get_tuning", "pg_net_set_tuning",
            "pg_reconstruct_experts", "pg_mis_create", "pg_mis_accumulate", "pg_mis_update", "pg_mis_sample",
            "pg_mis_eval", "pg_progress_create", "pg_progress_add_photons", "pg_progress_reconstruct",
            "pg_progress_view", "pg_build_grid_kd", "pg_progress_add_photons_normals"]
PG_NOALLOC_MAX_PHOTONS = 1 << 20


class PgError(RuntimeError):
    def __init__(self, status, what=""):
        self.status = status
        name = STATUS.get(status, str(status))
        super().__init__(f"{what}: {name} ({_lib.pg_status_string(status).decode() if _lib else ''})")


class pg_grid_params(ctypes.Structure):
    _fields_ = [("lo", ctypes.c_float * 3), ("hi", ctypes.c_float * 3), ("max_depth", ctypes.c_int32),
                ("min_depth", ctypes.c_int32), ("split_threshold", ctypes.c_uint32)]


class pg_kd_params(ctypes.Structure):
    _fields_ = [("lo", ctypes.c_float * 3), ("hi", ctypes.c_float * 3), ("resolution", ctypes.c_int32),
                ("max_depth", ctypes.c_int32), ("split_threshold", ctypes.c_uint32),
                ("normal_variance_threshold", ctypes.c_float)]


class pg_progress_params(ctypes.Structure):
    _fields_ = [("lo", ctypes.c_float * 3), ("hi", ctypes.c_float * 3), ("max_depth", ctypes.c_int32),
                ("min_depth", ctypes.c_int32), ("split_c", ctypes.c_double), ("refine_iterations", ctypes.c_int32),
                ("H", ctypes.c_int32), ("W", ctypes.c_int32), ("frac_bits", ctypes.c_int32),
                ("max_photons", ctypes.c_uint64), ("grid_rule", ctypes.c_int32), ("resolution", ctypes.c_int32),
                ("normal_variance_threshold", ctypes.c_float)]


_lib = None


def load(path: str = LIB_PATH):
    """Loads libpg.so; raises if it has not been built."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"libpg.so not built ({path}); run __graft_entry__.build()")
    L = ctypes.CDLL(path)
    P, u64, u32, i32, sz = ctypes.c_void_p, ctypes.c_uint64, ctypes.c_uint32, ctypes.c_int, ctypes.c_size_t
    PP = ctypes.POINTER(ctypes.c_void_p)
    sig = {
        "pg_create": [PP, P, sz], "pg_destroy": [P], "pg_set_stream": [P, P], "pg_sync": [P],
        "pg_bytes_in_use": [P, ctypes.POINTER(u64)],
        "pg_build_grid": [P, P, u64, ctypes.POINTER(pg_grid_params), PP],
        "pg_splat_photons": [P, P, P, u64, u64, i32, i32, i32, PP],
        "pg_net_load": [P, P, sz, PP], "pg_reconstruct": [P, P, P, i32, PP],
        "pg_map_import": [P, P, u64, i32, i32, PP], "pg_build_cdf": [P, P, PP],
        "pg_sample_dirs": [P, P, P, P, u64, u64, u32, P, P, P, P],
        "pg_eval_pdf": [P, P, P, P, P, u64, P],
        "pg_info": [P, i32, ctypes.POINTER(u64)], "pg_export": [P, P, i32, P, sz],
        "pg_sort_photons_noalloc": [P, u64, ctypes.POINTER(pg_grid_params), P, P, P],
        "pg_autotune": [P, P, P, i32],
        "pg_build_grid_batched": [P, P, u64, P, u32, P, PP],
        "pg_splat_photons_batched": [P, P, P, u64, P, i32, i32, i32, PP],
        "pg_sample_dirs_batched": [P, P, P, P, P, u64, u64, P, P, P, P, P],
        "pg_eval_pdf_batched": [P, P, P, P, P, P, u64, P],
        "pg_launch_count": [P, ctypes.POINTER(u64)],
        "pg_reconstruct_experts": [P, P, P, i32, P, i32, PP],
        "pg_mis_create": [P, P, PP], "pg_mis_accumulate": [P, P, P, P, P, P, u64],
        "pg_mis_update": [P, P, u32, ctypes.c_float, ctypes.c_float],
        "pg_mis_sample": [P, P, P, P, P, P, u64, u64, u32, P, P, P],
        "pg_mis_eval": [P, P, P, P, P, P, P, u64, P],
        "pg_progress_create": [P, ctypes.POINTER(pg_progress_params), PP],
        "pg_progress_add_photons": [P, P, P, u64], "pg_progress_reconstruct": [P, P, P, i32],
        "pg_progress_add_photons_normals": [P, P, P, P, u64],
        "pg_progress_view": [P, PP, PP, PP, PP],
        "pg_build_grid_kd": [P, P, P, u64, ctypes.POINTER(pg_kd_params), PP],
        "pg_net_get_tuning": [P, P, sz, ctypes.POINTER(sz)], "pg_net_set_tuning": [P, P, sz],
        "pg_budget_create": [u64, PP], "pg_budget_destroy": [P], "pg_ctx_attach_budget": [P, P],
        "pg_budget_charge": [P, u64], "pg_budget_release": [P, u64],
        "pg_budget_wait": [P, u64, ctypes.POINTER(u64), u32],
        "pg_budget_query": [P, ctypes.POINTER(u64), ctypes.POINTER(u64), ctypes.POINTER(u64)],
    }
    for name, args in sig.items():
        f = getattr(L, name)
        f.argtypes = args
        f.restype = ctypes.c_int
    L.pg_free.argtypes = [P]
    L.pg_free.restype = None
    L.pg_status_string.argtypes = [ctypes.c_int]
    L.pg_status_string.restype = ctypes.c_char_p
    _lib = L
    return L


def _check(status, what):
    if status != 0:
        raise PgError(status, what)


def _ptr(x):
    """Address of a torch tensor / numpy array / int (None -> NULL)."""
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if hasattr(x, "data_ptr"):
        assert x.is_contiguous(), "arrays must be contiguous"
        return x.data_ptr()
    if isinstance(x, np.ndarray):
        assert x.flags["C_CONTIGUOUS"], "arrays must be contiguous"
        return x.ctypes.data
    raise TypeError(f"cannot take the address of {type(x)}")


class Handle:
    """Owns one library handle; freed with pg_free (before its context)."""

    def __init__(self, ctx, ptr, kind):
        self.ctx, self.ptr, self.kind = ctx, ptr, kind
        ctx._handles.add(self)

    def info(self, what):
        v = ctypes.c_uint64()
        _check(_lib.pg_info(self.ptr, what, ctypes.byref(v)), "pg_info")
        return v.value

    def export(self, what, dtype, count):
        out = np.empty(count, dtype=dtype)
        if count:
            _check(_lib.pg_export(self.ctx.ptr, self.ptr, what, out.ctypes.data, out.nbytes), "pg_export")
        return out

    def free(self):
        if self.ptr and self.ctx.ptr:
            _lib.pg_free(self.ptr)
        self.ptr = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


class Borrowed(Handle):
    """A handle lent by another handle (a progress state's grid, planes, maps,
    tables): never freed here, and it keeps its owner alive."""

    def __init__(self, ctx, ptr, kind, owner):
        self.ctx, self.ptr, self.kind, self.owner = ctx, ptr, kind, owner

    def free(self):
        self.ptr = None


class Context:
    """A pg_ctx bound to a CUDA stream (torch's current stream by default)."""

    def __init__(self, stream=None, hbm_budget=0):
        load()
        self.ptr = None
        self._handles = weakref.WeakSet()
        if stream is None:
            import torch
            stream = torch.cuda.current_stream().cuda_stream
        p = ctypes.c_void_p()
        _check(_lib.pg_create(ctypes.byref(p), ctypes.c_void_p(stream), hbm_budget), "pg_create")
        self.ptr = p.value

    def sync(self):
        _check(_lib.pg_sync(self.ptr), "pg_sync")

    def bytes_in_use(self):
        v = ctypes.c_uint64()
        _check(_lib.pg_bytes_in_use(self.ptr, ctypes.byref(v)), "pg_bytes_in_use")
        return v.value

    def launch_count(self):
        v = ctypes.c_uint64()
        _check(_lib.pg_launch_count(self.ptr, ctypes.byref(v)), "pg_launch_count")
        return v.value

    def set_stream(self, stream):
        _check(_lib.pg_set_stream(self.ptr, ctypes.c_void_p(stream)), "pg_set_stream")

    def destroy(self):
        """Frees every live handle of this context, then the context."""
        if self.ptr:
            for h in list(self._handles):
                h.free()
            _lib.pg_destroy(self.ptr)
            self.ptr = None

    def __del__(self):
        try:
            self.destroy()
        except Exception:
            pass


class Budget:
    """A pg_budget: one HBM byte budget shared by several contexts."""

    def __init__(self, capacity):
        load()
        p = ctypes.c_void_p()
        _check(_lib.pg_budget_create(capacity, ctypes.byref(p)), "pg_budget_create")
        self.ptr = p.value
        self.capacity = capacity

    def attach(self, ctx):
        _check(_lib.pg_ctx_attach_budget(ctx.ptr, self.ptr), "pg_ctx_attach_budget")

    @staticmethod
    def detach(ctx):
        _check(_lib.pg_ctx_attach_budget(ctx.ptr, None), "pg_ctx_attach_budget")

    def charge(self, nbytes) -> bool:
        """Charges nbytes if they fit; False (nothing charged) otherwise."""
        st = _lib.pg_budget_charge(self.ptr, nbytes)
        if st == 3:
            return False
        _check(st, "pg_budget_charge")
        return True

    def release(self, nbytes):
        _check(_lib.pg_budget_release(self.ptr, nbytes), "pg_budget_release")

    def query(self):
        """(in_use, capacity, generation)."""
        a, b, g = ctypes.c_uint64(), ctypes.c_uint64(), ctypes.c_uint64()
        _check(_lib.pg_budget_query(self.ptr, ctypes.byref(a), ctypes.byref(b), ctypes.byref(g)), "pg_budget_query")
        return a.value, b.value, g.value

    def wait(self, nbytes, generation, timeout_ms) -> tuple:
        """Blocks (GIL released) until nbytes fit or a release happened after
        `generation`; returns (fits_or_released, new_generation)."""
        g = ctypes.c_uint64(generation)
        st = _lib.pg_budget_wait(self.ptr, nbytes, ctypes.byref(g), timeout_ms)
        if st not in (0, 6):
            _check(st, "pg_budget_wait")
        return st == 0, g.value

    def destroy(self):
        if self.ptr:
            _check(_lib.pg_budget_destroy(self.ptr), "pg_budget_destroy")
            self.ptr = None


def pg_create(stream=None, hbm_budget=0) -> Context:
    return Context(stream, hbm_budget)


def pg_build_grid(ctx, photons, n, lo, hi, max_depth, min_depth, split_threshold) -> Handle:
    prm = pg_grid_params((ctypes.c_float * 3)(*lo), (ctypes.c_float * 3)(*hi), max_depth, min_depth,
                         split_threshold)
    out = ctypes.c_void_p()
    _check(_lib.pg_build_grid(ctx.ptr, _ptr(photons), n, ctypes.byref(prm), ctypes.byref(out)), "pg_build_grid")
    return Handle(ctx, out.value, "grid")


def pg_splat_photons(ctx, grid, photons, n, n_prev, H, W, frac_bits=32) -> Handle:
    out = ctypes.c_void_p()
    _check(_lib.pg_splat_photons(ctx.ptr, grid.ptr, _ptr(photons), n, n_prev, H, W, frac_bits, ctypes.byref(out)),
           "pg_splat_photons")
    return Handle(ctx, out.value, "hist")


def pg_net_load(ctx, blob: bytes) -> Handle:
    out = ctypes.c_void_p()
    buf = ctypes.create_string_buffer(blob, len(blob))
    _check(_lib.pg_net_load(ctx.ptr, buf, len(blob), ctypes.byref(out)), "pg_net_load")
    return Handle(ctx, out.value, "net")


def pg_reconstruct(ctx, hist, net, precision=PG_FP32) -> Handle:
    out = ctypes.c_void_p()
    _check(_lib.pg_reconstruct(ctx.ptr, hist.ptr, net.ptr, precision, ctypes.byref(out)), "pg_reconstruct")
    return Handle(ctx, out.value, "map")


def pg_build_grid_batched(ctx, photons, n, scene_begin, los, his, max_depth, min_depth, split_threshold) -> Handle:
    """scene_begin: S+1 uint32 offsets (array or tensor); los/his: S x 3."""
    S = len(los)
    prm = (pg_grid_params * S)()
    for s in range(S):
        prm[s] = pg_grid_params((ctypes.c_float * 3)(*[float(v) for v in los[s]]),
                                (ctypes.c_float * 3)(*[float(v) for v in his[s]]), max_depth, min_depth,
                                split_threshold)
    out = ctypes.c_void_p()
    _check(_lib.pg_build_grid_batched(ctx.ptr, _ptr(photons), n, _ptr(scene_begin), S, prm, ctypes.byref(out)),
           "pg_build_grid_batched")
    return Handle(ctx, out.value, "grid")


def pg_splat_photons_batched(ctx, grid, photons, n, n_prev, H, W, frac_bits=32) -> Handle:
    out = ctypes.c_void_p()
    _check(_lib.pg_splat_photons_batched(ctx.ptr, grid.ptr, _ptr(photons), n, _ptr(n_prev), H, W, frac_bits,
                                         ctypes.byref(out)), "pg_splat_photons_batched")
    return Handle(ctx, out.value, "hist")


def pg_sample_dirs_batched(ctx, grid, tables, pos, query_begin, q, seed, stream_ids, dirs, pdf, leaf, bins=None):
    _check(_lib.pg_sample_dirs_batched(ctx.ptr, grid.ptr, tables.ptr, _ptr(pos), _ptr(query_begin), q, seed,
                                       _ptr(stream_ids), _ptr(dirs), _ptr(pdf), _ptr(leaf), _ptr(bins)),
           "pg_sample_dirs_batched")


def pg_eval_pdf_batched(ctx, grid, tables, pos, dirs, query_begin, q, pdf):
    _check(_lib.pg_eval_pdf_batched(ctx.ptr, grid.ptr, tables.ptr, _ptr(pos), _ptr(dirs), _ptr(query_begin), q,
                                    _ptr(pdf)), "pg_eval_pdf_batched")


PAPER_EXPERT_BOUNDS = (100, 500, 1000, 5000)  # photon-count ranges of the 5 experts (Sec. 8)


def pg_reconstruct_experts(ctx, hist, nets, count_bounds=PAPER_EXPERT_BOUNDS, precision=PG_FP32) -> Handle:
    """Map of every leaf from the net of its photon-count range (len(nets)
    experts, len(nets) - 1 ascending bounds)."""
    arr = (ctypes.c_void_p * len(nets))(*[n.ptr for n in nets])
    b = np.ascontiguousarray(np.asarray(count_bounds, dtype=np.uint32))
    out = ctypes.c_void_p()
    _check(_lib.pg_reconstruct_experts(ctx.ptr, hist.ptr, arr, len(nets), b.ctypes.data if b.size else None,
                                       precision, ctypes.byref(out)), "pg_reconstruct_experts")
    return Handle(ctx, out.value, "map")


def pg_mis_create(ctx, grid) -> Handle:
    out = ctypes.c_void_p()
    _check(_lib.pg_mis_create(ctx.ptr, grid.ptr, ctypes.byref(out)), "pg_mis_create")
    return Handle(ctx, out.value, "mis")


def pg_mis_accumulate(ctx, mis, grid, pos, strategy, contrib, q):
    _check(_lib.pg_mis_accumulate(ctx.ptr, mis.ptr, grid.ptr, _ptr(pos), _ptr(strategy), _ptr(contrib), q),
           "pg_mis_accumulate")


def pg_mis_update(ctx, mis, min_count=50, alpha_lo=0.2, alpha_hi=0.8):
    _check(_lib.pg_mis_update(ctx.ptr, mis.ptr, min_count, alpha_lo, alpha_hi), "pg_mis_update")


def pg_mis_sample(ctx, grid, tables, mis, pos, normal, q, seed, stream_id, dirs, pdf, strategy):
    _check(_lib.pg_mis_sample(ctx.ptr, grid.ptr, tables.ptr, mis.ptr, _ptr(pos), _ptr(normal), q, seed, stream_id,
                              _ptr(dirs), _ptr(pdf), _ptr(strategy)), "pg_mis_sample")


def pg_mis_eval(ctx, grid, tables, mis, pos, normal, dirs, q, pdf):
    _check(_lib.pg_mis_eval(ctx.ptr, grid.ptr, tables.ptr, mis.ptr, _ptr(pos), _ptr(normal), _ptr(dirs), q,
                            _ptr(pdf)), "pg_mis_eval")


def export_mis(m):
    L = m.info(PG_INFO_N_LEAVES)
    return dict(nu_b=m.export(PG_MIS_NU_B, np.float64, L), nu_g=m.export(PG_MIS_NU_G, np.float64, L),
                q_b=m.export(PG_MIS_Q_B, np.uint32, L), q_g=m.export(PG_MIS_Q_G, np.uint32, L),
                alpha=m.export(PG_MIS_ALPHA, np.float32, L))


def pg_autotune(ctx, hist, net, precision):
    _check(_lib.pg_autotune(ctx.ptr, hist.ptr, net.ptr, precision), "pg_autotune")


def pg_net_get_tuning(net) -> np.ndarray:
    need = ctypes.c_size_t()
    _check(_lib.pg_net_get_tuning(net.ptr, None, 0, ctypes.byref(need)), "pg_net_get_tuning")
    out = np.zeros(need.value, np.int32)
    _check(_lib.pg_net_get_tuning(net.ptr, out.ctypes.data, out.size, ctypes.byref(need)), "pg_net_get_tuning")
    return out


def pg_net_set_tuning(net, values):
    v = np.ascontiguousarray(values, dtype=np.int32)
    _check(_lib.pg_net_set_tuning(net.ptr, v.ctypes.data, v.size), "pg_net_set_tuning")


def pg_map_import(ctx, y, n_maps, H, W) -> Handle:
    out = ctypes.c_void_p()
    _check(_lib.pg_map_import(ctx.ptr, _ptr(y), n_maps, H, W, ctypes.byref(out)), "pg_map_import")
    return Handle(ctx, out.value, "map")


def pg_build_cdf(ctx, m) -> Handle:
    out = ctypes.c_void_p()
    _check(_lib.pg_build_cdf(ctx.ptr, m.ptr, ctypes.byref(out)), "pg_build_cdf")
    return Handle(ctx, out.value, "tables")


def pg_sample_dirs(ctx, grid, tables, pos, q, seed, stream_id, dirs, pdf, leaf, bins=None):
    _check(_lib.pg_sample_dirs(ctx.ptr, grid.ptr, tables.ptr, _ptr(pos), q, seed, stream_id, _ptr(dirs), _ptr(pdf),
                               _ptr(leaf), _ptr(bins)), "pg_sample_dirs")


def pg_eval_pdf(ctx, grid, tables, pos, dirs, q, pdf):
    _check(_lib.pg_eval_pdf(ctx.ptr, grid.ptr, tables.ptr, _ptr(pos), _ptr(dirs), q, _ptr(pdf)), "pg_eval_pdf")


def pg_sort_photons_noalloc(photons, n, lo, hi, max_depth, codes, perm, stream=0):
    """Morton codes and stable sort permutation with no device allocation
    (scratch is a static device array; n <= PG_NOALLOC_MAX_PHOTONS)."""
    load()
    prm = pg_grid_params((ctypes.c_float * 3)(*lo), (ctypes.c_float * 3)(*hi), max_depth, 0, 0)
    _check(_lib.pg_sort_photons_noalloc(_ptr(photons), n, ctypes.byref(prm), _ptr(codes), _ptr(perm),
                                        ctypes.c_void_p(stream)), "pg_sort_photons_noalloc")


def pg_sync(ctx):
    ctx.sync()


def pg_free(handle):
    handle.free()


# ------------------------------------------------------------------ exports
def export_grid(g):
    n, L, A = g.info(PG_INFO_N_PHOTONS), g.info(PG_INFO_N_LEAVES), g.info(PG_INFO_N_ACTIVE)
    return dict(codes=g.export(PG_GRID_CODES, np.uint64, n), perm=g.export(PG_GRID_PERM, np.uint32, n),
                leaf_of=g.export(PG_GRID_LEAF_OF, np.uint32, n),
                leaf_code=g.export(PG_GRID_LEAF_CODE, np.uint64, L),
                leaf_depth=g.export(PG_GRID_LEAF_DEPTH, np.int32, L),
                leaf_begin=g.export(PG_GRID_LEAF_BEGIN, np.uint32, L),
                leaf_end=g.export(PG_GRID_LEAF_END, np.uint32, L),
                active=g.export(PG_GRID_ACTIVE, np.uint32, A),
                slot_of_leaf=g.export(PG_GRID_SLOT_OF_LEAF, np.int32, L), L=L, A=A)


def export_hist(h):
    A, H, W = h.info(PG_INFO_N_ACTIVE), h.info(PG_INFO_H), h.info(PG_INFO_W)
    c = A * H * W
    return dict(pow_cur=h.export(PG_HIST_POW_CUR, np.uint64, c).reshape(A, H * W),
                cnt_cur=h.export(PG_HIST_CNT_CUR, np.uint32, c).reshape(A, H * W),
                pow_prev=h.export(PG_HIST_POW_PREV, np.uint64, c).reshape(A, H * W),
                cnt_prev=h.export(PG_HIST_CNT_PREV, np.uint32, c).reshape(A, H * W), H=H, W=W)


def export_map(m):
    A, H, W = m.info(PG_INFO_N_ACTIVE), m.info(PG_INFO_H), m.info(PG_INFO_W)
    return m.export(PG_MAP_Y, np.float32, A * H * W).reshape(A, H, W)


def export_tables(t):
    A, H, W = t.info(PG_INFO_N_ACTIVE), t.info(PG_INFO_H), t.info(PG_INFO_W)
    return dict(P=t.export(PG_TAB_P, np.float32, A * H * W).reshape(A, H, W),
                cdf_phi=t.export(PG_TAB_CDF_PHI, np.float32, A * H * W).reshape(A, H, W),
                cdf_z=t.export(PG_TAB_CDF_Z, np.float32, A * H).reshape(A, H),
                valid=t.export(PG_TAB_VALID, np.uint8, A), H=H, W=W)


# ---------------------------------------------------------------- progressive iterations
def pg_progress_create(ctx, lo, hi, max_depth, min_depth, H, W, max_photons, split_c=500.0, refine_iterations=2,
                       frac_bits=32, grid_rule=0, resolution=100, normal_variance_threshold=0.5) -> Handle:
    p = pg_progress_params((ctypes.c_float * 3)(*lo), (ctypes.c_float * 3)(*hi), max_depth, min_depth, split_c,
                           refine_iterations, H, W, frac_bits, max_photons, grid_rule, resolution,
                           normal_variance_threshold)
    out = ctypes.c_void_p()
    _check(_lib.pg_progress_create(ctx.ptr, ctypes.byref(p), ctypes.byref(out)), "pg_progress_create")
    return Handle(ctx, out.value, "progress")


def pg_progress_add_photons(ctx, state, photons, n, normals=None):
    if normals is None:
        _check(_lib.pg_progress_add_photons(ctx.ptr, state.ptr, _ptr(photons), n), "pg_progress_add_photons")
    else:
        _check(_lib.pg_progress_add_photons_normals(ctx.ptr, state.ptr, _ptr(photons), _ptr(normals), n),
               "pg_progress_add_photons_normals")


def pg_progress_reconstruct(ctx, state, net, precision):
    _check(_lib.pg_progress_reconstruct(ctx.ptr, state.ptr, net.ptr, precision), "pg_progress_reconstruct")


def pg_progress_view(state):
    """(grid, planes, maps, tables) borrowed from the state (tables is None
    before the first reconstruct); valid until the state's next call."""
    ptrs = [ctypes.c_void_p() for _ in range(4)]
    _check(_lib.pg_progress_view(state.ptr, *[ctypes.byref(p) for p in ptrs]), "pg_progress_view")
    kinds = ("grid", "hist", "map", "tables")
    return tuple(Borrowed(state.ctx, p.value, k, state) if p.value else None for p, k in zip(ptrs, kinds))


def export_progress_updated(state) -> np.ndarray:
    return state.export(PG_PROGRESS_UPDATED, np.uint32, state.info(PG_INFO_N_UPDATED))


# ---------------------------------------------------------------- the paper's grid rule
def pg_build_grid_kd(ctx, photons, normals, n, lo, hi, resolution=100, max_depth=8, split_threshold=500,
                     normal_variance_threshold=0.5) -> Handle:
    p = pg_kd_params((ctypes.c_float * 3)(*lo), (ctypes.c_float * 3)(*hi), resolution, max_depth, split_threshold,
                     normal_variance_threshold)
    out = ctypes.c_void_p()
    _check(_lib.pg_build_grid_kd(ctx.ptr, _ptr(photons), _ptr(normals), n, ctypes.byref(p), ctypes.byref(out)),
           "pg_build_grid_kd")
    return Handle(ctx, out.value, "grid")


def export_kd(g):
    """Leaf table and tree of a grid of the paper's form."""
    n, L, N = g.info(PG_INFO_N_PHOTONS), g.info(PG_INFO_N_LEAVES), g.info(PG_INFO_KD_NODES)
    return dict(cells=g.export(PG_GRID_CODES, np.uint64, n), perm=g.export(PG_GRID_PERM, np.uint32, n),
                leaf_of=g.export(PG_GRID_LEAF_OF, np.uint32, n), leaf_cell=g.export(PG_GRID_LEAF_CODE, np.uint64, L),
                leaf_depth=g.export(PG_GRID_LEAF_DEPTH, np.int32, L),
                leaf_begin=g.export(PG_GRID_LEAF_BEGIN, np.uint32, L),
                leaf_end=g.export(PG_GRID_LEAF_END, np.uint32, L),
                node_axis=g.export(PG_GRID_KD_AXIS, np.uint8, N), node_tau=g.export(PG_GRID_KD_TAU, np.float32, N),
                node_link=g.export(PG_GRID_KD_LINK, np.int32, N), L=L, A=g.info(PG_INFO_N_ACTIVE))
