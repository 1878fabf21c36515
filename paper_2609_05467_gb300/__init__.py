"""GB300 (sm_103a) hemispherical ray-casting for milling accessibility.

A thin binding over the C ABI of ``include/rc.h`` (``librc.so``, built
in-tree by :mod:`paper_2609_05467_gb300.build`).  Every function here has
the name of the C entry point it calls and does argument marshalling only:
torch CUDA tensors are passed as raw device pointers together with the
current CUDA stream, and every per-face, per-point and per-ray step runs in
the library's CUDA kernels.  There is no CPU fallback: if the library or a
CUDA device is missing, the calls raise.

Paper: Baltadouros, Lauwers, Duflou, "Hemispherical Ray-Casting Analysis for
Milling Configuration Classification and Machinability Assessment"
(Section 3.1 hemispherical accessibility, Section 3.2 directional
accessibility, Section 3.3 indicators, classification and setups).
"""
from __future__ import annotations

import ctypes
import os
import threading

__all__ = [
    "RcError", "Params", "Summary", "Setups", "BvhInfo", "load", "lib_path",
    "rc_params_default", "rc_build_bvh", "rc_refit_bvh", "rc_destroy_bvh", "rc_bvh_get_info",
    "rc_sample_points", "rc_direction_table", "rc_hemisphere_cast", "rc_hemisphere_cast_retests", "rc_direction_variability",
    "rc_direction_variability_noalloc",
    "rc_classify", "rc_orthogonal_cast", "rc_min_setups", "rc_setup_cover", "rc_analyze_part",
    "rc_launch_count", "rc_stream_status", "rc_bvh_validate", "Bvh", "PartResult", "rc_batch_create", "rc_batch_add_part", "rc_batch_clear",
    "rc_batch_set_params", "rc_batch_launch", "rc_batch_poll", "rc_batch_add_analysis", "rc_batch_results", "rc_batch_autotune", "rc_batch_destroy", "rc_server_create",
    "rc_server_submit", "rc_server_wait", "rc_server_read_bits", "rc_server_get_stats", "rc_server_destroy",
]

_HERE = os.path.dirname(os.path.abspath(__file__))
_lib = None
_lock = threading.Lock()

STATUS = {0: "RC_OK", 1: "RC_E_ARG", 2: "RC_E_CUDA", 3: "RC_E_OOM", 4: "RC_E_TIMEOUT",
          5: "RC_E_DEGENERATE", 6: "RC_E_UNSUPPORTED", 7: "RC_E_DEVICE"}
RC_SAMPLE_AREA_RANDOM, RC_SAMPLE_FACE_CENTROID = 0, 1


class RcError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("%s: %s" % (STATUS.get(status, status), msg))
        self.status = status


class Params(ctypes.Structure):
    _fields_ = [
        ("n_dirs", ctypes.c_int32), ("sample_mode", ctypes.c_int32), ("origin_offset", ctypes.c_double),
        ("seed", ctypes.c_uint64), ("frame", ctypes.c_float * 9), ("tool_length", ctypes.c_float),
        ("conc_mode", ctypes.c_int32), ("t_acc", ctypes.c_double), ("t_share", ctypes.c_double),
        ("t_conc", ctypes.c_double), ("block_threads", ctypes.c_int32), ("blocks_per_sm", ctypes.c_int32),
        ("collect_stats", ctypes.c_int32), ("always_setups", ctypes.c_int32), ("point_order", ctypes.c_int32),
        ("tile_mode", ctypes.c_int32), ("points_per_item", ctypes.c_int32), ("launch_mode", ctypes.c_int32),
        ("fetch_mode", ctypes.c_int32), ("tree_width", ctypes.c_int32), ("parallel_tol", ctypes.c_double),
    ]


class Summary(ctypes.Structure):
    _fields_ = [
        ("overall_access", ctypes.c_double), ("overall_access_unweighted", ctypes.c_double),
        ("axis_share", ctypes.c_double * 3), ("mean_conc", ctypes.c_double),
        ("n_points", ctypes.c_int64), ("n_counted", ctypes.c_int64), ("n_zero_visible", ctypes.c_int64),
        ("dom_count", ctypes.c_int64 * 3), ("count_sum", ctypes.c_int64), ("weighted_count", ctypes.c_double),
        ("weight_sum", ctypes.c_double), ("conc_sum_q", ctypes.c_int64),
    ]

    def as_dict(self):
        return {
            "overall_access": self.overall_access,
            "overall_access_unweighted": self.overall_access_unweighted,
            "axis_share": list(self.axis_share), "mean_conc": self.mean_conc,
            "n_points": self.n_points, "n_counted": self.n_counted, "n_zero_visible": self.n_zero_visible,
            "dom_count": list(self.dom_count), "count_sum": self.count_sum,
        }


class Setups(ctypes.Structure):
    _fields_ = [
        ("setups_exact", ctypes.c_int32), ("setups_greedy", ctypes.c_int32), ("chosen_exact", ctypes.c_uint8),
        ("chosen_greedy", ctypes.c_uint8), ("pad", ctypes.c_uint8 * 6), ("class_counts", ctypes.c_int64 * 4),
        ("mask_hist", ctypes.c_int64 * 64),
    ]


RC_MAX_FRAMES = 6
RC_BOX_STEPS = 128
RC_FRAME_GIVEN, RC_FRAME_PRINCIPAL, RC_FRAME_NORMALS, RC_FRAME_BOX = 0, 1, 2, 3


class Frames(ctypes.Structure):
    """Candidate machining frames and their setups (``rc_frames``)."""
    _fields_ = [
        ("k", ctypes.c_int32), ("best", ctypes.c_int32), ("source", ctypes.c_int32 * RC_MAX_FRAMES),
        ("box_axis", ctypes.c_int32 * RC_MAX_FRAMES), ("box_step", ctypes.c_int32 * RC_MAX_FRAMES),
        ("frame", (ctypes.c_float * 9) * RC_MAX_FRAMES), ("volume", ctypes.c_double * RC_MAX_FRAMES),
        ("principal", ctypes.c_double * 3), ("setups", Setups * RC_MAX_FRAMES),
    ]

    def frame_array(self, c):
        import numpy as np
        return np.array(list(self.frame[c]), np.float32)


class PartResult(ctypes.Structure):
    _fields_ = [
        ("summary", Summary), ("setups", Setups), ("label", ctypes.c_int32), ("setups_ran", ctypes.c_int32),
        ("cast_counters", ctypes.c_int64 * 4), ("ortho_counters", ctypes.c_int64 * 4),
    ]


class ServerConfig(ctypes.Structure):
    _fields_ = [("slots", ctypes.c_int32), ("cast_blocks_per_sm", ctypes.c_int32),
                ("hbm_budget_bytes", ctypes.c_int64), ("small_rays", ctypes.c_int64),
                ("incremental", ctypes.c_int32), ("pad", ctypes.c_int32)]


class RequestResult(ctypes.Structure):
    _fields_ = [
        ("request_id", ctypes.c_int64), ("part_key", ctypes.c_uint64), ("status", ctypes.c_int),
        ("slot", ctypes.c_int32), ("rebuilt", ctypes.c_int32), ("priority_level", ctypes.c_int32),
        ("updated", ctypes.c_int32), ("pad", ctypes.c_int32), ("t_submit", ctypes.c_double), ("t_admit", ctypes.c_double), ("t_start", ctypes.c_double),
        ("t_end", ctypes.c_double), ("resident_bytes", ctypes.c_int64), ("result", PartResult),
        ("message", ctypes.c_char * 128),
    ]


class ServerStats(ctypes.Structure):
    _fields_ = [(k, ctypes.c_int64) for k in ("submitted", "completed", "failed", "rejected", "evicted", "running",
                                               "queued", "resident_parts", "used_bytes")]


class BvhInfo(ctypes.Structure):
    _fields_ = [
        ("n_tris", ctypes.c_int64), ("n_nodes", ctypes.c_int64), ("node_bytes", ctypes.c_int64),
        ("tri_bytes", ctypes.c_int64), ("max_depth", ctypes.c_int32), ("leaf_size", ctypes.c_int32),
        ("scene_lo", ctypes.c_float * 3), ("scene_hi", ctypes.c_float * 3),
    ]


def lib_path():
    return os.path.join(_HERE, "librc.so")


def load(build_if_missing=True):
    """Load ``librc.so`` (building it first if it is missing or stale)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if build_if_missing:
            from . import build as _b
            _b.build()
        path = lib_path()
        if not os.path.exists(path):
            raise RcError(2, "librc.so is not built (run paper_2609_05467_gb300.build.build())")
        L = ctypes.CDLL(path)
        P, i64, i32 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32
        st = ctypes.c_int
        sig = {
            "rc_params_default": ([ctypes.POINTER(Params)], st),
            "rc_last_error": ([], ctypes.c_char_p),
            "rc_launch_count": ([], i64),
            "rc_stream_status": ([P], st),
            "rc_build_bvh": ([P, i64, P, i64, P, ctypes.POINTER(P)], st),
            "rc_build_bvh_ex": ([P, i64, P, i64, i32, P, ctypes.POINTER(P)], st),
            "rc_refit_bvh": ([P, P, P], st),
            "rc_destroy_bvh": ([P], st),
            "rc_bvh_get_info": ([P, ctypes.POINTER(BvhInfo)], st),
            "rc_bvh_validate": ([P, P, P], st),
            "rc_sample_points": ([P, i64, ctypes.POINTER(Params), P, P, P, P, P], st),
            "rc_direction_table": ([i32, P], st),
            "rc_hemisphere_cast": ([P, P, P, i64, ctypes.POINTER(Params), P, P, P, P], st),
            "rc_hemisphere_cast_retests": ([P, P, P, i64, ctypes.POINTER(Params), P, P, P, P, i64, P], st),
            "rc_direction_variability": ([P, P, P, i64, ctypes.POINTER(Params), P, P, P, P,
                                          ctypes.POINTER(Summary), P], st),
            "rc_direction_variability_noalloc": ([P, P, P, i64, ctypes.POINTER(Params), P, P, P, P,
                                                  ctypes.POINTER(Summary), P], st),
            "rc_classify": ([ctypes.POINTER(Summary), ctypes.POINTER(Params), ctypes.POINTER(i32)], st),
            "rc_orthogonal_cast": ([P, P, P, i64, ctypes.POINTER(Params), P, P, P, P], st),
            "rc_min_setups": ([P, P, P, P, i64, ctypes.POINTER(Params), P, ctypes.POINTER(Setups), P], st),
            "rc_setup_cover": ([P, ctypes.POINTER(Setups)], st),
            "rc_batch_create": ([ctypes.POINTER(Params), i64, ctypes.POINTER(P)], st),
            "rc_batch_poll": ([P, i64, ctypes.POINTER(i32)], st),
            "rc_batch_add_analysis": ([P, P, P, P, P, i64, P, P, ctypes.POINTER(i64)], st),
            "rc_batch_results": ([P, ctypes.POINTER(PartResult), i64], st),
            "rc_batch_add_part": ([P, P, P, P, i64, P, P, P, ctypes.POINTER(i64)], st),
            "rc_batch_clear": ([P], st),
            "rc_batch_set_params": ([P, ctypes.POINTER(Params)], st),
            "rc_batch_launch": ([P, P], st),
            "rc_batch_autotune": ([P, P, i32, ctypes.POINTER(Params)], st),
            "rc_batch_destroy": ([P], st),
            "rc_server_create": ([ctypes.POINTER(Params), ctypes.POINTER(ServerConfig), ctypes.POINTER(P)], st),
            "rc_server_submit": ([P, ctypes.c_uint64, P, i64, P, i64, i64, ctypes.POINTER(i64)], st),
            "rc_server_wait": ([P, i64, ctypes.c_double, ctypes.POINTER(RequestResult)], st),
            "rc_server_read_bits": ([P, ctypes.c_uint64, P, i64, P, i64], st),
            "rc_server_get_stats": ([P, ctypes.POINTER(ServerStats)], st),
            "rc_server_destroy": ([P], st),
            "rc_analyze_part": ([P, i64, P, i64, i64, ctypes.POINTER(Params), P, P, P, P,
                                 ctypes.POINTER(PartResult), P], st),
            "rc_frame_candidates": ([P, ctypes.POINTER(Params), ctypes.POINTER(Frames), P], st),
            "rc_sample_points_on_faces": ([P, i64, ctypes.POINTER(Params), P, P, P, P], st),
            "rc_changed_faces": ([P, P, i64, P, i64, P, P, ctypes.POINTER(i64), P], st),
            "rc_hemisphere_update": ([P, P, P, P, i64, P, P, ctypes.POINTER(Params), P, P, P, P], st),
            "rc_frame_select": ([P, P, P, P, i64, ctypes.POINTER(Params), ctypes.POINTER(Frames), P, P], st),
            "rc_probe_l2": ([i64, i32, i32, ctypes.POINTER(ctypes.c_double), P], st),
            "rc_probe_fp32": ([i32, ctypes.POINTER(ctypes.c_double), P], st),
            "rc_tool_cast": ([P, P, P, i64, ctypes.POINTER(Params), ctypes.c_double, i32, P, P, P], st),
            "rc_stl_read": ([ctypes.c_char_p, P, i64, P, i64, ctypes.POINTER(i64), ctypes.POINTER(i64)], st),
            "rc_analyze_stl": ([ctypes.c_char_p, i64, ctypes.POINTER(Params), ctypes.POINTER(PartResult), P], st),
        }
        for name, (args, res) in sig.items():
            fn = getattr(L, name)
            fn.argtypes = args
            fn.restype = res
        _lib = L
        return _lib


def _check(status):
    if status != 0:
        msg = load().rc_last_error()
        raise RcError(status, msg.decode() if msg else "")


def _ptr(t):
    """Device pointer of a CUDA tensor (None -> NULL); checks contiguity."""
    if t is None:
        return None
    if not t.is_cuda:
        raise ValueError("expected a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError("expected a contiguous tensor")
    return ctypes.c_void_p(t.data_ptr())


def _stream(stream=None):
    import torch
    s = torch.cuda.current_stream() if stream is None else stream
    return ctypes.c_void_p(s.cuda_stream)


# ---------------------------------------------------------------------------
# the C ABI, one function per entry point
# ---------------------------------------------------------------------------

def rc_params_default(**kw):
    """Default :class:`Params` with keyword overrides (``frame`` takes 9
    floats, row-major)."""
    p = Params()
    _check(load().rc_params_default(ctypes.byref(p)))
    for k, v in kw.items():
        if k == "frame":
            for i, x in enumerate(v):
                p.frame[i] = float(x)
        else:
            setattr(p, k, v)
    return p


def rc_build_bvh(V, F, stream=None):
    """Build the device BVH of mesh ``V`` (float32 [nV,3] CUDA) / ``F``
    (int32 [T,3] CUDA); returns an opaque handle (int)."""
    h = ctypes.c_void_p()
    _check(load().rc_build_bvh(_ptr(V), V.shape[0], _ptr(F), F.shape[0], _stream(stream), ctypes.byref(h)))
    return h.value


RC_BUILDER_KARRAS, RC_BUILDER_PLOC = 0, 1


def rc_build_bvh_ex(V, F, builder, stream=None):
    """rc_build_bvh with a choice of binary builder (RC_BUILDER_*)."""
    h = ctypes.c_void_p()
    _check(load().rc_build_bvh_ex(_ptr(V), V.shape[0], _ptr(F), F.shape[0], builder, _stream(stream),
                                  ctypes.byref(h)))
    return h.value


def rc_refit_bvh(h, V, stream=None):
    _check(load().rc_refit_bvh(ctypes.c_void_p(h), _ptr(V), _stream(stream)))


def rc_destroy_bvh(h):
    _check(load().rc_destroy_bvh(ctypes.c_void_p(h)))


def rc_bvh_get_info(h):
    info = BvhInfo()
    _check(load().rc_bvh_get_info(ctypes.c_void_p(h), ctypes.byref(info)))
    return info


def rc_sample_points(h, n, params, P, N, face, weight=None, stream=None):
    _check(load().rc_sample_points(ctypes.c_void_p(h), n, ctypes.byref(params), _ptr(P), _ptr(N), _ptr(face),
                                   _ptr(weight), _stream(stream)))


def rc_direction_table(n_dirs):
    """Canonical fp32 direction table [n_dirs, 3] (host numpy array)."""
    import numpy as np
    out = np.zeros((n_dirs, 3), np.float32)
    _check(load().rc_direction_table(n_dirs, out.ctypes.data_as(ctypes.c_void_p)))
    return out


def rc_hemisphere_cast(h, P, N, params, bits, count, counters=None, stream=None):
    _check(load().rc_hemisphere_cast(ctypes.c_void_p(h), _ptr(P), _ptr(N), P.shape[0], ctypes.byref(params),
                                     _ptr(bits), _ptr(count), _ptr(counters), _stream(stream)))


def rc_hemisphere_cast_retests(h, P, N, params, bits, count, counters, lst, stream=None):
    """Instrumented cast listing the rays an FP64 re-test took part in
    (i * 65536 + j in `lst`, counters[6] = their total)."""
    _check(load().rc_hemisphere_cast_retests(ctypes.c_void_p(h), _ptr(P), _ptr(N), P.shape[0],
                                             ctypes.byref(params), _ptr(bits), _ptr(count), _ptr(counters),
                                             _ptr(lst), lst.numel() if lst is not None else 0, _stream(stream)))


def rc_direction_variability(bits, N, params, weight=None, acc=None, dom=None, conc=None, dir_area=None,
                             summary=True, stream=None):
    s = Summary() if summary else None
    _check(load().rc_direction_variability(_ptr(bits), _ptr(N), _ptr(weight), N.shape[0], ctypes.byref(params),
                                           _ptr(acc), _ptr(dom), _ptr(conc), _ptr(dir_area),
                                           ctypes.byref(s) if s is not None else None, _stream(stream)))
    return s


def rc_direction_variability_noalloc(bits, N, params, weight=None, acc=None, dom=None, conc=None,
                                     dir_area=None, summary=True, stream=None):
    """As :func:`rc_direction_variability`, using the library's static
    device scratch instead of allocating (see include/rc.h)."""
    s = Summary() if summary else None
    _check(load().rc_direction_variability_noalloc(_ptr(bits), _ptr(N), _ptr(weight), N.shape[0],
                                                   ctypes.byref(params), _ptr(acc), _ptr(dom), _ptr(conc),
                                                   _ptr(dir_area), ctypes.byref(s) if s is not None else None,
                                                   _stream(stream)))
    return s


def rc_classify(summary, params):
    lab = ctypes.c_int32()
    _check(load().rc_classify(ctypes.byref(summary), ctypes.byref(params), ctypes.byref(lab)))
    return lab.value


def rc_orthogonal_cast(h, P, N, params, mask, travel, counters=None, stream=None):
    _check(load().rc_orthogonal_cast(ctypes.c_void_p(h), _ptr(P), _ptr(N), P.shape[0], ctypes.byref(params),
                                     _ptr(mask), _ptr(travel), _ptr(counters), _stream(stream)))


def rc_tool_cast(h, P, N, params, tool_radius, ring_rays, mask, counters=None, stream=None):
    _check(load().rc_tool_cast(ctypes.c_void_p(h), _ptr(P), _ptr(N), P.shape[0], ctypes.byref(params),
                               float(tool_radius), int(ring_rays), _ptr(mask), _ptr(counters), _stream(stream)))


def rc_probe_l2(buffer_bytes=64 << 20, record_bytes=128, reads_per_thread=256, stream=None):
    """Random-record read bandwidth of an L2-resident buffer (GB/s)."""
    g = ctypes.c_double()
    _check(load().rc_probe_l2(buffer_bytes, record_bytes, reads_per_thread, ctypes.byref(g), _stream(stream)))
    return g.value


def rc_probe_fp32(iters=4096, stream=None):
    """FP32 FMA throughput (TFLOP/s)."""
    t = ctypes.c_double()
    _check(load().rc_probe_fp32(iters, ctypes.byref(t), _stream(stream)))
    return t.value


def rc_min_setups(h, mask, travel, face, params, cls=None, stream=None):
    out = Setups()
    _check(load().rc_min_setups(ctypes.c_void_p(h), _ptr(mask), _ptr(travel), _ptr(face), mask.shape[0],
                                ctypes.byref(params), _ptr(cls), ctypes.byref(out), _stream(stream)))
    return out


def rc_setup_cover(mask_hist):
    """Exact and greedy covers from a 64-bin histogram (host only)."""
    import numpy as np
    h = np.ascontiguousarray(mask_hist, dtype=np.int64)
    if h.shape != (64,):
        raise ValueError("mask_hist must have 64 bins")
    out = Setups()
    _check(load().rc_setup_cover(h.ctypes.data_as(ctypes.c_void_p), ctypes.byref(out)))
    return out


def rc_frame_candidates(h, params, stream=None):
    """Candidate machining frames of the part (see include/rc.h)."""
    out = Frames()
    _check(load().rc_frame_candidates(ctypes.c_void_p(h), ctypes.byref(params), ctypes.byref(out),
                                      _stream(stream)))
    return out


def rc_frame_select(h, P, N, face, params, frames, counters=None, stream=None):
    """Evaluate ``frames`` (a :class:`Frames`, updated in place) on the
    sample points and choose one; returns ``frames``."""
    _check(load().rc_frame_select(ctypes.c_void_p(h), _ptr(P), _ptr(N), _ptr(face), P.shape[0],
                                  ctypes.byref(params), ctypes.byref(frames), _ptr(counters), _stream(stream)))
    return frames


def rc_sample_points_on_faces(h, params, face, P, N, stream=None):
    _check(load().rc_sample_points_on_faces(ctypes.c_void_p(h), face.shape[0], ctypes.byref(params), _ptr(face),
                                            _ptr(P), _ptr(N), _stream(stream)))


def rc_changed_faces(V_old, V_new, F, changed, stream=None):
    """Returns (number of changed faces, box as a list lo xyz + hi xyz)."""
    box = (ctypes.c_float * 6)()
    nc = ctypes.c_int64()
    _check(load().rc_changed_faces(_ptr(V_old), _ptr(V_new), V_old.shape[0], _ptr(F), F.shape[0], _ptr(changed),
                                   box, ctypes.byref(nc), _stream(stream)))
    return nc.value, list(box)


def rc_hemisphere_update(h, P, N, face, changed, box, params, bits, count, counters=None, stream=None):
    b = (ctypes.c_float * 6)(*[float(x) for x in box])
    _check(load().rc_hemisphere_update(ctypes.c_void_p(h), _ptr(P), _ptr(N), _ptr(face), P.shape[0], _ptr(changed),
                                       b, ctypes.byref(params), _ptr(bits), _ptr(count), _ptr(counters),
                                       _stream(stream)))


def rc_stl_read(path):
    """Read an STL file (binary or ASCII): returns (V float32 [nV,3], F
    int32 [T,3]) as numpy arrays, vertices merged as include/rc.h says."""
    import numpy as np
    b = os.fsencode(path)
    nV, T = ctypes.c_int64(), ctypes.c_int64()
    _check(load().rc_stl_read(b, None, 0, None, 0, ctypes.byref(nV), ctypes.byref(T)))
    V = np.zeros((nV.value, 3), np.float32)
    F = np.zeros((T.value, 3), np.int32)
    _check(load().rc_stl_read(b, V.ctypes.data_as(ctypes.c_void_p), nV.value, F.ctypes.data_as(ctypes.c_void_p),
                              T.value, ctypes.byref(nV), ctypes.byref(T)))
    return V, F


def rc_analyze_stl(path, n, params, stream=None):
    """The paper's per-part analysis of an STL file: returns a PartResult."""
    out = PartResult()
    _check(load().rc_analyze_stl(os.fsencode(path), n, ctypes.byref(params), ctypes.byref(out), _stream(stream)))
    return out


def _hptr(a):
    """Host pointer of a numpy array or CPU tensor (None -> NULL)."""
    if a is None:
        return None
    if hasattr(a, "data_ptr"):
        if a.is_cuda or not a.is_contiguous():
            raise ValueError("expected a contiguous CPU tensor")
        return ctypes.c_void_p(a.data_ptr())
    if not a.flags["C_CONTIGUOUS"]:
        raise ValueError("expected a C-contiguous array")
    return a.ctypes.data_as(ctypes.c_void_p)


def rc_analyze_part(V, F, n, params, bits=None, count=None, mask=None, cls=None, stream=None):
    """Whole pipeline on HOST arrays (numpy or pinned CPU tensors): returns a
    :class:`PartResult`; the optional per-point outputs are host arrays."""
    out = PartResult()
    _check(load().rc_analyze_part(_hptr(V), V.shape[0], _hptr(F), F.shape[0], n, ctypes.byref(params),
                                  _hptr(bits), _hptr(count), _hptr(mask), _hptr(cls), ctypes.byref(out),
                                  _stream(stream)))
    return out


def rc_batch_create(params, hbm_budget_bytes=0):
    b = ctypes.c_void_p()
    _check(load().rc_batch_create(ctypes.byref(params), int(hbm_budget_bytes), ctypes.byref(b)))
    return b.value


def rc_batch_add_analysis(b, h, P, N, face, bits, count):
    """Add a part whose launch runs the whole path (cast, reduction,
    orthogonal cast, classes); returns its id."""
    pid = ctypes.c_int64()
    _check(load().rc_batch_add_analysis(ctypes.c_void_p(b), ctypes.c_void_p(h), _ptr(P), _ptr(N), _ptr(face),
                                        P.shape[0], _ptr(bits), _ptr(count), ctypes.byref(pid)))
    return pid.value


def rc_batch_results(b, n_parts):
    """Part-level results of the last launch, one PartResult per part."""
    out = (PartResult * n_parts)()
    _check(load().rc_batch_results(ctypes.c_void_p(b), out, n_parts))
    return list(out)


def rc_batch_poll(b, part_id):
    """1 once the last launch of the batch (this part included) has completed, else 0."""
    done = ctypes.c_int32()
    _check(load().rc_batch_poll(ctypes.c_void_p(b), int(part_id), ctypes.byref(done)))
    return done.value


def rc_batch_add_part(b, h, P, N, bits, count, counters=None):
    pid = ctypes.c_int64()
    _check(load().rc_batch_add_part(ctypes.c_void_p(b), ctypes.c_void_p(h), _ptr(P), _ptr(N), P.shape[0], _ptr(bits),
                                    _ptr(count), _ptr(counters), ctypes.byref(pid)))
    return pid.value


def rc_batch_clear(b):
    _check(load().rc_batch_clear(ctypes.c_void_p(b)))


def rc_batch_set_params(b, params):
    _check(load().rc_batch_set_params(ctypes.c_void_p(b), ctypes.byref(params)))


def rc_batch_launch(b, stream=None):
    _check(load().rc_batch_launch(ctypes.c_void_p(b), _stream(stream)))


def rc_batch_autotune(b, repeats=2, stream=None):
    best = Params()
    _check(load().rc_batch_autotune(ctypes.c_void_p(b), _stream(stream), repeats, ctypes.byref(best)))
    return best


def rc_batch_destroy(b):
    _check(load().rc_batch_destroy(ctypes.c_void_p(b)))


def rc_server_create(params, slots=4, hbm_budget_bytes=120 << 30, cast_blocks_per_sm=0, small_rays=0,
                     incremental=0):
    cfg = ServerConfig(slots, cast_blocks_per_sm, hbm_budget_bytes, small_rays, incremental, 0)
    s = ctypes.c_void_p()
    _check(load().rc_server_create(ctypes.byref(params), ctypes.byref(cfg), ctypes.byref(s)))
    return s.value


def rc_server_submit(s, part_key, V, F, n):
    """Queue an analysis of host mesh (numpy float32 [nV,3], int32 [T,3])."""
    import numpy as np
    V = np.ascontiguousarray(V, np.float32)
    F = np.ascontiguousarray(F, np.int32)
    rid = ctypes.c_int64()
    _check(load().rc_server_submit(ctypes.c_void_p(s), ctypes.c_uint64(part_key), _hptr(V), V.shape[0], _hptr(F),
                                   F.shape[0], n, ctypes.byref(rid)))
    return rid.value


def rc_server_wait(s, req_id, timeout_s=60.0):
    out = RequestResult()
    _check(load().rc_server_wait(ctypes.c_void_p(s), req_id, float(timeout_s), ctypes.byref(out)))
    return out


def rc_server_read_bits(s, part_key, n, n_dirs):
    import numpy as np
    bits = np.zeros((n, (n_dirs + 31) // 32), np.uint32)
    cnt = np.zeros(n, np.int32)
    _check(load().rc_server_read_bits(ctypes.c_void_p(s), ctypes.c_uint64(part_key), _hptr(bits), bits.size,
                                      _hptr(cnt), n))
    return bits, cnt


def rc_server_get_stats(s):
    out = ServerStats()
    _check(load().rc_server_get_stats(ctypes.c_void_p(s), ctypes.byref(out)))
    return out


def rc_server_destroy(s):
    _check(load().rc_server_destroy(ctypes.c_void_p(s)))


def rc_bvh_validate(h, stream=None):
    """Index checks of a built tree; returns a dict of violation counts
    (all zero for a sound tree) and the number of 4-wide nodes reached."""
    import numpy as np
    out = np.zeros(6, np.int64)
    _check(load().rc_bvh_validate(ctypes.c_void_p(h), out.ctypes.data_as(ctypes.c_void_p), _stream(stream)))
    keys = ("wide_child", "wide_leaf", "wide_box", "binary_child", "tri_face", "nodes_seen")
    return {k: int(v) for k, v in zip(keys, out)}


def rc_launch_count():
    return int(load().rc_launch_count())


def rc_stream_status(stream=None):
    """Wait for `stream` (default: the current torch stream) and raise
    RcError if asynchronous work queued on it failed."""
    _check(load().rc_stream_status(_stream(stream)))


class Bvh:
    """Owning wrapper of an ``rc_bvh`` handle (destroyed on ``close``)."""

    def __init__(self, V, F, stream=None, builder=None):
        self.h = rc_build_bvh(V, F, stream) if builder is None else rc_build_bvh_ex(V, F, builder, stream)
        self.T = F.shape[0]

    def close(self):
        if self.h:
            rc_destroy_bvh(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
