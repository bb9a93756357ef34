"""ctypes binding of libhpm (include/hpm.h): argument marshalling only.

Every step of the solve runs in the CUDA library. Torch tensors are accepted
for device buffers and passed as raw pointers with the current CUDA stream.
Importing this module fails loudly if the compiled library is missing.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libhpm.so")

HPM_OK = 0
STATUS = {0: "HPM_OK", -1: "HPM_ERR_INVALID_ARG", -2: "HPM_ERR_OUT_OF_DOMAIN", -3: "HPM_ERR_OOM",
          -4: "HPM_ERR_CUDA", -5: "HPM_ERR_TIMEOUT", -6: "HPM_ERR_NOT_BUILT", -7: "HPM_ERR_BUSY",
          -8: "HPM_ERR_UNSUPPORTED"}
HPM_GREEN_PLUMMER, HPM_GREEN_NEWTON, HPM_GREEN_YUKAWA, HPM_GREEN_USER = 0, 1, 2, 3
HPM_FLAG_TIMINGS = 1
HPM_FLAG_GENERIC_M2L = 2
HPM_FLAG_XTRANSFORM_M2L = 4
HPM_FLAG_FFT_M2L = 8
HPM_FLAG_EXTENDED_GRIDLET = 16
HPM_STAGE_MASSES, HPM_STAGE_M2L, HPM_STAGE_LOCAL = 1, 2, 3

# Every symbol include/hpm.h declares, with its ctypes signature.
_vp, _i32, _i64, _f64 = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_double


class hpm_domain(ctypes.Structure):
    _fields_ = [("origin", ctypes.c_double * 3), ("side", ctypes.c_double)]


USER_G = ctypes.CFUNCTYPE(ctypes.c_double, ctypes.c_double, ctypes.c_void_p)   # double (*)(double r, void *ctx)


class hpm_green(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int), ("eps", ctypes.c_double), ("lam", ctypes.c_double),
                ("user_g", USER_G), ("ctx", ctypes.c_void_p)]


class Green:
    """A Green function descriptor (hpm_green): Plummer (default), Newton, Yukawa, or a user
    kernel given as a C function pointer ``double g(double r, void *ctx)`` (a ctypes
    function from a shared library, or a ``USER_G`` wrapping a Python callable; the library
    calls it only while a plan is made)."""

    def __init__(self, kind=HPM_GREEN_PLUMMER, eps=0.0, lam=0.0, user_g=None, ctx=None):
        self.kind, self.eps, self.lam, self.ctx = kind, float(eps), float(lam), ctx
        self.user_g = None if user_g is None else ctypes.cast(user_g, USER_G)
        self._keep = (user_g, ctx)

    @classmethod
    def plummer(cls, eps):
        return cls(HPM_GREEN_PLUMMER, eps)

    @classmethod
    def newton(cls):
        return cls(HPM_GREEN_NEWTON)

    @classmethod
    def yukawa(cls, lam, eps=0.0):
        return cls(HPM_GREEN_YUKAWA, eps, lam)

    @classmethod
    def user(cls, fn, ctx=None):
        return cls(HPM_GREEN_USER, user_g=fn, ctx=ctx)

    def struct(self) -> hpm_green:
        g = hpm_green(self.kind, self.eps, self.lam)
        if self.user_g is not None:
            g.user_g = self.user_g
        if self.ctx is not None:
            g.ctx = ctypes.cast(self.ctx, ctypes.c_void_p)
        return g


def _green(eps, green) -> hpm_green:
    return (green if green is not None else Green.plummer(eps)).struct()


class hpm_plan_opts(ctypes.Structure):
    _fields_ = [("leaf_max", ctypes.c_int), ("flags", ctypes.c_int)]


class hpm_problem(ctypes.Structure):
    _fields_ = [("d_pos", ctypes.c_void_p), ("d_mass", ctypes.c_void_p), ("n", ctypes.c_int64),
                ("d_phi", ctypes.c_void_p), ("d_acc", ctypes.c_void_p)]


class hpm_server_opts(ctypes.Structure):
    _fields_ = [("dom", hpm_domain), ("max_depth", ctypes.c_int), ("gridlet_order", ctypes.c_int),
                ("green", hpm_green), ("leaf_max", ctypes.c_int), ("workers", ctypes.c_int),
                ("max_batch", ctypes.c_int), ("hbm_budget_bytes", ctypes.c_int64),
                ("bytes_per_particle", ctypes.c_double), ("max_batch_particles", ctypes.c_int64)]


class hpm_request(ctypes.Structure):
    _fields_ = [("pos", ctypes.c_void_p), ("mass", ctypes.c_void_p), ("n", ctypes.c_int64),
                ("phi", ctypes.c_void_p), ("acc", ctypes.c_void_p)]


class hpm_server_stats(ctypes.Structure):
    _fields_ = [(k, ctypes.c_int64) for k in ("submitted", "completed", "rejected", "cancelled", "failed",
                                              "batches", "queued", "in_flight_bytes", "particles")] + \
               [(k, ctypes.c_double) for k in ("p50_ms", "p99_ms", "mean_ms", "particles_per_s",
                                               "bytes_per_particle")]


class hpm_lists_info(ctypes.Structure):
    _fields_ = [("n_particles", ctypes.c_int64), ("n_cells", ctypes.c_int64), ("n_targets", ctypes.c_int64),
                ("n_leaves", ctypes.c_int64), ("n_boxes", ctypes.c_int64), ("max_depth", ctypes.c_int),
                ("depth_reached", ctypes.c_int)]


class hpm_stats(ctypes.Structure):
    _fields_ = [(k, ctypes.c_float) for k in ("ms_tree", "ms_p2g", "ms_m2m", "ms_m2l", "ms_l2l", "ms_g2p",
                                              "ms_p2p", "ms_total")] + \
               [("launches", ctypes.c_int64), ("m2l_launches", ctypes.c_int64), ("m2l_targets", ctypes.c_int64),
                ("ms_m2l_kernel", ctypes.c_float), ("m2l_parents", ctypes.c_int64), ("p2p_pairs", ctypes.c_int64),
                ("table_bytes", ctypes.c_int64), ("work_bytes", ctypes.c_int64)]


class hpm_tuning(ctypes.Structure):
    _fields_ = [("level_blocks_per_sm", ctypes.c_int), ("gridlet_warps", ctypes.c_int),
                ("m2l_ctas_per_sm", ctypes.c_int), ("m2l_block_order", ctypes.c_int),
                ("m2l_tile_parents", ctypes.c_int)]


class hpm_alu_peaks(ctypes.Structure):
    _fields_ = [(k, ctypes.c_double) for k in ("fp32_tflops", "fp64_tflops", "rsqrt_gops", "ms_fp32", "ms_fp64",
                                               "ms_rsqrt")] + [("sm_count", ctypes.c_int)]


SIGNATURES = {
    "hpm_plan": ([ctypes.POINTER(hpm_domain), _i32, _i32, ctypes.POINTER(hpm_green),
                  ctypes.POINTER(hpm_plan_opts), ctypes.POINTER(_vp)], _i32),
    "hpm_build_tree": ([_vp, _vp, _i64, _vp], _i32),
    "hpm_solve": ([_vp, _vp, _vp, _vp, _vp, _vp], _i32),
    "hpm_solve_host": ([_vp, _vp, _vp, _i64, _vp, _vp, _vp], _i32),
    "hpm_build_tree_batch": ([_vp, _vp, _vp, _i32, _vp], _i32),
    "hpm_solve_batch": ([_vp, ctypes.POINTER(hpm_problem), _i32, _vp], _i32),
    "hpm_get_lists_info": ([_vp, ctypes.POINTER(hpm_lists_info)], _i32),
    "hpm_get_lists": ([_vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp], _i32),
    "hpm_get_stats": ([_vp, ctypes.POINTER(hpm_stats)], _i32),
    "hpm_get_boxes": ([_vp, _vp, _vp, _vp], _i32),
    "hpm_get_stage": ([_vp, _i32, _vp, _i64], _i32),
    "hpm_sort_particles_static": ([ctypes.POINTER(hpm_domain), _i32, _vp, _i64, _vp, _vp, _vp], _i32),
    "hpm_server_create": ([ctypes.POINTER(hpm_server_opts), ctypes.POINTER(_vp)], _i32),
    "hpm_server_submit": ([_vp, ctypes.POINTER(hpm_request), ctypes.POINTER(ctypes.c_uint64)], _i32),
    "hpm_server_poll": ([_vp, ctypes.c_uint64, ctypes.POINTER(_i32), ctypes.POINTER(_f64)], _i32),
    "hpm_server_wait": ([_vp, ctypes.c_uint64, _i32, ctypes.POINTER(_f64)], _i32),
    "hpm_server_cancel": ([_vp, ctypes.c_uint64], _i32),
    "hpm_server_get_stats": ([_vp, ctypes.POINTER(hpm_server_stats)], _i32),
    "hpm_server_reset_stats": ([_vp], _i32),
    "hpm_server_destroy": ([_vp], _i32),
    "hpm_set_tuning": ([_vp, ctypes.POINTER(hpm_tuning)], _i32),
    "hpm_get_tuning": ([_vp, ctypes.POINTER(hpm_tuning)], _i32),
    "hpm_tune": ([_vp, _vp, _vp, _i64, _vp, ctypes.POINTER(hpm_tuning)], _i32),
    "hpm_test_stall": ([_vp, _i32, ctypes.c_longlong], _i32),
    "hpm_measure_alu_peaks": ([ctypes.POINTER(hpm_alu_peaks), _vp], _i32),
    "hpm_check_conversions": ([_vp, _i64, _vp, _i64, ctypes.POINTER(ctypes.c_int64), _vp], _i32),
    "hpm_destroy": ([_vp], _i32),
    "hpm_status_str": ([_i32], ctypes.c_char_p),
    "hpm_last_cuda_error": ([], ctypes.c_char_p),
}


class HpmError(RuntimeError):
    def __init__(self, call: str, status: int):
        self.status = status
        detail = ""
        if status == -4 and _lib is not None:
            detail = " (" + _lib.hpm_last_cuda_error().decode() + ")"
        super().__init__(f"{call}: {STATUS.get(status, status)}{detail}")


_lib = None


def load(path: str = LIB_PATH) -> ctypes.CDLL:
    """Loads libhpm; raises if it has not been built (no fallback exists)."""
    global _lib
    if _lib is None:
        if not os.path.exists(path):
            raise RuntimeError(f"libhpm is not built ({path}); run __graft_entry__.build()")
        L = ctypes.CDLL(path)
        for name, (args, res) in SIGNATURES.items():
            fn = getattr(L, name)
            fn.argtypes = args
            fn.restype = res
        _lib = L
    return _lib


def _check(call: str, status: int):
    if status != HPM_OK:
        raise HpmError(call, status)


def _ptr(t) -> int:
    """Device pointer of a torch tensor (or an int address); None -> NULL."""
    if t is None:
        return None
    if isinstance(t, int):
        return t
    return t.data_ptr()


def _stream(stream) -> int:
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def hpm_plan(origin=(0.0, 0.0, 0.0), side=1.0, max_depth=3, gridlet_order=4, eps=0.0, leaf_max=0,
             flags=0, green: Green | None = None) -> int:
    """A plan (hpm_plan). The kernel is `green` if given, else Plummer with softening eps."""
    L = load()
    dom = hpm_domain((ctypes.c_double * 3)(*origin), side)
    green = _green(eps, green)
    opts = hpm_plan_opts(leaf_max, flags)
    out = _vp()
    _check("hpm_plan", L.hpm_plan(ctypes.byref(dom), max_depth, gridlet_order, ctypes.byref(green),
                                  ctypes.byref(opts), ctypes.byref(out)))
    return out.value


def hpm_build_tree(plan: int, d_pos, n: int, stream=None):
    _check("hpm_build_tree", load().hpm_build_tree(plan, _ptr(d_pos), n, _stream(stream)))


def hpm_solve(plan: int, d_pos, d_mass, d_phi, d_acc, stream=None):
    _check("hpm_solve", load().hpm_solve(plan, _ptr(d_pos), _ptr(d_mass), _ptr(d_phi), _ptr(d_acc),
                                         _stream(stream)))


def hpm_build_tree_batch(plan: int, d_pos, offsets, stream=None):
    """Trees of P problems packed in d_pos; offsets: P + 1 int64 (host)."""
    off = np.ascontiguousarray(offsets, dtype=np.int64)
    _check("hpm_build_tree_batch", load().hpm_build_tree_batch(plan, _ptr(d_pos), off.ctypes.data, off.shape[0] - 1,
                                                               _stream(stream)))


def hpm_solve_batch(plan: int, problems, stream=None):
    """problems: sequence of (d_pos, d_mass, d_phi, d_acc) torch tensors (phi/acc may be None)."""
    arr = (hpm_problem * len(problems))()
    for k, (pos, mass, phi, acc) in enumerate(problems):
        arr[k] = hpm_problem(_ptr(pos), _ptr(mass), int(pos.shape[0]), _ptr(phi), _ptr(acc))
    _check("hpm_solve_batch", load().hpm_solve_batch(plan, arr, len(problems), _stream(stream)))


def hpm_solve_host(plan: int, h_pos: np.ndarray, h_mass: np.ndarray, h_phi: np.ndarray = None,
                   h_acc: np.ndarray = None, stream=None):
    """Host-memory solve: numpy (or pinned-memory) arrays in and out."""
    n = int(h_pos.shape[0])
    assert h_pos.dtype == np.float64 and h_pos.flags["C_CONTIGUOUS"]
    assert h_mass.dtype == np.float64 and h_mass.flags["C_CONTIGUOUS"]
    for a in (h_phi, h_acc):
        assert a is None or (a.dtype == np.float32 and a.flags["C_CONTIGUOUS"])
    addr = lambda a: None if a is None else a.ctypes.data
    _check("hpm_solve_host", load().hpm_solve_host(plan, addr(h_pos), addr(h_mass), n, addr(h_phi),
                                                   addr(h_acc), _stream(stream)))


def hpm_get_lists_info(plan: int) -> dict:
    info = hpm_lists_info()
    _check("hpm_get_lists_info", load().hpm_get_lists_info(plan, ctypes.byref(info)))
    return {k: getattr(info, k) for k, _ in hpm_lists_info._fields_}


def hpm_get_lists(plan: int) -> dict:
    info = hpm_get_lists_info(plan)
    nc, nt, nl, n = info["n_cells"], info["n_targets"], info["n_leaves"], info["n_particles"]
    out = {"level": np.zeros(nc, np.int32), "key": np.zeros(nc, np.uint64), "begin": np.zeros(nc, np.int64),
           "end": np.zeros(nc, np.int64), "leaf": np.zeros(nc, np.uint8), "iz": np.zeros((nt, 4), np.uint64),
           "near": np.zeros(nl, np.uint32), "perm": np.zeros(n, np.int64)}
    a = lambda k: out[k].ctypes.data if out[k].size else None
    _check("hpm_get_lists", load().hpm_get_lists(plan, a("level"), a("key"), a("begin"), a("end"), a("leaf"),
                                                 a("iz"), a("near"), a("perm")))
    return out


def hpm_get_boxes(plan: int) -> dict:
    nb = hpm_get_lists_info(plan)["n_boxes"]
    out = {"level": np.zeros(nb, np.int32), "key": np.zeros(nb, np.uint64), "flags": np.zeros(nb, np.uint8)}
    a = lambda k: out[k].ctypes.data if nb else None
    _check("hpm_get_boxes", load().hpm_get_boxes(plan, a("level"), a("key"), a("flags")))
    return out


def hpm_get_stage(plan: int, stage: int, ng: int, ng_target: int | None = None) -> np.ndarray:
    """Stage buffer as float32: (rows, Ng^3) for masses; (targets, Nt^3 + 1) otherwise
    (values then the constant), Nt = ng_target (Ng + 2 for widened target gridlets)."""
    info = hpm_get_lists_info(plan)
    m3 = ng ** 3 if stage == HPM_STAGE_MASSES else (ng_target or ng) ** 3
    if stage == HPM_STAGE_MASSES:
        boxes = hpm_get_boxes(plan)
        rows = int(np.sum(boxes["level"] >= 2))
        out = np.zeros(max(rows * m3, 1), np.float32)
        _check("hpm_get_stage", load().hpm_get_stage(plan, stage, out.ctypes.data, out.size))
        return out[:rows * m3].reshape(rows, m3)
    nt = info["n_targets"]
    out = np.zeros(max(nt * (m3 + 1), 1), np.float32)
    _check("hpm_get_stage", load().hpm_get_stage(plan, stage, out.ctypes.data, out.size))
    vals = out[:nt * m3].reshape(nt, m3)
    const = out[nt * m3:nt * m3 + nt]
    return np.concatenate([vals, const[:, None]], axis=1)


def hpm_set_tuning(plan: int, level_blocks_per_sm=0, gridlet_warps=0, m2l_ctas_per_sm=0, m2l_block_order=0,
                   m2l_tile_parents=0):
    t = hpm_tuning(level_blocks_per_sm, gridlet_warps, m2l_ctas_per_sm, m2l_block_order, m2l_tile_parents)
    _check("hpm_set_tuning", load().hpm_set_tuning(plan, ctypes.byref(t)))


def hpm_get_tuning(plan: int) -> dict:
    t = hpm_tuning()
    _check("hpm_get_tuning", load().hpm_get_tuning(plan, ctypes.byref(t)))
    return {k: getattr(t, k) for k, _ in hpm_tuning._fields_}


def hpm_tune(plan: int, d_pos, d_mass, stream=None) -> dict:
    """Autotunes the plan's launch shapes on this input; returns the chosen shapes."""
    t = hpm_tuning()
    _check("hpm_tune", load().hpm_tune(plan, _ptr(d_pos), _ptr(d_mass), int(d_pos.shape[0]), _stream(stream),
                                       ctypes.byref(t)))
    return {k: getattr(t, k) for k, _ in hpm_tuning._fields_}


def hpm_test_stall(plan: int, on: bool, wait_limit_cycles: int = 0):
    """Failure test hook: the next solves' source-to-target kernel waits on a barrier that
    nothing arrives at (bounded by wait_limit_cycles), gives up and records a timeout."""
    _check("hpm_test_stall", load().hpm_test_stall(plan, 1 if on else 0, int(wait_limit_cycles)))


def hpm_get_stats(plan: int) -> dict:
    st = hpm_stats()
    _check("hpm_get_stats", load().hpm_get_stats(plan, ctypes.byref(st)))
    return {k: getattr(st, k) for k, _ in hpm_stats._fields_}


def _addr(a):
    """Address of a torch tensor or numpy array (host or device); None -> NULL."""
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        assert a.flags["C_CONTIGUOUS"]
        return a.ctypes.data
    return a.data_ptr()


class Server:
    """Continuous-batching solver service (hpm_server_*). Buffers of a request may be
    host numpy arrays or device tensors and must stay alive until it is done."""

    def __init__(self, max_depth=12, gridlet_order=4, eps=1e-4, leaf_max=32, workers=2, max_batch=64,
                 hbm_budget_bytes=150 << 30, origin=(0.0, 0.0, 0.0), side=1.0, green: Green | None = None,
                 bytes_per_particle=0.0, max_batch_particles=0):
        L = load()
        opts = hpm_server_opts(hpm_domain((ctypes.c_double * 3)(*origin), side), max_depth, gridlet_order,
                               _green(eps, green), leaf_max, workers, max_batch, hbm_budget_bytes,
                               bytes_per_particle, max_batch_particles)
        h = _vp()
        _check("hpm_server_create", L.hpm_server_create(ctypes.byref(opts), ctypes.byref(h)))
        self.h = h.value
        self._keep = {}

    def submit(self, pos, mass, phi, acc) -> int:
        req = hpm_request(_addr(pos), _addr(mass), int(pos.shape[0]), _addr(phi), _addr(acc))
        t = ctypes.c_uint64()
        _check("hpm_server_submit", load().hpm_server_submit(self.h, ctypes.byref(req), ctypes.byref(t)))
        self._keep[t.value] = (pos, mass, phi, acc)
        return t.value

    def poll(self, ticket):
        d, lat = _i32(), _f64()
        _check("hpm_server_poll", load().hpm_server_poll(self.h, ticket, ctypes.byref(d), ctypes.byref(lat)))
        return d.value, lat.value

    def wait(self, ticket, timeout_ms=60000):
        lat = _f64()
        _check("hpm_server_wait", load().hpm_server_wait(self.h, ticket, timeout_ms, ctypes.byref(lat)))
        self._keep.pop(ticket, None)
        return lat.value

    def cancel(self, ticket):
        _check("hpm_server_cancel", load().hpm_server_cancel(self.h, ticket))

    def stats(self) -> dict:
        st = hpm_server_stats()
        _check("hpm_server_get_stats", load().hpm_server_get_stats(self.h, ctypes.byref(st)))
        return {k: getattr(st, k) for k, _ in hpm_server_stats._fields_}

    def reset_stats(self):
        _check("hpm_server_reset_stats", load().hpm_server_reset_stats(self.h))

    def close(self):
        if self.h:
            _check("hpm_server_destroy", load().hpm_server_destroy(self.h))
            self.h = 0

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


HPM_STATIC_SORT_MAX_N = 1048576


def hpm_sort_particles_static(d_pos, n: int, d_keys, d_perm, max_depth: int, origin=(0.0, 0.0, 0.0),
                              side=1.0, stream=None):
    """Morton keys and stable sort into caller buffers, no allocation (scratch is static)."""
    dom = hpm_domain((ctypes.c_double * 3)(*origin), side)
    _check("hpm_sort_particles_static",
           load().hpm_sort_particles_static(ctypes.byref(dom), max_depth, _ptr(d_pos), n, _ptr(d_keys),
                                            _ptr(d_perm), _stream(stream)))


def hpm_destroy(plan: int):
    _check("hpm_destroy", load().hpm_destroy(plan))


def hpm_status_str(status: int) -> str:
    return load().hpm_status_str(status).decode()


class Solver:
    """Convenience owner of one plan: build + solve on torch device tensors."""

    def __init__(self, max_depth, gridlet_order=4, eps=0.0, leaf_max=0, origin=(0.0, 0.0, 0.0), side=1.0,
                 timings=False, flags=0, green: Green | None = None):
        self.ng = gridlet_order
        self.ng_target = gridlet_order + (2 if flags & HPM_FLAG_EXTENDED_GRIDLET else 0)
        self.plan = hpm_plan(origin, side, max_depth, gridlet_order, eps, leaf_max,
                             (HPM_FLAG_TIMINGS if timings else 0) | flags, green)

    def __call__(self, pos, mass, phi=None, acc=None, stream=None):
        import torch
        n = pos.shape[0]
        if phi is None:
            phi = torch.empty(n, dtype=torch.float32, device=pos.device)
        if acc is None:
            acc = torch.empty((n, 3), dtype=torch.float32, device=pos.device)
        hpm_build_tree(self.plan, pos, n, stream)
        hpm_solve(self.plan, pos, mass, phi, acc, stream)
        return phi, acc

    def lists(self):
        return hpm_get_lists(self.plan)

    def boxes(self):
        return hpm_get_boxes(self.plan)

    def stage(self, which):
        return hpm_get_stage(self.plan, which, self.ng, self.ng_target)

    def close(self):
        if self.plan:
            hpm_destroy(self.plan)
            self.plan = 0

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def hpm_measure_alu_peaks(stream=None) -> dict:
    """Measured FP32 / FP64 FMA and rsqrt rates of the current device (see include/hpm.h)."""
    out = hpm_alu_peaks()
    _check("hpm_measure_alu_peaks", load().hpm_measure_alu_peaks(ctypes.byref(out), _stream(stream)))
    return {k: getattr(out, k) for k, _ in hpm_alu_peaks._fields_}


def hpm_check_conversions(d, f, stream=None) -> int:
    """Bits in which the library's integer-unit float <-> double conversions differ from the
    hardware's, over device tensors d (float64) and f (float32): the count of such inputs."""
    out = ctypes.c_int64(0)
    _check("hpm_check_conversions", load().hpm_check_conversions(_ptr(d), int(d.numel()), _ptr(f), int(f.numel()),
                                                                 ctypes.byref(out), _stream(stream)))
    return int(out.value)
