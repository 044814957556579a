"""Thin ctypes binding of libzbus (include/zbus.h).

Argument marshalling only: every step of the solve runs in the library's CUDA
kernels.  Device buffers are torch tensors (complex128 for complex arrays),
streams are torch.cuda streams.  If libzbus.so is missing or cannot be loaded
every call raises; there is no fallback.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
# ZBUS_LIB selects another build of the library (the checked build)
LIB_PATH = os.environ.get("ZBUS_LIB") or os.path.join(_HERE, "libzbus.so")

ZBUS_OK = 0
STATUS = {0: "ZBUS_OK", 1: "ZBUS_ERR_ARG", 2: "ZBUS_ERR_SINGULAR", 3: "ZBUS_ERR_OOM",
          4: "ZBUS_ERR_CUDA", 5: "ZBUS_ERR_TIMEOUT", 6: "ZBUS_ERR_DEVICE",
          7: "ZBUS_ERR_UNSUPPORTED", 8: "ZBUS_ERR_SOURCE"}
PRECISION = {"fp64": 0, "bf16x2": 1, "fp16_scaled": 2, "tree": 3}
RULE = {"maxabs": 0, "summag": 1}


class ZbusError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{STATUS.get(status, status)}: {message}")
        self.status = status


class zbus_solve_opts(C.Structure):
    _fields_ = [("precision", C.c_int32), ("conv_rule", C.c_int32),
                ("mismatch_tol", C.c_double), ("max_correction", C.c_int32),
                ("profile", C.c_int32), ("fp32_start", C.c_int32), ("reserved_i", C.c_int32),
                ("reserved", C.c_double * 3)]


class zbus_batch_item(C.Structure):
    _fields_ = [("net", C.c_void_p), ("B", C.c_int64), ("S_wye", C.c_void_p),
                ("S_delta", C.c_void_p), ("V_init", C.c_void_p), ("V_out", C.c_void_p),
                ("iters", C.c_void_p), ("converged", C.c_void_p)]


class zbus_request(C.Structure):
    _fields_ = [("feeder", C.c_int32), ("B", C.c_int64), ("S_wye", C.c_void_p),
                ("S_delta", C.c_void_p), ("V_out", C.c_void_p), ("iters", C.c_void_p),
                ("converged", C.c_void_p), ("warm_start", C.c_int32), ("reserved0", C.c_int32),
                ("tag", C.c_uint64), ("t_arrival", C.c_double)]


class zbus_request_result(C.Structure):
    _fields_ = [("status", C.c_int), ("n_converged", C.c_int32), ("max_iters", C.c_int32),
                ("operands_formed", C.c_int32), ("t_admit", C.c_double), ("t_done", C.c_double),
                ("V", C.c_void_p), ("iters", C.c_void_p), ("converged", C.c_void_p)]


class zbus_serve_config(C.Structure):
    _fields_ = [("hbm_budget_bytes", C.c_uint64), ("max_slots", C.c_int32),
                ("precision", C.c_int32), ("conv_rule", C.c_int32), ("max_iter", C.c_int32),
                ("tol", C.c_double), ("mismatch_tol", C.c_double),
                ("max_admit_per_sweep", C.c_int32), ("max_correction", C.c_int32),
                ("fp32_start", C.c_int32)]


class zbus_nr_opts(C.Structure):
    _fields_ = [("gmres_restart", C.c_int32), ("gmres_max_restarts", C.c_int32),
                ("gmres_tol", C.c_double), ("precision", C.c_int32), ("reserved0", C.c_int32),
                ("reserved", C.c_double * 3)]


NR_PRECISION = {"fp64": 0, "mixed": 1}


SOURCE_FN = C.CFUNCTYPE(C.c_int32, C.c_void_p, C.c_double, C.POINTER(zbus_request))
SINK_FN = C.CFUNCTYPE(None, C.c_void_p, C.POINTER(zbus_request), C.POINTER(zbus_request_result))

_lib = None

_P = C.c_void_p
_SIGS = {
    "zbus_solve_opts_default": (None, [C.POINTER(zbus_solve_opts)]),
    "zbus_network_create": (C.c_int, [C.c_int32, C.c_int64, _P, _P, _P, _P, _P, _P,
                                      C.POINTER(_P)]),
    "zbus_network_create_phased": (C.c_int, [C.c_int32, C.c_int64, _P, _P, _P, _P, _P, _P, _P,
                                             C.POINTER(_P)]),
    "zbus_network_destroy": (None, [_P]),
    "zbus_network_size": (C.c_int32, [_P]),
    "zbus_network_get_z": (C.c_int, [_P, _P, _P, _P]),
    "zbus_network_reserve": (C.c_int, [_P, C.c_int64, C.c_int32]),
    "zbus_solve": (C.c_int, [_P, C.c_int64, _P, _P, _P, C.c_double, C.c_int32,
                             C.POINTER(zbus_solve_opts), _P, _P, _P, _P]),
    "zbus_power_mismatch": (C.c_int, [_P, C.c_int64, _P, _P, _P, _P, _P]),
    "zbus_last_profile": (C.c_int, [_P, C.c_int32, _P, _P, _P]),
    "zbus_solve_noalloc": (C.c_int, [_P, C.c_int64, _P, _P, _P, C.c_double, C.c_int32,
                                     C.c_int32, _P, _P, _P, _P]),
    "zbus_solve_batched": (C.c_int, [C.POINTER(zbus_batch_item), C.c_int32, C.c_double,
                                     C.c_int32, C.POINTER(zbus_solve_opts), _P]),
    "zbus_autotune": (C.c_int, [C.POINTER(zbus_batch_item), C.c_int32,
                                C.POINTER(zbus_solve_opts), C.c_double, C.c_int32, C.c_int32,
                                _P, C.POINTER(C.c_int32), C.POINTER(C.c_int32)]),
    "zbus_tune_variants": (C.c_int32, [C.c_int32, C.POINTER(C.c_int32), C.POINTER(C.c_int32),
                                       C.c_int32]),
    "zbus_tune_set": (C.c_int, [C.c_int32, C.c_int32, C.c_int64, C.c_int32, C.c_int32]),
    "zbus_serve": (C.c_int, [C.POINTER(zbus_serve_config), C.POINTER(C.c_void_p), C.c_int32,
                             SOURCE_FN, SINK_FN, C.c_void_p, C.c_void_p]),
    "zbus_last_device_status": (C.c_int, [_P, _P]),
    "zbus_probe_fp64_rate": (C.c_int, [C.POINTER(C.c_double), C.POINTER(C.c_float), _P]),
    "zbus_checked_set_wait": (C.c_int, [C.c_uint64]),
    "zbus_serve_footprint": (C.c_int, [_P, C.c_int32, C.POINTER(C.c_uint64),
                                       C.POINTER(C.c_uint64), C.POINTER(C.c_uint64)]),
    "zbus_solve_adjoint": (C.c_int, [_P, C.c_int64, _P, _P, _P, _P, C.c_double, C.c_int32,
                                     C.POINTER(zbus_solve_opts), _P, _P, _P, _P, _P]),
    "zbus_nr_opts_default": (None, [C.POINTER(zbus_nr_opts)]),
    "zbus_nr_network_create": (C.c_int, [C.c_int32, C.c_int64, _P, _P, _P, _P, _P, C.c_double,
                                         _P, C.POINTER(_P)]),
    "zbus_nr_network_destroy": (None, [_P]),
    "zbus_nr_network_info": (C.c_int, [_P, C.POINTER(C.c_int32), C.POINTER(C.c_int32),
                                       C.POINTER(C.c_int64), C.POINTER(C.c_int32)]),
    "zbus_nr_solve": (C.c_int, [_P, C.c_int64, _P, _P, C.c_double, C.c_int32,
                                C.POINTER(zbus_nr_opts), _P, _P, _P, _P, _P]),
    "zbus_checked_status": (C.c_int32, [C.POINTER(C.c_uint32)]),
    "zbus_status_string": (C.c_char_p, [C.c_int]),
    "zbus_last_error": (C.c_char_p, []),
}


def lib():
    """The loaded libzbus (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"libzbus.so not found at {LIB_PATH}; build it with "
                               "paper_2605_14103_gb300.build.build()")
        L = C.CDLL(LIB_PATH)
        for name, (res, args) in _SIGS.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def _check(status: int):
    if status != ZBUS_OK:
        msg = lib().zbus_last_error().decode(errors="replace")
        raise ZbusError(status, msg)


def _stream(stream) -> int | None:
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return s.cuda_stream or None


def _dptr(t, name, dtype=None, shape=None, host_ok=False):
    """Pointer of a contiguous tensor (None passes through): CUDA memory, or
    host memory where the call accepts it (host_ok)."""
    if t is None:
        return None
    if not t.is_cuda and not host_ok:
        raise ValueError(f"{name} must be a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if dtype is not None and t.dtype != dtype:
        raise ValueError(f"{name} must have dtype {dtype}, got {t.dtype}")
    if shape is not None and tuple(t.shape) != tuple(shape):
        raise ValueError(f"{name} must have shape {tuple(shape)}, got {tuple(t.shape)}")
    return t.data_ptr()


# ---------------------------------------------------------------------------
# Functions with the C ABI's names.
# ---------------------------------------------------------------------------

def zbus_solve_opts_default() -> zbus_solve_opts:
    o = zbus_solve_opts()
    lib().zbus_solve_opts_default(C.byref(o))
    return o


def zbus_network_create(n_total, row, col, val, slack_idx, v_slack, stream=None,
                        bus_phase=None) -> int:
    """Host COO (numpy) -> network handle (an integer).  With bus_phase
    (int32[n_total], 3 * bus + phase of every global index) the network may
    have partial-phase buses (zbus_network_create_phased)."""
    row = np.ascontiguousarray(row, dtype=np.int32)
    col = np.ascontiguousarray(col, dtype=np.int32)
    val = np.ascontiguousarray(val, dtype=np.complex128)
    sl = np.ascontiguousarray(slack_idx, dtype=np.int32)
    vs = np.ascontiguousarray(v_slack, dtype=np.complex128)
    if not (row.shape == col.shape == val.shape) or sl.shape != (3,) or vs.shape != (3,):
        raise ValueError("row/col/val must have equal length; slack_idx and v_slack 3 entries")
    h = _P()
    if bus_phase is None:
        _check(lib().zbus_network_create(int(n_total), int(row.size), row.ctypes.data,
                                         col.ctypes.data, val.ctypes.data, sl.ctypes.data,
                                         vs.ctypes.data, _stream(stream), C.byref(h)))
    else:
        bp = np.ascontiguousarray(bus_phase, dtype=np.int32)
        if bp.shape != (int(n_total),):
            raise ValueError("bus_phase must have n_total entries")
        _check(lib().zbus_network_create_phased(int(n_total), int(row.size), row.ctypes.data,
                                                col.ctypes.data, val.ctypes.data,
                                                sl.ctypes.data, vs.ctypes.data, bp.ctypes.data,
                                                _stream(stream), C.byref(h)))
    return h.value


def zbus_network_destroy(h):
    if h:
        lib().zbus_network_destroy(h)


def zbus_network_size(h) -> int:
    return int(lib().zbus_network_size(h))


def zbus_network_get_z(h, Z_out=None, w_out=None, stream=None):
    import torch
    n = zbus_network_size(h)
    _check(lib().zbus_network_get_z(h, _dptr(Z_out, "Z_out", torch.complex128, (n, n)),
                                    _dptr(w_out, "w_out", torch.complex128, (n,)),
                                    _stream(stream)))


def zbus_network_reserve(h, B, precision="fp64"):
    _check(lib().zbus_network_reserve(h, int(B), PRECISION[precision]))


def zbus_solve(h, S_wye, S_delta, V_init, tol, max_iter, opts, V_out, iters, converged,
               stream=None):
    import torch
    n = zbus_network_size(h)
    B = V_out.shape[0]
    c128 = torch.complex128
    # all buffers on the device, or all in host memory (then the library stages
    # them through the device, overlapping the copies with the sweeps)
    _check(lib().zbus_solve(
        h, int(B), _dptr(S_wye, "S_wye", c128, (B, n), True),
        _dptr(S_delta, "S_delta", c128, (B, n), True),
        _dptr(V_init, "V_init", c128, (B, n), True), float(tol), int(max_iter),
        C.byref(opts) if opts is not None else None,
        _dptr(V_out, "V_out", c128, (B, n), True), _dptr(iters, "iters", torch.int32, (B,), True),
        _dptr(converged, "converged", torch.uint8, (B,), True), _stream(stream)))


def zbus_last_device_status(h, stream=None) -> int:
    """ZBUS_OK (0), or the status of an error the device detected in the last solve."""
    return int(lib().zbus_last_device_status(h, _stream(stream)))


def zbus_serve_footprint(h, precision="fp16_scaled"):
    """(operand bytes while cached, extra bytes while forming, bytes per slot)."""
    a, b, c = C.c_uint64(0), C.c_uint64(0), C.c_uint64(0)
    _check(lib().zbus_serve_footprint(h, PRECISION[precision], C.byref(a), C.byref(b),
                                      C.byref(c)))
    return a.value, b.value, c.value


def zbus_probe_fp64_rate(stream=None):
    """(TFLOP/s, ms) of the device's FP64 fused multiply-add rate (DFMA chains)."""
    t = C.c_double(0.0)
    ms = C.c_float(0.0)
    _check(lib().zbus_probe_fp64_rate(C.byref(t), C.byref(ms), _stream(stream)))
    return t.value, ms.value


def zbus_solve_noalloc(h, S_wye, S_delta, V_init, tol, max_iter, rule, V_out, iters, converged,
                       stream=None):
    """The FP64 solve with library-static scratch (no device allocation)."""
    import torch
    n = zbus_network_size(h)
    B = V_out.shape[0]
    c128 = torch.complex128
    _check(lib().zbus_solve_noalloc(
        h, int(B), _dptr(S_wye, "S_wye", c128, (B, n)), _dptr(S_delta, "S_delta", c128, (B, n)),
        _dptr(V_init, "V_init", c128, (B, n)), float(tol), int(max_iter), RULE[rule],
        _dptr(V_out, "V_out", c128, (B, n)), _dptr(iters, "iters", torch.int32, (B,)),
        _dptr(converged, "converged", torch.uint8, (B,)), _stream(stream)))


def zbus_solve_adjoint(h, S_wye, S_delta, V, G, tol, max_iter, opts, dS_wye, dS_delta, iters,
                       converged, stream=None):
    """Load gradient dL/dS at converged voltages V given G = dL/dV (device tensors)."""
    import torch
    n = zbus_network_size(h)
    B = V.shape[0]
    c128 = torch.complex128
    _check(lib().zbus_solve_adjoint(
        h, int(B), _dptr(S_wye, "S_wye", c128, (B, n)), _dptr(S_delta, "S_delta", c128, (B, n)),
        _dptr(V, "V", c128, (B, n)), _dptr(G, "G", c128, (B, n)), float(tol), int(max_iter),
        C.byref(opts) if opts is not None else None, _dptr(dS_wye, "dS_wye", c128, (B, n)), _dptr(dS_delta, "dS_delta", c128, (B, n)),
        _dptr(iters, "iters", torch.int32, (B,)), _dptr(converged, "converged", torch.uint8, (B,)),
        _stream(stream)))


def zbus_power_mismatch(h, V, S_wye, S_delta, out, stream=None):
    import torch
    n = zbus_network_size(h)
    B = V.shape[0]
    c128 = torch.complex128
    _check(lib().zbus_power_mismatch(
        h, int(B), _dptr(V, "V", c128, (B, n)), _dptr(S_wye, "S_wye", c128, (B, n)),
        _dptr(S_delta, "S_delta", c128, (B, n)), _dptr(out, "out", torch.float64, (B,)),
        _stream(stream)))


def zbus_last_profile(h, max_n):
    """(ms [sweeps, 3] float32, active [sweeps] int32) of the last profiled solve."""
    ms = np.zeros((max_n, 3), dtype=np.float32)
    act = np.zeros(max_n, dtype=np.int32)
    sw = C.c_int32(0)
    _check(lib().zbus_last_profile(h, int(max_n), ms.ctypes.data, act.ctypes.data,
                                   C.byref(sw)))
    m = min(max_n, sw.value)
    return ms[:m], act[:m]


def _batch_array(items):
    """items: list of (handle, S_wye, S_delta, V_init, V_out, iters, converged) tensors."""
    import torch
    arr = (zbus_batch_item * len(items))()
    c128 = torch.complex128
    for k, (h, sw, sd, v0, vo, it, cv) in enumerate(items):
        n = zbus_network_size(h)
        B = vo.shape[0]
        arr[k].net = h
        arr[k].B = B
        arr[k].S_wye = _dptr(sw, "S_wye", c128, (B, n))
        arr[k].S_delta = _dptr(sd, "S_delta", c128, (B, n))
        arr[k].V_init = _dptr(v0, "V_init", c128, (B, n))
        arr[k].V_out = _dptr(vo, "V_out", c128, (B, n))
        arr[k].iters = _dptr(it, "iters", torch.int32, (B,))
        arr[k].converged = _dptr(cv, "converged", torch.uint8, (B,))
    return arr


def zbus_solve_batched(items, tol, max_iter, opts, stream=None):
    arr = _batch_array(items)
    _check(lib().zbus_solve_batched(arr, len(items), float(tol), int(max_iter),
                                    C.byref(opts) if opts is not None else None, _stream(stream)))


def zbus_autotune(items, opts, tol, max_iter, reps=3, stream=None):
    """Times every compiled contraction variant on these items; returns (BN, stages)."""
    arr = _batch_array(items)
    bn = C.c_int32(0)
    stg = C.c_int32(0)
    _check(lib().zbus_autotune(arr, len(items), C.byref(opts), float(tol), int(max_iter),
                               int(reps), _stream(stream), C.byref(bn), C.byref(stg)))
    return bn.value, stg.value


def zbus_tune_variants(precision):
    """The compiled contraction variants of a mixed precision: [(BN, stages)]."""
    p = PRECISION[precision] if isinstance(precision, str) else int(precision)
    m = lib().zbus_tune_variants(p, None, None, 0)
    if m <= 0:
        return []
    bn = (C.c_int32 * m)()
    st = (C.c_int32 * m)()
    lib().zbus_tune_variants(p, bn, st, m)
    return list(zip(bn, st))


def zbus_tune_set(precision, max_n, total_B, BN, stages):
    """Use variant (BN, stages) for the size bucket of (max_n, total_B); BN = 0 clears it."""
    p = PRECISION[precision] if isinstance(precision, str) else int(precision)
    _check(lib().zbus_tune_set(p, int(max_n), int(total_B), int(BN), int(stages)))


def solve_batched(networks, loads, tol=1e-8, max_iter=50, precision="fp16_scaled",
                  rule="maxabs", mismatch_tol=1e-6, max_correction=8, fp32_start=True,
                  stream=None):
    """networks: [Network]; loads: [(S_wye, S_delta)] device tensors.  Returns [(V, iters, conv)]."""
    import torch
    o = zbus_solve_opts_default()
    o.precision = PRECISION[precision]
    o.conv_rule = RULE[rule]
    o.mismatch_tol = mismatch_tol
    o.max_correction = max_correction
    o.fp32_start = 1 if fp32_start else 0
    items, outs = [], []
    for net, (sw, sd) in zip(networks, loads):
        ref = sw if sw is not None else sd
        B = ref.shape[0]
        out = (torch.empty((B, net.n), dtype=torch.complex128, device=ref.device),
               torch.empty((B,), dtype=torch.int32, device=ref.device),
               torch.empty((B,), dtype=torch.uint8, device=ref.device))
        items.append((net.handle, sw, sd, None) + out)
        outs.append(out)
    zbus_solve_batched(items, tol, max_iter, o, stream)
    return outs


def zbus_serve(cfg, pool_handles, source, sink, stream=None):
    """Raw call: source(now) -> zbus_request | None | -1; sink(req, res)."""
    arr = (C.c_void_p * len(pool_handles))(*pool_handles)
    errors = []   # exceptions of the callbacks, raised again when the loop returns

    @SOURCE_FN
    def _src(user, now, out):
        try:
            r = source(now)
        except BaseException as e:   # the source failed: stop taking requests
            errors.append(e)
            return -2
        if r is None:
            return 0
        if isinstance(r, int):
            return r
        out[0] = r
        return 1

    @SINK_FN
    def _snk(user, req, res):
        try:
            sink(req[0], res[0])
        except BaseException as e:
            errors.append(e)

    status = lib().zbus_serve(C.byref(cfg), arr, len(pool_handles), _src, _snk, None,
                              _stream(stream))
    if errors:
        raise errors[0]
    _check(status)


def serve(networks, requests, hbm_budget_bytes=120 << 30, max_slots=4096,
          precision="fp16_scaled", tol=1e-8, max_iter=50, mismatch_tol=1e-6, rule="maxabs",
          keep_results=True, max_admit_per_sweep=0, max_correction=8, fp32_start=True,
          stream=None):
    """Serve a list of requests over a pool of networks.

    requests: dicts with keys feeder, S_wye, S_delta (device tensors [B, n]),
    arrival (seconds after the start), optional warm_start.  Returns one dict
    per request (in input order): status, t_arrival, t_admit, t_done,
    n_converged, max_iters and, with keep_results, V / iters / converged.
    """
    import torch
    order = sorted(range(len(requests)), key=lambda i: requests[i].get("arrival", 0.0))
    out = [None] * len(requests)
    keep = []
    structs = []
    for i in order:
        q = requests[i]
        ref = q["S_wye"] if q.get("S_wye") is not None else q["S_delta"]
        B, n = ref.shape
        r = zbus_request()
        r.feeder = q["feeder"]
        r.B = B
        r.S_wye = q["S_wye"].data_ptr() if q.get("S_wye") is not None else None
        r.S_delta = q["S_delta"].data_ptr() if q.get("S_delta") is not None else None
        if keep_results:
            V = torch.empty((B, n), dtype=torch.complex128, device=ref.device)
            it = torch.empty((B,), dtype=torch.int32, device=ref.device)
            cv = torch.empty((B,), dtype=torch.uint8, device=ref.device)
            keep.append((i, V, it, cv))
            r.V_out, r.iters, r.converged = V.data_ptr(), it.data_ptr(), cv.data_ptr()
        r.warm_start = 1 if q.get("warm_start") else 0
        r.tag = i
        r.t_arrival = float(q.get("arrival", 0.0))
        structs.append(r)
    pos = [0]

    def source(now):
        if pos[0] >= len(structs):
            return -1
        r = structs[pos[0]]
        if r.t_arrival <= now:
            pos[0] += 1
            return r
        return None

    def sink(req, res):
        out[req.tag] = {"status": res.status, "t_arrival": req.t_arrival, "t_admit": res.t_admit,
                        "t_done": res.t_done, "n_converged": res.n_converged,
                        "max_iters": res.max_iters, "B": req.B,
                        "operands_formed": res.operands_formed}

    cfg = zbus_serve_config()
    cfg.hbm_budget_bytes = int(hbm_budget_bytes)
    cfg.max_slots = int(max_slots)
    cfg.precision = PRECISION[precision]
    cfg.conv_rule = RULE[rule]
    cfg.max_iter = int(max_iter)
    cfg.tol = float(tol)
    cfg.mismatch_tol = float(mismatch_tol)
    cfg.max_admit_per_sweep = int(max_admit_per_sweep)
    cfg.max_correction = int(max_correction)
    cfg.fp32_start = 1 if fp32_start else 0
    zbus_serve(cfg, [net.handle for net in networks], source, sink, stream)
    for i, V, it, cv in keep:
        if out[i] is not None:
            out[i].update(V=V, iters=it, converged=cv)
    return out


def zbus_checked_status():
    """(1 if the checked build else 0, first check code recorded since the last call)."""
    w = C.c_uint32(0)
    flag = lib().zbus_checked_status(C.byref(w))
    return int(flag), int(w.value)


def zbus_status_string(s: int) -> str:
    return lib().zbus_status_string(int(s)).decode()


def zbus_last_error() -> str:
    return lib().zbus_last_error().decode(errors="replace")


# ---------------------------------------------------------------------------
# Convenience wrapper.
# ---------------------------------------------------------------------------

class Network:
    """One feeder's Z-bus data on the current CUDA device."""

    def __init__(self, n_total, row, col, val, slack_idx, v_slack, stream=None, bus_phase=None):
        self.handle = zbus_network_create(n_total, row, col, val, slack_idx, v_slack, stream,
                                          bus_phase)
        self.n = zbus_network_size(self.handle)

    @classmethod
    def from_feeder(cls, f, stream=None):
        return cls(f.n_total, f.Y_row, f.Y_col, f.Y_val, f.slack_idx, f.v_slack, stream,
                   getattr(f, "bus_phase", None))

    def close(self):
        if self.handle:
            zbus_network_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def get_z(self, stream=None):
        import torch
        Z = torch.empty((self.n, self.n), dtype=torch.complex128, device="cuda")
        w = torch.empty((self.n,), dtype=torch.complex128, device="cuda")
        zbus_network_get_z(self.handle, Z, w, stream)
        return Z, w

    def reserve(self, B, precision="fp64"):
        zbus_network_reserve(self.handle, B, precision)

    def solve(self, S_wye, S_delta=None, V_init=None, tol=1e-8, max_iter=50,
              precision="fp64", rule="maxabs", mismatch_tol=1e-6, max_correction=8,
              profile=False, out=None, stream=None, fp32_start=True):
        """Returns (V [B,n] complex128, iters int32[B], converged uint8[B]) where the
        loads live: on the device, or in host memory (results valid once the
        stream has synchronised)."""
        import torch
        B = (S_wye if S_wye is not None else S_delta).shape[0]
        dev = (S_wye if S_wye is not None else S_delta).device
        if out is None:
            out = (torch.empty((B, self.n), dtype=torch.complex128, device=dev),
                   torch.empty((B,), dtype=torch.int32, device=dev),
                   torch.empty((B,), dtype=torch.uint8, device=dev))
        o = zbus_solve_opts_default()
        o.precision = PRECISION[precision]
        o.conv_rule = RULE[rule]
        o.mismatch_tol = mismatch_tol
        o.max_correction = max_correction
        o.profile = 1 if profile else 0
        o.fp32_start = 1 if fp32_start else 0
        V, it, cv = out
        zbus_solve(self.handle, S_wye, S_delta, V_init, tol, max_iter, o, V, it, cv, stream)
        return V, it, cv

    def device_status(self, stream=None):
        """Status of the device-side checks of the last solve (after a sync)."""
        return zbus_last_device_status(self.handle, stream)

    def last_profile(self, max_n=1024):
        return zbus_last_profile(self.handle, max_n)

    def power_mismatch(self, V, S_wye=None, S_delta=None, stream=None):
        import torch
        out = torch.empty((V.shape[0],), dtype=torch.float64, device=V.device)
        zbus_power_mismatch(self.handle, V, S_wye, S_delta, out, stream)
        return out

    def solve_adjoint(self, V, G, S_wye=None, S_delta=None, tol=1e-12, max_iter=200,
                      wye=True, delta=True, precision="fp64", stream=None):
        """Load gradient at converged voltages V given G = dL/dV; precision
        "fp64" (dense Z^T sweeps) or "tree" (radial networks).  Returns
        (dS_wye or None, dS_delta or None, iters, converged)."""
        import torch
        B = V.shape[0]
        c128 = torch.complex128
        dw = torch.empty((B, self.n), dtype=c128, device=V.device) if wye else None
        dd = torch.empty((B, self.n), dtype=c128, device=V.device) if delta else None
        it = torch.empty((B,), dtype=torch.int32, device=V.device)
        cv = torch.empty((B,), dtype=torch.uint8, device=V.device)
        o = zbus_solve_opts_default()
        o.precision = PRECISION[precision]
        zbus_solve_adjoint(self.handle, S_wye, S_delta, V, G, tol, max_iter, o, dw, dd, it, cv,
                           stream)
        return dw, dd, it, cv


def _solve_function():
    import torch

    class SolveFn(torch.autograd.Function):
        """v*(S) with its gradient by zbus_solve_adjoint (argument marshalling)."""

        @staticmethod
        def forward(ctx, S_wye, S_delta, net, opts):
            tol, max_iter, precision, adj_tol, adj_max_iter, adj_precision = opts
            V, it, cv = net.solve(S_wye, S_delta, tol=tol, max_iter=max_iter,
                                  precision=precision)
            ctx.save_for_backward(S_wye, S_delta, V)
            ctx.net = net
            ctx.adj = (adj_tol, adj_max_iter, adj_precision)
            ctx.mark_non_differentiable(it, cv)
            return V, it, cv

        @staticmethod
        def backward(ctx, gV, g_it, g_cv):
            S_wye, S_delta, V = ctx.saved_tensors
            want_w, want_d = ctx.needs_input_grad[0], ctx.needs_input_grad[1]
            dw, dd, it, cv = ctx.net.solve_adjoint(
                V, gV.contiguous(), S_wye, S_delta, tol=ctx.adj[0], max_iter=ctx.adj[1],
                wye=want_w, delta=want_d, precision=ctx.adj[2])
            ctx.net.last_adjoint = (it, cv)
            return dw, dd, None, None

    return SolveFn


_SOLVE_FN = None


def solve_differentiable(net, S_wye, S_delta=None, tol=1e-10, max_iter=50, precision="fp64",
                         adj_tol=1e-12, adj_max_iter=200, adj_precision="fp64"):
    """(V, iters, converged) of net.solve, with V differentiable in S_wye and
    S_delta through zbus_solve_adjoint (torch autograd; adj_precision "fp64"
    or "tree").  After a backward pass, net.last_adjoint holds the adjoint's
    (iters, converged)."""
    global _SOLVE_FN
    if _SOLVE_FN is None:
        _SOLVE_FN = _solve_function()
    return _SOLVE_FN.apply(S_wye, S_delta, net,
                           (tol, max_iter, precision, adj_tol, adj_max_iter, adj_precision))


# ---------------------------------------------------------------------------
# Transmission grids: batched Newton-Raphson (Sec. II-A).
# ---------------------------------------------------------------------------

def zbus_nr_opts_default() -> zbus_nr_opts:
    o = zbus_nr_opts()
    lib().zbus_nr_opts_default(C.byref(o))
    return o


def zbus_nr_network_create(N, row, col, val, bus_type, v_set, eps=1e-8, stream=None) -> int:
    row = np.ascontiguousarray(row, dtype=np.int32)
    col = np.ascontiguousarray(col, dtype=np.int32)
    val = np.ascontiguousarray(val, dtype=np.complex128)
    bt = np.ascontiguousarray(bus_type, dtype=np.int32)
    vs = np.ascontiguousarray(v_set, dtype=np.float64)
    if not (row.shape == col.shape == val.shape) or bt.shape != (N,) or vs.shape != (N,):
        raise ValueError("row/col/val must have equal length; bus_type and v_set N entries")
    h = _P()
    _check(lib().zbus_nr_network_create(int(N), int(row.size), row.ctypes.data, col.ctypes.data,
                                        val.ctypes.data, bt.ctypes.data, vs.ctypes.data,
                                        float(eps), _stream(stream), C.byref(h)))
    return h.value


def zbus_nr_network_destroy(h):
    if h:
        lib().zbus_nr_network_destroy(h)


def zbus_nr_network_info(h):
    """(n_theta, n_q, factor_nnz, factor_levels)."""
    a, b, c, d = C.c_int32(0), C.c_int32(0), C.c_int64(0), C.c_int32(0)
    _check(lib().zbus_nr_network_info(h, C.byref(a), C.byref(b), C.byref(c), C.byref(d)))
    return a.value, b.value, c.value, d.value


def zbus_nr_solve(h, N, P, Q, tol, max_iter, opts, V_out, iters, converged, gmres_iters=None,
                  stream=None):
    import torch
    B = V_out.shape[0]
    f64 = torch.float64
    _check(lib().zbus_nr_solve(
        h, int(B), _dptr(P, "P", f64, (B, N)), _dptr(Q, "Q", f64, (B, N)), float(tol),
        int(max_iter), C.byref(opts) if opts is not None else None,
        _dptr(V_out, "V_out", torch.complex128, (B, N)),
        _dptr(iters, "iters", torch.int32, (B,)), _dptr(converged, "converged", torch.uint8, (B,)),
        _dptr(gmres_iters, "gmres_iters", torch.int32, (B,)), _stream(stream)))


class NrNetwork:
    """One transmission grid for the batched Newton-Raphson solve."""

    def __init__(self, N, row, col, val, bus_type, v_set, eps=1e-8, stream=None):
        self.N = int(N)
        self.handle = zbus_nr_network_create(N, row, col, val, bus_type, v_set, eps, stream)

    @classmethod
    def from_grid(cls, g, eps=1e-8, stream=None):
        return cls(g.N, g.Y_row, g.Y_col, g.Y_val, g.bus_type, g.v_set, eps, stream)

    def close(self):
        if self.handle:
            zbus_nr_network_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def info(self):
        return zbus_nr_network_info(self.handle)

    def solve(self, P, Q, tol=1e-10, max_iter=20, gmres_restart=30, gmres_max_restarts=4,
              gmres_tol=1e-6, precision="fp64", out=None, stream=None):
        """Returns (V [B,N] complex128, iters, converged, gmres_iters) on P's device."""
        import torch
        B = P.shape[0]
        if out is None:
            out = (torch.empty((B, self.N), dtype=torch.complex128, device=P.device),
                   torch.empty((B,), dtype=torch.int32, device=P.device),
                   torch.empty((B,), dtype=torch.uint8, device=P.device),
                   torch.empty((B,), dtype=torch.int32, device=P.device))
        o = zbus_nr_opts_default()
        o.gmres_restart = gmres_restart
        o.gmres_max_restarts = gmres_max_restarts
        o.gmres_tol = gmres_tol
        o.precision = NR_PRECISION[precision]
        V, it, cv, gm = out
        zbus_nr_solve(self.handle, self.N, P, Q, tol, max_iter, o, V, it, cv, gm, stream)
        return V, it, cv, gm
