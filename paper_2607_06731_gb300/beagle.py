"""Thin Python binding of libbeagle.so (include/beagle.h), same names as the C ABI.

Only argument marshalling happens here: pointers of torch CUDA tensors (or numpy arrays for
host calls), sizes and the current torch stream are passed through ctypes. Every step of
scoring runs in the library's CUDA kernels. There is no CPU fallback: if the library has not
been built, every call raises.
"""
from __future__ import annotations

import ctypes
import os
import re

import numpy as np

from . import build as _build

OK = 0
ERR_OOM = -4
ERR_TIMEOUT = -6
ERRORS = {-1: "BEAGLE_ERR_ARG", -2: "BEAGLE_ERR_PROGRAM", -3: "BEAGLE_ERR_DATASET",
          -4: "BEAGLE_ERR_OOM", -5: "BEAGLE_ERR_CUDA", -6: "BEAGLE_ERR_TIMEOUT",
          -7: "BEAGLE_ERR_BUSY", -8: "BEAGLE_ERR_LIMIT"}
FP32_COMPENSATED, FP64 = 0, 1
FLAG_INVALID, FLAG_DEGENERATE, FLAG_MALFORMED, FLAG_TIMEOUT = 1, 2, 4, 8
MAX_VARS, MAX_DEPTH, MAX_LENGTH = 16, 32, 256

# beagle_fitness: {double mse; double one_minus_r2; uint32 flags; uint32 reserved}
FITNESS_DTYPE = np.dtype([("mse", "<f8"), ("one_minus_r2", "<f8"), ("flags", "<u4"),
                          ("reserved", "<u4")])

# The paper's fitness functions (beagle_score_fit)
FIT_CORRELATION, FIT_STD, FIT_STD_SQUARE, FIT_STD_CUBE, FIT_STD_HYPER, FIT_VALIDATE = range(1, 7)
FLAG_PERFECT = 16
DATASET_INVALID_TARGETS = 1
# beagle_fit_result: {double score, asr, r2, taxed_score; int64 c1, c2; uint32 flags, reserved}
FIT_RESULT_DTYPE = np.dtype([("score", "<f8"), ("asr", "<f8"), ("r2", "<f8"),
                             ("taxed_score", "<f8"), ("c1", "<i8"), ("c2", "<i8"),
                             ("flags", "<u4"), ("reserved", "<u4")])


class FitConfig(ctypes.Structure):
    """beagle_fit_config."""
    _fields_ = [("kind", ctypes.c_int32), ("max_score", ctypes.c_int32),
                ("tax_per_token", ctypes.c_double)]


HEADER = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                      "include", "beagle.h")


class BeagleError(RuntimeError):
    def __init__(self, code: int, message: str):
        super().__init__(f"{ERRORS.get(code, code)}: {message}")
        self.code = code


_lib = None
_vp, _i32, _i64, _u8p = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_void_p

_SIGNATURES = {
    "beagle_upload_dataset": ([_vp, _vp, _i64, _i32, _i32, _vp, _vp], _i32),
    "beagle_upload_dataset_ex": ([_vp, _vp, _i64, _i32, _i32, ctypes.c_uint32, _vp, _vp], _i32),
    "beagle_score_fit": ([_vp, _vp, _vp, _vp, _i64, _i32, _vp, _vp, _i32, _vp], _i32),
    "beagle_release_dataset": ([_i32], _i32),
    "beagle_dataset_info": ([_i32, _vp, _vp, _vp, _vp], _i32),
    "beagle_validate_programs": ([_vp, _vp, _vp, _i64, _i32, _i32, _vp], _i32),
    "beagle_validate_programs_ex": ([_vp, _vp, _vp, _i64, _i32, _i32, _vp, _i32, _vp], _i32),
    "beagle_score": ([_vp, _vp, _vp, _vp, _i64, _i32, _vp, _i32, _vp], _i32),
    "beagle_score_static": ([_vp, _vp, _vp, _vp, _i64, _i32, _vp, _i32, _vp], _i32),
    "beagle_eval": ([_vp, _vp, _vp, _vp, _i64, _i32, _vp, _vp, _i32, _vp], _i32),
    "beagle_score_host": ([_vp, _vp, _vp, _vp, _i64, _i64, _i32, _vp, _i32, _vp], _i32),
    "beagle_score_batch": ([_vp, _i32, _i32, _vp], _i32),
    "beagle_batch_plan_create": ([_vp, _i32, _i32, _vp], _i32),
    "beagle_batch_plan_launch": ([_vp, _vp], _i32),
    "beagle_batch_plan_destroy": ([_vp], _i32),
    "beagle_autotune": ([_vp, _i32, _i32, _i32, _vp, _vp, _vp], _i32),
    "beagle_autotune_clear": ([], _i32),
    "beagle_serve_create": ([_vp, _vp], _i32),
    "beagle_serve_submit": ([_vp, _vp, _vp], _i32),
    "beagle_serve_poll": ([_vp, ctypes.c_uint64, _vp, _vp], _i32),
    "beagle_serve_wait": ([_vp, ctypes.c_uint64, _vp, _i64], _i32),
    "beagle_serve_stats": ([_vp, _vp], _i32),
    "beagle_serve_timing": ([_vp, ctypes.c_uint64, _vp, _vp, _vp, _vp], _i32),
    "beagle_rank": ([_vp, _i64, _i32, _i64, _vp, _i32, _vp, _vp, _vp, _vp], _i32),
    "beagle_shard_by_cost": ([_vp, _i64, _i32, _vp], _i32),
    "beagle_serve_destroy": ([_vp], _i32),
    "beagle_set_launch_config": ([_vp], _i32),
    "beagle_get_launch_config": ([_vp], _i32),
    "beagle_measure_op_rates": ([_vp, _i32, ctypes.c_double, _vp], _i32),
    "beagle_set_invalid_early_exit": ([_i32], _i32),
    "beagle_count_cases": ([_vp, _i64], _i32),
    "beagle_kernel_timing": ([_i32], _i32),
    "beagle_kernel_time": ([_vp, _vp], _i32),
    "beagle_last_error": ([], ctypes.c_char_p),
    "beagle_version": ([], _i32),
}


def lib_path() -> str:
    return _build.LIB


def lib():
    """The loaded library. Raises if it has not been built (no fallback exists)."""
    global _lib
    if _lib is None:
        if not os.path.exists(_build.LIB):
            raise RuntimeError(f"{_build.LIB} is missing: build it first "
                               "(python -m paper_2607_06731_gb300.build)")
        L = ctypes.CDLL(_build.LIB)
        for name, (args, res) in _SIGNATURES.items():
            fn = getattr(L, name)
            fn.argtypes = args
            fn.restype = res
        _lib = L
    return _lib


def header_functions() -> list[str]:
    """Names of the functions include/beagle.h declares."""
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(beagle_[a-z_0-9]+)\s*\(", text)))


def last_error() -> str:
    return lib().beagle_last_error().decode()


def version() -> int:
    return int(lib().beagle_version())


def check(rc: int):
    if rc != OK:
        raise BeagleError(rc, last_error())


def _stream_handle(stream):
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def _ptr(t):
    if t is None:
        return None
    if isinstance(t, np.ndarray):
        return t.ctypes.data
    return t.data_ptr()


# ----------------------------------------------------------------------------- datasets
class Dataset:
    """A dataset resident on the current device (beagle_upload_dataset)."""

    def __init__(self, X, y, stream=None, invalid_targets: bool = False):
        import torch
        on_device = isinstance(X, torch.Tensor) and X.is_cuda
        if on_device:
            X = X.detach().to(torch.float32).contiguous()
            y = y.detach().to(torch.float32).contiguous()
        else:
            X = np.ascontiguousarray(X, np.float32)
            y = np.ascontiguousarray(y, np.float32)
        if X.ndim == 1:
            X = X.reshape(1, -1)
        d, N = int(X.shape[0]), int(X.shape[1])
        if int(y.shape[0]) != N:
            raise ValueError("y must have N entries")
        out = ctypes.c_int32()
        check(lib().beagle_upload_dataset_ex(_ptr(X), _ptr(y), N, d, int(on_device),
                                             DATASET_INVALID_TARGETS if invalid_targets else 0,
                                             _stream_handle(stream) if on_device else None,
                                             ctypes.byref(out)))
        self.id = int(out.value)
        self.N, self.d = N, d
        yb, syy = ctypes.c_double(), ctypes.c_double()
        check(lib().beagle_dataset_info(self.id, None, None, ctypes.byref(yb), ctypes.byref(syy)))
        self.ybar, self.syy = yb.value, syy.value

    def release(self):
        if self.id:
            check(lib().beagle_release_dataset(self.id))
            self.id = 0


def upload_dataset(X, y, stream=None) -> Dataset:
    return Dataset(X, y, stream)


def release_dataset(ds: Dataset):
    ds.release()


# ----------------------------------------------------------------------------- programs
def validate_programs(ops, offsets, lengths, d: int, max_depth: int = MAX_DEPTH,
                      allowed=None):
    """Host structural check (beagle_validate_programs_ex): -1 if all programs are valid,
    else the first bad index. allowed: optional opcode whitelist."""
    ops = np.ascontiguousarray(ops, np.uint8)
    offsets = np.ascontiguousarray(offsets, np.int64)
    lengths = np.ascontiguousarray(lengths, np.int32)
    first = ctypes.c_int64(-1)
    al = np.ascontiguousarray(allowed if allowed is not None else [], np.uint8)
    rc = lib().beagle_validate_programs_ex(_ptr(ops), _ptr(offsets), _ptr(lengths),
                                           len(lengths), d, max_depth,
                                           _ptr(al) if len(al) else None, len(al),
                                           ctypes.byref(first))
    if rc not in (OK, -2):
        check(rc)
    return int(first.value)


class DevicePrograms:
    """A population copied to the device in the wire format (torch tensors)."""

    def __init__(self, progs, device="cuda"):
        import torch
        self.ops = torch.from_numpy(np.ascontiguousarray(progs.ops, np.uint8)).to(device)
        self.offsets = torch.from_numpy(np.ascontiguousarray(progs.offsets, np.int64)).to(device)
        self.lengths = torch.from_numpy(np.ascontiguousarray(progs.lengths, np.int32)).to(device)
        self.consts = torch.from_numpy(np.ascontiguousarray(progs.consts, np.float32)).to(device)
        self.P = int(progs.lengths.shape[0])
        self.tokens = int(progs.ops.shape[0])


def _precision(p) -> int:
    if p in (FP32_COMPENSATED, "fp32c", "fp32"):
        return FP32_COMPENSATED
    if p in (FP64, "fp64"):
        return FP64
    raise ValueError(p)


def score(programs, offsets, lengths, consts, dataset: Dataset, out=None,
          precision="fp32c", stream=None):
    """beagle_score on device tensors. Returns (and fills) a [P, 3] float64 CUDA tensor whose
    rows are the 24-byte beagle_fitness records (see unpack_fitness)."""
    import torch
    P = int(lengths.shape[0])
    if out is None:
        out = torch.empty((P, 3), dtype=torch.float64, device=lengths.device)
    check(lib().beagle_score(_ptr(programs), _ptr(offsets), _ptr(lengths), _ptr(consts), P,
                             dataset.id, _ptr(out), _precision(precision),
                             _stream_handle(stream)))
    return out


def score_fit(dp: "DevicePrograms", dataset: "Dataset", kind: int, max_score: int = 10_000,
              tax_per_token: float = 0.0, precision="fp32c", out=None, stream=None):
    """beagle_score_fit: the paper's fitness functions. Returns (and fills) a [P, 7] float64
    CUDA tensor whose rows are the 56-byte beagle_fit_result records (see unpack_fit)."""
    import torch
    if out is None:
        out = torch.empty((dp.P, 7), dtype=torch.float64, device=dp.lengths.device)
    cfg = FitConfig(kind, max_score, tax_per_token)
    check(lib().beagle_score_fit(_ptr(dp.ops), _ptr(dp.offsets), _ptr(dp.lengths),
                                 _ptr(dp.consts), dp.P, dataset.id, ctypes.byref(cfg), _ptr(out),
                                 _precision(precision), _stream_handle(stream)))
    return out


def unpack_fit(out):
    """Structured numpy array (FIT_RESULT_DTYPE) from a [P, 7] tensor."""
    a = out.detach().cpu().numpy()
    return np.ascontiguousarray(a).view(FIT_RESULT_DTYPE).reshape(-1).copy()


def eval_programs(dp: "DevicePrograms", dataset: "Dataset", precision="fp32c", stream=None):
    """beagle_eval: per-case outputs [P, N] (float32 or float64 CUDA tensor) and fitness."""
    import torch
    prec = _precision(precision)
    dt = torch.float64 if prec == FP64 else torch.float32
    outputs = torch.full((dp.P, dataset.N), float("nan"), dtype=dt, device=dp.lengths.device)
    fit = torch.empty((dp.P, 3), dtype=torch.float64, device=dp.lengths.device)
    check(lib().beagle_eval(_ptr(dp.ops), _ptr(dp.offsets), _ptr(dp.lengths), _ptr(dp.consts),
                            dp.P, dataset.id, _ptr(outputs), _ptr(fit), prec,
                            _stream_handle(stream)))
    return outputs, fit


def score_programs(dp: DevicePrograms, dataset: Dataset, out=None, precision="fp32c",
                   stream=None):
    return score(dp.ops, dp.offsets, dp.lengths, dp.consts, dataset, out, precision, stream)


def score_host(progs, dataset: Dataset, out=None, precision="fp32c", stream=None):
    """beagle_score_host: host arrays in, host fitness records out (numpy structured array)."""
    ops = np.ascontiguousarray(progs.ops, np.uint8)
    offs = np.ascontiguousarray(progs.offsets, np.int64)
    lens = np.ascontiguousarray(progs.lengths, np.int32)
    cs = np.ascontiguousarray(progs.consts, np.float32)
    P = len(lens)
    if out is None:
        out = np.zeros(P, FITNESS_DTYPE)
    check(lib().beagle_score_host(_ptr(ops), _ptr(offs), _ptr(lens), _ptr(cs), P, len(ops),
                                  dataset.id, _ptr(out), _precision(precision),
                                  _stream_handle(stream)))
    return out


def unpack_fitness(out):
    """(mse, one_minus_r2, flags) numpy arrays from a [P, 3] tensor or a structured array."""
    if isinstance(out, np.ndarray) and out.dtype == FITNESS_DTYPE:
        return out["mse"].copy(), out["one_minus_r2"].copy(), out["flags"].copy()
    a = out.detach().cpu().numpy()
    rec = np.ascontiguousarray(a).view(FITNESS_DTYPE).reshape(-1)
    return rec["mse"].copy(), rec["one_minus_r2"].copy(), rec["flags"].copy()


# ----------------------------------------------------------------------------- measurement
def measure_op_rates(seconds_hint: float = 1.0, stream=None) -> dict:
    """Operator evaluations per second on the current device, keyed by opcode."""
    rates = (ctypes.c_double * 16)()
    check(lib().beagle_measure_op_rates(rates, 16, seconds_hint, _stream_handle(stream)))
    return {i: float(rates[i]) for i in range(16) if rates[i] > 0}


def set_invalid_early_exit(enable: bool):
    """beagle_set_invalid_early_exit: stop evaluating a program once a case makes it invalid."""
    check(lib().beagle_set_invalid_early_exit(1 if enable else 0))


def count_cases(cases_run=None):
    """beagle_count_cases: add each program's evaluated cases to cases_run (a CUDA int64
    tensor of P), or stop counting (None)."""
    if cases_run is None:
        check(lib().beagle_count_cases(None, 0))
    else:
        check(lib().beagle_count_cases(_ptr(cases_run), int(cases_run.numel())))


def kernel_timing(enable: bool):
    check(lib().beagle_kernel_timing(1 if enable else 0))


def kernel_time():
    """(total ms, launches) of the scoring kernels timed since the previous call."""
    ms, n = ctypes.c_double(), ctypes.c_int64()
    check(lib().beagle_kernel_time(ctypes.byref(ms), ctypes.byref(n)))
    return ms.value, int(n.value)


class LaunchConfig(ctypes.Structure):
    """beagle_launch_config (0 = automatic)."""
    _fields_ = [("cases_per_lane", ctypes.c_int32), ("tile", ctypes.c_int32),
                ("group", ctypes.c_int32), ("warps", ctypes.c_int32), ("grid", ctypes.c_int32),
                ("keep_order", ctypes.c_int32)]


def set_launch_config(cases_per_lane=0, tile=0, group=0, warps=0, grid=0, keep_order=0):
    cfg = LaunchConfig(cases_per_lane, tile, group, warps, grid, keep_order)
    check(lib().beagle_set_launch_config(ctypes.byref(cfg)))


def reset_launch_config():
    check(lib().beagle_set_launch_config(None))


def get_launch_config() -> dict:
    cfg = LaunchConfig()
    check(lib().beagle_get_launch_config(ctypes.byref(cfg)))
    return {k: getattr(cfg, k) for k, _ in LaunchConfig._fields_}


# ----------------------------------------------------------------------------- batches
class Job(ctypes.Structure):
    """beagle_job: one (population, dataset) pair of a batch (device pointers)."""
    _fields_ = [("programs", ctypes.c_void_p), ("offsets", ctypes.c_void_p),
                ("lengths", ctypes.c_void_p), ("consts", ctypes.c_void_p),
                ("P", ctypes.c_int64), ("dataset_id", ctypes.c_int32),
                ("reserved", ctypes.c_int32), ("fitness_out", ctypes.c_void_p)]


def make_jobs(items):
    """items: sequence of (DevicePrograms, Dataset, out tensor [P, 3] float64)."""
    arr = (Job * len(items))()
    for i, (dp, ds, out) in enumerate(items):
        arr[i] = Job(_ptr(dp.ops), _ptr(dp.offsets), _ptr(dp.lengths), _ptr(dp.consts), dp.P,
                     ds.id, 0, _ptr(out))
    return arr


def score_batch(items, precision="fp32c", stream=None):
    """beagle_score_batch over (DevicePrograms, Dataset, out) triples."""
    jobs = make_jobs(items)
    check(lib().beagle_score_batch(jobs, len(items), _precision(precision),
                                   _stream_handle(stream)))


class BatchPlan:
    """beagle_batch_plan: a batch captured in a CUDA graph, replayed with launch()."""

    def __init__(self, items, precision="fp32c"):
        self._items = list(items)          # keep the buffers alive with the plan
        jobs = make_jobs(self._items)
        h = ctypes.c_void_p()
        check(lib().beagle_batch_plan_create(jobs, len(self._items), _precision(precision),
                                             ctypes.byref(h)))
        self.handle = h

    def launch(self, stream=None):
        check(lib().beagle_batch_plan_launch(self.handle, _stream_handle(stream)))

    def destroy(self):
        if self.handle:
            check(lib().beagle_batch_plan_destroy(self.handle))
            self.handle = None


def autotune(items, precision="fp32c", max_trials=0, stream=None):
    """beagle_autotune: returns (best launch config dict, ms per call)."""
    jobs = make_jobs(items)
    cfg = LaunchConfig()
    ms = ctypes.c_double()
    check(lib().beagle_autotune(jobs, len(items), _precision(precision), max_trials,
                                _stream_handle(stream), ctypes.byref(cfg), ctypes.byref(ms)))
    return {k: getattr(cfg, k) for k, _ in LaunchConfig._fields_}, ms.value


def autotune_clear():
    check(lib().beagle_autotune_clear())


# ----------------------------------------------------------------------------- serving
class ServeConfig(ctypes.Structure):
    _fields_ = [("hbm_budget_bytes", ctypes.c_int64), ("max_inflight", ctypes.c_int32),
                ("max_batch_jobs", ctypes.c_int32), ("precision", ctypes.c_int32),
                ("reserved", ctypes.c_int32)]


class Request(ctypes.Structure):
    _fields_ = [("programs", ctypes.c_void_p), ("offsets", ctypes.c_void_p),
                ("lengths", ctypes.c_void_p), ("consts", ctypes.c_void_p),
                ("P", ctypes.c_int64), ("n_tokens", ctypes.c_int64),
                ("dataset_id", ctypes.c_int32), ("reserved", ctypes.c_int32)]


class ServeStats(ctypes.Structure):
    _fields_ = [(n, ctypes.c_int64) for n in
                ("submitted", "completed", "rejected", "queued", "inflight_launches",
                 "launches", "node_evals", "bytes_in_use", "peak_bytes", "budget_bytes")] + \
               [(n, ctypes.c_double) for n in ("gpops", "p50_us", "p99_us", "max_us")]


class Server:
    """beagle_serve_*: continuous-batching scoring server (host-memory requests)."""

    def __init__(self, hbm_budget_bytes=0, max_inflight=0, max_batch_jobs=0,
                 precision="fp32c"):
        cfg = ServeConfig(hbm_budget_bytes, max_inflight, max_batch_jobs,
                          _precision(precision), 0)
        h = ctypes.c_void_p()
        check(lib().beagle_serve_create(ctypes.byref(cfg), ctypes.byref(h)))
        self.handle = h
        self._keep = {}

    def submit(self, progs, dataset: "Dataset") -> int:
        ops = np.ascontiguousarray(progs.ops, np.uint8)
        offs = np.ascontiguousarray(progs.offsets, np.int64)
        lens = np.ascontiguousarray(progs.lengths, np.int32)
        cs = np.ascontiguousarray(progs.consts, np.float32)
        req = Request(_ptr(ops), _ptr(offs), _ptr(lens), _ptr(cs), len(lens), len(ops),
                      dataset.id, 0)
        t = ctypes.c_uint64()
        check(lib().beagle_serve_submit(self.handle, ctypes.byref(req), ctypes.byref(t)))
        self._keep[t.value] = len(lens)
        return t.value

    def poll(self, ticket: int):
        """None while running, else the structured fitness array."""
        P = self._keep.get(ticket, 0)     # unknown tickets: the library reports the error
        out = np.zeros(P, FITNESS_DTYPE)
        done = ctypes.c_int32()
        rc = lib().beagle_serve_poll(self.handle, ticket, _ptr(out) if P else None,
                                     ctypes.byref(done))
        if rc == OK and not done.value:
            return None
        self._keep.pop(ticket, None)   # finished (or failed): the ticket is retired
        check(rc)
        return out

    def wait(self, ticket: int, timeout_us: int = -1):
        P = self._keep.get(ticket, 0)
        out = np.zeros(P, FITNESS_DTYPE)
        rc = lib().beagle_serve_wait(self.handle, ticket, _ptr(out) if P else None,
                                     timeout_us)
        if rc != ERR_TIMEOUT:
            self._keep.pop(ticket, None)   # a timed-out ticket stays valid
        check(rc)
        return out

    def timing(self, ticket: int) -> dict:
        """Queue time and latency (us, host clock) and the device's %globaltimer stamps (ns) of
        a finished request (beagle_serve_timing)."""
        q, lat = ctypes.c_double(), ctypes.c_double()
        g0, g1 = ctypes.c_uint64(), ctypes.c_uint64()
        check(lib().beagle_serve_timing(self.handle, ticket, ctypes.byref(q), ctypes.byref(lat),
                                        ctypes.byref(g0), ctypes.byref(g1)))
        return {"queue_us": q.value, "latency_us": lat.value, "gpu_start_ns": g0.value,
                "gpu_end_ns": g1.value}

    def stats(self) -> dict:
        st = ServeStats()
        check(lib().beagle_serve_stats(self.handle, ctypes.byref(st)))
        return {k: getattr(st, k) for k, _ in ServeStats._fields_}

    def destroy(self):
        if self.handle:
            check(lib().beagle_serve_destroy(self.handle))
            self.handle = None


# ----------------------------------------------------------------------------- a generation
def rank(fitness, sample, u, field: str = "mse", stream=None):
    """beagle_rank (Monte-Carlo ranking) over fitness records on the device: a [P, 3] tensor
    of beagle_fitness (field "mse" or "one_minus_r2": lower is better) or a [P, 7] tensor of
    beagle_fit_result (field "score", "asr" or "taxed_score": higher is better). sample: 100
    device int64 indices; u: [P] device float32 uniforms. Returns (group uint8, children int32)
    device tensors."""
    import torch
    P = int(fitness.shape[0])
    if fitness.shape[1] == 3:
        off = {"mse": 0, "one_minus_r2": 8}[field]
        stride, neg = 24, 1
    else:
        off = {"score": 0, "asr": 8, "taxed_score": 24}[field]
        stride, neg = 56, 0
    group = torch.empty(P, dtype=torch.uint8, device=fitness.device)
    children = torch.empty(P, dtype=torch.int32, device=fitness.device)
    check(lib().beagle_rank(_ptr(fitness) + off, stride, neg, P, _ptr(sample), int(sample.numel()),
                            _ptr(u), _ptr(group), _ptr(children), _stream_handle(stream)))
    return group, children


def shard_by_cost(lengths, n_shards: int):
    """beagle_shard_by_cost: [n_shards + 1] int64 range edges of programs split by summed
    length."""
    lengths = np.ascontiguousarray(lengths, np.int32)
    bounds = np.zeros(n_shards + 1, np.int64)
    check(lib().beagle_shard_by_cost(_ptr(lengths), len(lengths), n_shards, _ptr(bounds)))
    return bounds
