"""Thin ctypes binding of libpf.so (include/pf.h).

Argument marshalling only: every step of the particle-learning cycle runs in
the library's CUDA kernels.  PyTorch supplies device memory (through the
allocator callbacks) and streams.  Importing this module loads libpf.so and
raises if it has not been built; there is no fallback path.
"""
import ctypes as C
import struct
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libpf.so")

if not os.path.exists(LIB_PATH):
    raise ImportError("libpf.so is not built: run __graft_entry__.build() "
                      "(or python paper_1212_1639_gb300/build.py)")

_lib = C.CDLL(LIB_PATH)

PF_OK, PF_ERR_INVALID, PF_ERR_OOM, PF_ERR_CUDA, PF_ERR_NUMERIC, PF_ERR_TIMEOUT, PF_ERR_BUSY = range(7)
STATUS_NAMES = {0: "PF_OK", 1: "PF_ERR_INVALID", 2: "PF_ERR_OOM", 3: "PF_ERR_CUDA",
                4: "PF_ERR_NUMERIC", 5: "PF_ERR_TIMEOUT", 6: "PF_ERR_BUSY"}
MULTINOMIAL, SYSTEMATIC, MULTINOMIAL_CUTPOINT, SYSTEMATIC_CUTPOINT = 0, 1, 2, 3
SCHEMES = {"multinomial": 0, "systematic": 1, "multinomial_cutpoint": 2, "systematic_cutpoint": 3,
           "stratified": 4}
FP32, FP64 = 0, 1
MAX_PARTICLES = 1 << 26
NOALLOC_MAX_PARTICLES = 1 << 20

ALLOC_FN = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p, C.c_void_p)
FREE_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_void_p, C.c_void_p)


class PfConfig(C.Structure):
    _fields_ = [("n_particles", C.c_uint64), ("seed", C.c_uint64), ("filter_id", C.c_uint32),
                ("scheme", C.c_int32), ("precision", C.c_int32),
                ("known_variances", C.c_int32),
                ("x0_mean", C.c_double), ("x0_var", C.c_double),
                ("a_sigma", C.c_double), ("b_sigma", C.c_double),
                ("a_tau", C.c_double), ("b_tau", C.c_double),
                ("sigma2", C.c_double), ("tau2", C.c_double),
                ("stream", C.c_void_p), ("alloc", ALLOC_FN), ("free", FREE_FN),
                ("alloc_ctx", C.c_void_p), ("algorithm", C.c_int32), ("ess_frac", C.c_double)]

ALGORITHMS = {"pl": 0, "particle_learning": 0, "bootstrap": 1}


class PfEstimates(C.Structure):
    _fields_ = [("t", C.c_uint64), ("x_mean", C.c_double), ("x_var", C.c_double),
                ("sigma2_mean", C.c_double), ("sigma2_var", C.c_double),
                ("tau2_mean", C.c_double), ("tau2_var", C.c_double),
                ("log_marglik", C.c_double)]


class PfBatchOpts(C.Structure):
    _fields_ = [("max_filters", C.c_uint32), ("hbm_budget_bytes", C.c_uint64),
                ("scheme", C.c_int32), ("precision", C.c_int32), ("autotune", C.c_int32),
                ("stream", C.c_void_p), ("alloc", ALLOC_FN), ("free", FREE_FN),
                ("alloc_ctx", C.c_void_p), ("adaptive", C.c_int32)]


BATCH_MAX_SHAPES = 16


class PfBatchTuning(C.Structure):
    _fields_ = [("n_shapes", C.c_uint32), ("block", C.c_uint32 * BATCH_MAX_SHAPES),
                ("grid", C.c_uint32 * BATCH_MAX_SHAPES), ("cluster", C.c_uint32 * BATCH_MAX_SHAPES),
                ("big_min", C.c_uint32 * BATCH_MAX_SHAPES), ("ms", C.c_float * BATCH_MAX_SHAPES),
                ("chosen", C.c_uint32)]


class PfBatchInfo(C.Structure):
    _fields_ = [("max_filters", C.c_uint32), ("resident", C.c_uint32),
                ("pool_particles", C.c_uint64), ("used_particles", C.c_uint64),
                ("bytes_per_particle", C.c_uint64), ("pool_bytes", C.c_uint64),
                ("grid", C.c_uint32), ("block", C.c_uint32), ("cluster", C.c_uint32),
                ("big_min", C.c_uint32), ("tuned", C.c_uint32), ("cycles", C.c_uint64)]


class PfServerOpts(C.Structure):
    _fields_ = [("max_streams", C.c_uint32), ("hbm_budget_bytes", C.c_uint64),
                ("scheme", C.c_int32), ("precision", C.c_int32),
                ("max_inflight", C.c_uint32), ("keep_results", C.c_int32),
                ("block", C.c_uint32), ("grid", C.c_uint32),
                ("cluster", C.c_uint32), ("big_min", C.c_uint32), ("warmup_s", C.c_double),
                ("stream", C.c_void_p), ("alloc", ALLOC_FN), ("free", FREE_FN),
                ("alloc_ctx", C.c_void_p), ("adaptive", C.c_int32)]


class PfServerResult(C.Structure):
    _fields_ = [("stream_id", C.c_uint64), ("seq", C.c_uint64), ("est", PfEstimates),
                ("latency_us", C.c_float), ("status", C.c_int32)]


class PfServerStats(C.Structure):
    _fields_ = [("submitted", C.c_uint64), ("completed", C.c_uint64),
                ("cycles", C.c_uint64), ("particle_steps", C.c_uint64),
                ("streams_opened", C.c_uint64), ("streams_closed", C.c_uint64),
                ("admitted", C.c_uint64), ("admitted_after_wait", C.c_uint64),
                ("waiting", C.c_uint32), ("resident", C.c_uint32),
                ("pool_particles", C.c_uint64), ("used_particles", C.c_uint64),
                ("mean_cycle_streams", C.c_double), ("max_cycle_streams", C.c_uint32),
                ("mean_admission_wait_us", C.c_double), ("replay_max_lag_us", C.c_double),
                ("wall_s", C.c_double), ("particle_steps_per_s", C.c_double),
                ("obs_per_s", C.c_double), ("mean_us", C.c_double), ("p50_us", C.c_double),
                ("p90_us", C.c_double), ("p99_us", C.c_double), ("max_us", C.c_double),
                ("steady_count", C.c_uint64), ("steady_p50_us", C.c_double),
                ("steady_p90_us", C.c_double), ("steady_p99_us", C.c_double),
                ("grid", C.c_uint32), ("block", C.c_uint32), ("cluster", C.c_uint32)]


EVENT_OBS, EVENT_CLOSE, EVENT_OPEN = 0, 1, 2

_V = C.c_void_p
_SIGS = {
    "pf_create": [C.POINTER(PfConfig), C.POINTER(_V)],
    "pf_step": [_V, C.c_double],
    "pf_step_ahead": [_V, C.c_double, C.c_double],
    "pf_run": [_V, _V, C.c_uint32],
    "pf_estimate": [_V, C.POINTER(PfEstimates)],
    "pf_step_estimate": [_V, C.c_double, C.POINTER(PfEstimates)],
    "pf_sync": [_V],
    "pf_step_profiled": [_V, C.c_double, C.POINTER(C.c_float), C.POINTER(C.c_char_p), C.c_int,
                         C.POINTER(C.c_int)],
    "pf_step_ahead_profiled": [_V, C.c_double, C.c_double, C.POINTER(C.c_float),
                               C.POINTER(C.c_char_p), C.c_int, C.POINTER(C.c_int)],
    "pf_get_particles": [_V, _V, _V, _V, _V, _V],
    "pf_get_ancestors": [_V, _V, _V],
    "pf_destroy": [_V],
    "pf_checkpoint_size": [_V, C.POINTER(C.c_size_t)],
    "pf_checkpoint": [_V, _V, C.c_size_t],
    "pf_restore": [C.POINTER(PfConfig), _V, C.c_size_t, C.POINTER(_V)],
    "pf_resample": [_V, C.c_uint64, C.c_uint64, C.c_uint32, C.c_uint32, C.c_int32, _V, _V],
    "pf_resample_noalloc": [_V, C.c_uint64, C.c_uint64, C.c_uint32, C.c_uint32, C.c_int32, _V,
                            _V],
    "pf_cdf": [_V, C.c_uint64, _V, _V],
    "pf_diag_cdf_wait": [_V, C.c_uint64, C.c_uint32, C.c_uint32, _V, _V],
    "pf_cutpoint_search": [_V, C.c_uint64, _V, _V],
    "pf_cutpoint_method": [_V, C.c_uint64, _V, _V, C.c_uint64, _V, _V],
    "pf_batch_create": [C.POINTER(PfConfig), C.c_uint32, C.POINTER(PfBatchOpts), C.POINTER(_V)],
    "pf_batch_add": [_V, C.POINTER(PfConfig), C.POINTER(C.c_uint32)],
    "pf_batch_remove": [_V, C.c_uint32],
    "pf_batch_step": [_V, _V, _V],
    "pf_batch_estimate": [_V, _V, C.POINTER(PfEstimates)],
    "pf_batch_tune": [_V, _V, _V, C.POINTER(PfBatchTuning)],
    "pf_batch_set_shape": [_V, C.c_uint32, C.c_uint32, C.c_uint32, C.c_uint32],
    "pf_batch_sync": [_V],
    "pf_batch_get_particles": [_V, C.c_uint32, _V, _V, _V, _V, _V],
    "pf_batch_get_ancestors": [_V, C.c_uint32, _V, _V],
    "pf_batch_get_info": [_V, C.POINTER(PfBatchInfo)],
    "pf_batch_destroy": [_V],
    "pf_server_create": [C.POINTER(PfServerOpts), C.POINTER(_V)],
    "pf_server_open": [_V, C.c_uint64, C.POINTER(PfConfig)],
    "pf_server_submit": [_V, C.c_uint64, C.c_double],
    "pf_server_close": [_V, C.c_uint64],
    "pf_server_replay": [_V, C.c_uint64, _V, _V, _V, _V, _V, C.c_uint64],
    "pf_server_drain": [_V, C.c_double],
    "pf_server_poll": [_V, C.POINTER(PfServerResult), C.c_uint32, C.POINTER(C.c_uint32)],
    "pf_server_get_stats": [_V, C.POINTER(PfServerStats)],
    "pf_server_destroy": [_V],
}
for _name, _args in _SIGS.items():
    _f = getattr(_lib, _name)
    _f.argtypes = _args
    _f.restype = C.c_int
_lib.pf_last_error.restype = C.c_char_p
_lib.pf_last_error.argtypes = []


class PfError(RuntimeError):
    def __init__(self, status, where):
        self.status = status
        msg = _lib.pf_last_error().decode(errors="replace")
        super().__init__("%s: %s (%s)" % (where, STATUS_NAMES.get(status, status), msg))


def _check(status, where):
    if status != PF_OK:
        raise PfError(status, where)


def last_error():
    return _lib.pf_last_error().decode(errors="replace")


def _torch():
    import torch
    return torch


def _stream_ptr(stream):
    torch = _torch()
    s = stream if stream is not None else torch.cuda.current_stream()
    return C.c_void_p(s.cuda_stream)


def _ptr(t):
    return C.c_void_p(t.data_ptr())


class TorchAllocator:
    """Device allocations of a filter handle through torch's caching allocator."""

    def __init__(self):
        torch = _torch()
        self.device = torch.cuda.current_device()

        def _alloc(nbytes, stream, ctx):
            try:
                return torch.cuda.caching_allocator_alloc(int(nbytes), self.device, stream)
            except Exception:
                return None

        def _free(ptr, stream, ctx):
            try:
                torch.cuda.caching_allocator_delete(ptr)
            except Exception:
                pass

        self.alloc = ALLOC_FN(_alloc)
        self.free = FREE_FN(_free)


def filter_config(n, seed=1212, filter_id=0, scheme="systematic", precision="fp32",
                  x0_mean=0.0, x0_var=10.0, a_sigma=3.0, b_sigma=2.0, a_tau=3.0, b_tau=2.0,
                  known_variances=False, sigma2=1.0, tau2=0.1, ess_frac=0.0):
    """A pf_config for one filter (stream and allocator fields left empty);
    ess_frac > 0: adaptive resampling (batches and servers created with
    adaptive=True)."""
    return PfConfig(n_particles=int(n), seed=int(seed), filter_id=int(filter_id),
                    scheme=SCHEMES[scheme] if isinstance(scheme, str) else int(scheme),
                    precision=FP64 if precision in ("fp64", FP64) else FP32,
                    known_variances=int(bool(known_variances)), x0_mean=x0_mean, x0_var=x0_var,
                    a_sigma=a_sigma, b_sigma=b_sigma, a_tau=a_tau, b_tau=b_tau,
                    sigma2=sigma2, tau2=tau2, ess_frac=float(ess_frac))


# Checkpoint header: magic, format version, header size, n, seed, filter id,
# scheme, precision, known variances, algorithm, pad, eight prior/variance
# doubles, t, log-ML, ess_frac, carried weights' sum, total size (see
# pf_checkpoint).
_CKPT_FMT = "<QIIQQIiiiii8dQdddQ"
_CKPT_HEAD = struct.calcsize(_CKPT_FMT)


def _ckpt_fields(head):
    v = struct.unpack(_CKPT_FMT, head[:_CKPT_HEAD])
    return int(v[3]), int(v[6]), int(v[7])


class Filter:
    """One particle-learning filter (paper Section 2, Algorithm "Particle Learning")."""

    def __init__(self, n, seed=1212, filter_id=0, scheme="systematic", precision="fp32",
                 x0_mean=0.0, x0_var=10.0, a_sigma=3.0, b_sigma=2.0, a_tau=3.0, b_tau=2.0,
                 known_variances=False, sigma2=1.0, tau2=0.1, stream=None, torch_alloc=True,
                 algorithm="pl", ess_frac=0.0):
        """algorithm: "pl" (Algorithm "Particle Learning") or "bootstrap"
        (Algorithm "Particle Filtering", with known_variances=True).
        ess_frac > 0: adaptive resampling (pf_config.ess_frac)."""
        torch = _torch()
        self.n = int(n)
        self.precision = FP64 if precision in ("fp64", FP64) else FP32
        self.scheme = SCHEMES[scheme] if isinstance(scheme, str) else int(scheme)
        # a real (non-legacy) stream: the cycle is captured as a CUDA graph on it
        self.stream = stream if stream is not None else torch.cuda.Stream()
        if self.stream.cuda_stream == 0:
            raise ValueError("pass a non-default torch.cuda.Stream (the cycle is graph-captured)")
        # torch_alloc: True for torch's caching allocator, False for the
        # library's own cudaMallocAsync, or an object with ctypes callbacks
        # .alloc / .free (ALLOC_FN / FREE_FN)
        self._alloc = TorchAllocator() if torch_alloc is True else (torch_alloc or None)
        cfg = PfConfig(n_particles=self.n, seed=seed, filter_id=filter_id, scheme=self.scheme,
                       precision=self.precision, known_variances=int(bool(known_variances)),
                       x0_mean=x0_mean, x0_var=x0_var, a_sigma=a_sigma, b_sigma=b_sigma,
                       a_tau=a_tau, b_tau=b_tau, sigma2=sigma2, tau2=tau2,
                       stream=C.c_void_p(self.stream.cuda_stream),
                       algorithm=ALGORITHMS[algorithm] if isinstance(algorithm, str) else int(algorithm),
                       ess_frac=float(ess_frac))
        if self._alloc is not None:
            cfg.alloc = self._alloc.alloc
            cfg.free = self._alloc.free
        self._cfg = cfg
        h = C.c_void_p()
        _check(_lib.pf_create(C.byref(cfg), C.byref(h)), "pf_create")
        self.h = h

    def step(self, y):
        _check(_lib.pf_step(self.h, float(y)), "pf_step")

    def step_ahead(self, y, y_next):
        """One cycle for y whose propagation also weighs the particles against
        y_next, the next call's observation (pf_step_ahead)."""
        _check(_lib.pf_step_ahead(self.h, float(y), float(y_next)), "pf_step_ahead")

    def run(self, y):
        """y: a float64 CUDA tensor (device-resident observations) or array-like."""
        torch = _torch()
        if isinstance(y, torch.Tensor) and y.is_cuda:
            y = y.to(torch.float64).contiguous()
            if self.stream != torch.cuda.current_stream():
                self.stream.wait_stream(torch.cuda.current_stream())
                y.record_stream(self.stream)
            _check(_lib.pf_run(self.h, _ptr(y), y.numel()), "pf_run")
        else:
            arr = np.ascontiguousarray(np.asarray(y, dtype=np.float64))
            _check(_lib.pf_run(self.h, arr.ctypes.data_as(C.c_void_p), arr.size), "pf_run")

    def sync(self):
        _check(_lib.pf_sync(self.h), "pf_sync")

    def step_profiled(self, y, y_next=None):
        """One cycle with per-kernel CUDA-event timing: {kernel name: ms}.
        With y_next, the cycle of step_ahead(y, y_next)."""
        ms = (C.c_float * 8)()
        names = (C.c_char_p * 8)()
        cnt = C.c_int()
        if y_next is None:
            _check(_lib.pf_step_profiled(self.h, float(y), ms, names, 8, C.byref(cnt)),
                   "pf_step_profiled")
        else:
            _check(_lib.pf_step_ahead_profiled(self.h, float(y), float(y_next), ms, names, 8,
                                               C.byref(cnt)), "pf_step_ahead_profiled")
        return {names[i].decode(): float(ms[i]) for i in range(cnt.value)}

    def estimate(self):
        e = PfEstimates()
        _check(_lib.pf_estimate(self.h, C.byref(e)), "pf_estimate")
        return {f: getattr(e, f) for f, _ in PfEstimates._fields_}

    def step_estimate(self, y):
        """One cycle and its posterior summaries (pf_step_estimate)."""
        e = PfEstimates()
        _check(_lib.pf_step_estimate(self.h, float(y), C.byref(e)), "pf_step_estimate")
        return {f: getattr(e, f) for f, _ in PfEstimates._fields_}

    def particles(self):
        torch = _torch()
        rt = torch.float64 if self.precision == FP64 else torch.float32
        bt = torch.float64 if self.precision == FP64 else torch.int64  # uint64 bits
        out = [torch.empty(self.n, dtype=rt, device="cuda") for _ in range(3)]
        out += [torch.empty(self.n, dtype=bt, device="cuda") for _ in range(2)]
        _check(_lib.pf_get_particles(self.h, *[_ptr(t) for t in out]), "pf_get_particles")
        return dict(zip(("x", "sigma2", "tau2", "b_sigma", "b_tau"), out))

    def ancestors(self, with_cdf=False):
        torch = _torch()
        anc = torch.empty(self.n, dtype=torch.int32, device="cuda")
        Q = torch.empty(self.n, dtype=torch.int64, device="cuda") if with_cdf else None
        _check(_lib.pf_get_ancestors(self.h, _ptr(anc), _ptr(Q) if Q is not None else None),
               "pf_get_ancestors")
        return (anc, Q) if with_cdf else anc

    def checkpoint(self, device=False):
        """The filter's checkpoint (pf_checkpoint): a numpy uint8 array, or a
        CUDA uint8 tensor with device=True."""
        torch = _torch()
        nb = C.c_size_t()
        _check(_lib.pf_checkpoint_size(self.h, C.byref(nb)), "pf_checkpoint_size")
        if device:
            buf = torch.empty(nb.value, dtype=torch.uint8, device="cuda")
            _check(_lib.pf_checkpoint(self.h, _ptr(buf), nb.value), "pf_checkpoint")
        else:
            buf = np.empty(nb.value, dtype=np.uint8)
            _check(_lib.pf_checkpoint(self.h, buf.ctypes.data_as(C.c_void_p), nb.value),
                   "pf_checkpoint")
        return buf

    @classmethod
    def restore(cls, blob, stream=None, torch_alloc=True):
        """A filter continuing from a checkpoint (pf_restore); blob is a numpy
        uint8 array or a CUDA uint8 tensor."""
        torch = _torch()
        self = cls.__new__(cls)
        self.h = None
        is_dev = isinstance(blob, torch.Tensor) and blob.is_cuda
        head = blob[:_CKPT_HEAD].cpu().numpy() if is_dev else np.asarray(blob[:_CKPT_HEAD])
        if head.size < _CKPT_HEAD:
            raise PfError(PF_ERR_INVALID, "pf_restore: checkpoint truncated")
        n, scheme, precision = _ckpt_fields(head.tobytes())
        self.n, self.scheme, self.precision = n, scheme, precision
        self.stream = stream if stream is not None else torch.cuda.Stream()
        if self.stream.cuda_stream == 0:
            raise ValueError("pass a non-default torch.cuda.Stream (the cycle is graph-captured)")
        # torch_alloc: True for torch's caching allocator, False for the
        # library's own cudaMallocAsync, or an object with ctypes callbacks
        # .alloc / .free (ALLOC_FN / FREE_FN)
        self._alloc = TorchAllocator() if torch_alloc is True else (torch_alloc or None)
        cfg = PfConfig(stream=C.c_void_p(self.stream.cuda_stream))
        if self._alloc is not None:
            cfg.alloc = self._alloc.alloc
            cfg.free = self._alloc.free
        self._cfg = cfg
        if is_dev:
            ptr, size = _ptr(blob), blob.numel()
        else:
            arr = np.ascontiguousarray(blob, dtype=np.uint8)
            ptr, size = arr.ctypes.data_as(C.c_void_p), arr.size
        h = C.c_void_p()
        _check(_lib.pf_restore(C.byref(cfg), ptr, size, C.byref(h)), "pf_restore")
        self.h = h
        return self

    def close(self):
        if getattr(self, "h", None):
            _lib.pf_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Batch:
    """Many independent filters advanced by one persistent launch per cycle
    (pf_batch_*).  `filters` is a list of dicts of filter_config() keyword
    arguments (n, seed, filter_id, priors, ...); scheme and precision are the
    batch's.  Slots are indexed 0..max_filters-1; the initial filters take
    slots 0..len(filters)-1."""

    def __init__(self, filters=(), scheme="systematic", precision="fp32", max_filters=0,
                 hbm_budget_bytes=0, autotune=False, stream=None, torch_alloc=True,
                 adaptive=False):
        torch = _torch()
        self.scheme = SCHEMES[scheme] if isinstance(scheme, str) else int(scheme)
        self.precision = FP64 if precision in ("fp64", FP64) else FP32
        self.stream = stream if stream is not None else torch.cuda.Stream()
        if self.stream.cuda_stream == 0:
            raise ValueError("pass a non-default torch.cuda.Stream (the cycle is graph-captured)")
        self._alloc = TorchAllocator() if torch_alloc is True else (torch_alloc or None)
        cfgs = [self._cfg(f) for f in filters]
        arr = (PfConfig * max(len(cfgs), 1))(*cfgs)
        opts = PfBatchOpts(max_filters=int(max_filters), hbm_budget_bytes=int(hbm_budget_bytes),
                           scheme=self.scheme, precision=self.precision,
                           autotune=int(bool(autotune)), adaptive=int(bool(adaptive)),
                           stream=C.c_void_p(self.stream.cuda_stream))
        if self._alloc is not None:
            opts.alloc = self._alloc.alloc
            opts.free = self._alloc.free
        self._opts = opts
        h = C.c_void_p()
        _check(_lib.pf_batch_create(arr, len(cfgs), C.byref(opts), C.byref(h)), "pf_batch_create")
        self.h = h
        self.max_filters = self.info()["max_filters"]
        self._n = {}
        for i, f in enumerate(filters):
            self._n[i] = int(f["n"])

    def _cfg(self, f):
        kw = dict(f)
        kw["scheme"] = self.scheme
        kw["precision"] = self.precision
        return filter_config(**kw)

    def add(self, **f):
        """Admit one filter; returns its slot, or raises PfError (PF_ERR_BUSY
        when the pool or the slots are full)."""
        cfg = self._cfg(f)
        slot = C.c_uint32()
        _check(_lib.pf_batch_add(self.h, C.byref(cfg), C.byref(slot)), "pf_batch_add")
        self._n[slot.value] = int(f["n"])
        return slot.value

    def try_add(self, **f):
        """add(), but None instead of an exception when admission is refused."""
        cfg = self._cfg(f)
        slot = C.c_uint32()
        st = _lib.pf_batch_add(self.h, C.byref(cfg), C.byref(slot))
        if st == PF_ERR_BUSY:
            return None
        _check(st, "pf_batch_add")
        self._n[slot.value] = int(f["n"])
        return slot.value

    def remove(self, slot):
        _check(_lib.pf_batch_remove(self.h, int(slot)), "pf_batch_remove")
        self._n.pop(int(slot), None)

    def step(self, y, mask=None):
        """y: float64 array of max_filters observations (indexed by slot);
        mask: optional uint8/bool array selecting the filters to step."""
        y = np.ascontiguousarray(np.asarray(y, dtype=np.float64))
        assert y.size >= self.max_filters
        mp = None
        if mask is not None:
            mask = np.ascontiguousarray(np.asarray(mask, dtype=np.uint8))
            assert mask.size >= self.max_filters
            mp = mask.ctypes.data_as(C.c_void_p)
        _check(_lib.pf_batch_step(self.h, y.ctypes.data_as(C.c_void_p), mp), "pf_batch_step")

    def sync(self):
        _check(_lib.pf_batch_sync(self.h), "pf_batch_sync")

    def tune(self, y, mask=None):
        """Time the candidate launch shapes on trial cycles (which change no
        result) and keep the fastest; returns [(block, grid, ms)] and the
        chosen index."""
        y = np.ascontiguousarray(np.asarray(y, dtype=np.float64))
        mp = None
        if mask is not None:
            mask = np.ascontiguousarray(np.asarray(mask, dtype=np.uint8))
            mp = mask.ctypes.data_as(C.c_void_p)
        out = PfBatchTuning()
        _check(_lib.pf_batch_tune(self.h, y.ctypes.data_as(C.c_void_p), mp, C.byref(out)),
               "pf_batch_tune")
        shapes = [dict(block=out.block[i], grid=out.grid[i], cluster=out.cluster[i],
                       big_min=out.big_min[i], ms=out.ms[i]) for i in range(out.n_shapes)]
        return shapes, out.chosen

    def set_shape(self, block, grid, cluster=1, big_min=0):
        _check(_lib.pf_batch_set_shape(self.h, int(block), int(grid), int(cluster), int(big_min)),
               "pf_batch_set_shape")

    def estimates(self, mask=None):
        """{slot: summaries dict} for the selected resident filters."""
        out = (PfEstimates * self.max_filters)()
        mp = None
        if mask is not None:
            mask = np.ascontiguousarray(np.asarray(mask, dtype=np.uint8))
            mp = mask.ctypes.data_as(C.c_void_p)
        _check(_lib.pf_batch_estimate(self.h, mp, out), "pf_batch_estimate")
        sel = [s for s in self._n if mask is None or mask[s]]
        return {s: {f: getattr(out[s], f) for f, _ in PfEstimates._fields_} for s in sel}

    def particles(self, slot):
        torch = _torch()
        n = self._n[int(slot)]
        rt = torch.float64 if self.precision == FP64 else torch.float32
        bt = torch.float64 if self.precision == FP64 else torch.int64
        out = [torch.empty(n, dtype=rt, device="cuda") for _ in range(3)]
        out += [torch.empty(n, dtype=bt, device="cuda") for _ in range(2)]
        _check(_lib.pf_batch_get_particles(self.h, int(slot), *[_ptr(t) for t in out]),
               "pf_batch_get_particles")
        return dict(zip(("x", "sigma2", "tau2", "b_sigma", "b_tau"), out))

    def ancestors(self, slot, with_cdf=False):
        torch = _torch()
        n = self._n[int(slot)]
        anc = torch.empty(n, dtype=torch.int32, device="cuda")
        Q = torch.empty(n, dtype=torch.int64, device="cuda") if with_cdf else None
        _check(_lib.pf_batch_get_ancestors(self.h, int(slot), _ptr(anc),
                                           _ptr(Q) if Q is not None else None),
               "pf_batch_get_ancestors")
        return (anc, Q) if with_cdf else anc

    def info(self):
        i = PfBatchInfo()
        _check(_lib.pf_batch_get_info(self.h, C.byref(i)), "pf_batch_get_info")
        return {f: getattr(i, f) for f, _ in PfBatchInfo._fields_}

    def close(self):
        if getattr(self, "h", None):
            _lib.pf_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Server:
    """Continuous-batching server of filter streams (pf_server_*): streams
    open, receive observations at any time and close; a library worker thread
    batches the pending observations of all resident streams into batched
    cycles; streams are admitted in FIFO order within an HBM budget."""

    def __init__(self, max_streams, hbm_budget_bytes, scheme="systematic", precision="fp32",
                 max_inflight=2, keep_results=False, block=0, grid=0, cluster=0, big_min=0,
                 warmup_s=0.0, stream=None, torch_alloc=True, adaptive=False):
        torch = _torch()
        self.scheme = SCHEMES[scheme] if isinstance(scheme, str) else int(scheme)
        self.precision = FP64 if precision in ("fp64", FP64) else FP32
        self.stream = stream if stream is not None else torch.cuda.Stream()
        if self.stream.cuda_stream == 0:
            raise ValueError("pass a non-default torch.cuda.Stream (cycles are graph-captured)")
        self._alloc = TorchAllocator() if torch_alloc else None
        opts = PfServerOpts(max_streams=int(max_streams), hbm_budget_bytes=int(hbm_budget_bytes),
                            scheme=self.scheme, precision=self.precision,
                            max_inflight=int(max_inflight), keep_results=int(bool(keep_results)),
                            block=int(block), grid=int(grid), cluster=int(cluster),
                            big_min=int(big_min), warmup_s=float(warmup_s),
                            adaptive=int(bool(adaptive)),
                            stream=C.c_void_p(self.stream.cuda_stream))
        if self._alloc is not None:
            opts.alloc = self._alloc.alloc
            opts.free = self._alloc.free
        self._opts = opts
        h = C.c_void_p()
        _check(_lib.pf_server_create(C.byref(opts), C.byref(h)), "pf_server_create")
        self.h = h

    def config(self, **f):
        kw = dict(f)
        kw["scheme"] = self.scheme
        kw["precision"] = self.precision
        return filter_config(**kw)

    def open(self, stream_id, **f):
        cfg = self.config(**f)
        _check(_lib.pf_server_open(self.h, int(stream_id), C.byref(cfg)), "pf_server_open")

    def submit(self, stream_id, y):
        _check(_lib.pf_server_submit(self.h, int(stream_id), float(y)), "pf_server_submit")

    def close_stream(self, stream_id):
        _check(_lib.pf_server_close(self.h, int(stream_id)), "pf_server_close")

    def replay(self, t_s, kind, ids, y, cfgs=()):
        """Events at times t_s (seconds from now): kind EVENT_OBS (submit y to
        ids), EVENT_CLOSE, EVENT_OPEN (with cfgs[id], a list of dicts)."""
        t_s = np.ascontiguousarray(t_s, dtype=np.float64)
        kind = np.ascontiguousarray(kind, dtype=np.uint8)
        ids = np.ascontiguousarray(ids, dtype=np.uint64)
        y = np.ascontiguousarray(y, dtype=np.float64)
        arr = (PfConfig * max(len(cfgs), 1))(*[self.config(**c) for c in cfgs])
        _check(_lib.pf_server_replay(self.h, t_s.size, t_s.ctypes.data_as(C.c_void_p),
                                     kind.ctypes.data_as(C.c_void_p),
                                     ids.ctypes.data_as(C.c_void_p), y.ctypes.data_as(C.c_void_p),
                                     arr, len(cfgs)), "pf_server_replay")

    def drain(self, timeout_s=600.0):
        _check(_lib.pf_server_drain(self.h, float(timeout_s)), "pf_server_drain")

    def poll(self, max_results=1 << 16):
        """Finished results: list of (stream_id, seq, summaries dict, latency_us, status)."""
        buf = (PfServerResult * max_results)()
        out = []
        while True:
            n = C.c_uint32()
            _check(_lib.pf_server_poll(self.h, buf, max_results, C.byref(n)), "pf_server_poll")
            for i in range(n.value):
                r = buf[i]
                est = {f: getattr(r.est, f) for f, _ in PfEstimates._fields_}
                out.append((r.stream_id, r.seq, est, r.latency_us, r.status))
            if n.value < max_results:
                return out

    def stats(self):
        st = PfServerStats()
        _check(_lib.pf_server_get_stats(self.h, C.byref(st)), "pf_server_get_stats")
        return {f: getattr(st, f) for f, _ in PfServerStats._fields_}

    def close(self):
        if getattr(self, "h", None):
            _lib.pf_server_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _resample_out(w, out):
    """The caller's int32 output on w's device with room for n ancestors, or a
    new one."""
    torch = _torch()
    assert w.is_cuda and w.dtype == torch.float32 and w.is_contiguous()
    n = w.numel()
    if out is None:
        return torch.empty(n, dtype=torch.int32, device=w.device)
    if out.dtype != torch.int32 or out.device != w.device or not out.is_contiguous():
        raise ValueError("out must be a contiguous int32 tensor on %s" % w.device)
    if out.numel() < n:
        raise ValueError("out holds %d ancestors, %d needed" % (out.numel(), n))
    return out


def _on_device(dev, fn):
    """fn() with dev current (the library works on the current device)."""
    torch = _torch()
    if dev.index == torch.cuda.current_device():
        return fn()
    with torch.cuda.device(dev):
        return fn()


def resample(w, seed, filter_id=0, t=0, scheme="systematic", out=None, stream=None):
    """Ancestors (int32 CUDA tensor viewed as uint32) for float32 CUDA weights w."""
    anc = _resample_out(w, out)
    sch = SCHEMES[scheme] if isinstance(scheme, str) else int(scheme)
    _check(_on_device(w.device, lambda: _lib.pf_resample(
        _ptr(w), w.numel(), seed, filter_id, t, sch, _ptr(anc), _stream_ptr(stream))), "pf_resample")
    return anc


def resample_noalloc(w, seed, filter_id=0, t=0, scheme="systematic", out=None, stream=None):
    """As resample(), through pf_resample_noalloc: the library allocates nothing
    (its scratch is a fixed device array, n <= NOALLOC_MAX_PARTICLES); `out`,
    when given, is the caller's preallocated int32 output."""
    anc = _resample_out(w, out)
    sch = SCHEMES[scheme] if isinstance(scheme, str) else int(scheme)
    _check(_on_device(w.device, lambda: _lib.pf_resample_noalloc(  # the fixed array of w's device
        _ptr(w), w.numel(), seed, filter_id, t, sch, _ptr(anc), _stream_ptr(stream))),
        "pf_resample_noalloc")
    return anc


def cdf(w, stream=None):
    torch = _torch()
    assert w.is_cuda and w.dtype == torch.float32 and w.is_contiguous()
    Q = torch.empty(w.numel(), dtype=torch.int64, device=w.device)
    _check(_lib.pf_cdf(_ptr(w), w.numel(), _ptr(Q), _stream_ptr(stream)), "pf_cdf")
    return Q


def diag_cdf_wait(w, withhold_tile, spin_limit, stream=None):
    """pf_diag_cdf_wait: pf_cdf with the look-back wait's test settings.
    Returns (status code, Q); Q is valid only when the status is PF_OK."""
    torch = _torch()
    assert w.is_cuda and w.dtype == torch.float32 and w.is_contiguous()
    Q = torch.empty(w.numel(), dtype=torch.int64, device=w.device)
    with torch.cuda.device(w.device):
        st = _lib.pf_diag_cdf_wait(_ptr(w), w.numel(), int(withhold_tile), int(spin_limit), _ptr(Q),
                                   _stream_ptr(stream))
    return st, Q


def cutpoint_search(Q, stream=None):
    torch = _torch()
    I = torch.empty(Q.numel(), dtype=torch.int32, device=Q.device)
    _check(_lib.pf_cutpoint_search(_ptr(Q), Q.numel(), _ptr(I), _stream_ptr(stream)),
           "pf_cutpoint_search")
    return I


def cutpoint_method(Q, I, U, stream=None):
    torch = _torch()
    anc = torch.empty(U.numel(), dtype=torch.int32, device=Q.device)
    _check(_lib.pf_cutpoint_method(_ptr(Q), Q.numel(), _ptr(I), _ptr(U), U.numel(), _ptr(anc),
                                   _stream_ptr(stream)), "pf_cutpoint_method")
    return anc
