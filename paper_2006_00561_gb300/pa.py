"""Python binding of the C ABI in include/pa.h (ctypes, argument marshalling only).

Every step of the method runs in the CUDA kernels of libpa_gb300.so; this
module only converts arguments.  PyTorch provides the device workspace
(``torch.empty(..., dtype=torch.uint8, device='cuda')``) and the stream.
Importing the module works without a GPU (the host-only entry points
pa_workspace_size / pa_tables / pa_num_bins need none); creating a run needs
the library and a CUDA device and raises if either is missing.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libpa_gb300.so")

PA_OK = 0
ERRORS = {
    -1: "PA_ERR_INVALID_ARG", -2: "PA_ERR_ODD_L", -3: "PA_ERR_UNSUPPORTED", -4: "PA_ERR_CAPACITY",
    -5: "PA_ERR_TIMEOUT", -6: "PA_ERR_CUDA", -7: "PA_ERR_WORKSPACE", -8: "PA_ERR_DONE",
    -9: "PA_ERR_EMPTY", -10: "PA_ERR_INVARIANT",
}
MODEL_FERRO, MODEL_PMJ = 0, 1
INIT_RANDOM, INIT_GROUND = 0, 1
RESAMPLE_NEAREST, RESAMPLE_POISSON, RESAMPLE_MULTINOMIAL = 0, 1, 2
LAYOUT_INT8, LAYOUT_PACKED = 0, 1
(DUMP_SPINS, DUMP_EBIN, DUMP_MAG, DUMP_HIST, DUMP_COUNTS, DUMP_OFFSETS, DUMP_TAB_N, DUMP_TAB_F,
 DUMP_COUPLINGS, DUMP_SPINS_RAW, DUMP_STATE) = range(11)

EXPORTS = [
    "pa_workspace_size", "pa_init", "pa_resample", "pa_sweep", "pa_step", "pa_run_steps",
    "pa_observables", "pa_observables_history", "pa_status", "pa_dump_size", "pa_dump",
    "pa_dump_range", "pa_load", "pa_profile", "pa_profile_read",
    "pa_tables", "pa_num_bins", "pa_free", "pa_strerror", "pa_copy_counts_scan_noalloc",
    "pa_batch_workspace_size", "pa_batch_init", "pa_batch_step", "pa_batch_run_steps",
    "pa_batch_sync", "pa_batch_num_classes", "pa_batch_class_info", "pa_batch_set_shape",
    "pa_batch_free", "pa_checkpoint_size", "pa_checkpoint", "pa_restore",
    "pa_adaptive_beta", "pa_resample_to", "pa_poisson1_table", "pa_step_stream", "pa_debug",
    "pa_bench_philox_threads", "pa_bench_philox", "pa_bench_intops_threads",
    "pa_bench_intops_per_iter", "pa_bench_intops", "pa_batch_profile", "pa_batch_profile_read",
    "pa_resample_begin", "pa_resample_finish", "pa_batch_init_async",
]
MAX_SEGMENTS = 1024
(INTOPS_LOP3, INTOPS_IMAD, INTOPS_WIDE, INTOPS_LOP3_IMAD, INTOPS_LOP3_WIDE,
 INTOPS_MULWIDE_XOR) = range(6)
DEBUG_WITHHOLD_PREFIX = 1
NOALLOC_MAX_REPLICAS = 8388608


class PaError(RuntimeError):
    def __init__(self, code: int, what: str = ""):
        self.code = code
        super().__init__(f"{what}: {ERRORS.get(code, code)} ({strerror(code)})")


class Config(C.Structure):
    _fields_ = [
        ("dim", C.c_int32), ("L", C.c_int32), ("model", C.c_int32), ("layout", C.c_int32),
        ("K", C.c_int32), ("theta", C.c_int32), ("instance_id", C.c_int32),
        ("init", C.c_int32), ("R0", C.c_int64), ("capacity", C.c_int64),
        ("beta0", C.c_double), ("beta_max", C.c_double),
        ("seed", C.c_uint64), ("coupling_seed", C.c_uint64),
        ("resample", C.c_int32), ("reserved", C.c_int32),
    ]


class Obs(C.Structure):
    _fields_ = [
        ("step", C.c_int64), ("R", C.c_int64),
        ("sumE", C.c_int64), ("sumE2", C.c_int64), ("sumAbsM", C.c_int64), ("sumM2", C.c_int64),
        ("beta", C.c_double), ("lnQ", C.c_double), ("lnZ", C.c_double),
        ("e", C.c_double), ("cv", C.c_double), ("m_abs", C.c_double), ("chi", C.c_double),
    ]

    def as_dict(self) -> dict:
        return {n: getattr(self, n) for n, _ in self._fields_}


class State(C.Structure):
    _fields_ = [
        ("step", C.c_int64), ("R", C.c_int64), ("R_prev", C.c_int64), ("kref", C.c_int64),
        ("sweeps_done", C.c_int64), ("status_bits", C.c_int64),
        ("lnQ", C.c_double), ("lnZ", C.c_double), ("S", C.c_double),
        ("N", C.c_int64), ("bins", C.c_int64), ("stride", C.c_int64), ("capacity", C.c_int64),
        ("parity", C.c_int64), ("sources", C.c_int64),
    ]

    def as_dict(self) -> dict:
        return {n: getattr(self, n) for n, _ in self._fields_}


def make_config(dim=2, L=16, model=MODEL_FERRO, layout=LAYOUT_PACKED, K=100, theta=10,
                instance_id=0, R0=1000, capacity=0, beta0=0.0, beta_max=1.0, seed=1,
                coupling_seed=0, init=INIT_RANDOM, resample=RESAMPLE_NEAREST) -> Config:
    return Config(dim, L, model, layout, K, theta, instance_id, init, R0, capacity, beta0,
                  beta_max, seed, coupling_seed, resample, 0)


_lib = None


def lib():
    """The loaded engine; raises if libpa_gb300.so was not built."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(
                f"{LIB_PATH} is missing: build it with paper_2006_00561_gb300.build.build()")
        L = C.CDLL(LIB_PATH)
        vp, cfgp = C.c_void_p, C.POINTER(Config)
        L.pa_workspace_size.argtypes = [cfgp]
        L.pa_workspace_size.restype = C.c_size_t
        L.pa_init.argtypes = [cfgp, vp, C.c_size_t, vp, C.POINTER(vp)]
        for n in ("pa_resample", "pa_step", "pa_status", "pa_resample_begin"):
            getattr(L, n).argtypes = [vp]
        L.pa_resample_finish.argtypes = [vp, C.c_int32, C.POINTER(C.c_int64),
                                         C.POINTER(C.c_int64)]
        L.pa_sweep.argtypes = [vp, C.c_int32]
        L.pa_run_steps.argtypes = [vp, C.c_int32]
        L.pa_step_stream.argtypes = [vp, vp, C.c_size_t, C.c_int32, vp, C.POINTER(C.c_int64)]
        L.pa_debug.argtypes = [vp, C.c_uint32]
        L.pa_bench_philox_threads.argtypes = []
        L.pa_bench_philox_threads.restype = C.c_int64
        L.pa_bench_philox.argtypes = [C.c_uint64, C.c_int32, vp, C.c_int64, vp]
        for n in ("pa_bench_intops_threads", "pa_bench_intops_per_iter"):
            getattr(L, n).argtypes = []
            getattr(L, n).restype = C.c_int64
        L.pa_bench_intops.argtypes = [C.c_int32, C.c_int32, vp, C.c_int64, vp]
        L.pa_observables.argtypes = [vp, C.POINTER(Obs)]
        L.pa_observables_history.argtypes = [vp, C.c_int32, C.c_int32, C.POINTER(Obs)]
        L.pa_dump_size.argtypes = [vp, C.c_int32]
        L.pa_dump_size.restype = C.c_int64
        L.pa_dump.argtypes = [vp, C.c_int32, vp, C.c_size_t]
        L.pa_dump_range.argtypes = [vp, C.c_int32, C.c_int64, C.c_int64, vp, C.c_size_t]
        L.pa_load.argtypes = [vp, C.c_int32, vp, C.c_int64, C.c_size_t]
        L.pa_profile.argtypes = [vp, C.c_int32]
        L.pa_profile_read.argtypes = [vp, C.POINTER(C.c_int64), C.POINTER(C.c_double), C.c_int32]
        L.pa_tables.argtypes = [cfgp, C.c_int32, C.POINTER(C.c_uint64), C.POINTER(C.c_double),
                                C.c_int64]
        L.pa_poisson1_table.argtypes = [C.POINTER(C.c_uint32), C.c_int32]
        L.pa_num_bins.argtypes = [C.c_int32, C.c_int32]
        L.pa_num_bins.restype = C.c_int64
        L.pa_free.argtypes = [vp]
        L.pa_free.restype = None
        L.pa_copy_counts_scan_noalloc.argtypes = [vp, C.c_int64, vp, vp, C.c_int64, C.c_uint64,
                                                   C.c_int32, C.c_int32, vp, vp, vp, vp]
        L.pa_batch_workspace_size.argtypes = [C.c_int32]
        L.pa_batch_workspace_size.restype = C.c_size_t
        L.pa_batch_init.argtypes = [C.POINTER(vp), C.c_int32, vp, C.c_size_t, vp, C.POINTER(vp)]
        L.pa_batch_init_async.argtypes = [C.POINTER(vp), C.c_int32, C.POINTER(C.c_int32), vp,
                                          C.c_size_t, vp, C.POINTER(vp)]
        for n in ("pa_batch_step", "pa_batch_sync", "pa_batch_num_classes"):
            getattr(L, n).argtypes = [vp]
        L.pa_batch_run_steps.argtypes = [vp, C.c_int32]
        L.pa_batch_profile.argtypes = [vp, C.c_int32]
        L.pa_batch_profile_read.argtypes = [vp, C.POINTER(C.c_int64), C.POINTER(C.c_double),
                                            C.c_int32]
        L.pa_batch_class_info.argtypes = [vp, C.c_int32, C.POINTER(C.c_int32)]
        L.pa_batch_set_shape.argtypes = [vp, C.c_int32, C.c_int32, C.c_int32]
        L.pa_batch_free.argtypes = [vp]
        L.pa_batch_free.restype = None
        L.pa_adaptive_beta.argtypes = [vp, C.c_double, C.c_double, C.POINTER(C.c_double)]
        L.pa_resample_to.argtypes = [vp, C.c_double]
        L.pa_checkpoint_size.argtypes = [vp]
        L.pa_checkpoint_size.restype = C.c_int64
        L.pa_checkpoint.argtypes = [vp, vp, C.c_size_t]
        L.pa_restore.argtypes = [vp, vp, C.c_size_t]
        L.pa_strerror.argtypes = [C.c_int]
        L.pa_strerror.restype = C.c_char_p
        _lib = L
    return _lib


def strerror(code: int) -> str:
    try:
        return lib().pa_strerror(code).decode()
    except Exception:
        return ERRORS.get(code, "unknown")


def _check(rc: int, what: str):
    if rc != PA_OK:
        raise PaError(rc, what)


# ---- the C ABI, name for name ------------------------------------------------
def pa_workspace_size(cfg: Config) -> int:
    return int(lib().pa_workspace_size(C.byref(cfg)))


def pa_poisson1_table() -> np.ndarray:
    T = np.zeros(32, dtype=np.uint32)
    n = lib().pa_poisson1_table(T.ctypes.data_as(C.POINTER(C.c_uint32)), 32)
    if n < 0:
        raise PaError(n, "pa_poisson1_table")
    return T[:n].copy()


def pa_num_bins(dim: int, L: int) -> int:
    return int(lib().pa_num_bins(dim, L))


def pa_tables(cfg: Config, step: int, bins: int | None = None):
    """(T[3] uint64, D[bins] float64) exactly as the engine uploads them."""
    if bins is None:
        bins = pa_num_bins(cfg.dim, cfg.L)
    T = np.zeros(3, dtype=np.uint64)
    D = np.zeros(bins, dtype=np.float64)
    _check(lib().pa_tables(C.byref(cfg), step, T.ctypes.data_as(C.POINTER(C.c_uint64)),
                           D.ctypes.data_as(C.POINTER(C.c_double)), bins), "pa_tables")
    return T, D


def pa_init(cfg: Config, workspace_ptr: int, nbytes: int, stream_handle: int) -> int:
    h = C.c_void_p()
    _check(lib().pa_init(C.byref(cfg), C.c_void_p(workspace_ptr), nbytes,
                         C.c_void_p(stream_handle), C.byref(h)), "pa_init")
    return h.value


def pa_resample(h: int):
    _check(lib().pa_resample(C.c_void_p(h)), "pa_resample")


def pa_sweep(h: int, nsweeps: int):
    _check(lib().pa_sweep(C.c_void_p(h), nsweeps), "pa_sweep")


def pa_step(h: int):
    _check(lib().pa_step(C.c_void_p(h)), "pa_step")


def pa_run_steps(h: int, nsteps: int):
    _check(lib().pa_run_steps(C.c_void_p(h), nsteps), "pa_run_steps")


def pa_bench_philox_threads() -> int:
    return int(lib().pa_bench_philox_threads())


def pa_bench_philox(seed: int, halfsweeps: int, out_ptr: int, out_words: int, stream_handle: int):
    """The register kernels' generator alone: one xor word per thread at out_ptr."""
    _check(lib().pa_bench_philox(seed, halfsweeps, C.c_void_p(out_ptr), out_words,
                                 C.c_void_p(stream_handle)), "pa_bench_philox")


def pa_bench_intops_threads() -> int:
    return int(lib().pa_bench_intops_threads())


def pa_bench_intops_per_iter() -> int:
    return int(lib().pa_bench_intops_per_iter())


def pa_bench_intops(kind: int, iters: int, out_ptr: int, out_words: int, stream_handle: int):
    _check(lib().pa_bench_intops(kind, iters, C.c_void_p(out_ptr), out_words,
                                 C.c_void_p(stream_handle)), "pa_bench_intops")


def pa_debug(h: int, flags: int):
    """Test hooks of the failure paths (DEBUG_WITHHOLD_PREFIX)."""
    _check(lib().pa_debug(C.c_void_p(h), flags), "pa_debug")


def pa_step_stream(h: int, host_ptr: int, nbytes: int, chunks: int, copy_stream_handle: int) -> int:
    """pa_step with the population copied to host_ptr range by range; returns R_i."""
    R = C.c_int64(-1)
    _check(lib().pa_step_stream(C.c_void_p(h), C.c_void_p(host_ptr), nbytes, chunks,
                                C.c_void_p(copy_stream_handle), C.byref(R)), "pa_step_stream")
    return R.value


def pa_observables(h: int, check: bool = True) -> dict:
    o = Obs()
    rc = lib().pa_observables(C.c_void_p(h), C.byref(o))
    if check:
        _check(rc, "pa_observables")
    return o.as_dict()


def pa_observables_history(h: int, first: int, n: int) -> list:
    arr = (Obs * max(n, 1))()
    _check(lib().pa_observables_history(C.c_void_p(h), first, n, arr), "pa_observables_history")
    return [arr[i].as_dict() for i in range(n)]


def pa_status(h: int) -> int:
    return int(lib().pa_status(C.c_void_p(h)))


_DUMP_DTYPES = {
    DUMP_SPINS: np.int8, DUMP_EBIN: np.uint32, DUMP_MAG: np.int32, DUMP_HIST: np.uint32,
    DUMP_COUNTS: np.uint32, DUMP_OFFSETS: np.uint32, DUMP_TAB_N: np.uint32, DUMP_TAB_F: np.uint32,
    DUMP_COUPLINGS: np.int8, DUMP_SPINS_RAW: np.uint8,
}


def pa_dump(h: int, what: int):
    n = int(lib().pa_dump_size(C.c_void_p(h), what))
    if n < 0:
        raise PaError(-1, "pa_dump_size")
    if what == DUMP_STATE:
        s = State()
        _check(lib().pa_dump(C.c_void_p(h), what, C.byref(s), C.sizeof(s)), "pa_dump")
        return s.as_dict()
    buf = np.zeros(max(n, 1), dtype=np.uint8)
    _check(lib().pa_dump(C.c_void_p(h), what, C.c_void_p(buf.ctypes.data), buf.size), "pa_dump")
    return buf[:n].view(_DUMP_DTYPES[what]).copy()


def pa_dump_range(h: int, what: int, first: int, count: int, N: int = 0, stride: int = 0):
    per = {DUMP_SPINS: N, DUMP_SPINS_RAW: stride}.get(what, 4)
    buf = np.zeros(max(count * per, 1), dtype=np.uint8)
    _check(lib().pa_dump_range(C.c_void_p(h), what, first, count, C.c_void_p(buf.ctypes.data),
                               buf.size), "pa_dump_range")
    out = buf[:count * per].view(_DUMP_DTYPES[what]).copy()
    return out.reshape(count, -1) if what in (DUMP_SPINS, DUMP_SPINS_RAW) else out


def pa_load(h: int, what: int, src: np.ndarray, count: int):
    """Uploads `count` replicas from host array `src` (int8 site order or raw layout)."""
    assert src.flags.c_contiguous
    _check(lib().pa_load(C.c_void_p(h), what, C.c_void_p(src.ctypes.data), count, src.nbytes),
           "pa_load")


def pa_load_ptr(h: int, what: int, ptr: int, count: int, nbytes: int):
    """Same as pa_load from a raw host pointer (e.g. pinned torch memory)."""
    _check(lib().pa_load(C.c_void_p(h), what, C.c_void_p(ptr), count, nbytes), "pa_load")


def pa_profile(h: int, enable: bool):
    _check(lib().pa_profile(C.c_void_p(h), 1 if enable else 0), "pa_profile")


def pa_profile_read(h: int, reset: bool = True):
    n = (C.c_int64 * 4)()
    ms = (C.c_double * 4)()
    _check(lib().pa_profile_read(C.c_void_p(h), n, ms, 1 if reset else 0), "pa_profile_read")
    kinds = ("tau", "resample", "sweep", "obs")
    return {k: (int(n[i]), float(ms[i])) for i, k in enumerate(kinds)}


def pa_free(h: int):
    if h:
        lib().pa_free(C.c_void_p(h))


def pa_copy_counts_scan_noalloc(ebin_ptr: int, R: int, tab_n_ptr: int, tab_F_ptr: int, bins: int,
                                seed: int, step: int, instance_id: int, counts_ptr: int,
                                offsets_ptr: int, total_ptr: int, stream_handle: int):
    """Copy counts + exclusive scan into caller-owned device buffers (device
    pointers as ints); allocates nothing.  See include/pa.h."""
    _check(lib().pa_copy_counts_scan_noalloc(
        C.c_void_p(ebin_ptr), R, C.c_void_p(tab_n_ptr), C.c_void_p(tab_F_ptr), bins, seed, step,
        instance_id, C.c_void_p(counts_ptr), C.c_void_p(offsets_ptr), C.c_void_p(total_ptr),
        C.c_void_p(stream_handle)), "pa_copy_counts_scan_noalloc")


# ---- convenience: a run that owns its torch workspace ------------------------
class Run:
    """One PA run on the current CUDA device.

    The workspace is a torch uint8 tensor (the library never allocates device
    memory); the stream defaults to torch's current stream.
    """

    def __init__(self, cfg: Config, stream=None, workspace=None):
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("a CUDA device is required")
        lib()
        self.cfg = cfg
        self.nbytes = pa_workspace_size(cfg)
        if self.nbytes == 0:
            raise PaError(-1, "pa_workspace_size")
        if workspace is None:
            workspace = torch.empty(self.nbytes, dtype=torch.uint8, device="cuda")
        self.workspace = workspace
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        self.h = pa_init(cfg, workspace.data_ptr(), workspace.numel(), self.stream.cuda_stream)
        self.N = cfg.L ** cfg.dim

    def close(self):
        if getattr(self, "h", None):
            pa_free(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def resample(self):
        pa_resample(self.h)

    def resample_begin(self):
        """Reweight, copy counts and scan of the next step, gather pending."""
        _check(lib().pa_resample_begin(C.c_void_p(self.h)), "pa_resample_begin")

    def resample_finish(self, segments):
        """Gather of the pending resample into the slot order given by
        [(first new slot, length), ...] (post-exchange order)."""
        seg = np.asarray(segments, dtype=np.int64).reshape(-1, 2)
        src = np.ascontiguousarray(seg[:, 0])
        ln = np.ascontiguousarray(seg[:, 1])
        _check(lib().pa_resample_finish(C.c_void_p(self.h), int(seg.shape[0]),
                                        src.ctypes.data_as(C.POINTER(C.c_int64)),
                                        ln.ctypes.data_as(C.POINTER(C.c_int64))),
               "pa_resample_finish")

    def sweep(self, n: int):
        pa_sweep(self.h, n)

    def step(self):
        pa_step(self.h)

    def run_steps(self, n: int):
        pa_run_steps(self.h, n)

    def step_stream(self, host, chunks: int, copy_stream) -> int:
        """pa_step_stream into a pinned host uint8 tensor of at least
        capacity * stride bytes, copies on copy_stream; returns R_i."""
        return pa_step_stream(self.h, host.data_ptr(), host.numel() * host.element_size(), chunks,
                              copy_stream.cuda_stream)

    def observables(self, check: bool = True) -> dict:
        return pa_observables(self.h, check)

    def history(self, first: int, n: int) -> list:
        return pa_observables_history(self.h, first, n)

    def status(self) -> int:
        return pa_status(self.h)

    def state(self) -> dict:
        return pa_dump(self.h, DUMP_STATE)

    def spins(self) -> np.ndarray:
        a = pa_dump(self.h, DUMP_SPINS)
        return a.reshape(-1, self.N)

    def dump(self, what: int) -> np.ndarray:
        return pa_dump(self.h, what)

    def adaptive_beta(self, overlap_target: float, beta_end: float) -> float:
        out = C.c_double()
        _check(lib().pa_adaptive_beta(C.c_void_p(self.h), overlap_target, beta_end,
                                      C.byref(out)), "pa_adaptive_beta")
        return out.value

    def resample_to(self, beta_next: float):
        _check(lib().pa_resample_to(C.c_void_p(self.h), beta_next), "pa_resample_to")

    def checkpoint(self) -> bytes:
        n = int(lib().pa_checkpoint_size(C.c_void_p(self.h)))
        if n < 0:
            raise PaError(-1, "pa_checkpoint_size")
        buf = np.zeros(n, dtype=np.uint8)
        _check(lib().pa_checkpoint(C.c_void_p(self.h), C.c_void_p(buf.ctypes.data), n),
               "pa_checkpoint")
        return buf.tobytes()

    def restore(self, blob: bytes):
        buf = np.frombuffer(blob, dtype=np.uint8).copy()
        _check(lib().pa_restore(C.c_void_p(self.h), C.c_void_p(buf.ctypes.data), buf.size),
               "pa_restore")

    def load(self, what: int, src: np.ndarray, count: int):
        pa_load(self.h, what, src, count)

    def dump_range(self, what: int, first: int, count: int) -> np.ndarray:
        stride = self.state()["stride"] if what == DUMP_SPINS_RAW else 0
        return pa_dump_range(self.h, what, first, count, self.N, stride)


# ---- batched form ---------------------------------------------------------------
class Batch:
    """Several runs stepped together (pa_batch_* of include/pa.h)."""

    def __init__(self, runs, stream=None, steps_left=None, workspace=None):
        """steps_left: remaining steps of every run, known to the caller (the
        batch is then built without waiting for the device, pa_batch_init_async);
        workspace: a device tensor of at least pa_batch_workspace_size bytes
        (allocated here when None)."""
        import torch
        self.runs = list(runs)
        n = len(self.runs)
        nbytes = int(lib().pa_batch_workspace_size(n))
        if nbytes == 0:
            raise PaError(-1, "pa_batch_workspace_size")
        if workspace is None:
            workspace = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
        self.workspace = workspace
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        handles = (C.c_void_p * n)(*[r.h for r in self.runs])
        h = C.c_void_p()
        if steps_left is None:
            _check(lib().pa_batch_init(handles, n, C.c_void_p(self.workspace.data_ptr()), nbytes,
                                       C.c_void_p(self.stream.cuda_stream), C.byref(h)),
                   "pa_batch_init")
        else:
            left = (C.c_int32 * n)(*[int(x) for x in steps_left])
            _check(lib().pa_batch_init_async(handles, n, left,
                                             C.c_void_p(self.workspace.data_ptr()), nbytes,
                                             C.c_void_p(self.stream.cuda_stream), C.byref(h)),
                   "pa_batch_init_async")
        self.h = h.value

    def close(self):
        if getattr(self, "h", None):
            lib().pa_batch_free(C.c_void_p(self.h))
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def step(self):
        _check(lib().pa_batch_step(C.c_void_p(self.h)), "pa_batch_step")

    def run_steps(self, n: int):
        _check(lib().pa_batch_run_steps(C.c_void_p(self.h), n), "pa_batch_run_steps")

    def sync(self) -> int:
        return int(lib().pa_batch_sync(C.c_void_p(self.h)))

    def classes(self) -> list:
        out = []
        for c in range(int(lib().pa_batch_num_classes(C.c_void_p(self.h)))):
            info = (C.c_int32 * 8)()
            _check(lib().pa_batch_class_info(C.c_void_p(self.h), c, info), "pa_batch_class_info")
            out.append(dict(zip(("layout", "dim", "L", "model", "runs", "warps", "slots",
                                 "chunk"), list(info))))
        return out

    def profile(self, enable: bool):
        _check(lib().pa_batch_profile(C.c_void_p(self.h), 1 if enable else 0),
               "pa_batch_profile")

    def profile_read(self, reset: bool = True) -> dict:
        """Timed steps and summed device ms per phase (non-graph steps)."""
        n = C.c_int64()
        ms = (C.c_double * 4)()
        _check(lib().pa_batch_profile_read(C.c_void_p(self.h), C.byref(n), ms, 1 if reset else 0),
               "pa_batch_profile_read")
        return {"steps": n.value, "reweight": ms[0], "resample": ms[1], "sweep": ms[2],
                "obs": ms[3]}

    def set_shape(self, cls: int, warps: int = 0, chunk: int = 0):
        _check(lib().pa_batch_set_shape(C.c_void_p(self.h), cls, warps, chunk),
               "pa_batch_set_shape")

    def set_warps(self, cls: int, warps: int):
        self.set_shape(cls, warps, 0)
