"""ctypes view of the C oracle (oracle/pa_oracle.c).

TEST INFRASTRUCTURE ONLY: imported by tests/, by ``__graft_entry__.smoke()``
and by the ``cpu_baseline`` leg / ``--impl reference`` arm of bench.py.  The
product package never imports it.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "liboracle.so")
SRC = os.path.join(HERE, "pa_oracle.c")

MODEL_FERRO = 0
MODEL_PMJ = 1


def build(force: bool = False) -> str:
    """Compile the oracle with IEEE double semantics (no FP contraction)."""
    if force or not os.path.exists(LIB_PATH) or os.path.getmtime(LIB_PATH) < max(
        os.path.getmtime(SRC), os.path.getmtime(os.path.join(HERE, "pa_oracle.h"))
    ):
        tmp = LIB_PATH + f".{os.getpid()}.tmp"
        cmd = ["gcc", "-O2", "-std=c99", "-ffp-contract=off", "-fno-fast-math", "-fPIC",
               "-shared", "-Wall", "-o", tmp, SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, LIB_PATH)
    return LIB_PATH


class Config(C.Structure):
    _fields_ = [
        ("dim", C.c_int32), ("L", C.c_int32), ("model", C.c_int32), ("K", C.c_int32),
        ("theta", C.c_int32), ("instance_id", C.c_int32),
        ("R0", C.c_int64), ("capacity", C.c_int64),
        ("beta0", C.c_double), ("beta_max", C.c_double),
        ("seed", C.c_uint64), ("coupling_seed", C.c_uint64),
        ("init", C.c_int32), ("resample", C.c_int32),
    ]


INIT_RANDOM, INIT_GROUND = 0, 1
RESAMPLE_NEAREST, RESAMPLE_POISSON, RESAMPLE_MULTINOMIAL = 0, 1, 2


class Obs(C.Structure):
    _fields_ = [
        ("step", C.c_int64), ("R", C.c_int64),
        ("sumE", C.c_int64), ("sumE2", C.c_int64), ("sumAbsM", C.c_int64), ("sumM2", C.c_int64),
        ("beta", C.c_double), ("lnQ", C.c_double), ("lnZ", C.c_double),
        ("e", C.c_double), ("cv", C.c_double), ("m_abs", C.c_double), ("chi", C.c_double),
    ]

    def as_dict(self) -> dict:
        return {name: getattr(self, name) for name, _ in self._fields_}


_lib = None


def lib():
    global _lib
    if _lib is None:
        path = os.environ.get("PA_ORACLE_LIB") or build()
        L = C.CDLL(path)
        u32p, i8p, dp, u64p = (C.POINTER(C.c_uint32), C.POINTER(C.c_int8),
                               C.POINTER(C.c_double), C.POINTER(C.c_uint64))
        i64p = C.POINTER(C.c_int64)
        L.or_philox4x32_10.argtypes = [u32p, u32p, u32p]
        L.or_beta.argtypes = [C.POINTER(Config), C.c_int32]
        L.or_beta.restype = C.c_double
        L.or_threshold.argtypes = [C.c_double, C.c_int32]
        L.or_threshold.restype = C.c_uint64
        L.or_weight.argtypes = [C.c_double, C.c_int64]
        L.or_weight.restype = C.c_double
        L.or_num_bins.argtypes = [C.c_int32, C.c_int32]
        L.or_num_bins.restype = C.c_int64
        L.or_init_couplings.argtypes = [C.POINTER(Config), i8p]
        L.or_init_replica.argtypes = [C.POINTER(Config), C.c_int64, i8p]
        L.or_energy.argtypes = [C.c_int32, C.c_int32, i8p, i8p, i64p, i64p]
        L.or_delta_e.argtypes = [C.c_int32, C.c_int32, i8p, i8p, C.c_int64]
        L.or_delta_e.restype = C.c_int64
        L.or_sweep_replica.argtypes = [C.POINTER(Config), i8p, i8p, C.c_int64, C.c_int64,
                                       C.c_int32, u64p]
        L.or_sweep_replica.restype = C.c_int64
        L.or_tau_table.argtypes = [u32p, C.c_int64, dp, C.c_int64, C.c_int32, u32p, u32p, i64p]
        L.or_tau_table.restype = C.c_double
        L.or_copy_counts.argtypes = [C.POINTER(Config), C.c_int32, u32p, C.c_int64, u32p, u32p,
                                     u32p]
        L.or_copy_counts_poisson.argtypes = [C.POINTER(Config), C.c_int32, u32p, C.c_int64,
                                             u32p, u32p, u32p]
        L.or_copy_counts_multinomial.argtypes = [C.POINTER(Config), C.c_int32, u32p, C.c_int64,
                                                 u32p, u32p, u32p]
        L.or_poisson1_thresholds.argtypes = [u32p, C.c_int32]
        L.or_poisson1_thresholds.restype = C.c_int32
        L.or_derive_obs.argtypes = [C.POINTER(Obs), C.c_int64]
        L.or_overlap.argtypes = [u32p, C.c_int64, C.c_int64, C.c_double]
        L.or_overlap.restype = C.c_double
        L.or_adaptive_next.argtypes = [u32p, C.c_int64, C.c_int64, C.c_double, C.c_double,
                                       C.c_double]
        L.or_adaptive_next.restype = C.c_double
        L.or_resample_to.argtypes = [C.c_void_p, C.c_double]
        L.or_resample_to.restype = C.c_int
        L.or_current_beta.argtypes = [C.c_void_p]
        L.or_current_beta.restype = C.c_double
        L.or_create.argtypes = [C.POINTER(Config)]
        L.or_create.restype = C.c_void_p
        L.or_destroy.argtypes = [C.c_void_p]
        for name in ("or_resample", "or_step"):
            getattr(L, name).argtypes = [C.c_void_p]
            getattr(L, name).restype = C.c_int
        L.or_sweep.argtypes = [C.c_void_p, C.c_int32]
        L.or_sweep.restype = C.c_int
        L.or_permute.argtypes = [C.c_void_p, C.c_int32, C.POINTER(C.c_int64),
                                 C.POINTER(C.c_int64)]
        L.or_permute.restype = C.c_int
        L.or_observables.argtypes = [C.c_void_p, C.POINTER(Obs)]
        for name in ("or_R", "or_N", "or_bins", "or_sweep_counter", "or_R_prev", "or_kref",
                     "or_parity", "or_check_failures"):
            getattr(L, name).argtypes = [C.c_void_p]
            getattr(L, name).restype = C.c_int64
        L.or_step_index.argtypes = [C.c_void_p]
        L.or_step_index.restype = C.c_int32
        for name in ("or_S", "or_lnQ", "or_lnZ"):
            getattr(L, name).argtypes = [C.c_void_p]
            getattr(L, name).restype = C.c_double
        for name, t in (("or_spins", i8p), ("or_ebin", u32p), ("or_mag", C.POINTER(C.c_int32)),
                        ("or_hist", u32p), ("or_counts", u32p), ("or_offsets", u32p),
                        ("or_tab_n", u32p), ("or_tab_F", u32p), ("or_couplings", i8p)):
            getattr(L, name).argtypes = [C.c_void_p]
            getattr(L, name).restype = t
        _lib = L
    return _lib


def _ptr(a: np.ndarray, ctype):
    return a.ctypes.data_as(C.POINTER(ctype))


def make_config(dim=2, L=16, model=MODEL_FERRO, K=100, theta=10, instance_id=0, R0=1000,
                capacity=0, beta0=0.0, beta_max=1.0, seed=1, coupling_seed=0,
                init=INIT_RANDOM, resample=RESAMPLE_NEAREST) -> Config:
    return Config(dim, L, model, K, theta, instance_id, R0, capacity, beta0, beta_max, seed,
                  coupling_seed, init, resample)


# ---------------------------------------------------------------------------
# building blocks
# ---------------------------------------------------------------------------
def philox(ctr, key) -> np.ndarray:
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.zeros(4, dtype=np.uint32)
    lib().or_philox4x32_10(_ptr(c, C.c_uint32), _ptr(k, C.c_uint32), _ptr(out, C.c_uint32))
    return out


def beta(cfg: Config, i: int) -> float:
    return lib().or_beta(C.byref(cfg), i)


def threshold(b: float, dE: int) -> int:
    return int(lib().or_threshold(b, dE))


def weight(dbeta: float, j: int) -> float:
    return lib().or_weight(dbeta, j)


def num_bins(dim: int, L: int) -> int:
    return int(lib().or_num_bins(dim, L))


def couplings(cfg: Config) -> np.ndarray:
    N = cfg.L ** cfg.dim
    J = np.zeros(N * cfg.dim, dtype=np.int8)
    lib().or_init_couplings(C.byref(cfg), _ptr(J, C.c_int8))
    return J


def init_replica(cfg: Config, slot: int) -> np.ndarray:
    s = np.zeros(cfg.L ** cfg.dim, dtype=np.int8)
    lib().or_init_replica(C.byref(cfg), slot, _ptr(s, C.c_int8))
    return s


def energy(dim: int, L: int, J: np.ndarray, spins: np.ndarray):
    U = C.c_int64()
    M = C.c_int64()
    J = np.ascontiguousarray(J, dtype=np.int8)
    spins = np.ascontiguousarray(spins, dtype=np.int8)
    lib().or_energy(dim, L, _ptr(J, C.c_int8), _ptr(spins, C.c_int8), C.byref(U), C.byref(M))
    return U.value, M.value


def delta_e(dim: int, L: int, J: np.ndarray, spins: np.ndarray, s: int) -> int:
    J = np.ascontiguousarray(J, dtype=np.int8)
    spins = np.ascontiguousarray(spins, dtype=np.int8)
    return int(lib().or_delta_e(dim, L, _ptr(J, C.c_int8), _ptr(spins, C.c_int8), s))


def sweep_replica(cfg: Config, J: np.ndarray, spins: np.ndarray, slot: int, g0: int,
                  nsweeps: int, T) -> int:
    """Runs nsweeps sweeps on ``spins`` in place; returns the tracked change of U."""
    assert spins.dtype == np.int8 and spins.flags.c_contiguous
    Jc = np.ascontiguousarray(J, dtype=np.int8)
    Ta = np.ascontiguousarray(T, dtype=np.uint64)
    assert Ta.size >= 3
    return int(lib().or_sweep_replica(C.byref(cfg), _ptr(Jc, C.c_int8), _ptr(spins, C.c_int8),
                                      slot, g0, nsweeps, _ptr(Ta, C.c_uint64)))


def tau_table(H: np.ndarray, Dtab: np.ndarray, R0: int, heating: bool = False):
    H = np.ascontiguousarray(H, dtype=np.uint32)
    Dtab = np.ascontiguousarray(Dtab, dtype=np.float64)
    bins = H.size
    n = np.zeros(bins, dtype=np.uint32)
    F = np.zeros(bins, dtype=np.uint32)
    kref = C.c_int64()
    S = lib().or_tau_table(_ptr(H, C.c_uint32), bins, _ptr(Dtab, C.c_double), R0,
                           1 if heating else 0, _ptr(n, C.c_uint32), _ptr(F, C.c_uint32),
                           C.byref(kref))
    return S, kref.value, n, F


def copy_counts(cfg: Config, step: int, ebin: np.ndarray, n: np.ndarray, F: np.ndarray):
    ebin = np.ascontiguousarray(ebin, dtype=np.uint32)
    n = np.ascontiguousarray(n, dtype=np.uint32)
    F = np.ascontiguousarray(F, dtype=np.uint32)
    r = np.zeros(ebin.size, dtype=np.uint32)
    lib().or_copy_counts(C.byref(cfg), step, _ptr(ebin, C.c_uint32), ebin.size,
                         _ptr(n, C.c_uint32), _ptr(F, C.c_uint32), _ptr(r, C.c_uint32))
    return r


def copy_counts_poisson(cfg: Config, step: int, ebin: np.ndarray, n: np.ndarray,
                        F: np.ndarray):
    ebin = np.ascontiguousarray(ebin, dtype=np.uint32)
    n = np.ascontiguousarray(n, dtype=np.uint32)
    F = np.ascontiguousarray(F, dtype=np.uint32)
    r = np.zeros(ebin.size, dtype=np.uint32)
    lib().or_copy_counts_poisson(C.byref(cfg), step, _ptr(ebin, C.c_uint32), ebin.size,
                                 _ptr(n, C.c_uint32), _ptr(F, C.c_uint32), _ptr(r, C.c_uint32))
    return r


def copy_counts_multinomial(cfg: Config, step: int, ebin: np.ndarray, n: np.ndarray,
                            F: np.ndarray):
    ebin = np.ascontiguousarray(ebin, dtype=np.uint32)
    n = np.ascontiguousarray(n, dtype=np.uint32)
    F = np.ascontiguousarray(F, dtype=np.uint32)
    r = np.zeros(ebin.size, dtype=np.uint32)
    lib().or_copy_counts_multinomial(C.byref(cfg), step, _ptr(ebin, C.c_uint32), ebin.size,
                                     _ptr(n, C.c_uint32), _ptr(F, C.c_uint32),
                                     _ptr(r, C.c_uint32))
    return r


def poisson1_thresholds() -> np.ndarray:
    T = np.zeros(64, dtype=np.uint32)
    m = lib().or_poisson1_thresholds(_ptr(T, C.c_uint32), 64)
    return T[:m].copy()


def overlap(H: np.ndarray, R: int, dbeta: float) -> float:
    H = np.ascontiguousarray(H, dtype=np.uint32)
    return float(lib().or_overlap(_ptr(H, C.c_uint32), H.size, R, dbeta))


def adaptive_next(H: np.ndarray, R: int, beta: float, beta_end: float, target: float) -> float:
    H = np.ascontiguousarray(H, dtype=np.uint32)
    return float(lib().or_adaptive_next(_ptr(H, C.c_uint32), H.size, R, beta, beta_end, target))


def derive_obs(sums: dict, N: int) -> dict:
    o = Obs()
    for k in ("step", "R", "sumE", "sumE2", "sumAbsM", "sumM2", "beta", "lnQ", "lnZ"):
        if k in sums:
            setattr(o, k, sums[k])
    lib().or_derive_obs(C.byref(o), N)
    return o.as_dict()


# ---------------------------------------------------------------------------
# a whole run
# ---------------------------------------------------------------------------
class Run:
    """One PA run on the CPU oracle."""

    def __init__(self, cfg: Config):
        self.cfg = cfg
        self._h = lib().or_create(C.byref(cfg))
        if not self._h:
            raise ValueError("oracle rejected the configuration")

    def close(self):
        if self._h:
            lib().or_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def resample(self) -> int:
        return lib().or_resample(self._h)

    def sweep(self, n: int) -> int:
        return lib().or_sweep(self._h, n)

    def permute(self, segments) -> int:
        """Replica exchange (Sec. 3): new slot order from [(old first slot,
        length), ...]."""
        seg = np.asarray(segments, dtype=np.int64).reshape(-1, 2)
        src = np.ascontiguousarray(seg[:, 0])
        ln = np.ascontiguousarray(seg[:, 1])
        return lib().or_permute(self._h, int(seg.shape[0]), _ptr(src, C.c_int64),
                                _ptr(ln, C.c_int64))

    def resample_to(self, beta_next: float) -> int:
        return lib().or_resample_to(self._h, beta_next)

    @property
    def beta(self) -> float:
        return float(lib().or_current_beta(self._h))

    def step(self) -> int:
        return lib().or_step(self._h)

    def observables(self) -> dict:
        o = Obs()
        lib().or_observables(self._h, C.byref(o))
        return o.as_dict()

    @property
    def R(self) -> int:
        return int(lib().or_R(self._h))

    @property
    def R_prev(self) -> int:
        return int(lib().or_R_prev(self._h))

    @property
    def N(self) -> int:
        return int(lib().or_N(self._h))

    @property
    def bins(self) -> int:
        return int(lib().or_bins(self._h))

    @property
    def step_index(self) -> int:
        return int(lib().or_step_index(self._h))

    @property
    def sweep_counter(self) -> int:
        return int(lib().or_sweep_counter(self._h))

    @property
    def kref(self) -> int:
        return int(lib().or_kref(self._h))

    @property
    def S(self) -> float:
        return float(lib().or_S(self._h))

    @property
    def lnQ(self) -> float:
        return float(lib().or_lnQ(self._h))

    @property
    def lnZ(self) -> float:
        return float(lib().or_lnZ(self._h))

    @property
    def parity(self) -> int:
        return int(lib().or_parity(self._h))

    @property
    def check_failures(self) -> int:
        return int(lib().or_check_failures(self._h))

    def _view(self, fn, n, dtype):
        p = getattr(lib(), fn)(self._h)
        return np.ctypeslib.as_array(p, shape=(n,)).astype(dtype, copy=True)

    def spins(self) -> np.ndarray:
        return self._view("or_spins", self.R * self.N, np.int8).reshape(self.R, self.N)

    def ebin(self) -> np.ndarray:
        return self._view("or_ebin", self.R, np.uint32)

    def mag(self) -> np.ndarray:
        return self._view("or_mag", self.R, np.int32)

    def hist(self) -> np.ndarray:
        return self._view("or_hist", self.bins, np.uint32)

    def counts(self) -> np.ndarray:
        return self._view("or_counts", self.R_prev, np.uint32)

    def offsets(self) -> np.ndarray:
        return self._view("or_offsets", self.R_prev, np.uint32)

    def tab_n(self) -> np.ndarray:
        return self._view("or_tab_n", self.bins, np.uint32)

    def tab_F(self) -> np.ndarray:
        return self._view("or_tab_F", self.bins, np.uint32)

    def couplings(self) -> np.ndarray:
        return self._view("or_couplings", self.N * self.cfg.dim, np.int8)


if __name__ == "__main__":  # pragma: no cover - manual build helper
    print(build(force="--force" in sys.argv))
