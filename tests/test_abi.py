"""C-ABI checks that need no GPU: the library loads, exports every entry point
include/pa.h declares, validates configurations, and builds host tables that
are bit-identical to the oracle's (thresholds and Eq. 3 weights are compared
before any kernel runs)."""
from __future__ import annotations

import ctypes
import os
import re

import numpy as np
import pytest

from oracle import oracle as O

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def P():
    from paper_2006_00561_gb300 import build as B
    B.build()
    from paper_2006_00561_gb300 import pa
    return pa


def declared_symbols():
    src = open(os.path.join(ROOT, "include", "pa.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(pa_[a-z0-9_]+)\s*\(", src)))


def test_library_exports_every_declared_symbol(P):
    names = declared_symbols()
    assert len(names) >= 14
    lib = ctypes.CDLL(P.LIB_PATH)
    for n in names:
        assert hasattr(lib, n), n
    assert set(P.EXPORTS) == set(names)


def test_num_bins(P):
    assert P.pa_num_bins(2, 64) == 4097
    assert P.pa_num_bins(2, 16) == 257
    assert P.pa_num_bins(3, 10) == 1501
    assert P.pa_num_bins(2, 128) == 16385
    for dim, L in [(2, 4), (2, 64), (3, 2), (3, 6), (3, 10)]:
        assert P.pa_num_bins(dim, L) == O.num_bins(dim, L)


@pytest.mark.parametrize("kw,code", [
    (dict(L=5), -2), (dict(L=6), -3), (dict(L=0), -1), (dict(dim=4), -1), (dict(K=0), -1),
    (dict(R0=0), -1), (dict(theta=-1), -1), (dict(beta0=-1.0), -1), (dict(init=2), -1),
    (dict(init=1, model=1), -1),
    (dict(instance_id=1 << 28), -1), (dict(layout=7), -1), (dict(model=3), -1),
    (dict(capacity=10, R0=100), -1), (dict(dim=3, L=14), -3), (dict(R0=(1 << 31) + 1), -1),
])
def test_invalid_configurations_are_rejected(P, kw, code):
    cfg = P.make_config(**kw)
    assert P.pa_workspace_size(cfg) == 0
    with pytest.raises(P.PaError) as e:
        P.pa_tables(cfg, 0, 4)
    assert e.value.code == code


def test_workspace_size_grows_with_capacity(P):
    a = P.pa_workspace_size(P.make_config(dim=2, L=64, R0=1 << 17, K=200))
    b = P.pa_workspace_size(P.make_config(dim=2, L=64, R0=1 << 21, K=400))
    assert 0 < a < b
    # two 512-byte spin buffers dominate at L = 64
    cap = (1 << 21) + 16 * 1449 + 1024
    assert b >= 2 * cap * 512 and b < 2 * cap * 512 * 1.1


@pytest.mark.parametrize("spec", [
    dict(dim=2, L=16, K=100, beta_max=1.0), dict(dim=2, L=64, K=400, beta_max=1.0),
    dict(dim=3, L=10, K=150, beta_max=3.0), dict(dim=2, L=128, K=300, beta_max=3.0),
    dict(dim=2, L=64, K=7, beta0=0.25, beta_max=0.9),
    dict(dim=2, L=16, K=50, beta0=2.0, beta_max=0.0),
])
def test_host_tables_bitwise_equal_to_oracle(P, spec):
    cfg = P.make_config(**spec)
    ocfg = O.make_config(dim=spec["dim"], L=spec["L"], K=spec["K"], beta0=spec.get("beta0", 0.0),
                         beta_max=spec["beta_max"])
    bins = P.pa_num_bins(cfg.dim, cfg.L)
    for step in sorted({0, 1, 2, cfg.K // 2, cfg.K - 1, cfg.K}):
        T, D = P.pa_tables(cfg, step, bins)
        b = O.beta(ocfg, step)
        assert [int(t) for t in T] == [O.threshold(b, 4 * (c + 1)) for c in range(3)]
        if step >= 1:
            db = O.beta(ocfg, step) - O.beta(ocfg, step - 1)
            want = np.array([O.weight(db, j) for j in range(bins)])
            assert np.array_equal(D.view(np.uint64), want.view(np.uint64))


def test_poisson1_table_equals_oracle_and_exact(P):
    """The engine's host-built Poisson(1) inversion table equals the oracle's
    (which is pinned to 40-digit sums) entry for entry."""
    T = P.pa_poisson1_table()
    assert T.dtype == np.uint32 and len(T) == 13 and T[-1] == 2 ** 32 - 1
    assert np.array_equal(T, O.poisson1_thresholds())


def test_resample_rule_is_validated(P):
    assert P.pa_workspace_size(P.make_config(resample=1)) > 0
    # multinomial runs add the cumulative weights (8 B per slot) and tile prefixes
    cap = 1000 + 16 * 32 + 1024
    assert (P.pa_workspace_size(P.make_config(R0=1000, resample=2)) >=
            P.pa_workspace_size(P.make_config(R0=1000, resample=0)) + 8 * cap)
    for bad in (dict(resample=3), dict(resample=-1)):
        assert P.pa_workspace_size(P.make_config(**bad)) == 0
    cfg = P.make_config()
    cfg.reserved = 1
    assert P.pa_workspace_size(cfg) == 0
