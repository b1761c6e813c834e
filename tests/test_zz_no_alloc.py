"""pa_copy_counts_scan_noalloc: copy counts and their exclusive scan for
callers that cannot allocate device memory (code running under CUDA graph
capture, plugins whose host process owns every allocation, fixed-budget
embedded callers).  Its scratch is a static device array inside the library,
so the caller passes only inputs and outputs.

Checked through the C ABI, bit for bit (integers), on two calls in a row (the
second call reuses the static scratch the first one left behind):
  * against the CPU oracle's copy counts (or_copy_counts, the nearest-integer
    rule of the resampling step) and the exclusive cumulative sum of those
    counts, for a population of a real run and for R = 300 000 replicas with
    synthetic levels and tables (about 150 scan tiles, so the lookback spans
    many tiles);
  * against the regular resample (pa_resample) on the same population."""
from __future__ import annotations

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    from paper_2006_00561_gb300 import build as B
    B.build()
    from paper_2006_00561_gb300 import pa
    return pa


def _dev(a: np.ndarray):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.uint32).view(np.int32)).cuda()


def _oracle_counts(seed, instance_id, step, ebin, n, F):
    from oracle import oracle as O
    cfg = O.make_config(seed=seed, instance_id=instance_id)
    r = O.copy_counts(cfg, step, ebin, n, F)
    o = np.zeros_like(r)
    np.cumsum(r[:-1], out=o[1:], dtype=np.uint32)
    return r, o, int(r.astype(np.int64).sum())


def _call(P, ebin, n, F, seed, step, instance_id, counts, offsets, total):
    import torch
    d_ebin, d_n, d_F = _dev(ebin), _dev(n), _dev(F)
    P.pa_copy_counts_scan_noalloc(d_ebin.data_ptr(), ebin.size, d_n.data_ptr(), d_F.data_ptr(),
                                  n.size, seed, step, instance_id, counts.data_ptr(),
                                  offsets.data_ptr(), total.data_ptr(),
                                  torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    R = ebin.size
    return (counts[:R].cpu().numpy().view(np.uint32), offsets[:R].cpu().numpy().view(np.uint32),
            int(total.cpu().numpy().view(np.uint32)[0]))


def test_noalloc_counts_and_offsets_match_oracle_and_resample_two_calls(P):
    import torch
    cfg = P.make_config(dim=2, L=16, layout=P.LAYOUT_PACKED, R0=5000, K=20, theta=2,
                        beta_max=1.5, seed=21, instance_id=7)
    run = P.Run(cfg)
    cap = run.state()["capacity"]
    counts = torch.full((cap,), -1, dtype=torch.int32, device="cuda")
    offsets = torch.full((cap,), -1, dtype=torch.int32, device="cuda")
    total = torch.full((1,), -1, dtype=torch.int32, device="cuda")
    for call in range(2):
        run.step()
        R = run.state()["R"]
        ebin = run.dump(P.DUMP_EBIN)  # population about to be resampled
        run.resample()
        st = run.state()
        assert st["status_bits"] == 0
        n, F = run.dump(P.DUMP_TAB_N), run.dump(P.DUMP_TAB_F)
        got_r, got_o, got_total = _call(P, ebin, n, F, cfg.seed, st["step"], cfg.instance_id,
                                        counts, offsets, total)
        want_r, want_o, want_total = _oracle_counts(cfg.seed, cfg.instance_id, st["step"], ebin,
                                                    n, F)
        assert np.array_equal(got_r, want_r), f"call {call}: counts differ from the oracle"
        assert np.array_equal(got_o, want_o), f"call {call}: offsets differ from the cumsum"
        assert got_total == want_total == st["R"], f"call {call}"
        assert np.array_equal(got_r, run.dump(P.DUMP_COUNTS)), f"call {call}"
        assert np.array_equal(got_o, run.dump(P.DUMP_OFFSETS)), f"call {call}"
        assert R > 2048  # more than one scan tile
        run.sweep(cfg.theta)
    run.close()


def test_noalloc_many_tiles_match_oracle_two_calls(P):
    """R = 300 000 synthetic replicas (levels and tables from a seeded numpy
    generator), about 150 scan tiles, two calls with different inputs."""
    import torch
    R, bins = 300_000, 4097
    counts = torch.full((R,), -1, dtype=torch.int32, device="cuda")
    offsets = torch.full((R,), -1, dtype=torch.int32, device="cuda")
    total = torch.full((1,), -1, dtype=torch.int32, device="cuda")
    rng = np.random.default_rng(2006)
    for call, (seed, step, inst) in enumerate(((3, 17, 0), (0x123456789ABCDEF, 401, 5))):
        ebin = rng.integers(0, bins, size=R, dtype=np.uint32)
        n = rng.integers(0, 3, size=bins, dtype=np.uint32)
        F = rng.integers(0, 1 << 32, size=bins, dtype=np.uint64).astype(np.uint32)
        got_r, got_o, got_total = _call(P, ebin, n, F, seed, step, inst, counts, offsets, total)
        want_r, want_o, want_total = _oracle_counts(seed, inst, step, ebin, n, F)
        assert np.array_equal(got_r, want_r), f"call {call}: counts differ from the oracle"
        assert np.array_equal(got_o, want_o), f"call {call}: offsets differ from the cumsum"
        assert got_total == want_total, f"call {call}"


def test_noalloc_rejects_sizes_above_its_static_scratch(P):
    import torch
    one = torch.zeros(4, dtype=torch.int32, device="cuda")
    s = torch.cuda.current_stream().cuda_stream
    with pytest.raises(P.PaError) as e:
        P.pa_copy_counts_scan_noalloc(one.data_ptr(), P.NOALLOC_MAX_REPLICAS + 1, one.data_ptr(),
                                      one.data_ptr(), 4, 1, 1, 0, one.data_ptr(), one.data_ptr(),
                                      one.data_ptr(), s)
    assert e.value.code == -1
    # an empty population is fine and reports 0 replicas
    total = torch.full((1,), 7, dtype=torch.int32, device="cuda")
    P.pa_copy_counts_scan_noalloc(one.data_ptr(), 0, one.data_ptr(), one.data_ptr(), 4, 1, 1, 0,
                                  one.data_ptr(), one.data_ptr(), total.data_ptr(), s)
    torch.cuda.synchronize()
    assert int(total.item()) == 0
