"""pa_copy_counts_scan_noalloc: copy counts and their exclusive scan for
callers that cannot allocate device memory (code running under CUDA graph
capture, plugins whose host process owns every allocation, fixed-budget
embedded callers).  Its scratch is a static device array inside the library,
so the caller passes only inputs and outputs.

Checked through the C ABI against the regular resample (pa_resample), which
computes the same counts and offsets with scratch from the run's workspace:
integers, so bit for bit, on two calls in a row (the second call reuses the
static scratch the first one left behind)."""
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
    return torch.from_numpy(np.ascontiguousarray(a).view(np.int32)).cuda()


def test_noalloc_counts_and_offsets_match_resample_two_calls(P):
    import torch
    cfg = P.make_config(dim=2, L=16, layout=P.LAYOUT_PACKED, R0=5000, K=20, theta=2,
                        beta_max=1.5, seed=21, instance_id=7)
    run = P.Run(cfg)
    stream = torch.cuda.current_stream()
    bins = P.pa_num_bins(cfg.dim, cfg.L)
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
        want_counts = run.dump(P.DUMP_COUNTS)
        want_offsets = run.dump(P.DUMP_OFFSETS)
        d_ebin, d_n, d_F = _dev(ebin), _dev(run.dump(P.DUMP_TAB_N)), _dev(run.dump(P.DUMP_TAB_F))
        P.pa_copy_counts_scan_noalloc(d_ebin.data_ptr(), R, d_n.data_ptr(), d_F.data_ptr(), bins,
                                      cfg.seed, st["step"], cfg.instance_id, counts.data_ptr(),
                                      offsets.data_ptr(), total.data_ptr(), stream.cuda_stream)
        torch.cuda.synchronize()
        got_counts = counts[:R].cpu().numpy().view(np.uint32)
        got_offsets = offsets[:R].cpu().numpy().view(np.uint32)
        assert np.array_equal(got_counts, want_counts), f"call {call}"
        assert np.array_equal(got_offsets, want_offsets), f"call {call}"
        assert int(total.item()) == st["R"], f"call {call}"
        assert R > 2048  # more than one scan tile
        run.sweep(cfg.theta)
    run.close()


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
