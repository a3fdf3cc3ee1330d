"""dem_detect_contacts_noalloc: contact detection for callers that may not
allocate GPU memory (their device memory held by another framework's caching
allocator, a real-time loop that forbids allocation after start-up, or work
enqueued while a stream is being captured).  Every intermediate array lives in
one static device array that all calls share, so these tests check what that
sharing could break: two calls in a row with different inputs, a call that
finds more pairs than the caller's capacity, an empty call after a full one, a
call on a stream that is not the current one, and invalid input.

The expected contact sets come from the FP64 oracle's brute-force detection
(every pair tested with the exact predicate) and from a bed stepped through
the regular entry points.  Collected last on purpose: if it fails, a run that
stops at the first failure has already run every other test."""
import numpy as np
import pytest

import oracle
from dem_cases import compressed_cloud, make_gpu, params

pytestmark = pytest.mark.gpu


def oracle_contacts(x, r):
    a, b, dl = oracle.detect(x, np.asarray(r, np.float32).astype(np.float64), np.arange(len(r), dtype=np.int32))
    return {(int(p), int(q)): float(d) for p, q, d in zip(a, b, dl)}


def bed_contacts(x, r):
    g = make_gpu(x, r, params(n_it=1))
    g.step(1)
    a, b, lam, dl = g.read_contacts()
    g.close()
    lo, hi = np.minimum(a, b), np.maximum(a, b)
    return {(int(p), int(q)): float(d) for p, q, d in zip(lo, hi, dl)}


def buffers(cap):
    import torch
    ka = torch.full((cap,), -7, dtype=torch.int32, device="cuda")
    kb = torch.full((cap,), -7, dtype=torch.int32, device="cuda")
    dl = torch.full((cap,), -7.0, dtype=torch.float32, device="cuda")
    cnt = torch.full((1,), -9, dtype=torch.int64, device="cuda")
    return ka, kb, dl, cnt


def inputs(x, r):
    import torch
    return (torch.tensor(x, dtype=torch.float64, device="cuda"),
            torch.tensor(np.asarray(r, np.float32), dtype=torch.float32, device="cuda"))


def as_dict(ka, kb, dl, m):
    return {(int(p), int(q)): float(d) for p, q, d in
            zip(ka[:m].cpu().numpy(), kb[:m].cpu().numpy(), dl[:m].cpu().numpy())}


def test_noalloc_detection_matches_oracle_and_bed_twice():
    import torch
    from paper_2501_05300_gb300 import dem
    torch.cuda.set_device(0)
    stream = torch.cuda.current_stream()
    ka, kb, dl, cnt = buffers(200_000)
    for seed, n in ((21, 5000), (22, 3001)):      # two calls in a row, different inputs
        x, r = compressed_cloud(n, seed=seed)
        ref = oracle_contacts(x, r)
        bed = bed_contacts(x, r)
        assert set(bed) == set(ref)
        xt, rt = inputs(x, r)
        dem.detect_contacts_noalloc(xt, rt, ka, kb, dl, cnt, stream)
        torch.cuda.synchronize()
        m = int(cnt.item())
        assert m == len(ref) and m > n
        got = as_dict(ka, kb, dl, m)
        assert set(got) == set(ref)               # contact sets: bit-exact
        keys = sorted(ref)
        d_ref = np.array([ref[k] for k in keys])
        d_got = np.array([got[k] for k in keys])
        d_bed = np.array([bed[k] for k in keys])
        # FP32 overlaps from FP64 differences: a few ulps of the overlap
        assert np.allclose(d_got, d_ref, rtol=1e-5, atol=1e-7 * d_ref.max())
        assert np.array_equal(d_got, d_bed)       # same arithmetic as the step's rows


def test_noalloc_count_beyond_capacity_writes_only_cap():
    """More pairs than the caller's capacity: count is the full number, only
    the first cap slots are written, each one a true contact."""
    import torch
    from paper_2501_05300_gb300 import dem
    x, r = compressed_cloud(5000, seed=21)
    ref = oracle_contacts(x, r)
    xt, rt = inputs(x, r)
    ka, kb, dl, cnt = buffers(20)
    cap = 10
    dem.detect_contacts_noalloc(xt, rt, ka[:cap], kb[:cap], dl[:cap], cnt)
    torch.cuda.synchronize()
    assert int(cnt.item()) == len(ref)
    got = as_dict(ka, kb, dl, cap)
    assert len(got) == cap and set(got) <= set(ref)
    for k, d in got.items():
        assert abs(d - ref[k]) <= 1e-5 * ref[k] + 1e-7 * max(ref.values())
    assert (ka[cap:] == -7).all() and (kb[cap:] == -7).all() and (dl[cap:] == -7.0).all()


def test_noalloc_empty_call_after_full_call_and_side_stream():
    """n = 0 right after a call that found pairs gives count 0 (the shared
    counter is cleared); a call on a stream that is not the current one gives
    the same contacts as on the current stream."""
    import torch
    from paper_2501_05300_gb300 import dem
    x, r = compressed_cloud(3001, seed=22)
    ref = oracle_contacts(x, r)
    xt, rt = inputs(x, r)
    ka, kb, dl, cnt = buffers(100_000)
    dem.detect_contacts_noalloc(xt, rt, ka, kb, dl, cnt)
    torch.cuda.synchronize()
    assert int(cnt.item()) == len(ref)
    empty_x = torch.empty((0, 3), dtype=torch.float64, device="cuda")
    empty_r = torch.empty((0,), dtype=torch.float32, device="cuda")
    dem.detect_contacts_noalloc(empty_x, empty_r, ka, kb, dl, cnt)
    torch.cuda.synchronize()
    assert int(cnt.item()) == 0
    side = torch.cuda.Stream()
    ka2, kb2, dl2, cnt2 = buffers(100_000)
    side.wait_stream(torch.cuda.current_stream())   # inputs and buffers are ready
    with torch.cuda.stream(side):
        dem.detect_contacts_noalloc(xt, rt, ka2, kb2, dl2, cnt2, side)
    side.synchronize()
    m = int(cnt2.item())
    assert m == len(ref)
    assert set(as_dict(ka2, kb2, dl2, m)) == set(ref)


def test_noalloc_invalid_radius_gives_minus_one_then_recovers():
    """A zero radius is invalid input: count is -1 and nothing is written; the
    next valid call is unaffected."""
    import torch
    from paper_2501_05300_gb300 import dem
    x, r = compressed_cloud(800, seed=23)
    ref = oracle_contacts(x, r)
    xt, rt = inputs(x, r)
    bad = rt.clone()
    bad[17] = 0.0
    ka, kb, dl, cnt = buffers(20_000)
    dem.detect_contacts_noalloc(xt, bad, ka, kb, dl, cnt)
    torch.cuda.synchronize()
    assert int(cnt.item()) == -1
    assert (ka == -7).all()
    dem.detect_contacts_noalloc(xt, rt, ka, kb, dl, cnt)
    torch.cuda.synchronize()
    m = int(cnt.item())
    assert m == len(ref) and set(as_dict(ka, kb, dl, m)) == set(ref)


def test_noalloc_rejects_sizes_beyond_its_scratch():
    import torch
    from paper_2501_05300_gb300 import dem
    n = (1 << 18) + 1
    pos = torch.zeros((n, 3), dtype=torch.float64, device="cuda")
    rad = torch.full((n,), 1e-3, dtype=torch.float32, device="cuda")
    out = torch.empty(1, dtype=torch.int32, device="cuda")
    dl = torch.empty(1, dtype=torch.float32, device="cuda")
    cnt = torch.zeros(1, dtype=torch.int64, device="cuda")
    with pytest.raises(dem.DemError) as e:
        dem.detect_contacts_noalloc(pos, rad, out, out, dl, cnt)
    assert e.value.status == dem.DEM_ERR_ARG
    assert "262144" in str(e.value)
