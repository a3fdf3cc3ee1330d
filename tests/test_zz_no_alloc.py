"""dem_detect_contacts_noalloc: the allocation-free detection entry point
gives the same contacts as a bed created and stepped through the regular
entry points, on two calls in a row (the shared scratch array must be reset
between calls).  Collected last on purpose."""
import numpy as np
import pytest

from dem_cases import compressed_cloud, make_gpu, params

pytestmark = pytest.mark.gpu


def bed_contacts(x, r):
    g = make_gpu(x, r, params(n_it=1))
    g.step(1)
    a, b, lam, dl = g.read_contacts()
    g.close()
    lo, hi = np.minimum(a, b), np.maximum(a, b)
    return {(int(p), int(q)): float(d) for p, q, d in zip(lo, hi, dl)}


def test_noalloc_detection_matches_bed_contacts_twice():
    import torch
    from paper_2501_05300_gb300 import dem
    torch.cuda.set_device(0)
    stream = torch.cuda.current_stream()
    cap = 200_000
    ka = torch.empty(cap, dtype=torch.int32, device="cuda")
    kb = torch.empty(cap, dtype=torch.int32, device="cuda")
    dl = torch.empty(cap, dtype=torch.float32, device="cuda")
    cnt = torch.zeros(1, dtype=torch.int64, device="cuda")
    for seed, n in ((21, 5000), (22, 3001)):      # two calls in a row, different inputs
        x, r = compressed_cloud(n, seed=seed)
        ref = bed_contacts(x, r)
        xt = torch.tensor(x, dtype=torch.float64, device="cuda")
        rt = torch.tensor(r, dtype=torch.float32, device="cuda")
        dem.detect_contacts_noalloc(xt, rt, ka, kb, dl, cnt, stream)
        torch.cuda.synchronize()
        m = int(cnt.item())
        assert m == len(ref) and m > n
        got = {(int(p), int(q)): float(d) for p, q, d in
               zip(ka[:m].cpu().numpy(), kb[:m].cpu().numpy(), dl[:m].cpu().numpy())}
        assert set(got) == set(ref)               # contact sets: bit-exact
        d_ref = np.array([ref[k] for k in sorted(ref)])
        d_got = np.array([got[k] for k in sorted(ref)])
        assert np.allclose(d_got, d_ref, rtol=1e-6, atol=1e-7 * d_ref.max())


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
