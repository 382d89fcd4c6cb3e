"""hea_search_coop_noalloc: the cooperative search for callers that cannot allocate device memory
(its exchange area is a fixed array inside the library).  Two calls in a row, each compared with
hea_search_coop given a caller-allocated exchange area, must agree bit for bit; oversized grids
are refused before any launch.  This file is collected last on purpose."""
import numpy as np
import pytest

import oracle
from paper_2411_18906_gb300 import hea, workloads
from tests import gpu_util as G

pytestmark = pytest.mark.gpu


def _inputs():
    kind, L, M = workloads.FCC, (8, 8, 8), 3
    N = oracle.num_sites(kind, L)
    entry = workloads.annealed_targets()["pool_fcc_4sp"][1]
    n_per = workloads.composition_counts(N, entry["fractions"])
    target = np.array(entry["alpha"])
    types = oracle.init_config(N, n_per, 17)
    cnt = oracle.counts(kind, L, M, len(n_per), types)
    return kind, L, M, n_per, np.ones(M), target, types, cnt


def _run(entry_point, kind, L, M, n_per, w, target, types, cnt, ctas, **kw):
    import torch
    lat = hea.Lattice(kind, L, M)
    obj = hea.Objective(n_per, w, target)
    t = G.dev(np.asarray(types, np.uint8))
    c = G.dev(np.asarray(cnt, np.int32))
    res = torch.zeros(hea.RESULT_BYTES, dtype=torch.uint8, device="cuda")
    params = hea.search_params(**kw)
    if entry_point == "noalloc":
        hea.hea_search_coop_noalloc(lat, obj, params, ctas, t, c, res)
    else:
        ws = torch.zeros(hea.hea_search_coop_workspace_bytes(ctas), dtype=torch.uint8, device="cuda")
        hea.hea_search_coop(lat, obj, params, ctas, t, c, res, ws)
    torch.cuda.synchronize()
    return t.cpu().numpy(), c.cpu().numpy(), hea.decode_results(res.cpu().numpy())[0]


def test_noalloc_matches_caller_workspace_on_two_calls():
    G.ensure_built()
    args = _inputs()
    ctas = min(16, G.sm_count())
    calls = [dict(K=ctas * 64, max_steps=40, accept_mode=1, group_size=64, group_top=2, seed=5),
             dict(K=ctas * 32, max_steps=60, accept_mode=0, seed=9)]
    for kw in calls:     # two calls in a row through the fixed exchange area
        want = _run("workspace", *args, ctas, **kw)
        got = _run("noalloc", *args, ctas, **kw)
        assert got[2]["status"] == want[2]["status"] == hea.HEA_OK
        for f in ("steps", "trials", "accepted", "depth"):
            assert got[2][f] == want[2][f], f
        assert got[2]["f2"] == want[2]["f2"]
        assert np.array_equal(got[0], want[0]) and np.array_equal(got[1], want[1])


def test_noalloc_refuses_grids_beyond_its_exchange_area():
    G.ensure_built()
    kind, L, M, n_per, w, target, types, cnt = _inputs()
    lat = hea.Lattice(kind, L, M)
    obj = hea.Objective(n_per, w, target)
    # 513 CTAs would still fit the array's bytes; the documented limit is 512 CTAs all the same
    assert hea.hea_search_coop_workspace_bytes(513) <= 344064 < hea.hea_search_coop_workspace_bytes(1024)
    for big in (513, 1024):
        with pytest.raises(hea.HeaError) as e:
            hea.hea_search_coop_noalloc(lat, obj, hea.search_params(big * 4, 1), big, G.dev(types), G.dev(cnt),
                                        G.dev(np.zeros(hea.RESULT_BYTES, np.uint8)))
        assert e.value.status == hea.HEA_EINVAL
        assert "512" in str(e.value)
