"""Serving loop: continuous batching, admission against an HBM budget, fault isolation.  Each
request's result must be the same alone (reindex_mesh) and in the mix."""
import numpy as np
import pytest

import oracle
from paper_2109_09812_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rx():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_2109_09812_gb300 import build

    build.build()
    import paper_2109_09812_gb300 as rx

    return rx


def make_requests(n, seed):
    rng = np.random.default_rng(seed)
    reqs = []
    for r in range(n):
        if r % 3 == 2:
            L = int(rng.integers(1, 9))
            v, i = synth.tet_soup_gpu(L, float(rng.uniform(0, 0.1)), seed * 1000 + r)
        else:
            G, Gy = int(rng.integers(1, 60)), int(rng.integers(1, 60))
            v, i = synth.heightfield_soup_gpu(G, Gy, float(rng.uniform(0, 0.1)), seed * 1000 + r)
        reqs.append((v.view(torch.int32), i))
    torch.cuda.synchronize()
    return reqs


def collect(server, n, timeout_s=120):
    import time

    got, t0 = {}, time.time()
    while len(got) < n:
        for res in server.poll(wait_ms=50):
            got[res["id"]] = res
        assert time.time() - t0 < timeout_s, f"only {len(got)} of {n} finished"
    return got


def test_alone_and_in_the_mix_are_identical(rx):
    reqs = make_requests(60, 1)
    with rx.Server(hbm_budget_bytes=1 << 30, max_batch_requests=7, num_streams=3) as srv:
        ids = [srv.submit(v, i) for v, i in reqs]
        got = collect(srv, len(ids))
        stats = srv.stats()
        assert stats["batches"] >= len(ids) // 7 and stats["requests_failed"] == 0
        for rid, (v, i) in zip(ids, reqs):
            res = got[rid]
            assert res["status"] == 0
            alone_v, alone_n, alone_i = rx.reindex_mesh(v, i)
            torch.cuda.synchronize()
            D = int(alone_n.item())
            assert res["n_out"] == D
            assert torch.equal(res["out_vtx"], alone_v[:D]) and torch.equal(res["out_idx"], alone_i)
            srv.release(rid)
        assert srv.stats()["arena_bytes_in_use"] == 0


def test_results_match_oracle(rx):
    reqs = make_requests(9, 2)
    with rx.Server(hbm_budget_bytes=1 << 28, max_batch_requests=4, num_streams=2) as srv:
        ids = [srv.submit(v, i) for v, i in reqs]
        got = collect(srv, len(ids))
        for rid, (v, i) in zip(ids, reqs):
            ov, oi = oracle.reindex_sort(v.cpu().numpy().view(np.uint32), i.cpu().numpy())
            np.testing.assert_array_equal(got[rid]["out_vtx"].cpu().numpy().view(np.uint32), ov)
            np.testing.assert_array_equal(got[rid]["out_idx"].cpu().numpy().reshape(-1), oi)
            srv.release(rid)


def test_admission_under_a_tight_budget(rx):
    """Requests of ~2.5 MB each against a 16 MiB budget: they are admitted a few at a time as
    memory is released, and all finish."""
    reqs = [synth.heightfield_soup_gpu(64, 64, 0.05, 50 + r) for r in range(24)]
    reqs = [(v.view(torch.int32), i) for v, i in reqs]
    torch.cuda.synchronize()
    with rx.Server(hbm_budget_bytes=16 << 20, max_batch_requests=64, num_streams=2) as srv:
        ids = [srv.submit(v, i) for v, i in reqs]
        done = 0
        import time

        t0 = time.time()
        while done < len(ids):
            for res in srv.poll(wait_ms=50):
                assert res["status"] == 0 and res["n_out"] == 65 * 65
                srv.release(res["id"])  # frees memory for the next requests
                done += 1
            assert time.time() - t0 < 120
        st = srv.stats()
        assert st["batches"] >= 3 and st["arena_bytes_in_use"] == 0


def test_request_larger_than_budget_is_refused(rx):
    v, i = synth.heightfield_soup_gpu(200, 200, 0.0, 3)
    with rx.Server(hbm_budget_bytes=2 << 20) as srv:
        with pytest.raises(rx.ReindexError) as e:
            srv.submit(v.view(torch.int32), i)
        assert e.value.code == rx.REINDEX_ERR_OOM
        assert srv.stats()["requests_rejected"] == 1


def test_faulty_request_is_isolated(rx):
    reqs = make_requests(8, 3)
    bad = 4
    v, i = reqs[bad]
    i = i.clone()
    i.view(-1)[1] = v.shape[0]  # out of range
    reqs[bad] = (v, i)
    with rx.Server(hbm_budget_bytes=1 << 28, max_batch_requests=16, num_streams=1) as srv:
        ids = [srv.submit(v, i) for v, i in reqs]
        got = collect(srv, len(ids))
        for r, rid in enumerate(ids):
            if r == bad:
                assert got[rid]["status"] == rx.REINDEX_ERR_INDEX_RANGE
            else:
                assert got[rid]["status"] == 0
                ov, oi = oracle.reindex_sort(reqs[r][0].cpu().numpy().view(np.uint32), reqs[r][1].cpu().numpy())
                np.testing.assert_array_equal(got[rid]["out_idx"].cpu().numpy().reshape(-1), oi)
        assert srv.stats()["batches_split"] >= 1
    rx.reindex_stream_status()  # clear the sticky error
