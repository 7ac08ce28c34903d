"""Batched persistent launch and the request loop (continuous batching).

Each ray owns a counter-addressed Philox stream and images are integer, so a
job's image must not depend on which other jobs share the launch, on how its
rays are sliced into rounds, or on admission order: the tests check bit
identity between "alone" and "in the mix"."""
import time

import numpy as np
import pytest

from paper_2503_16955_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def H():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    import paper_2503_16955_gb300 as H
    return H


def _mix(n_jobs, seed, ray_range):
    jobs = W.batched_64(seed=seed, n_configs=n_jobs, ray_range=ray_range)
    return jobs


def _img(H, spec, torch):
    return torch.zeros(spec.shape, dtype=torch.int64 if spec.count_dtype == "int64" else torch.int32,
                       device="cuda")


def test_batch_alone_equals_mixed_and_matches_single_launches(H):
    import torch
    jobs = _mix(12, 33, (1e4, 3e5))
    specs = [H.heart_spectrometer_create(j["spec"]) for j in jobs]
    imgs = [_img(H, s, torch) for s in specs]
    tall = H.heart_trace_batch(specs, [j["source"] for j in jobs], [j["n_rays"] for j in jobs],
                               [j["seed"] for j in jobs], imgs)
    for i in (0, 5, 11):
        alone = _img(H, specs[i], torch)
        t1 = H.heart_trace_batch([specs[i]], [jobs[i]["source"]], [jobs[i]["n_rays"]], [jobs[i]["seed"]], [alone])[0]
        assert torch.equal(alone, imgs[i]), i
        assert t1 == tall[i]
    for i, (j, t) in enumerate(zip(jobs, tall)):
        assert t["emitted"] == j["n_rays"]
        assert t["emitted"] == (t["miss"] + t["absorbed"] + t["exit_front"] + t["exit_back"] + t["exit_side"] +
                                t["capped"] + t["stuck"])
        assert t["det_hits"] == int(imgs[i].sum())
        # the specialised single-job kernel computes the same rays; allow only
        # rounding-level decision differences between the two instantiations
        single = _img(H, specs[i], torch)
        ts = H.heart_trace(specs[i], j["source"], j["n_rays"], j["seed"], 0, single, precision="fp32")
        diff = int((single.to(torch.int64) - imgs[i].to(torch.int64)).abs().sum())
        assert diff <= 2 + 1e-4 * j["n_rays"], (i, diff)
        assert abs(ts["collisions"] - t["collisions"]) <= 1e-4 * max(1, t["collisions"]) + 50
    for s in specs:
        s.close()


def test_batch_large_jobs_equal_their_single_traces(H):
    # jobs of 2^18 rays or more run as two-pass traces inside the batch: image and
    # tallies equal to heart_trace of the same job; the small jobs in the same call
    # still equal the batch of themselves alone
    import torch
    jobs = _mix(4, 55, (1e4, 2e5))
    jobs[1]["n_rays"] = 5_000_000
    jobs[2]["n_rays"] = 1 << 18
    specs = [H.heart_spectrometer_create(j["spec"]) for j in jobs]
    imgs = [_img(H, s, torch) for s in specs]
    tall = H.heart_trace_batch(specs, [j["source"] for j in jobs], [j["n_rays"] for j in jobs],
                               [j["seed"] for j in jobs], imgs)
    for i in (1, 2):
        single = _img(H, specs[i], torch)
        t1 = H.heart_trace(specs[i], jobs[i]["source"], jobs[i]["n_rays"], jobs[i]["seed"], 0, single)
        assert torch.equal(single, imgs[i]), i
        assert t1 == tall[i], i
        assert tall[i]["emitted"] == jobs[i]["n_rays"]
    small = [0, 3]
    sim = [_img(H, specs[i], torch) for i in small]
    ts = H.heart_trace_batch([specs[i] for i in small], [jobs[i]["source"] for i in small],
                             [jobs[i]["n_rays"] for i in small], [jobs[i]["seed"] for i in small], sim)
    for k, i in enumerate(small):
        assert torch.equal(sim[k], imgs[i]) and ts[k] == tall[i], i
    for s in specs:
        s.close()


def test_batch_with_empty_and_single_ray_jobs(H):
    # degenerate jobs inside one batch call: jobs of no rays leave their images and
    # tallies untouched, a one-ray job traces its one ray, and the other jobs equal
    # the batch of themselves alone
    import torch
    jobs = _mix(5, 77, (1e4, 1e5))
    jobs[0]["n_rays"] = 0
    jobs[2]["n_rays"] = 1
    jobs[4]["n_rays"] = 0
    specs = [H.heart_spectrometer_create(j["spec"]) for j in jobs]
    imgs = [_img(H, s, torch) for s in specs]
    for i in (0, 4):
        imgs[i].fill_(7)
    tall = H.heart_trace_batch(specs, [j["source"] for j in jobs], [j["n_rays"] for j in jobs],
                               [j["seed"] for j in jobs], imgs)
    for i in (0, 4):
        assert int((imgs[i] != 7).sum()) == 0
        assert all(v == 0 for k, v in tall[i].items() if k != "refl_hist") and not any(tall[i]["refl_hist"])
    t = tall[2]
    assert t["emitted"] == 1 == (t["miss"] + t["absorbed"] + t["exit_front"] + t["exit_back"] + t["exit_side"] +
                                 t["capped"] + t["stuck"])
    assert int(imgs[2].sum()) == t["det_hits"] <= 1
    rest = [1, 2, 3]
    sim = [_img(H, specs[i], torch) for i in rest]
    ts = H.heart_trace_batch([specs[i] for i in rest], [jobs[i]["source"] for i in rest],
                             [jobs[i]["n_rays"] for i in rest], [jobs[i]["seed"] for i in rest], sim)
    for k, i in enumerate(rest):
        assert torch.equal(sim[k], imgs[i]) and ts[k] == tall[i], i
    for s in specs:
        s.close()


def test_server_results_identical_alone_and_in_the_mix(H):
    import torch
    jobs = _mix(10, 44, (5e4, 2e6))
    jobs[3]["n_rays"] = 30_000_000          # sliced over several rounds when mixed
    jobs[7]["n_rays"] = 20_000_000
    specs = [H.heart_spectrometer_create(j["spec"]) for j in jobs]
    # alone: one job per server
    alone = []
    for s, j in zip(specs, jobs):
        srv = H.heart_server_create(1 << 30)
        jid = srv.submit(s, j["source"], j["n_rays"], j["seed"])
        st, t, ptr = srv.poll(jid, timeout_ms=120_000)
        assert st == "HEART_OK"
        out = srv.fetch(jid, _img(H, s, torch))
        alone.append((out, t))
        srv.release(jid)
        srv.close()
    # mixed: staggered submissions into one server whose cap admits 3 images
    cap = 3 * max(s.shape[0] * s.shape[1] * 4 for s in specs)
    srv = H.heart_server_create(cap)
    ids = []
    for s, j in zip(specs, jobs):
        ids.append(srv.submit(s, j["source"], j["n_rays"], j["seed"]))
        time.sleep(0.002)
    for i, jid in enumerate(ids):
        st, t, ptr = srv.poll(jid, timeout_ms=300_000)
        assert st == "HEART_OK"
        out = srv.fetch(jid, _img(H, specs[i], torch))
        assert torch.equal(out, alone[i][0]), i
        assert t == alone[i][1], i
        assert srv.latency(jid) > 0
        srv.release(jid)            # frees memory so queued jobs can be admitted
    srv.close()
    for s in specs:
        s.close()


def test_server_errors(H):
    w = W.flat_hopg_mono()
    s = H.heart_spectrometer_create(w["spec"])
    srv = H.heart_server_create(1024)                  # too small for a 256^2 int32 image
    with pytest.raises(H.HeartError) as e:
        srv.submit(s, w["source"], 1000, 1)
    assert e.value.status == 2
    srv.close()
    srv = H.heart_server_create(1 << 28)
    with pytest.raises(H.HeartError) as e:
        srv.poll(12345)
    assert e.value.status == 7
    jid = srv.submit(s, w["source"], 50_000_000, 1)
    st, t, _ = srv.poll(jid, timeout_ms=0)
    assert st in ("HEART_EBUSY", "HEART_OK")
    st, t, _ = srv.poll(jid, timeout_ms=120_000)
    assert st == "HEART_OK" and t["emitted"] == 50_000_000
    srv.release(jid)
    with pytest.raises(H.HeartError) as e:
        srv.release(jid)
    assert e.value.status == 7
    srv.close()
    s.close()
