"""heart_trace_batch_static: the batched trace for callers that cannot
allocate device memory while they run (for example an application that gave
all free device memory to its own pool, or a loop that must not risk an
allocation failure).  It runs the same kernel as heart_trace_batch on a fixed
device work area, so on the same inputs it must give the same integer images
and tallies, on every call: the work area keeps the previous call's contents
and each call has to start its counters from zero.

Collected last on purpose (file name), so that a stopping run has already run
every other test."""
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


def _zeros(spec, torch):
    dt = torch.int64 if spec.count_dtype == "int64" else torch.int32
    return torch.zeros(spec.shape, dtype=dt, device="cuda")


def test_static_batch_equals_allocating_batch_on_two_calls_in_a_row(H):
    import torch
    jobs = W.batched_64(seed=7, n_configs=5, ray_range=(2e4, 2.5e5))
    specs = [H.heart_spectrometer_create(j["spec"]) for j in jobs]
    srcs = [j["source"] for j in jobs]
    nr = [j["n_rays"] for j in jobs]
    seeds = [j["seed"] for j in jobs]
    ref = [_zeros(s, torch) for s in specs]
    t_ref = H.heart_trace_batch(specs, srcs, nr, seeds, ref)
    for call in range(2):
        imgs = [_zeros(s, torch) for s in specs]
        t = H.heart_trace_batch_static(specs, srcs, nr, seeds, imgs)
        torch.cuda.synchronize()
        for i in range(len(jobs)):
            assert torch.equal(imgs[i], ref[i]), (call, i)
            assert t[i] == t_ref[i], (call, i)
            assert t[i]["emitted"] == nr[i]
    for s in specs:
        s.close()


def test_static_batch_rejects_more_jobs_than_its_work_area(H):
    import torch
    w = W.flat_hopg_mono()
    s = H.heart_spectrometer_create(w["spec"])
    img = _zeros(s, torch)
    n = H.STATIC_MAX_JOBS + 1
    with pytest.raises(H.HeartError) as e:
        H.heart_trace_batch_static([s] * n, [w["source"]] * n, [10] * n, [1] * n, [img] * n)
    assert e.value.status == 1 and "HEART_STATIC_MAX_JOBS" in str(e.value)
    assert int(img.sum()) == 0
    s.close()


def test_static_batch_with_a_large_job_allocates_nothing_and_matches_the_two_pass_trace(H):
    # heart_trace_batch runs a job of 2^19 rays as a two-pass trace (hit queue) and the small
    # ones in one persistent launch; the static call runs all of them on the persistent kernel,
    # which traces every ray as the two-pass trace does: the same images and tallies.  After a
    # first call on the device (which looks up the work area's address), a call changes the
    # device's free memory by nothing: it allocates no device memory.
    import torch
    jobs = W.batched_64(seed=9, n_configs=3, ray_range=(2e4, 6e4))
    big = W.von_hamos_hapg()
    specs = [H.heart_spectrometer_create(j["spec"]) for j in jobs] + [H.heart_spectrometer_create(big["spec"])]
    srcs = [j["source"] for j in jobs] + [big["source"]]
    nr = [j["n_rays"] for j in jobs] + [1 << 19]
    seeds = [j["seed"] for j in jobs] + [33]
    ref = [_zeros(s, torch) for s in specs]
    t_ref = H.heart_trace_batch(specs, srcs, nr, seeds, ref)
    for call in range(2):
        imgs = [_zeros(s, torch) for s in specs]
        torch.cuda.synchronize()
        free0 = torch.cuda.mem_get_info()[0]
        t = H.heart_trace_batch_static(specs, srcs, nr, seeds, imgs)
        torch.cuda.synchronize()
        free1 = torch.cuda.mem_get_info()[0]
        if call == 1:
            assert free1 == free0, (free0, free1)
        for i in range(len(specs)):
            assert torch.equal(imgs[i], ref[i]), (call, i)
            assert t[i] == t_ref[i], (call, i)
    assert t_ref[-1]["det_hits"] > 50
    for s in specs:
        s.close()


def test_static_batch_rejects_a_tabulated_spectrum(H):
    import numpy as np
    import torch
    w = W.flat_hopg_mono()
    s = H.heart_spectrometer_create(w["spec"])
    img = _zeros(s, torch)
    src = dict(w["source"], components=[dict(kind="table", weight=1.0)],
               table=(np.linspace(7.9, 8.1, 5), np.ones(5)))
    with pytest.raises(H.HeartError) as e:
        H.heart_trace_batch_static([s], [src], [1000], [1], [img])
    assert e.value.status == 1 and "tabulated" in str(e.value)
    torch.cuda.synchronize()
    assert int(img.sum()) == 0
    s.close()
