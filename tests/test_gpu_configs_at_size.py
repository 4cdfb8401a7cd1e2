"""Batched and served scans at the sizes of the mixed 2-D workload (GPU).

The mixed workload draws N from {128, 200, 256, 400} at a 512 mm field of view, 120-360 views,
n_b = the largest odd number <= 1.45 N (bin = pixel, so every view's pixel footprint spans at
most two bins: the KC = 2 gather) and 12-36 subsets, 10 iterations.  Each scan below is
reconstructed alone (pet_subiter), in one graph-replayed batch with all the others, and by the
FP64 oracle: the batch must give the same bits as the scan alone, and the image must be within
relative L2 1e-4 of the oracle after the 10 iterations.  The serving test puts the largest scan
and a clinical-size stacked 256^2 x 89 job into one server with other scans and checks that
each result is bitwise the one the scan gives alone.
"""
import time

import numpy as np
import pytest
import torch

import oracle
from paper_2111_07886_gb300 import pet, synth

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda:0")

# (N, views, subsets, counts): every image size and subset count of the mix, 120 and 360 views
SCANS = [(128, 150, 18, 2e5), (200, 120, 12, 1e5), (256, 360, 36, 1e7), (256, 200, 24, 3e6),
         (400, 360, 36, 5e6), (400, 120, 18, 1e6)]


def workload(N, V, M, counts, seed, iterations=10):
    nb = int(np.floor(1.45 * N))
    nb -= 1 - nb % 2
    p = synth.AlgoParams(iterations=iterations, beta=0.05, **synth.P2_WORKLOAD)
    return synth.Workload(f"mix_{N}_v{V}_b{nb}_m{M}", N, 1, 512.0 / N, V, nb, 512.0 / N, M,
                          counts, "ellipses2d", p, seed=seed)


def _upload(w, sc):
    g = pet.Geometry.from_dict(w.geometry(), sc["sens"])
    c = torch.from_numpy(sc["counts"]).to(DEV)
    gm = torch.from_numpy(sc["gamma"]).to(DEV)
    f0 = torch.ones((w.nplanes, w.n, w.n), device=DEV)
    return g, c, gm, f0


def _image(st, w):
    out = torch.empty((w.nplanes, w.n, w.n), device=DEV)
    st.read_image(out)
    torch.cuda.synchronize()
    return out.cpu().numpy()


@pytest.fixture(scope="module")
def mixed():
    ws = [workload(N, V, M, c, seed=700 + k) for k, (N, V, M, c) in enumerate(SCANS)]
    assert sorted({w.nbins for w in ws}) == [185, 289, 371, 579]
    scans = [synth.make_scan(w) for w in ws]
    alone = []
    for w, sc in zip(ws, scans):
        g, c, gm, f0 = _upload(w, sc)
        st = pet.State(g, c, gm, pet.make_params(w.params), f0)
        for _ in range(w.params.iterations * w.nsubsets):
            st.subiter()
        alone.append(_image(st, w))
        st.close()
    ref = []
    for w, sc in zip(ws, scans):
        og = oracle.geom_from(w.geometry(), sc["sens"])
        f, _ = oracle.reconstruct(og, sc["counts"], sc["gamma"], w.params,
                                  np.ones((w.nplanes, w.n, w.n)))
        ref.append(f)
    return ws, scans, alone, ref


def test_mixed_sizes_match_oracle(mixed):
    ws, scans, alone, ref = mixed
    for w, got, f in zip(ws, alone, ref):
        rel = np.linalg.norm(got - f) / np.linalg.norm(f)
        assert rel <= 1e-4, (w.name, rel)


def test_mixed_sizes_batched_bitwise_equal_alone(mixed):
    ws, scans, alone, _ = mixed
    stream = torch.cuda.Stream()
    batch = pet.Batch(capacity=len(ws), use_graph=True)
    keep = []
    for w, sc in zip(ws, scans):
        g, c, gm, f0 = _upload(w, sc)
        st = pet.State(g, c, gm, pet.make_params(w.params), f0)
        keep.append((g, c, gm, st))
        batch.add(st, with_objective=True, stream=stream)
    ticks = 1
    while batch.step(stream=stream) > 0:
        ticks += 1
    stream.synchronize()
    assert ticks == max(w.params.iterations * w.nsubsets for w in ws)
    for (g, c, gm, st), w, ref in zip(keep, ws, alone):
        np.testing.assert_array_equal(_image(st, w), ref, err_msg=w.name)
        obj = st.objective_history()
        assert np.all(np.isfinite(obj)) and obj[-1] < obj[0], (w.name, obj)


def _wait(server, tickets, timeout=600.0):
    out = {}
    t0 = time.time()
    while len(out) < len(tickets):
        for t in tickets:
            if t not in out:
                r = server.poll(t)
                if r is not None:
                    out[t] = r
        assert time.time() - t0 < timeout, "serving timed out"
        time.sleep(0.005)
    return out


def test_serving_mix_with_large_scan_and_stacked_job(mixed):
    """A 400^2 x 360-view scan, a clinical-size stacked 256^2 x 89 job (20 iterations) and the
    other mixed scans, submitted in a staggered stream: every result equals the scan alone."""
    ws, scans, alone, ref = mixed
    wst = synth.config_stacked_256x89(seed=21, iterations=20)
    sst = synth.make_scan(wst)
    g, c, gm, f0 = _upload(wst, sst)
    st = pet.State(g, c, gm, pet.make_params(wst.params), f0)
    for _ in range(wst.params.iterations * wst.nsubsets):
        st.subiter()
    stacked_alone = _image(st, wst)
    st.close()
    del g, c, gm, f0
    big = max(range(len(ws)), key=lambda k: ws[k].n * ws[k].nviews)
    order = [big, len(ws)] + [k for k in range(len(ws)) if k != big]
    server = pet.Server(hbm_budget_bytes=8 << 30, max_slots=4)
    tickets = []
    for k in order:
        w, sc = (wst, sst) if k == len(ws) else (ws[k], scans[k])
        tickets.append(server.submit(w.geometry(), sc["sens"], sc["counts"], sc["gamma"],
                                     pet.make_params(w.params)))
        time.sleep(0.003)
    res = _wait(server, tickets)
    for t, k in zip(tickets, order):
        want = stacked_alone if k == len(ws) else alone[k]
        np.testing.assert_array_equal(res[t][0], want, err_msg=str(k))
        obj = res[t][1]
        assert np.all(np.isfinite(obj)) and obj[-1] < obj[0]
    got_big = res[tickets[0]][0]
    assert np.linalg.norm(got_big - ref[big]) / np.linalg.norm(ref[big]) <= 1e-4
    s = server.stats()
    assert s["completed"] == len(order) and s["failed"] == 0
    server.close()
