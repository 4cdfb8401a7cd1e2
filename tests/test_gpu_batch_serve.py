"""Batched and served reconstruction (GPU): every scan gives the same bits alone and in a mix.

A batch advances many independent scans per step with persistent kernels (optionally
graph-replayed); the server admits requests continuously into such a batch.  Each scan keeps
its own launch shapes and reduction scratch, so the result must be bitwise identical to the
scan reconstructed on its own, and within the parity tolerance of the FP64 oracle.
"""
import time

import numpy as np
import pytest
import torch

import oracle
from paper_2111_07886_gb300 import pet, synth

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda:0")


def small_mix(seed=3, iterations=2):
    rng = np.random.default_rng(seed)
    ws = []
    for s in range(5):
        n = int(rng.choice([32, 48, 64]))
        v = int(rng.integers(18, 40))
        nb = (3 * n // 2) | 1
        m = int(rng.choice([3, 4, 6]))
        ws.append(synth.Workload(f"mix{s}", n, 1, 512.0 / n, v, nb, 512.0 / n, m,
                                 float(10 ** rng.uniform(5, 6)), "ellipses2d",
                                 synth.AlgoParams(iterations=iterations, J0=1), seed=seed * 10 + s))
    ws.append(synth.Workload("stacked", 40, 9, 8.0, 30, 61, 8.0, 5, 5e5, "ellipsoid3d",
                             synth.AlgoParams(iterations=iterations, J0=1), plane_mm=8.0, seed=99))
    return ws


def _state(w, scan):
    g = pet.Geometry.from_dict(w.geometry(), scan["sens"])
    counts = torch.from_numpy(scan["counts"]).to(DEV)
    gamma = torch.from_numpy(scan["gamma"]).to(DEV)
    f0 = torch.ones((w.nplanes, w.n, w.n), device=DEV)
    st = pet.State(g, counts, gamma, pet.make_params(w.params), f0)
    return g, st


def _image(st, w):
    out = torch.empty((w.nplanes, w.n, w.n), device=DEV)
    st.read_image(out)
    torch.cuda.synchronize()
    return out.cpu().numpy()


@pytest.fixture(scope="module")
def mix():
    ws = small_mix()
    scans = [synth.make_scan(w) for w in ws]
    alone = []
    for w, sc in zip(ws, scans):
        g, st = _state(w, sc)
        for _ in range(w.params.iterations * w.nsubsets):
            st.subiter()
        alone.append(_image(st, w))
    return ws, scans, alone


@pytest.mark.parametrize("use_graph", [True, False])
def test_batch_bitwise_equals_alone(mix, use_graph):
    ws, scans, alone = mix
    stream = torch.cuda.Stream()
    batch = pet.Batch(capacity=8, use_graph=use_graph)
    keep = []
    for w, sc in zip(ws, scans):
        g, st = _state(w, sc)
        keep.append((g, st))
        batch.add(st, with_objective=True, stream=stream)
    steps = 0
    while batch.step(stream=stream) > 0:
        steps += 1
    stream.synchronize()
    assert steps + 1 == max(w.params.iterations * w.nsubsets for w in ws)
    for (g, st), w, ref in zip(keep, ws, alone):
        np.testing.assert_array_equal(_image(st, w), ref)
        obj = st.objective_history()
        assert np.all(np.isfinite(obj)) and obj[-1] < obj[0]
    # objective history equals the one pet_reconstruct records for the same scan
    w, sc = ws[0], scans[0]
    g = pet.Geometry.from_dict(w.geometry(), sc["sens"])
    img = torch.ones((w.nplanes, w.n, w.n), device=DEV)
    obj_ref = pet.reconstruct(g, torch.from_numpy(sc["counts"]).to(DEV),
                              torch.from_numpy(sc["gamma"]).to(DEV), pet.make_params(w.params),
                              img, objective=True)
    assert keep[0][1].objective_history() == obj_ref


def test_batched_scans_match_oracle(mix):
    ws, scans, alone = mix
    for w, sc, got in list(zip(ws, scans, alone))[::2]:
        og = oracle.geom_from(w.geometry(), sc["sens"])
        ref, _ = oracle.reconstruct(og, sc["counts"], sc["gamma"], w.params,
                                    np.ones((w.nplanes, w.n, w.n)))
        assert np.linalg.norm(got - ref) / np.linalg.norm(ref) <= 1e-5


def _wait(server, tickets, timeout=180.0):
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


def test_serve_alone_equals_mix(mix):
    ws, scans, alone = mix
    server = pet.Server(hbm_budget_bytes=2 << 30, max_slots=4)
    # scan 0 alone
    t = server.submit(ws[0].geometry(), scans[0]["sens"], scans[0]["counts"], scans[0]["gamma"],
                      pet.make_params(ws[0].params))
    img_alone, obj_alone, lat = _wait(server, [t])[t]
    np.testing.assert_array_equal(img_alone, alone[0])
    assert lat > 0
    # a staggered stream of all scans (scan 0 among them) with fewer slots than requests
    tickets = []
    for w, sc in zip(ws, scans):
        tickets.append(server.submit(w.geometry(), sc["sens"], sc["counts"], sc["gamma"],
                                     pet.make_params(w.params)))
        time.sleep(0.002)
    res = _wait(server, tickets)
    for t, ref in zip(tickets, alone):
        np.testing.assert_array_equal(res[t][0], ref)
    assert res[tickets[0]][1] == obj_alone
    st = server.stats()
    assert st["completed"] == 1 + len(ws) and st["failed"] == 0
    assert 0 < st["p50_s"] <= st["p99_s"]
    server.close()


def test_serve_admission_and_errors(mix):
    ws, scans, _ = mix
    w, sc = ws[0], scans[0]
    server = pet.Server(hbm_budget_bytes=64 << 10, max_slots=2)    # 64 KiB: too small
    bad = sc["gamma"].copy()
    bad.flat[3] = 0.0
    with pytest.raises(pet.PetError) as e:
        server.submit(w.geometry(), sc["sens"], sc["counts"], bad, pet.make_params(w.params))
    assert e.value.status == pet.ERR_INVALID
    t = server.submit(w.geometry(), sc["sens"], sc["counts"], sc["gamma"], pet.make_params(w.params))
    t0 = time.time()
    while True:
        try:
            r = server.poll(t)
        except pet.PetError as err:
            assert err.status == pet.ERR_OOM
            break
        assert r is None and time.time() - t0 < 60
        time.sleep(0.01)
    with pytest.raises(pet.PetError) as e:
        server.poll(t)
    assert e.value.status == pet.ERR_NOT_FOUND
    server.close()
