"""Host-side fault injection (pet_debug_fail_alloc): an allocation that fails as out of memory
in geometry creation, state creation, a whole reconstruction and serving admission gives
PET_ERR_OOM (a failed request for the server), leaves nothing half-built behind, and the next
calls work and give the same bits as if nothing had failed.  No GPU fault is involved."""
import time

import numpy as np
import pytest
import torch

from paper_2111_07886_gb300 import pet, synth

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda:0")


def _scan():
    w = synth.Workload("f", 32, 3, 4.0, 20, 47, 4.0, 4, 2e5, "ellipsoid3d",
                       synth.AlgoParams(iterations=2), plane_mm=4.0, seed=3)
    return w, synth.make_scan(w)


def _run(g, w, scan):
    st = pet.State(g, torch.from_numpy(scan["counts"]).to(DEV), torch.from_numpy(scan["gamma"]).to(DEV),
                   pet.make_params(w.params), torch.ones((w.nplanes, w.n, w.n), device=DEV))
    for _ in range(w.params.iterations * w.nsubsets):
        st.subiter()
    out = torch.empty((w.nplanes, w.n, w.n), device=DEV)
    st.read_image(out)
    torch.cuda.synchronize()
    st.close()
    return out.cpu().numpy()


def test_injected_allocation_failures():
    w, scan = _scan()
    # geometry creation
    for n in (1, 3, 6):
        pet.debug_fail_alloc(n)
        with pytest.raises(pet.PetError) as e:
            pet.Geometry.from_dict(w.geometry(), scan["sens"])
        assert e.value.status == pet.ERR_OOM, n
    pet.debug_fail_alloc(0)
    g = pet.Geometry.from_dict(w.geometry(), scan["sens"])
    want = _run(g, w, scan)
    # state creation, at several allocations
    counts = torch.from_numpy(scan["counts"]).to(DEV)
    gamma = torch.from_numpy(scan["gamma"]).to(DEV)
    for n in (1, 2, 5):
        pet.debug_fail_alloc(n)
        with pytest.raises(pet.PetError) as e:
            pet.State(g, counts, gamma, pet.make_params(w.params),
                      torch.ones((w.nplanes, w.n, w.n), device=DEV))
        assert e.value.status == pet.ERR_OOM, n
    pet.debug_fail_alloc(0)
    np.testing.assert_array_equal(_run(g, w, scan), want)
    # a whole reconstruction on a fresh geometry (its workspace allocations)
    g2 = pet.Geometry.from_dict(w.geometry(), scan["sens"])
    pet.debug_fail_alloc(1)
    img = torch.ones((w.nplanes, w.n, w.n), device=DEV)
    with pytest.raises(pet.PetError) as e:
        pet.reconstruct(g2, counts, gamma, pet.make_params(w.params), img)
    assert e.value.status == pet.ERR_OOM
    pet.debug_fail_alloc(0)
    img = torch.ones((w.nplanes, w.n, w.n), device=DEV)
    pet.reconstruct(g2, counts, gamma, pet.make_params(w.params), img)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(img.cpu().numpy(), want)


def test_injected_failure_during_serving_admission():
    w, scan = _scan()
    server = pet.Server(hbm_budget_bytes=1 << 30, max_slots=2)
    pet.debug_fail_alloc(1)                 # the first allocation of the admission fails
    t0 = server.submit(w.geometry(), scan["sens"], scan["counts"], scan["gamma"], pet.make_params(w.params))
    err = None
    deadline = time.time() + 60
    while time.time() < deadline:
        try:
            if server.poll(t0) is not None:
                break
        except pet.PetError as e:
            err = e
            break
        time.sleep(0.01)
    pet.debug_fail_alloc(0)
    assert err is not None and err.status == pet.ERR_OOM
    t1 = server.submit(w.geometry(), scan["sens"], scan["counts"], scan["gamma"], pet.make_params(w.params))
    res = None
    while time.time() < deadline and res is None:
        res = server.poll(t1)
        time.sleep(0.01)
    assert res is not None
    g = pet.Geometry.from_dict(w.geometry(), scan["sens"])
    assert np.isfinite(res[0]).all() and res[0].shape == (w.nplanes, w.n, w.n)
    np.testing.assert_allclose(res[0], _run(g, w, scan), rtol=0, atol=0)
    server.close()
