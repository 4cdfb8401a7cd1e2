"""Scans with per-bin detection factors on the GPU (pet_state_create_attn / pet_reconstruct_attn)
against the FP64 oracle.

The data follow the paper's simulation model (Sec. IV-A): PSF-blurred trues attenuated by
uniform water on the body's support, smoothed scatter at SF = 0.25 and uniform randoms at
RF = 0.25.  The system matrix is diag(a) A with the water attenuation factors a, so p_j is
(A^T a)_j / M per voxel.  Checked: subiterations in each arithmetic (2-D and stacked, BSREM and
SDP-P2 through J0 and the dynamic-nu range), a whole reconstruction with its objective history,
the state objective, bitwise equality in a batch beside a plain scan, refused inputs, and that
a checkpoint does not cross between scans with and without factors.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2111_07886_gb300 import pet, synth

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda:0")


def to_dev(a, dtype=torch.float32):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV, dtype)


def rel_l2(got, ref):
    return float(np.linalg.norm(np.asarray(got, np.float64) - ref) / np.linalg.norm(ref))


def _work(N, P, V, NB, M, kind=4, iters=2, seed=5, counts=None):
    return synth.Workload("attn", N, P, 8.0, V, NB, 8.0, M, counts or 3e5 * P,
                          "ellipsoid3d" if P > 1 else "ellipses2d",
                          synth.AlgoParams(iterations=iters, precond=kind, J0=2, J1=6, a=0.2,
                                           beta=0.5),
                          plane_mm=8.0, seed=seed)


def _state(w, scan, precision, mult=True):
    g = pet.Geometry.from_dict(w.geometry(), scan["sens"])
    return g, pet.State(g, to_dev(scan["counts"], torch.int32), to_dev(scan["gamma"]),
                        pet.make_params(w.params, precision),
                        torch.ones((w.nplanes, w.n, w.n), device=DEV),
                        d_mult=to_dev(scan["mult"]) if mult else None)


@pytest.mark.parametrize("N,P,kind", [(48, 1, 4), (48, 1, 0), (40, 11, 4)])
def test_attn_subiterations(N, P, kind):
    """FP32 + Kahan <= 1e-5 and FP64 <= 1e-10 (relL2) against the oracle after 2, 5 and 9
    subiterations; the plain model on the same data is far from the factors' iterates."""
    w = _work(N, P, 30, 69 if P == 1 else 59, 5, kind=kind)
    scan = synth.make_scan_paper(w)
    og = oracle.geom_from(w.geometry(), scan["sens"])
    for nsub in (2, 5, 9):
        ref, _ = oracle.reconstruct(og, scan["counts"], scan["gamma"], w.params,
                                    np.ones((P, N, N)), nsub=nsub, mult=scan["mult"])
        for prec, tol in ((synth.PREC_FP32_KAHAN, 1e-5), (synth.PREC_FP64, 1e-10)):
            g, st = _state(w, scan, prec)
            for _ in range(nsub):
                st.subiter()
            out = torch.empty((P, N, N), dtype=torch.float64, device=DEV)
            st.read_image(out)
            torch.cuda.synchronize()
            assert rel_l2(out.cpu().numpy(), ref) <= tol, (nsub, prec, rel_l2(out.cpu().numpy(), ref))
            st.close()
    plain, _ = oracle.reconstruct(og, scan["counts"], scan["gamma"], w.params, np.ones((P, N, N)),
                                  nsub=9)
    assert rel_l2(plain, ref) > 1e-2


def test_attn_reconstruction_objective_and_batch():
    """64^2, 10 iterations of SDP-P2 with water attenuation: image relL2 <= 1e-4 and the
    objective history within 1e-6 of the oracle; Phi of the state within 1e-6; in a
    graph-replayed batch beside a plain scan of the same geometry, both give their bits alone."""
    w = _work(64, 1, 60, 91, 6, iters=10, seed=9, counts=1e6)
    scan = synth.make_scan_paper(w)
    og = oracle.geom_from(w.geometry(), scan["sens"])
    ref, obj_ref = oracle.reconstruct(og, scan["counts"], scan["gamma"], w.params,
                                      np.ones((1, 64, 64)), with_objective=True, mult=scan["mult"])
    g = pet.Geometry.from_dict(w.geometry(), scan["sens"])
    counts, gamma, mult = to_dev(scan["counts"], torch.int32), to_dev(scan["gamma"]), to_dev(scan["mult"])
    img = torch.ones((1, 64, 64), device=DEV)
    obj = pet.reconstruct(g, counts, gamma, pet.make_params(w.params), img, objective=True,
                          d_mult=mult)
    got = img.cpu().double().numpy()
    assert rel_l2(got, ref) <= 1e-4, rel_l2(got, ref)
    gap = np.max(np.abs(np.array(obj) - obj_ref) / np.abs(obj_ref))
    assert gap <= 1e-6, gap
    assert obj_ref[-1] < obj_ref[0]
    # the state objective at f^0
    st = pet.State(g, counts, gamma, pet.make_params(w.params), torch.ones((1, 64, 64), device=DEV),
                   d_mult=mult)
    phi, parts = st.objective()
    o = oracle.objective(og, scan["counts"], scan["gamma"], np.ones((1, 64, 64)), w.params.beta,
                         mult=scan["mult"])
    assert abs(phi - o["phi"]) <= 1e-6 * abs(o["phi"])
    assert abs(parts[0] - o["sum_af"]) <= 1e-6 * o["sum_af"]
    # batch: the attenuated scan beside a plain one (same geometry), each equal to itself alone
    alone = []
    for m in (mult, None):
        s1 = pet.State(g, counts, gamma, pet.make_params(w.params), torch.ones((1, 64, 64), device=DEV),
                       d_mult=m)
        for _ in range(w.params.iterations * w.nsubsets):
            s1.subiter()
        out = torch.empty((1, 64, 64), device=DEV)
        s1.read_image(out)
        torch.cuda.synchronize()
        alone.append(out.cpu().numpy())
        s1.close()
    assert rel_l2(alone[0], alone[1]) > 1e-2
    items = [pet.State(g, counts, gamma, pet.make_params(w.params), torch.ones((1, 64, 64), device=DEV),
                       d_mult=m) for m in (mult, None)]
    stream = torch.cuda.Stream()
    batch = pet.Batch(capacity=2, use_graph=True)
    for s1 in items:
        batch.add(s1, with_objective=True, stream=stream)
    while batch.step(stream=stream) > 0:
        pass
    stream.synchronize()
    for s1, want in zip(items, alone):
        out = torch.empty((1, 64, 64), device=DEV)
        s1.read_image(out)
        torch.cuda.synchronize()
        np.testing.assert_array_equal(out.cpu().numpy(), want)


def test_attn_refusals_and_checkpoint():
    w = _work(32, 1, 20, 47, 4, iters=2)
    scan = synth.make_scan_paper(w)
    g = pet.Geometry.from_dict(w.geometry(), scan["sens"])
    counts, gamma = to_dev(scan["counts"], torch.int32), to_dev(scan["gamma"])
    f0 = torch.ones((1, 32, 32), device=DEV)
    prm = pet.make_params(w.params)
    for bad in (-0.5, float("nan"), float("inf")):
        m = scan["mult"].copy()
        m[0, 3, 7] = bad
        with pytest.raises(pet.PetError) as e:
            pet.State(g, counts, gamma, prm, f0, d_mult=to_dev(m))
        assert e.value.status == pet.ERR_INVALID
    a = pet.State(g, counts, gamma, prm, f0, d_mult=to_dev(scan["mult"]))
    a.subiter()
    blob = a.export()
    b = pet.State(g, counts, gamma, prm, f0)
    with pytest.raises(pet.PetError) as e:
        b.load(blob)
    assert e.value.status == pet.ERR_INVALID
    c = pet.State(g, counts, gamma, prm, f0, d_mult=to_dev(scan["mult"]))
    c.load(blob)
    assert c.subiters == 1


def test_attn_served_equals_alone():
    """A scan with detection factors served (pet_request.h_mult) beside a plain one gives the
    bits of the same scan stepped alone, and its objective history is the diag(a) A one."""
    import time
    w = _work(48, 1, 30, 69, 5, iters=3, seed=13)
    scan = synth.make_scan_paper(w)
    g = pet.Geometry.from_dict(w.geometry(), scan["sens"])
    counts, gamma = to_dev(scan["counts"], torch.int32), to_dev(scan["gamma"])
    st = pet.State(g, counts, gamma, pet.make_params(w.params), torch.ones((1, 48, 48), device=DEV),
                   d_mult=to_dev(scan["mult"]))
    for _ in range(w.params.iterations * w.nsubsets):
        st.subiter()
    want = torch.empty((1, 48, 48), device=DEV)
    st.read_image(want)
    torch.cuda.synchronize()
    og = oracle.geom_from(w.geometry(), scan["sens"])
    _, obj_ref = oracle.reconstruct(og, scan["counts"], scan["gamma"], w.params, np.ones((1, 48, 48)),
                                    with_objective=True, mult=scan["mult"])
    server = pet.Server(hbm_budget_bytes=1 << 30, max_slots=4)
    t_plain = server.submit(w.geometry(), scan["sens"], scan["counts"], scan["gamma"],
                            pet.make_params(w.params))
    t_attn = server.submit(w.geometry(), scan["sens"], scan["counts"], scan["gamma"],
                           pet.make_params(w.params), mult=scan["mult"])
    res = {}
    deadline = time.time() + 120
    while len(res) < 2 and time.time() < deadline:
        for t in (t_plain, t_attn):
            if t not in res:
                r = server.poll(t)
                if r is not None:
                    res[t] = r
        time.sleep(0.005)
    server.close()
    img, obj, _ = res[t_attn]
    np.testing.assert_array_equal(img, want.cpu().numpy())
    assert np.max(np.abs(np.array(obj) - obj_ref) / np.abs(obj_ref)) <= 1e-6
    assert rel_l2(res[t_plain][0], want.cpu().numpy()) > 1e-2
    bad = scan["mult"].copy()
    bad[0, 0, 0] = -1.0
    server = pet.Server(hbm_budget_bytes=1 << 30, max_slots=2)
    with pytest.raises(pet.PetError) as e:
        server.submit(w.geometry(), scan["sens"], scan["counts"], scan["gamma"],
                      pet.make_params(w.params), mult=bad)
    assert e.value.status == pet.ERR_INVALID
    server.close()
