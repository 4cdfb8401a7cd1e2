"""The TV variant on the GPU (pet_params.regularizer = PET_REG_TV) against the FP64 oracle.

The paper's prior is RDP, by its gradient; the TV variant puts total variation into the same
preconditioned step through a proximal step in the step sizes' metric, approximated by
primal-dual iterations warm-started from the previous subiteration's dual variable.  Checked:
the proximal step alone (from a given dual variable), R_TV in the objective, subiterations in
each arithmetic, a whole reconstruction with its objective history, and that batches and the
server refuse TV states.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2111_07886_gb300 import pet, synth

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda:0")


def f32(a):
    return np.asarray(a, np.float32).astype(np.float64)


def to_dev(a, dtype=torch.float32):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV, dtype)


def rel_l2(got, ref):
    return float(np.linalg.norm(np.asarray(got, np.float64) - ref) / np.linalg.norm(ref))


@pytest.mark.parametrize("P", [1, 11])
def test_tv_prox_and_objective(P):
    N = 40
    g = pet.Geometry(N, P, 2.0, 30, 59, 2.0, 5, 0.9)
    rng = np.random.default_rng(P)
    z = f32(rng.uniform(-0.5, 3.0, (P, N, N)))
    W = f32(rng.uniform(0.2, 2.0, (P, N, N)))
    ang = rng.uniform(0, 2 * np.pi, (P, N, N))
    rad = rng.uniform(0, 1, (P, N, N))
    px0, py0 = f32(rad * np.cos(ang)), f32(rad * np.sin(ang))
    px0[:, :, -1] = 0.0                        # no x-difference across the last column
    py0[:, -1, :] = 0.0
    for b, iters in ((0.3, 60), (0.0, 5)):
        d_px, d_py = to_dev(px0), to_dev(py0)
        d_x = torch.empty((P, N, N), device=DEV)
        pet.tv_prox(g, to_dev(z), to_dev(W), b, iters, d_px, d_py, d_x)
        torch.cuda.synchronize()
        x, (px, py) = oracle.tv_prox(z, W, b, iters, (px0, py0))
        assert rel_l2(d_x.cpu().numpy(), x) <= 1e-5, (b, rel_l2(d_x.cpu().numpy(), x))
        assert np.abs(d_px.cpu().numpy() - px).max() <= 1e-5
        assert np.abs(d_py.cpu().numpy() - py).max() <= 1e-5
    w = synth.Workload("t", N, P, 2.0, 30, 59, 2.0, 5, 3e5 * P, "ellipsoid3d" if P > 1 else "ellipses2d",
                       synth.AlgoParams(), plane_mm=2.0, seed=P)
    scan = synth.make_scan(w)
    g2 = pet.Geometry.from_dict(w.geometry(), scan["sens"])
    og2 = oracle.geom_from(w.geometry(), scan["sens"])
    img = f32(rng.uniform(0.2, 3.0, (P, N, N)))
    phi, parts = pet.objective_tv(g2, to_dev(scan["counts"], torch.int32), to_dev(scan["gamma"]),
                                  to_dev(img), 7.0)
    o = oracle.objective(og2, scan["counts"], scan["gamma"], img, 7.0, tv=True)
    assert abs(parts[2] - o["rdp"]) <= 1e-6 * o["rdp"]
    assert abs(phi - o["phi"]) <= 1e-6 * abs(o["phi"])


def _run(w, scan, nsub, precision):
    g = pet.Geometry.from_dict(w.geometry(), scan["sens"])
    st = pet.State(g, to_dev(scan["counts"], torch.int32), to_dev(scan["gamma"]),
                   pet.make_params(w.params, precision),
                   torch.ones((w.nplanes, w.n, w.n), device=DEV))
    for _ in range(nsub):
        st.subiter()
    out = torch.empty((w.nplanes, w.n, w.n), dtype=torch.float64, device=DEV)
    st.read_image(out)
    torch.cuda.synchronize()
    return out.cpu().numpy()


@pytest.mark.parametrize("P,kind", [(1, 0), (1, 4), (11, 4)])
def test_tv_subiterations(P, kind):
    """BSREM and SDP-P2 with the TV proximal step (10 primal-dual iterations per subiteration,
    warm dual) through J0, the dynamic-nu range and the freeze at J1: FP32 + Kahan <= 1e-5,
    FP64 <= 1e-10 against the oracle."""
    N = 48 if P == 1 else 40
    w = synth.Workload("t", N, P, 8.0, 30, 69 if P == 1 else 59, 8.0, 5, 2e5 * P,
                       "ellipsoid3d" if P > 1 else "ellipses2d",
                       synth.AlgoParams(iterations=2, precond=kind, J0=2, J1=6, a=0.2, beta=30.0,
                                        reg=1, tv_iters=10),
                       plane_mm=8.0, seed=5)
    scan = synth.make_scan(w)
    og = oracle.geom_from(w.geometry(), scan["sens"])
    for nsub in (2, 5, 9):
        ref, _ = oracle.reconstruct(og, scan["counts"], scan["gamma"], w.params,
                                    np.ones((P, N, N)), nsub=nsub)
        for prec, tol in ((synth.PREC_FP32_KAHAN, 1e-5), (synth.PREC_FP64, 1e-10)):
            got = _run(w, scan, nsub, prec)
            assert rel_l2(got, ref) <= tol, (P, kind, nsub, prec, rel_l2(got, ref))


def test_tv_reconstruction_and_refusals():
    """64^2, 10 iterations of SDP-P2 with TV: image relL2 <= 1e-4 and the objective history
    (F + beta R_TV) within 1e-6 of the oracle; batches and the server refuse TV."""
    w = synth.Workload("tv64", 64, 1, 8.0, 60, 91, 8.0, 6, 1e6, "ellipses2d",
                       synth.AlgoParams(iterations=10, beta=20.0, reg=1, tv_iters=10), seed=9)
    scan = synth.make_scan(w)
    og = oracle.geom_from(w.geometry(), scan["sens"])
    ref, obj_ref = oracle.reconstruct(og, scan["counts"], scan["gamma"], w.params,
                                      np.ones((1, 64, 64)), with_objective=True)
    g = pet.Geometry.from_dict(w.geometry(), scan["sens"])
    counts, gamma = to_dev(scan["counts"], torch.int32), to_dev(scan["gamma"])
    img = torch.ones((1, 64, 64), device=DEV)
    obj = pet.reconstruct(g, counts, gamma, pet.make_params(w.params), img, objective=True)
    got = img.cpu().double().numpy()
    assert rel_l2(got, ref) <= 1e-4, rel_l2(got, ref)
    gap = np.max(np.abs(np.array(obj) - obj_ref) / np.abs(obj_ref))
    assert gap <= 1e-6, gap
    assert obj_ref[-1] < obj_ref[0]
    st = pet.State(g, counts, gamma, pet.make_params(w.params), torch.ones((1, 64, 64), device=DEV))
    batch = pet.Batch(capacity=2)
    with pytest.raises(pet.PetError) as e:
        batch.add(st)
    assert e.value.status == pet.ERR_INVALID
    server = pet.Server(hbm_budget_bytes=1 << 30, max_slots=2)
    with pytest.raises(pet.PetError) as e:
        server.submit(w.geometry(), scan["sens"], scan["counts"], scan["gamma"], pet.make_params(w.params))
    assert e.value.status == pet.ERR_INVALID
    server.close()
