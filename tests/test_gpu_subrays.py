"""The sub-ray system model on the GPU (pet_geometry_desc.subrays = R > 1) against the oracle.

Each bin is R parallel lines spread across its width (the paper's ray-driven model with parallel
rays per detector pair, Sec. IV-A, 32 there): the projector walks every line, the gather
backprojector sums the lines' lengths per (pixel, bin).  Checked per projection for every subset,
for adjointness, for the sensitivity, over subiterations and a whole reconstruction, and bitwise
between a batch and the scan alone.
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


def per_projection_rel(got, ref):
    den = np.abs(ref).max(axis=-1)
    num = np.abs(np.asarray(got, np.float64) - ref).max(axis=-1)
    ok = den > 0
    assert np.all(num[~ok] == 0)
    return float((num[ok] / den[ok]).max())


# (N, P, V, NB, M, rho, R): odd and even sides, planes in one and two groups, bins finer than pixels
GEOMS = [(48, 1, 30, 69, 4, 1.0, 32), (33, 11, 21, 47, 3, 1.0, 8), (40, 3, 18, 67, 3, 0.8, 5)]


@pytest.mark.parametrize("geom", GEOMS)
def test_subray_projectors(geom):
    N, P, V, NB, M, rho, R = geom
    g = pet.Geometry(N, P, 2.0, V, NB, rho * 2.0, M, 0.9, subrays=R)
    og = oracle.geom(N, P, V, NB, M, pixel_mm=2.0, bin_mm=rho * 2.0, sens=0.9, subrays=R)
    x = f32(synth.random_image((P, N, N), seed=R, lo=0.1, hi=2.0))
    for i in range(M):
        nv = g.subset_size(i)
        ref = oracle.forward(og, i, x)
        out = torch.empty((P, nv, NB), device=DEV)
        pet.forward_subset(g, i, to_dev(x), out)
        out64 = torch.empty((P, nv, NB), dtype=torch.float64, device=DEV)
        pet.forward_subset(g, i, to_dev(x, torch.float64), out64)
        torch.cuda.synchronize()
        assert per_projection_rel(out.cpu().numpy(), ref) <= 1e-5, i
        assert per_projection_rel(out64.cpu().numpy(), ref) <= 1e-11, i
        y = f32(synth.random_image((P, nv, NB), seed=i + 3, lo=0.0, hi=1.0))
        bref = oracle.back(og, i, y)
        b = torch.empty((P, N, N), device=DEV)
        pet.back_subset(g, i, to_dev(y), b)
        torch.cuda.synchronize()
        err = np.abs(b.cpu().numpy() - bref).max()
        assert err <= 1e-5 * np.abs(bref).max(), (i, err)
        # adjointness of the FP32 pair
        lhs = np.vdot(out.cpu().double().numpy(), y)
        rhs = np.vdot(x, b.cpu().double().numpy())
        assert abs(lhs - rhs) <= 1e-5 * abs(lhs)
    p = torch.empty((N, N), device=DEV)
    pet.sensitivity(g, p)
    torch.cuda.synchronize()
    np.testing.assert_allclose(p.cpu().numpy(), oracle.sensitivity(og), rtol=1e-6)


def _work(N, P, R, iters=3, seed=4):
    nb = int(1.45 * N) | 1
    return synth.Workload(f"sub{R}", N, P, 4.0, 36, nb, 4.0, 4, 2e5 * P,
                          "ellipsoid3d" if P > 1 else "ellipses2d",
                          synth.AlgoParams(iterations=iters, J0=2, J1=6, a=0.2), plane_mm=4.0,
                          seed=seed, subrays=R)


@pytest.mark.parametrize("N,P,R", [(48, 1, 32), (40, 11, 8)])
def test_subray_reconstruction(N, P, R):
    """SDP-P2 with sub-rays through J0 and the dynamic-nu range, then a whole reconstruction with
    its objective history, against the oracle; FP64 <= 1e-10 on the subiterations."""
    w = _work(N, P, R)
    scan = synth.make_scan(w)
    og = oracle.geom_from(w.geometry(), scan["sens"])
    g = pet.Geometry.from_dict(w.geometry(), scan["sens"])
    counts, gamma = to_dev(scan["counts"], torch.int32), to_dev(scan["gamma"])
    for nsub in (3, 7):
        ref, _ = oracle.reconstruct(og, scan["counts"], scan["gamma"], w.params,
                                    np.ones((P, N, N)), nsub=nsub)
        for prec, tol in ((synth.PREC_FP32_KAHAN, 1e-5), (synth.PREC_FP64, 1e-10)):
            st = pet.State(g, counts, gamma, pet.make_params(w.params, prec),
                           torch.ones((P, N, N), device=DEV))
            for _ in range(nsub):
                st.subiter()
            out = torch.empty((P, N, N), dtype=torch.float64, device=DEV)
            st.read_image(out)
            torch.cuda.synchronize()
            assert rel_l2(out.cpu().numpy(), ref) <= tol, (nsub, prec, rel_l2(out.cpu().numpy(), ref))
            st.close()
    ref, obj_ref = oracle.reconstruct(og, scan["counts"], scan["gamma"], w.params,
                                      np.ones((P, N, N)), with_objective=True)
    img = torch.ones((P, N, N), device=DEV)
    obj = pet.reconstruct(g, counts, gamma, pet.make_params(w.params), img, objective=True)
    assert rel_l2(img.cpu().numpy(), ref) <= 1e-4
    gap = np.max(np.abs(np.array(obj) - obj_ref) / np.abs(obj_ref))
    assert gap <= 1e-6, gap


def test_subray_scan_batched_beside_one_line_scan():
    """A sub-ray scan and a one-line scan of the same size in one graph-replayed batch: each gives
    the bits it gives alone."""
    ws = [_work(48, 1, 16, iters=2, seed=6), _work(48, 1, 1, iters=2, seed=6)]
    scans = [synth.make_scan(w) for w in ws]
    alone, items = [], []
    for w, sc in zip(ws, scans):
        g = pet.Geometry.from_dict(w.geometry(), sc["sens"])
        c, gm = to_dev(sc["counts"], torch.int32), to_dev(sc["gamma"])
        st = pet.State(g, c, gm, pet.make_params(w.params), torch.ones((1, 48, 48), device=DEV))
        for _ in range(w.params.iterations * w.nsubsets):
            st.subiter()
        out = torch.empty((1, 48, 48), device=DEV)
        st.read_image(out)
        torch.cuda.synchronize()
        alone.append(out.cpu().numpy())
        items.append((g, c, gm, pet.State(g, c, gm, pet.make_params(w.params),
                                          torch.ones((1, 48, 48), device=DEV))))
    assert rel_l2(alone[0], alone[1]) > 1e-3
    stream = torch.cuda.Stream()
    batch = pet.Batch(capacity=2, use_graph=True)
    for it in items:
        batch.add(it[3], with_objective=True, stream=stream)
    while batch.step(stream=stream) > 0:
        pass
    stream.synchronize()
    for it, ref in zip(items, alone):
        out = torch.empty((1, 48, 48), device=DEV)
        it[3].read_image(out)
        torch.cuda.synchronize()
        np.testing.assert_array_equal(out.cpu().numpy(), ref)
