"""Ring-sampled bins on the GPU (pet_geometry_desc.ring_mm > 0) against the FP64 oracle.

The bins of a view are the lines of a detector ring equally spaced in angle (the paper's
576-detector ring, Sec. IV-A), r_b = Rd sin(beta_b), each with R sub-rays over its width.
Checked: forward projection per projection and gather backprojection for every subset in FP32
and FP64, adjointness, sensitivity, subiterations and a whole reconstruction with its objective
history, ring + TOF, and bitwise equality in a batch beside a uniform-bin scan.
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
    got = np.asarray(got, np.float64).reshape(ref.shape[0], ref.shape[1], -1)
    ref = ref.reshape(ref.shape[0], ref.shape[1], -1)
    den = np.abs(ref).max(axis=-1)
    num = np.abs(got - ref).max(axis=-1)
    ok = den > 0
    assert np.all(num[~ok] <= 1e-30)
    return float((num[ok] / den[ok]).max())


# (N, P, V, NB, M, pixel_mm, bin_mm (arc), ring_mm, R): the paper's ring of 576 x 4 mm detectors
# (radius 366.7 mm) at 4 mm arc bins, tighter rings, sub-rays, one and two plane groups
GEOMS = [(48, 1, 36, 61, 4, 4.0, 4.0, 366.7, 1), (40, 11, 24, 67, 3, 4.0, 4.0, 220.0, 1),
         (33, 3, 21, 47, 3, 4.0, 4.0, 120.0, 8), (32, 1, 30, 41, 5, 4.0, 4.5, 366.7, 32)]


@pytest.mark.parametrize("geom", GEOMS)
def test_ring_projectors(geom):
    N, P, V, NB, M, px, bmm, rmm, R = geom
    g = pet.Geometry(N, P, px, V, NB, bmm, M, 0.9, subrays=R, ring_mm=rmm)
    og = oracle.geom(N, P, V, NB, M, pixel_mm=px, bin_mm=bmm, sens=0.9, subrays=R, ring_mm=rmm)
    x = f32(synth.random_image((P, N, N), seed=NB, lo=0.1, hi=2.0))
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
        b64 = torch.empty((P, N, N), dtype=torch.float64, device=DEV)
        pet.back_subset(g, i, to_dev(y, torch.float64), b64)
        torch.cuda.synchronize()
        assert np.abs(b.cpu().numpy() - bref).max() <= 1e-5 * np.abs(bref).max(), i
        assert np.abs(b64.cpu().numpy() - bref).max() <= 1e-11 * np.abs(bref).max(), i
        lhs = np.vdot(out.cpu().double().numpy(), y)
        rhs = np.vdot(x, b.cpu().double().numpy())
        assert abs(lhs - rhs) <= 1e-5 * abs(lhs)
    p = torch.empty((N, N), device=DEV)
    pet.sensitivity(g, p)
    torch.cuda.synchronize()
    np.testing.assert_allclose(p.cpu().numpy(), oracle.sensitivity(og), rtol=1e-6)


def _work(N, P, R=1, T=0, iters=2, seed=4, ring_mm=180.0):
    w = synth.Workload(f"ring{R}", N, P, 4.0, 30, int(1.45 * N) | 1, 4.0, 5, 3e5 * P,
                       "ellipsoid3d" if P > 1 else "ellipses2d",
                       synth.AlgoParams(iterations=iters, J0=2, J1=6, a=0.2, beta=0.5),
                       plane_mm=4.0, seed=seed, subrays=R, tof_bins=T,
                       tof_bin_mm=20.0 if T else 0.0, tof_fwhm_mm=45.0 if T else 0.0)
    geo = dict(w.geometry(), ring_mm=ring_mm)
    return w, geo


@pytest.mark.parametrize("N,P,R,T", [(48, 1, 1, 0), (40, 11, 4, 0), (40, 3, 1, 13)])
def test_ring_subiterations_and_reconstruction(N, P, R, T):
    """FP32 + Kahan <= 1e-5 and FP64 <= 1e-10 (relL2) against the oracle after 3 and 7
    subiterations; a whole reconstruction with its objective history (image <= 1e-4,
    objective <= 1e-6).  The data come from the uniform-bin analytic projections (a model
    mismatch that the comparison with the oracle does not care about)."""
    w, geo = _work(N, P, R, T)
    scan = synth.make_scan(w)
    og = oracle.geom_from(geo, scan["sens"])
    g = pet.Geometry.from_dict(geo, scan["sens"])
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
    assert np.max(np.abs(np.array(obj) - obj_ref) / np.abs(obj_ref)) <= 1e-6


def test_ring_scan_batched_beside_uniform_scan():
    """A ring-sampled scan and a uniform-bin scan of the same size in one graph-replayed batch:
    each gives the bits it gives alone."""
    items, alone = [], []
    for ring in (180.0, 0.0):
        w, geo = _work(48, 1, 1, 0, iters=2, seed=6, ring_mm=ring)
        sc = synth.make_scan(w)
        g = pet.Geometry.from_dict(geo, sc["sens"])
        c, gm = to_dev(sc["counts"], torch.int32), to_dev(sc["gamma"])
        st = pet.State(g, c, gm, pet.make_params(w.params), torch.ones((1, 48, 48), device=DEV))
        for _ in range(w.params.iterations * w.nsubsets):
            st.subiter()
        out = torch.empty((1, 48, 48), device=DEV)
        st.read_image(out)
        torch.cuda.synchronize()
        alone.append(out.cpu().numpy())
        items.append((g, pet.State(g, c, gm, pet.make_params(w.params),
                                   torch.ones((1, 48, 48), device=DEV))))
    assert rel_l2(alone[0], alone[1]) > 1e-3
    stream = torch.cuda.Stream()
    batch = pet.Batch(capacity=2, use_graph=True)
    for g, st in items:
        batch.add(st, with_objective=True, stream=stream)
    while batch.step(stream=stream) > 0:
        pass
    stream.synchronize()
    for (g, st), want in zip(items, alone):
        out = torch.empty((1, 48, 48), device=DEV)
        st.read_image(out)
        torch.cuda.synchronize()
        np.testing.assert_array_equal(out.cpu().numpy(), want)
