"""The fully 3-D prior on the GPU (pet_params.rdp_3d = 1) against the FP64 oracle.

RDP over the 26 neighbours of each voxel of the volume (Eqs. RDP and gradRD) and nu from the
volume's gradient (Sec. III), as for the paper's fully 3-D reconstructions (Sec. IV-C): single
steps, subiterations in each arithmetic, a whole reconstruction with its objective history, and a
3-D scan batched beside an in-plane one (bitwise equal alone).  Volumes with 11 and 20 planes
give plane groups whose neighbours sit in the next group and pad planes above the last one.
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


@pytest.mark.parametrize("P", [11, 20])
def test_rdp3d_gradient_nu_objective(P):
    N = 40
    g = pet.Geometry(N, P, 2.0, 30, 59, 2.0, 5, 0.9)
    og = oracle.geom(N, P, 30, 59, 5, pixel_mm=2.0, bin_mm=2.0, sens=0.9)
    x = f32(synth.random_image((P, N, N), seed=P, lo=0.2, hi=3.0))
    out = torch.empty((P, N, N), device=DEV)
    pet.rdp_gradient(g, to_dev(x), 2.0, 1e-12, out, three_d=True)
    torch.cuda.synchronize()
    ref = oracle.rdp_grad(x, 2.0, 1e-12, three_d=True)
    err = np.abs(out.cpu().numpy() - ref).max()
    assert err <= 1e-5 * np.abs(ref).max(), (err, np.abs(ref).max())
    # a volume with an edge across the planes and one across the columns: nu clamps active
    img = np.ones((P, N, N))
    img[:, :, 20:] += 1.5
    img[P // 2:] += 1.0
    img = f32(img + 0.05 * synth.random_image((P, N, N), seed=P + 1, lo=0.0, hi=1.0))
    pet.smoothness_nu(g, to_dev(img), 0.8, 2.2, out, three_d=True)
    torch.cuda.synchronize()
    ref = oracle.nu_from_image(img, 0.8, 2.2, three_d=True)
    err = np.abs(out.cpu().numpy() - ref)
    assert err.max() <= 1e-5, (err.max(), np.unravel_index(err.argmax(), err.shape))
    assert np.abs(ref - oracle.nu_from_image(img, 0.8, 2.2)).max() > 1e-2   # gz matters here
    w = synth.Workload("t", N, P, 2.0, 30, 59, 2.0, 5, 3e5 * P, "ellipsoid3d", synth.AlgoParams(),
                       plane_mm=2.0, seed=P)
    scan = synth.make_scan(w)
    g2 = pet.Geometry.from_dict(w.geometry(), scan["sens"])
    og2 = oracle.geom_from(w.geometry(), scan["sens"])
    phi, parts = pet.objective(g2, to_dev(scan["counts"], torch.int32), to_dev(scan["gamma"]),
                               to_dev(x), 0.05, 2.0, 1e-12, three_d=True)
    o = oracle.objective(og2, scan["counts"], scan["gamma"], x, 0.05, three_d=True)
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


@pytest.mark.parametrize("kind", [0, 3, 4])
def test_rdp3d_subiterations(kind):
    """BSREM, SDP-P1, SDP-P2 with the 3-D prior: through J0, the dynamic-nu range and the freeze
    at J1; FP32 + Kahan <= 1e-5, FP32 <= 1e-5, FP64 <= 1e-10 against the oracle."""
    w = synth.Workload("t", 33, 20, 8.0, 30, 47, 8.0, 5, 4e6, "ellipsoid3d",
                       synth.AlgoParams(iterations=2, precond=kind, J0=2, J1=6, a=0.2, beta=0.3,
                                        rdp3d=1),
                       plane_mm=8.0, seed=kind + 40)
    scan = synth.make_scan(w)
    og = oracle.geom_from(w.geometry(), scan["sens"])
    for nsub in (2, 5, 9):
        ref, _ = oracle.reconstruct(og, scan["counts"], scan["gamma"], w.params,
                                    np.ones((20, 33, 33)), nsub=nsub)
        ref2d, _ = oracle.reconstruct(og, scan["counts"], scan["gamma"],
                                      synth.AlgoParams(**{**w.params.__dict__, "rdp3d": 0}),
                                      np.ones((20, 33, 33)), nsub=nsub)
        assert rel_l2(ref2d, ref) > 1e-4                    # the 3-D prior changes the iterates
        for prec, tol in ((synth.PREC_FP32_KAHAN, 1e-5), (synth.PREC_FP32, 1e-5), (synth.PREC_FP64, 1e-10)):
            got = _run(w, scan, nsub, prec)
            assert rel_l2(got, ref) <= tol, (kind, nsub, prec, rel_l2(got, ref))


def test_rdp3d_reconstruction_and_batch():
    """A 64^2 x 24 volume, 8 iterations of SDP-P2 with the 3-D prior: image relL2 <= 1e-4 and
    the objective history within 1e-6 of the oracle; in a graph-replayed batch beside the same
    scan with the in-plane prior, each gives the same bits as alone."""
    w = synth.Workload("vol", 64, 24, 4.0, 72, 91, 4.0, 6, 2e7, "ellipsoid3d",
                       synth.AlgoParams(iterations=8, beta=0.3, rdp3d=1), plane_mm=4.0, seed=77)
    scan = synth.make_scan(w)
    og = oracle.geom_from(w.geometry(), scan["sens"])
    ref, obj_ref = oracle.reconstruct(og, scan["counts"], scan["gamma"], w.params,
                                      np.ones((24, 64, 64)), with_objective=True)
    g = pet.Geometry.from_dict(w.geometry(), scan["sens"])
    counts, gamma = to_dev(scan["counts"], torch.int32), to_dev(scan["gamma"])
    img = torch.ones((24, 64, 64), device=DEV)
    obj = pet.reconstruct(g, counts, gamma, pet.make_params(w.params), img, objective=True)
    got = img.cpu().double().numpy()
    assert rel_l2(got, ref) <= 1e-4, rel_l2(got, ref)
    gap = np.max(np.abs(np.array(obj) - obj_ref) / np.abs(obj_ref))
    assert gap <= 1e-6, gap
    # batched beside the in-plane twin
    w2 = synth.Workload("vol2d", 64, 24, 4.0, 72, 91, 4.0, 6, 2e7, "ellipsoid3d",
                        synth.AlgoParams(iterations=8, beta=0.3, rdp3d=0), plane_mm=4.0, seed=77)
    f0 = torch.ones((24, 64, 64), device=DEV)
    alone = []
    for ww in (w, w2):
        st = pet.State(g, counts, gamma, pet.make_params(ww.params), f0)
        for _ in range(ww.params.iterations * ww.nsubsets):
            st.subiter()
        out = torch.empty_like(f0)
        st.read_image(out)
        torch.cuda.synchronize()
        alone.append(out.cpu().numpy())
        st.close()
    assert rel_l2(alone[0], alone[1]) > 1e-4
    np.testing.assert_array_equal(alone[0], got.astype(np.float32))
    stream = torch.cuda.Stream()
    batch = pet.Batch(capacity=2, use_graph=True)
    states = [pet.State(g, counts, gamma, pet.make_params(ww.params), f0) for ww in (w, w2)]
    for st in states:
        batch.add(st, with_objective=True, stream=stream)
    while batch.step(stream=stream) > 0:
        pass
    stream.synchronize()
    for st, ref_img in zip(states, alone):
        out = torch.empty_like(f0)
        st.read_image(out)
        torch.cuda.synchronize()
        np.testing.assert_array_equal(out.cpu().numpy(), ref_img)
    assert states[0].objective_history() == obj
