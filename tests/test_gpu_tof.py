"""Time of flight on the GPU (pet_geometry_desc.tof_bins = T > 1) against the FP64 oracle.

Bin (v, b) splits into T TOF bins along its line; the system matrix weights each pixel's length
by the Gaussian timing kernel integrated over the TOF bin at the pixel's centre (the TOF data of
the clinical reconstructions, Sec. IV-C).  Checked: the forward projection per projection (one
view of one plane over its bins and TOF bins) and the gather backprojection for every subset in
FP32 and FP64, adjointness, the sensitivity, subiterations (2-D and stacked, BSREM and SDP-P2),
a whole reconstruction with its objective history, and the refusals (batches, the server,
sub-rays with TOF).
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


# (N, P, V, NB, M, rho, T, dtau_mm, fwhm_mm) at 4 mm pixels: odd and even sides, one and two
# plane groups, bins finer than pixels, TOF bins narrower and wider than the kernel
GEOMS = [(48, 1, 30, 69, 4, 1.0, 15, 20.0, 45.0), (33, 11, 21, 47, 3, 1.0, 9, 40.0, 30.0),
         (40, 3, 18, 67, 3, 0.8, 24, 9.0, 60.0)]


@pytest.mark.parametrize("geom", GEOMS)
def test_tof_projectors(geom):
    N, P, V, NB, M, rho, T, dt, fw = geom
    kw = dict(tof_bins=T, tof_bin_mm=dt, tof_fwhm_mm=fw)
    g = pet.Geometry(N, P, 4.0, V, NB, rho * 4.0, M, 0.9, **kw)
    og = oracle.geom(N, P, V, NB, M, pixel_mm=4.0, bin_mm=rho * 4.0, sens=0.9, **kw)
    x = f32(synth.random_image((P, N, N), seed=T, lo=0.1, hi=2.0))
    for i in range(M):
        nv = g.subset_size(i)
        ref = oracle.forward(og, i, x)
        out = torch.empty((P, nv, NB, T), device=DEV)
        pet.forward_subset(g, i, to_dev(x), out)
        out64 = torch.empty((P, nv, NB, T), dtype=torch.float64, device=DEV)
        pet.forward_subset(g, i, to_dev(x, torch.float64), out64)
        torch.cuda.synchronize()
        assert per_projection_rel(out.cpu().numpy(), ref) <= 1e-5, i
        assert per_projection_rel(out64.cpu().numpy(), ref) <= 1e-11, i
        y = f32(synth.random_image((P, nv, NB, T), seed=i + 3, lo=0.0, hi=1.0))
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


def _work(N, P, kind=4, iters=2, seed=4, T=15, dt=20.0, fw=45.0):
    nb = int(1.45 * N) | 1
    return synth.Workload(f"tof{T}", N, P, 4.0, 30, nb, 4.0, 5, 3e5 * P,
                          "ellipsoid3d" if P > 1 else "ellipses2d",
                          synth.AlgoParams(iterations=iters, precond=kind, J0=2, J1=6, a=0.2,
                                           beta=0.5),
                          plane_mm=4.0, seed=seed, tof_bins=T, tof_bin_mm=dt, tof_fwhm_mm=fw)


@pytest.mark.parametrize("N,P,kind", [(48, 1, 4), (48, 1, 0), (40, 11, 4)])
def test_tof_subiterations(N, P, kind):
    """FP32 + Kahan <= 1e-5 and FP64 <= 1e-10 (relL2) against the oracle after 2, 5 and 9
    subiterations (through J0 and the dynamic-nu range)."""
    w = _work(N, P, kind)
    scan = synth.make_scan(w)
    og = oracle.geom_from(w.geometry(), scan["sens"])
    g = pet.Geometry.from_dict(w.geometry(), scan["sens"])
    counts, gamma = to_dev(scan["counts"], torch.int32), to_dev(scan["gamma"])
    for nsub in (2, 5, 9):
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


def test_tof_reconstruction_batch_serve_and_refusals():
    """64^2, 10 iterations of SDP-P2 with 21 TOF bins: image relL2 <= 1e-4 and the objective
    history within 1e-6 of the oracle; in a graph-replayed batch beside a TOF scan of another
    timing resolution, and through the server, it gives its bits alone; TOF with sub-rays is
    refused."""
    import time
    w = synth.Workload("tof64", 64, 1, 4.0, 60, 91, 4.0, 6, 1e6, "ellipses2d",
                       synth.AlgoParams(iterations=10, beta=0.5), seed=9, tof_bins=21,
                       tof_bin_mm=18.0, tof_fwhm_mm=50.0)
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
    # alone, subiteration by subiteration (the bits batches and the server must give)
    w2 = synth.Workload("tof64b", 64, 1, 4.0, 60, 91, 4.0, 6, 1e6, "ellipses2d",
                        synth.AlgoParams(iterations=10, beta=0.5), seed=10, tof_bins=15,
                        tof_bin_mm=25.0, tof_fwhm_mm=70.0)
    scan2 = synth.make_scan(w2)
    runs = [(w, scan), (w2, scan2)]
    alone, states = [], []
    for ww, sc in runs:
        gg = pet.Geometry.from_dict(ww.geometry(), sc["sens"])
        c, gm = to_dev(sc["counts"], torch.int32), to_dev(sc["gamma"])
        st = pet.State(gg, c, gm, pet.make_params(ww.params), torch.ones((1, 64, 64), device=DEV))
        for _ in range(ww.params.iterations * ww.nsubsets):
            st.subiter()
        out = torch.empty((1, 64, 64), device=DEV)
        st.read_image(out)
        torch.cuda.synchronize()
        alone.append(out.cpu().numpy())
        states.append((gg, pet.State(gg, c, gm, pet.make_params(ww.params),
                                     torch.ones((1, 64, 64), device=DEV))))
    stream = torch.cuda.Stream()
    batch = pet.Batch(capacity=2, use_graph=True)
    for gg, st in states:
        batch.add(st, with_objective=True, stream=stream)
    while batch.step(stream=stream) > 0:
        pass
    stream.synchronize()
    for (gg, st), want in zip(states, alone):
        out = torch.empty((1, 64, 64), device=DEV)
        st.read_image(out)
        torch.cuda.synchronize()
        np.testing.assert_array_equal(out.cpu().numpy(), want)
    server = pet.Server(hbm_budget_bytes=1 << 30, max_slots=2)
    tickets = [server.submit(ww.geometry(), sc["sens"], sc["counts"], sc["gamma"],
                             pet.make_params(ww.params)) for ww, sc in runs]
    res = {}
    deadline = time.time() + 120
    while len(res) < 2 and time.time() < deadline:
        for t in tickets:
            if t not in res:
                r = server.poll(t)
                if r is not None:
                    res[t] = r
        time.sleep(0.005)
    server.close()
    for t, want in zip(tickets, alone):
        np.testing.assert_array_equal(res[t][0], want)
    assert np.max(np.abs(np.array(res[tickets[0]][1]) - obj_ref) / np.abs(obj_ref)) <= 1e-6
    with pytest.raises(pet.PetError) as e:
        pet.Geometry(32, 1, 4.0, 20, 47, 4.0, 4, 1.0, subrays=4, tof_bins=9, tof_bin_mm=20.0,
                     tof_fwhm_mm=40.0)
    assert e.value.status == pet.ERR_INVALID


def test_tof_with_attenuation_and_checkpoint():
    """TOF and per-bin detection factors together (the clinical path: attenuation-corrected TOF
    data): the factors of each bin repeated over its TOF bins, subiterations against the oracle;
    a checkpoint of the TOF state resumes to the same bits."""
    w = _work(40, 3, kind=4, iters=2, T=11, dt=30.0, fw=50.0)
    scan = synth.make_scan(w)
    body = [[(0.0, 0.0, 70.0, 55.0, 0.3, 1.0)]] * w.nplanes
    chord = synth.analytic_sinogram(body, w.nviews, w.nbins, w.bin_mm)
    mult = np.repeat(np.exp(-0.0096 * chord)[..., None], w.tof_bins, axis=-1).astype(np.float32)
    og = oracle.geom_from(w.geometry(), scan["sens"])
    g = pet.Geometry.from_dict(w.geometry(), scan["sens"])
    counts, gamma = to_dev(scan["counts"], torch.int32), to_dev(scan["gamma"])
    P, N = w.nplanes, w.n
    for nsub in (3, 7):
        ref, _ = oracle.reconstruct(og, scan["counts"], scan["gamma"], w.params,
                                    np.ones((P, N, N)), nsub=nsub, mult=mult)
        for prec, tol in ((synth.PREC_FP32_KAHAN, 1e-5), (synth.PREC_FP64, 1e-10)):
            st = pet.State(g, counts, gamma, pet.make_params(w.params, prec),
                           torch.ones((P, N, N), device=DEV), d_mult=to_dev(mult))
            for _ in range(nsub):
                st.subiter()
            out = torch.empty((P, N, N), dtype=torch.float64, device=DEV)
            st.read_image(out)
            torch.cuda.synchronize()
            assert rel_l2(out.cpu().numpy(), ref) <= tol, (nsub, prec, rel_l2(out.cpu().numpy(), ref))
            st.close()
    # checkpoint / resume
    prm = pet.make_params(w.params)
    total = w.params.iterations * w.nsubsets
    a = pet.State(g, counts, gamma, prm, torch.ones((P, N, N), device=DEV), d_mult=to_dev(mult))
    for _ in range(total):
        a.subiter()
    want = torch.empty((P, N, N), device=DEV)
    a.read_image(want)
    b = pet.State(g, counts, gamma, prm, torch.ones((P, N, N), device=DEV), d_mult=to_dev(mult))
    for _ in range(4):
        b.subiter()
    blob = b.export()
    c = pet.State(g, counts, gamma, prm, torch.ones((P, N, N), device=DEV), d_mult=to_dev(mult))
    c.load(blob)
    for _ in range(total - 4):
        c.subiter()
    got = torch.empty((P, N, N), device=DEV)
    c.read_image(got)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(got.cpu().numpy(), want.cpu().numpy())
