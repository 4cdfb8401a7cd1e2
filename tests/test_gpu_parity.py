"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle on seeded inputs.

Tolerances (stated by the target): per projection relative error <= 1e-5 (FP32 + Kahan),
image relative L2 <= 1e-4 after the configured iterations; the FP64 GPU path is held to
1e-10.  A "projection" is one view of one plane: max_b |y - y_ref| / max_b |y_ref|.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2111_07886_gb300 import pet, synth

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda:0")

# (N, P, V, NB, M, rho): several tiles, ragged subsets (V % M != 0), ragged plane groups
GEOMS = [
    (64, 1, 40, 91, 6, 1.0),
    (33, 1, 25, 47, 4, 1.0),      # odd N, even/odd mix
    (48, 11, 30, 69, 7, 1.0),     # two plane groups, 5 pad planes
    (40, 3, 18, 80, 3, 0.75),     # even NB, bins finer than pixels
    (24, 9, 16, 71, 2, 0.6),      # three candidate bins per view in the gather
    (5, 2, 7, 9, 3, 1.3),         # tiny image, coarse bins
]


def _geoms(N, P, V, NB, M, rho, pixel_mm=2.0, sens=0.9):
    g = pet.Geometry(N, P, pixel_mm, V, NB, rho * pixel_mm, M, sens)
    og = oracle.geom(N, P, V, NB, M, pixel_mm=pixel_mm, bin_mm=rho * pixel_mm, sens=sens)
    return g, og


def per_projection_rel(got, ref):
    got, ref = np.asarray(got, np.float64), np.asarray(ref, np.float64)
    den = np.abs(ref).max(axis=-1)
    num = np.abs(got - ref).max(axis=-1)
    ok = den > 0
    assert np.all(num[~ok] == 0)
    return float((num[ok] / den[ok]).max()) if ok.any() else 0.0


def rel_l2(got, ref):
    return float(np.linalg.norm(np.asarray(got, np.float64) - ref) / np.linalg.norm(ref))


def to_dev(a, dtype=torch.float32):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV, dtype)


def f32(a):
    """The float32 rounding of `a`, in float64: the exact input an FP32 kernel sees, so that
    both sides of a parity check get identical values."""
    return np.asarray(a, np.float32).astype(np.float64)


@pytest.mark.parametrize("geom", GEOMS)
def test_forward_parity(geom):
    g, og = _geoms(*geom)
    N, P, V, NB, M, _ = geom
    x = f32(synth.random_image((P, N, N), seed=N + P))
    xd = to_dev(x)
    for i in list(range(M)) + [-1]:
        nv = V if i < 0 else og and oracle.subset_size(og, i)
        ref = oracle.forward(og, i, x)
        out = torch.empty((P, nv, NB), dtype=torch.float32, device=DEV)
        pet.forward_subset(g, i, xd, out)
        torch.cuda.synchronize()
        assert per_projection_rel(out.cpu().numpy(), ref) <= 1e-5, (geom, i)
        out64 = torch.empty((P, nv, NB), dtype=torch.float64, device=DEV)
        pet.forward_subset(g, i, to_dev(x, torch.float64), out64)
        torch.cuda.synchronize()
        assert per_projection_rel(out64.cpu().numpy(), ref) <= 1e-10, (geom, i)


def test_set_ray_chunks():
    """Pinned ray chunks: invalid counts are rejected; every admissible count (and 0, the
    heuristic) gives the same projection within the parity bound."""
    g, og = _geoms(48, 11, 30, 69, 7, 1.0)            # 2 plane groups: S must divide 128
    for bad in (3, 9, 17, 32, -1):
        with pytest.raises(pet.PetError) as e:
            g.set_ray_chunks(bad)
        assert e.value.status == pet.ERR_INVALID
    x = f32(synth.random_image((11, 48, 48), seed=21))
    ref = oracle.forward(og, 2, x)
    for S in (1, 2, 8, 16, 0):
        g.set_ray_chunks(S)
        out = torch.empty(ref.shape, device=DEV)
        pet.forward_subset(g, 2, to_dev(x), out)
        torch.cuda.synchronize()
        assert per_projection_rel(out.cpu().numpy(), ref) <= 1e-5, S


@pytest.mark.parametrize("geom", GEOMS)
def test_back_parity(geom):
    g, og = _geoms(*geom)
    N, P, V, NB, M, _ = geom
    for i in list(range(M)) + [-1]:
        nv = V if i < 0 else oracle.subset_size(og, i)
        y = f32(synth.random_image((P, nv, NB), seed=7 * i + 100 + N))
        ref = oracle.back(og, i, y)
        out = torch.empty((P, N, N), dtype=torch.float32, device=DEV)
        pet.back_subset(g, i, to_dev(y), out)
        out64 = torch.empty((P, N, N), dtype=torch.float64, device=DEV)
        pet.back_subset(g, i, to_dev(y, torch.float64), out64)
        torch.cuda.synchronize()
        got, got64 = out.cpu().numpy(), out64.cpu().numpy()
        for p in range(P):
            scale = np.abs(ref[p]).max()
            assert np.abs(got[p] - ref[p]).max() <= 1e-5 * scale, (geom, i, p)
            assert np.abs(got64[p] - ref[p]).max() <= 1e-10 * scale, (geom, i, p)


def test_adjointness_gpu():
    g, og = _geoms(64, 11, 40, 91, 6, 1.0)
    x = f32(synth.random_image((11, 64, 64), seed=1))
    for i in range(6):
        nv = oracle.subset_size(og, i)
        y = f32(synth.random_image((11, nv, 91), seed=2 + i))
        ax = torch.empty((11, nv, 91), device=DEV)
        aty = torch.empty((11, 64, 64), device=DEV)
        pet.forward_subset(g, i, to_dev(x), ax)
        pet.back_subset(g, i, to_dev(y), aty)
        lhs = float(np.vdot(ax.cpu().double().numpy(), y))
        rhs = float(np.vdot(x, aty.cpu().double().numpy()))
        assert abs(lhs - rhs) <= 2e-6 * abs(lhs)


def test_axis_rays_on_pixel_edges():
    """Views at 0 and pi/2 put every ray of an even image / odd bin count on a grid line; the
    half-open rule gives each edge ray to the + side pixel only (dense clipping matrix)."""
    from test_oracle_pins import dense_A
    N, V, NB = 8, 4, 11
    g, og = _geoms(N, 1, V, NB, 1, 1.0, pixel_mm=1.0, sens=1.0)
    A = dense_A(N, V, NB)
    eye = np.eye(N * N).reshape(N * N, 1, N, N)
    cols = np.zeros((V * NB, N * N))
    out = torch.empty((1, V, NB), device=DEV)
    for j in range(N * N):
        pet.forward_subset(g, -1, to_dev(eye[j]), out)
        torch.cuda.synchronize()
        cols[:, j] = out.cpu().numpy().ravel()
    np.testing.assert_allclose(cols, A, rtol=0, atol=2e-7)


def test_sensitivity_parity():
    for geom in GEOMS[:4]:
        g, og = _geoms(*geom)
        p = torch.empty((geom[0], geom[0]), device=DEV)
        pet.sensitivity(g, p)
        torch.cuda.synchronize()
        ref = oracle.sensitivity(og)
        np.testing.assert_allclose(p.cpu().numpy(), ref, rtol=1e-6)


def test_rdp_gradient_and_nu_parity():
    g, og = _geoms(48, 11, 30, 69, 7, 1.0)
    x = f32(synth.random_image((11, 48, 48), seed=5, lo=0.2, hi=3.0))
    out = torch.empty((11, 48, 48), device=DEV)
    pet.rdp_gradient(g, to_dev(x), 2.0, 1e-12, out)
    torch.cuda.synchronize()
    ref = oracle.rdp_grad(x, 2.0, 1e-12)
    err = np.abs(out.cpu().numpy() - ref).max()
    assert err <= 1e-5 * np.abs(ref).max(), (err, np.abs(ref).max())
    # smooth image with an edge so that the clamp of nu is partly active
    img = np.ones((11, 48, 48))
    img[:, :, 20:] = 2.5
    img = f32(img + 0.05 * synth.random_image((11, 48, 48), seed=6, lo=0.0, hi=1.0))
    pet.smoothness_nu(g, to_dev(img), 0.8, 2.2, out)
    torch.cuda.synchronize()
    ref = oracle.nu_from_image(img, 0.8, 2.2)
    err = np.abs(out.cpu().numpy() - ref)
    assert err.max() <= 1e-5, (err.max(), np.unravel_index(err.argmax(), err.shape),
                               out.cpu().numpy().ravel()[err.argmax()], ref.ravel()[err.argmax()])


def test_nu_map_with_subnormal_gradients():
    """A background of ~1e-21 (what the iterates decay to outside the object after a few
    iterations) has squared gradients below the smallest normal float.  mu must stay
    max(0.01, |grad f| / mean f) = 0.01 there: a reciprocal square root that flushes them to zero
    turned |grad f| into inf, the sum of mu into inf and nu into nu2 everywhere."""
    g = pet.Geometry(48, 11, 2.0, 30, 69, 2.0, 5, 0.9)
    bg = 3e-21 * (1.0 + 0.5 * synth.random_image((11, 48, 48), seed=8, lo=0.0, hi=1.0))
    img = bg.copy()
    img[:, 12:36, 12:36] = 1.0 + synth.random_image((11, 24, 24), seed=9, lo=0.0, hi=1.5)
    img = f32(img)
    out = torch.empty((11, 48, 48), device=DEV)
    pet.smoothness_nu(g, to_dev(img), 0.8, 2.2, out)
    torch.cuda.synchronize()
    ref = oracle.nu_from_image(img, 0.8, 2.2)
    got = out.cpu().numpy()
    assert np.all(np.isfinite(got))
    err = np.abs(got - ref)
    assert err.max() <= 1e-5, (err.max(), np.unravel_index(err.argmax(), err.shape))


def test_objective_parity():
    w = synth.config_2d_128(seed=4)
    scan = synth.make_scan(w)
    g = pet.Geometry.from_dict(w.geometry(), scan["sens"])
    og = oracle.geom_from(w.geometry(), scan["sens"])
    x = f32(synth.random_image((1, w.n, w.n), seed=9, lo=0.5, hi=2.0))
    phi, parts = pet.objective(g, to_dev(scan["counts"], torch.int32), to_dev(scan["gamma"]),
                               to_dev(x), w.params.beta, 2.0, 1e-12)
    ref = oracle.objective(og, scan["counts"], scan["gamma"], x, w.params.beta)
    assert abs(parts[0] - ref["sum_af"]) <= 1e-6 * abs(ref["sum_af"])
    assert abs(parts[1] - ref["sum_glog"]) <= 1e-6 * abs(ref["sum_glog"])
    assert abs(parts[2] - ref["rdp"]) <= 1e-6 * abs(ref["rdp"])
    assert abs(phi - ref["phi"]) <= 1e-6 * abs(ref["phi"])


def _run_subiters(w, scan, nsub, precision):
    g = pet.Geometry.from_dict(w.geometry(), scan["sens"])
    prm = pet.make_params(w.params, precision)
    counts = to_dev(scan["counts"], torch.int32)
    gamma = to_dev(scan["gamma"])
    f0 = torch.ones((w.nplanes, w.n, w.n), device=DEV)
    st = pet.State(g, counts, gamma, prm, f0)
    for _ in range(nsub):
        st.subiter()
    out = torch.empty(f0.shape, dtype=torch.float64, device=DEV)
    st.read_image(out)
    torch.cuda.synchronize()
    return out.cpu().numpy()


@pytest.mark.parametrize("kind", [0, 1, 2, 3, 4])
def test_subiteration_parity_each_preconditioner(kind):
    """A few subiterations (through J0 into the dynamic-nu range) for BSREM, M1, M2, P1, P2."""
    w = synth.Workload("t", 48, 3, 8.0, 36, 69, 8.0, 4, 3e5, "ellipsoid3d",
                       synth.AlgoParams(iterations=2, precond=kind, J0=2, J1=5, a=0.2),
                       plane_mm=8.0, seed=2)
    scan = synth.make_scan(w)
    og = oracle.geom_from(w.geometry(), scan["sens"])
    for nsub in (1, 3, 8):
        ref, _ = oracle.reconstruct(og, scan["counts"], scan["gamma"], w.params,
                                    np.ones((3, 48, 48)), nsub=nsub)
        got = _run_subiters(w, scan, nsub, synth.PREC_FP32_KAHAN)
        assert rel_l2(got, ref) <= 1e-5, (kind, nsub, rel_l2(got, ref))
        got64 = _run_subiters(w, scan, nsub, synth.PREC_FP64)
        assert rel_l2(got64, ref) <= 1e-10, (kind, nsub, rel_l2(got64, ref))


@pytest.mark.parametrize("P", [5, 11, 20, 33])
def test_update_tiles_and_plane_chunks(P):
    """The 8-plane update kernel with 1, 2, 3 and 5 plane groups (pixel tiles of 256 / groups
    pixels, so tiles that straddle image rows and end raggedly; 33 planes leave 7 pad planes) on
    an odd image side: subiterations through J0, the dynamic-nu range, the freeze at J1 and
    beyond, against the oracle."""
    w = synth.Workload("t", 37, P, 8.0, 30, 53, 8.0, 5, 2e5 * P, "ellipsoid3d",
                       synth.AlgoParams(iterations=2, J0=2, J1=6, a=0.2), plane_mm=8.0, seed=P)
    scan = synth.make_scan(w)
    og = oracle.geom_from(w.geometry(), scan["sens"])
    for nsub in (3, 9):
        ref, _ = oracle.reconstruct(og, scan["counts"], scan["gamma"], w.params,
                                    np.ones((P, 37, 37)), nsub=nsub)
        got = _run_subiters(w, scan, nsub, synth.PREC_FP32_KAHAN)
        assert rel_l2(got, ref) <= 1e-5, (P, nsub, rel_l2(got, ref))
        got32 = _run_subiters(w, scan, nsub, synth.PREC_FP32)
        assert rel_l2(got32, ref) <= 1e-5, (P, nsub, rel_l2(got32, ref))


def test_upper_branch_and_clamp():
    """Small U: the (U - f)/p branch and the U - t clamp are active on both sides."""
    w = synth.Workload("t", 32, 1, 8.0, 24, 45, 8.0, 3, 3e5, "ellipses2d",
                       synth.AlgoParams(iterations=2, U=2.0, precond=4, J0=1), seed=8)
    scan = synth.make_scan(w)
    og = oracle.geom_from(w.geometry(), scan["sens"])
    ref, _ = oracle.reconstruct(og, scan["counts"], scan["gamma"], w.params, np.ones((1, 32, 32)))
    got = _run_subiters(w, scan, 6, synth.PREC_FP32_KAHAN)
    assert (ref > 1.0).any() and ref.max() < 2.0
    assert rel_l2(got, ref) <= 1e-5
    assert got.min() > 0 and got.max() < 2.0


def test_reconstruct_2d_128_full():
    """The 2-D workload (128^2, 180 x 185, 12 subsets, 10 iterations, SDP-P2(12)): image relL2
    <= 1e-4 and objective history within 1e-6 of the oracle, FP32 + Kahan; FP64 path 1e-9."""
    w = synth.config_2d_128(seed=0)
    scan = synth.make_scan(w)
    og = oracle.geom_from(w.geometry(), scan["sens"])
    ref, obj_ref = oracle.reconstruct(og, scan["counts"], scan["gamma"], w.params,
                                      np.ones((1, 128, 128)), with_objective=True)
    g = pet.Geometry.from_dict(w.geometry(), scan["sens"])
    counts = to_dev(scan["counts"], torch.int32)
    counts_before = counts.clone()
    for prec, tol in ((synth.PREC_FP32_KAHAN, 1e-4), (synth.PREC_FP32, 1e-4)):
        img = torch.ones((1, 128, 128), device=DEV)
        obj = pet.reconstruct(g, counts, to_dev(scan["gamma"]), pet.make_params(w.params, prec),
                              img, objective=True)
        got = img.cpu().double().numpy()
        assert rel_l2(got, ref) <= tol, (prec, rel_l2(got, ref))
        gap = np.max(np.abs(np.array(obj) - obj_ref) / np.abs(obj_ref))
        assert gap <= 1e-6, (prec, gap)
        assert got.min() > 0
    got64 = _run_subiters(w, scan, w.params.iterations * w.nsubsets, synth.PREC_FP64)
    assert rel_l2(got64, ref) <= 1e-9, rel_l2(got64, ref)
    assert torch.equal(counts, counts_before)          # counts are read-only, exact int32
    assert np.all(np.diff(obj_ref) < 0)


@pytest.mark.slow
def test_reconstruct_stacked_full_size():
    """Full clinical-size stacked workload (256^2 x 89, 288 x 357, 24 subsets, 20 iterations,
    SDP-P2(24)), the launch configuration the benchmark times: image relL2 <= 1e-4 and the
    objective history against the FP64 oracle."""
    w = synth.config_stacked_256x89(seed=0)
    scan = synth.make_scan(w)
    og = oracle.geom_from(w.geometry(), scan["sens"])
    ref, obj_ref = oracle.reconstruct(og, scan["counts"], scan["gamma"], w.params,
                                      np.ones((89, 256, 256)), with_objective=True)
    g = pet.Geometry.from_dict(w.geometry(), scan["sens"])
    img = torch.ones((89, 256, 256), device=DEV)
    obj = pet.reconstruct(g, to_dev(scan["counts"], torch.int32), to_dev(scan["gamma"]),
                          pet.make_params(w.params), img, objective=True)
    got = img.cpu().double().numpy()
    assert rel_l2(got, ref) <= 1e-4, rel_l2(got, ref)
    gap = np.max(np.abs(np.array(obj) - obj_ref) / np.abs(obj_ref))
    assert gap <= 1e-6, gap


def test_stacked_full_size_single_steps():
    """At the full stacked size: one subset projection and backprojection per projection
    <= 1e-5, and the first three subiterations relL2 <= 1e-5."""
    w = synth.config_stacked_256x89(seed=1)
    scan = synth.make_scan(w)
    og = oracle.geom_from(w.geometry(), scan["sens"])
    g = pet.Geometry.from_dict(w.geometry(), scan["sens"])
    x = f32(synth.random_image((89, 256, 256), seed=3))
    ref = oracle.forward(og, 5, x)
    out = torch.empty(ref.shape, device=DEV)
    pet.forward_subset(g, 5, to_dev(x), out)
    torch.cuda.synchronize()
    assert per_projection_rel(out.cpu().numpy(), ref) <= 1e-5
    bout = torch.empty((89, 256, 256), device=DEV)
    ref = f32(ref)
    bref = oracle.back(og, 5, ref)
    pet.back_subset(g, 5, to_dev(ref), bout)
    torch.cuda.synchronize()
    got = bout.cpu().numpy()
    assert np.abs(got - bref).max() <= 1e-5 * np.abs(bref).max()
    ref3, _ = oracle.reconstruct(og, scan["counts"], scan["gamma"], w.params,
                                 np.ones((89, 256, 256)), nsub=3)
    got3 = _run_subiters(w, scan, 3, synth.PREC_FP32_KAHAN)
    assert rel_l2(got3, ref3) <= 1e-5


def test_invalid_inputs_rejected():
    g, og = _geoms(16, 1, 8, 23, 2, 1.0)
    x = torch.ones((1, 16, 16), device=DEV)
    out = torch.empty((1, 4, 23), device=DEV)
    with pytest.raises(pet.PetError) as e:
        pet.forward_subset(g, 2, x, out)
    assert e.value.status == pet.ERR_INVALID
    counts = torch.zeros((1, 8, 23), dtype=torch.int32, device=DEV)
    gamma = torch.ones((1, 8, 23), device=DEV)
    gamma[0, 3, 4] = 0.0
    prm = pet.make_params(synth.AlgoParams(iterations=1))
    with pytest.raises(pet.PetError) as e:
        pet.State(g, counts, gamma, prm, x)
    assert e.value.status == pet.ERR_INVALID
    gamma[0, 3, 4] = 1.0
    counts[0, 1, 1] = -1
    with pytest.raises(pet.PetError):
        pet.reconstruct(g, counts, gamma, prm, x)
    bad = pet.make_params(synth.AlgoParams(iterations=1, t=2000.0))
    counts[0, 1, 1] = 0
    with pytest.raises(pet.PetError):
        pet.State(g, counts, gamma, bad, x)


def test_host_entry_matches_device_entry():
    w = synth.Workload("t", 40, 2, 8.0, 30, 57, 8.0, 5, 2e5, "ellipsoid3d",
                       synth.AlgoParams(iterations=2), plane_mm=8.0, seed=6)
    scan = synth.make_scan(w)
    g = pet.Geometry.from_dict(w.geometry(), scan["sens"])
    prm = pet.make_params(w.params)
    img = torch.ones((2, 40, 40), device=DEV)
    obj_d = pet.reconstruct(g, to_dev(scan["counts"], torch.int32), to_dev(scan["gamma"]), prm,
                            img, objective=True)
    h = np.ones((2, 40, 40), np.float32)
    obj_h = pet.reconstruct_host(g, scan["counts"], scan["gamma"], prm, h, objective=True)
    np.testing.assert_array_equal(h, img.cpu().numpy())
    assert obj_h == obj_d


def test_deterministic_repeat():
    """Same inputs, same bits: the gather and the reductions have a fixed order."""
    w = synth.config_2d_128(seed=2)
    w.params.iterations = 3
    scan = synth.make_scan(w)
    g = pet.Geometry.from_dict(w.geometry(), scan["sens"])
    outs = []
    for _ in range(2):
        img = torch.ones((1, 128, 128), device=DEV)
        obj = pet.reconstruct(g, to_dev(scan["counts"], torch.int32), to_dev(scan["gamma"]),
                              pet.make_params(w.params), img, objective=True)
        outs.append((img.cpu().numpy(), obj))
    np.testing.assert_array_equal(outs[0][0], outs[1][0])
    assert outs[0][1] == outs[1][1]
