"""Checkpoint / resume of a reconstruction state (GPU): a run interrupted after any subiteration
and resumed in a fresh state from pet_state_export's blob gives the bits of the uninterrupted
run (image and objective history), with the frozen nu (past J1) and the TV dual variable carried
over; a checkpoint of another geometry is refused."""
import numpy as np
import pytest
import torch

from paper_2111_07886_gb300 import pet, synth

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda:0")


def _image(st, w):
    out = torch.empty((w.nplanes, w.n, w.n), device=DEV)
    st.read_image(out)
    torch.cuda.synchronize()
    return out.cpu().numpy()


@pytest.mark.parametrize("reg,cut", [(0, 7), (0, 3), (1, 5)])
def test_resume_is_bitwise_the_uninterrupted_run(reg, cut):
    w = synth.Workload("ck", 40, 11, 8.0, 30, 59, 8.0, 5, 2e6, "ellipsoid3d",
                       synth.AlgoParams(iterations=4, J0=2, J1=6, beta=(20.0 if reg else 0.05),
                                        reg=reg, tv_iters=8), plane_mm=8.0, seed=12)
    scan = synth.make_scan(w)
    g = pet.Geometry.from_dict(w.geometry(), scan["sens"])
    counts = torch.from_numpy(scan["counts"]).to(DEV)
    gamma = torch.from_numpy(scan["gamma"]).to(DEV)
    f0 = torch.ones((w.nplanes, w.n, w.n), device=DEV)
    prm = pet.make_params(w.params)
    total = w.params.iterations * w.nsubsets
    a = pet.State(g, counts, gamma, prm, f0)
    for _ in range(total):
        a.subiter()
    want = _image(a, w)
    b = pet.State(g, counts, gamma, prm, f0)
    for _ in range(cut):
        b.subiter()
    blob = b.export()
    b.close()
    c = pet.State(g, counts, gamma, prm, f0)          # a fresh state at (0, 1)
    c.load(blob)
    assert c.subiters == cut
    for _ in range(total - cut):
        c.subiter()
    np.testing.assert_array_equal(_image(c, w), want)
    # a checkpoint of another geometry is refused
    w2 = synth.Workload("ck2", 32, 11, 8.0, 30, 59, 8.0, 5, 2e6, "ellipsoid3d", w.params,
                        plane_mm=8.0, seed=12)
    s2 = synth.make_scan(w2)
    g2 = pet.Geometry.from_dict(w2.geometry(), s2["sens"])
    d = pet.State(g2, torch.from_numpy(s2["counts"]).to(DEV), torch.from_numpy(s2["gamma"]).to(DEV),
                  prm, torch.ones((11, 32, 32), device=DEV))
    with pytest.raises(pet.PetError) as e:
        d.load(blob)
    assert e.value.status == pet.ERR_INVALID
