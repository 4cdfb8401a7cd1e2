"""The objective from the entry point that allocates nothing (pet_objective_static) matches
pet_objective and the FP64 oracle, on two calls in a row through the C ABI.

pet_objective_static exists for callers that may not allocate device memory when they need
the objective (a pipeline whose device memory belongs to a fixed pool, a real-time loop that
must not stall on an allocation); its reduction scratch is a static array in the library's
device memory, shared by every call.  On a freshly created geometry the static entry point is
called before anything else touches it: after a first call (which looks up the array's device
address), a second call must leave the device's free memory unchanged.  The second call also
checks that what the first call left in the shared array does not leak into its result.  This
file is collected last so that a run stopping at the first failure has run every other test.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2111_07886_gb300 import pet, synth

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda:0")
TOL = 1e-6          # objective parts and Phi, relative (the objective parity tolerance)


def _close(a, b, what):
    assert abs(a - b) <= TOL * abs(b), (what, a, b)


@pytest.mark.parametrize("make", [lambda: synth.config_2d_128(seed=5),
                                  lambda: synth.Workload("stacked_small", 64, 11, 4.0, 48, 91, 4.0, 6,
                                                         2e6, "ellipsoid3d", synth.AlgoParams(),
                                                         plane_mm=4.0, seed=5)])
def test_static_objective_matches_objective_twice(make):
    w = make()
    scan = synth.make_scan(w)
    g = pet.Geometry.from_dict(w.geometry(), scan["sens"])
    og = oracle.geom_from(w.geometry(), scan["sens"])
    counts = torch.from_numpy(scan["counts"]).to(DEV)
    gamma = torch.from_numpy(scan["gamma"]).to(DEV)
    rng = np.random.Generator(np.random.PCG64(11))
    imgs = [rng.uniform(0.5, 2.0, (w.nplanes, w.n, w.n)).astype(np.float32) for _ in range(2)]
    d_imgs = [torch.from_numpy(x).to(DEV) for x in imgs]
    torch.cuda.synchronize()
    # the static entry point first, on the fresh geometry: nothing else has allocated for it
    static = [pet.objective_static(g, counts, gamma, d_imgs[0], w.params.beta, 2.0, 1e-12)]
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info(DEV)[0]
    static.append(pet.objective_static(g, counts, gamma, d_imgs[1], w.params.beta, 2.0, 1e-12))
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info(DEV)[0] == free0, "pet_objective_static changed free device memory"
    for call, (x, d_x) in enumerate(zip(imgs, d_imgs)):
        phi_s, parts_s = static[call]
        phi, parts = pet.objective(g, counts, gamma, d_x, w.params.beta, 2.0, 1e-12)
        for a, b in zip(parts_s, parts):
            _close(a, b, ("vs pet_objective", call))
        _close(phi_s, phi, ("phi vs pet_objective", call))
        ref = oracle.objective(og, scan["counts"], scan["gamma"], x.astype(np.float64),
                               w.params.beta)
        for a, k in zip(parts_s, ("sum_af", "sum_glog", "rdp")):
            _close(a, ref[k], ("vs oracle", call, k))
        _close(phi_s, ref["phi"], ("phi vs oracle", call))
