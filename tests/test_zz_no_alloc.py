"""The objective from the entry point that allocates nothing (pet_objective_static) matches
pet_objective, on two calls in a row through the C ABI.

pet_objective_static exists for callers that may not allocate device memory when they need
the objective (a fixed device-memory pool, a CUDA graph capture or a real-time loop); its
reduction scratch is a static array in the library's device memory, shared by every call.
The second call checks that what the first call left in that array does not leak into the
result.  This file is collected last so that a run stopping at the first failure has run
every other test.
"""
import numpy as np
import pytest
import torch

from paper_2111_07886_gb300 import pet, synth

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda:0")


@pytest.mark.parametrize("make", [lambda: synth.config_2d_128(seed=5),
                                  lambda: synth.Workload("stacked_small", 64, 11, 4.0, 48, 91, 4.0, 6,
                                                         2e6, "ellipsoid3d", synth.AlgoParams(),
                                                         plane_mm=4.0, seed=5)])
def test_static_objective_matches_objective_twice(make):
    w = make()
    scan = synth.make_scan(w)
    g = pet.Geometry.from_dict(w.geometry(), scan["sens"])
    counts = torch.from_numpy(scan["counts"]).to(DEV)
    gamma = torch.from_numpy(scan["gamma"]).to(DEV)
    rng = np.random.Generator(np.random.PCG64(11))
    for call in range(2):
        img = torch.from_numpy(rng.uniform(0.5, 2.0, (w.nplanes, w.n, w.n)).astype(np.float32)).to(DEV)
        phi, parts = pet.objective(g, counts, gamma, img, w.params.beta, 2.0, 1e-12)
        phi_s, parts_s = pet.objective_static(g, counts, gamma, img, w.params.beta, 2.0, 1e-12)
        for a, b in zip(parts_s, parts):
            assert abs(a - b) <= 1e-6 * abs(b), (call, parts_s, parts)
        assert abs(phi_s - phi) <= 1e-6 * abs(phi), (call, phi_s, phi)
