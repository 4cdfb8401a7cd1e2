"""Precision study on the clinical-size stacked shapes (256^2 x 89, 288 x 357, 24 subsets,
20 iterations): FP32 sums, FP32 with compensated (Kahan) sums and the FP64 GPU path against the
FP64 CPU oracle, per outer iteration: relative L2 error of the image and the gap of the
objective Phi(f^k).  Counts stay int32 on every path.  The table is printed (run with -s) and,
when PET_PRECISION_OUT is set, written there as JSON."""
import json
import os

import numpy as np
import pytest
import torch

import oracle
from paper_2111_07886_gb300 import pet, synth

pytestmark = [pytest.mark.gpu, pytest.mark.slow]
DEV = torch.device("cuda:0")


def test_precision_study():
    w = synth.config_stacked_256x89(seed=0)
    scan = synth.make_scan(w)
    og = oracle.geom_from(w.geometry(), scan["sens"])
    T, M = w.params.iterations, w.nsubsets
    snaps, obj_ref = oracle.reconstruct_snapshots(og, scan["counts"], scan["gamma"], w.params,
                                                  np.ones((w.nplanes, w.n, w.n)))
    g = pet.Geometry.from_dict(w.geometry(), scan["sens"])
    counts = torch.from_numpy(scan["counts"]).to(DEV)
    gamma = torch.from_numpy(scan["gamma"]).to(DEV)
    table = {}
    for name, prec in (("fp32", synth.PREC_FP32), ("fp32_kahan", synth.PREC_FP32_KAHAN),
                       ("fp64", synth.PREC_FP64)):
        st = pet.State(g, counts, gamma, pet.make_params(w.params, prec),
                       torch.ones((w.nplanes, w.n, w.n), device=DEV))
        out = torch.empty((w.nplanes, w.n, w.n), dtype=torch.float64, device=DEV)
        rel, gap = [], []
        phi0, _ = st.objective()
        gap.append(abs(phi0 - obj_ref[0]) / abs(obj_ref[0]))
        for k in range(T):
            for _ in range(M):
                st.subiter()
            st.read_image(out)
            phi, _ = st.objective()
            got = out.cpu().numpy()
            rel.append(float(np.linalg.norm(got - snaps[k]) / np.linalg.norm(snaps[k])))
            gap.append(abs(phi - obj_ref[k + 1]) / abs(obj_ref[k + 1]))
        table[name] = {"relL2_per_iteration": rel, "objective_gap_per_iteration": gap}
    print(json.dumps({k: {"max_relL2": max(v["relL2_per_iteration"]),
                          "final_relL2": v["relL2_per_iteration"][-1],
                          "max_objective_gap": max(v["objective_gap_per_iteration"])}
                      for k, v in table.items()}, indent=1))
    if os.environ.get("PET_PRECISION_OUT"):
        with open(os.environ["PET_PRECISION_OUT"], "w") as fh:
            json.dump({"workload": w.name, "oracle_objective": list(obj_ref), **table}, fh)
    assert max(table["fp32_kahan"]["relL2_per_iteration"]) <= 1e-4
    assert max(table["fp32"]["relL2_per_iteration"]) <= 1e-4
    assert max(table["fp64"]["relL2_per_iteration"]) <= 1e-9
    assert max(table["fp32_kahan"]["objective_gap_per_iteration"]) <= 1e-6
    assert max(table["fp64"]["objective_gap_per_iteration"]) <= 1e-11
