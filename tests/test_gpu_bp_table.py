"""The packed FP32 update with the backprojection's (pixel, view) entries precomputed by
pet_geometry_create (8-plane geometries with uniform bins) against the same update computing
the entries per tile (geometries created under pet_debug_bp_table(0)): the same bits, alone and
in a graph-replayed batch, for two and four candidate bins per entry, and the entries' device
memory (16 or 32 bytes per pixel and view)."""
import numpy as np
import pytest
import torch

from paper_2111_07886_gb300 import pet, synth

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda:0")

# (N, P, V, NB, M, bin_mm / pixel_mm, bytes per entry): two tiles' entries (2 x views per subset
# x pixels per tile) fit the update's table, 1024 entries for two candidate bins, 512 for four
CASES = [(128, 11, 96, 181, 24, 1.0, 16),   # 128-pixel tiles, 4 views per subset
         (64, 19, 60, 91, 12, 1.0, 16),     # 3 plane groups (85-pixel tiles), 5 views
         (48, 17, 24, 113, 8, 0.6, 32)]     # bins finer than pixels: four candidates, 3 views


def _work(N, P, V, NB, M, rho):
    return synth.Workload(f"bp{N}_{P}", N, P, 4.0, V, NB, 4.0 * rho, M, 2e5 * P, "ellipsoid3d",
                          synth.AlgoParams(iterations=2, J0=2, J1=6, a=0.2, beta=0.5),
                          plane_mm=4.0, seed=N + P)


def _geometry(w, sens, table):
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    pet.debug_bp_table(table)
    try:
        g = pet.Geometry.from_dict(w.geometry(), sens)
    finally:
        pet.debug_bp_table(True)
    torch.cuda.synchronize()
    return g, free0 - torch.cuda.mem_get_info()[0]


def _state(g, w, scan):
    return pet.State(g, torch.from_numpy(scan["counts"]).to(DEV),
                     torch.from_numpy(scan["gamma"]).to(DEV), pet.make_params(w.params),
                     torch.ones((w.nplanes, w.n, w.n), device=DEV))


def _read(st, w):
    out = torch.empty((w.nplanes, w.n, w.n), device=DEV)
    st.read_image(out)
    torch.cuda.synchronize()
    return out.cpu().numpy()


@pytest.mark.parametrize("case", CASES)
def test_precomputed_entries_same_bits(case):
    N, P, V, NB, M, rho, esz = case
    w = _work(N, P, V, NB, M, rho)
    scan = synth.make_scan(w)
    nsub = w.params.iterations * M
    for table in (False, True):              # kernels loaded on first use, before measuring
        _geometry(w, scan["sens"], table)[0].close()
    images, used = {}, {}
    for table in (False, True):
        g, used[table] = _geometry(w, scan["sens"], table)
        st = _state(g, w, scan)
        for _ in range(nsub):
            st.subiter()
        images[table] = _read(st, w)
        st.close()
        if table:
            g_tab = g
    np.testing.assert_array_equal(images[True], images[False])
    assert np.isfinite(images[True]).all() and images[True].max() > 0
    # the entries: ceil(N^2 / TP) tiles x V views x TP pixels x esz bytes (allocation granularity
    # of a few MB on either side)
    TP = 256 // ((P + 7) // 8)
    want = -(-N * N // TP) * V * TP * esz
    extra = used[True] - used[False]
    assert want - (4 << 20) <= extra <= want + (4 << 20), (extra, want)
    # the same scan twice in one graph-replayed batch on the geometry with the entries
    items = [_state(g_tab, w, scan) for _ in range(2)]
    stream = torch.cuda.Stream()
    batch = pet.Batch(capacity=2, use_graph=True)
    for st in items:
        batch.add(st, with_objective=False, stream=stream)
    while batch.step(stream=stream) > 0:
        pass
    stream.synchronize()
    for st in items:
        np.testing.assert_array_equal(_read(st, w), images[False])
