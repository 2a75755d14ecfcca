"""pump_edge_masks_list (the per-(plan, edge) recomputation of the masks): every row equals the
graph's own mask of the listed edge, for repeated, culled and live edges, on box graphs of two
scenes; ids outside the graph leave their rows untouched and are counted."""
import numpy as np
import pytest

from paper_1607_06886_gb300 import inputs, pump

from _util import gpu_graph

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch
    assert torch.cuda.is_available()
    pump.load()
    pump.use_torch_allocator()
    yield


@pytest.mark.parametrize("name,seed,ns", [("indoor_4k", 3, 600), ("three_box_1k", 5, 400)])
def test_listed_masks_equal_the_edge_masks(name, seed, ns):
    import torch
    wl = inputs.make_workload(name, seed, ns)
    G = gpu_graph(wl)
    G.edge_masks()
    torch.cuda.synchronize()
    ref = G.export("masks")
    E, w = ref.shape[0], wl.n_particles // 32
    ref = ref.reshape(E, w)
    rng = np.random.default_rng(seed)
    # every edge once in reverse order, then random repeats (as a group's candidates repeat edges)
    elist = np.concatenate([np.arange(E)[::-1], rng.integers(0, E, size=3 * E)]).astype(np.int32)
    ed = torch.from_numpy(elist).cuda()
    out = torch.full((len(elist), w), -559038737, dtype=torch.int32).cuda()
    bad = torch.full((1,), 7, dtype=torch.int32).cuda()
    rc = G.edge_masks_list(ed.data_ptr(), len(elist), out.data_ptr(), bad.data_ptr())
    assert rc == pump.OK
    assert int(bad.item()) == 0
    got = out.cpu().numpy().view(np.uint32)
    np.testing.assert_array_equal(got, ref[elist])
    assert (ref != 0).any(axis=1).sum() > 0 and (ref == 0).all(axis=1).sum() > 0  # live and culled edges


def test_listed_masks_count_bad_ids():
    import torch
    wl = inputs.make_workload("three_box_1k", 2, 300)
    G = gpu_graph(wl)
    G.edge_masks()
    torch.cuda.synchronize()
    ref = G.export("masks")
    E = ref.shape[0]
    w = wl.n_particles // 32
    sentinel = -559038737
    for ids, n_bad in (([0, 1, E, 2], 1), ([0, -1, 1, E + 5], 2)):
        out = torch.full((4, w), sentinel, dtype=torch.int32).cuda()
        bad = torch.zeros((1,), dtype=torch.int32).cuda()
        ed = torch.tensor(ids, dtype=torch.int32).cuda()
        assert G.edge_masks_list(ed.data_ptr(), 4, out.data_ptr(), bad.data_ptr()) == pump.OK
        assert int(bad.item()) == n_bad
        got = out.cpu().numpy()
        for j, e in enumerate(ids):
            if 0 <= e < E:
                np.testing.assert_array_equal(got[j].view(np.uint32), ref[e])
            else:
                assert (got[j] == sentinel).all()
    ed = torch.tensor([0, 1, 2, 3], dtype=torch.int32).cuda()
    out = torch.zeros((4, w), dtype=torch.int32).cuda()
    assert G.edge_masks_list(ed.data_ptr(), 0, out.data_ptr()) == pump.OK
    assert G.edge_masks_list(ed.data_ptr(), -1, out.data_ptr()) == pump.ERR_INVALID_ARG
