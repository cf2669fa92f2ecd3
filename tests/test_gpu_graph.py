"""rec_graph_step (transport + rec_step captured as one CUDA graph, the
executable graph updated in place every step) against the same two calls
made directly: identical kernels and parameters, so the state after several
steps must agree bit for bit (single box and batch), and the misuse cases are
rejected."""
import numpy as np
import pytest

from gpu_helpers import make_fields

pytestmark = pytest.mark.gpu


def _zs(n_steps=6):
    from paper_2312_11448_gb300.inputs import z_schedule
    return z_schedule(1500.0, 1400.0, n_steps)


@pytest.mark.parametrize("precision,n,halo", [("mixed", 24, 0), ("fp64", 24, 0), ("mixed", 64, 8)])
def test_graph_steps_equal_direct_calls(precision, n, halo):
    """halo > 0: the region-sweep march (a memset and 22 kernel nodes) in the graph;
    the graph step after a change of halo re-instantiates the executable graph."""
    import torch
    from paper_2312_11448_gb300 import rec
    d, U = make_fields(n, 0.8, 2.0, seed=3)
    zs = _zs()
    boxes = []
    for _ in range(2):
        s = torch.cuda.Stream()
        b = rec.Box(n, d, U, 150_000, precision=precision, mixing="tally", seed=5, stream=s, n_stats=1)
        if halo:
            b.set_tuning(march_halo=halo, tile=16, march_blocks_per_sm=2)
        b.state_init(zs[0])
        boxes.append(b)
    direct, graph = boxes
    for k in range(len(zs) - 1):
        if halo and k == 3:  # sweeps off, then the graph changes its topology
            for b in boxes:
                b.set_tuning(march_halo=0)
        direct.transport(k, zs[k])
        direct.step(k, zs[k], zs[k + 1])
        graph.graph_step(k, zs[k], zs[k + 1])
    for name in ("x", "T", "vel4", "emis"):
        assert np.array_equal(direct.host(name), graph.host(name)), name
    sd, sg = direct.stats(), graph.stats()
    for key in ("emitted", "absorbed", "crossings", "queued", "X_e", "lam", "newton_passes"):
        assert sd[key] == sg[key], key
    direct.close()
    graph.close()


def test_graph_steps_batch():
    import torch
    from paper_2312_11448_gb300 import rec
    zs = _zs(4)
    specs = [(16, 0.5, 60_000), (13, 1.0, 20_000), (8, 0.3, 5)]
    out = []
    for use_graph in (False, True):
        boxes = []
        for i, (n, sig, npk) in enumerate(specs):
            d, U = make_fields(n, sig, 1.0, seed=40 + i)
            boxes.append((n, d, U, npk))
        b = rec.Batch(boxes, precision="mixed", mixing="tally", seed=9, stream=torch.cuda.Stream())
        b.state_init(zs[0])
        for k in range(len(zs) - 1):
            if use_graph:
                b.graph_step(k, zs[k], zs[k + 1])
            else:
                b.transport(k, zs[k])
                b.step(k, zs[k], zs[k + 1])
        out.append(([b.host("x", i) for i in range(len(specs))], b.stats()))
        b.close()
    for xa, xb in zip(out[0][0], out[1][0]):
        assert np.array_equal(xa, xb)
    for sa, sb in zip(out[0][1], out[1][1]):
        assert sa["absorbed"] == sb["absorbed"] and sa["X_e"] == sb["X_e"]


def test_graph_step_misuse():
    import torch
    from paper_2312_11448_gb300 import rec
    d, U = make_fields(8, 0.5, 1.0, seed=1)
    b = rec.Box(8, d, U, 1000, precision="mixed", seed=1, stream=torch.cuda.Stream())
    with pytest.raises(rec.RecError, match="rec_state_init"):
        b.graph_step(0, 1500.0, 1490.0)
    b.state_init(1500.0)
    b.timing(True)
    with pytest.raises(rec.RecError, match="timing"):
        b.graph_step(0, 1500.0, 1490.0)
    b.timing(False)
    with pytest.raises(rec.RecError, match="z_from > z_to"):
        b.graph_step(0, 1490.0, 1500.0)
    b.graph_step(0, 1500.0, 1490.0)
    b.close()
