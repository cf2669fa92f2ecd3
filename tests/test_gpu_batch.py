"""Batched contexts (several boxes of uneven sizes in one context, one launch
per phase): every box against the oracle on its own inputs with its own box
index in the random streams — tallies bit-identical, x_e / T within the
forms' tolerances — plus a box with no packets, a box with fewer packets than
a warp, and box 0 of a batch against the same box in a single-box context."""
import numpy as np
import pytest

import oracle as O
from gpu_helpers import make_fields
from paper_2312_11448_gb300.inputs import doppler_quantiles

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-9, "mixed": 1e-4}
# (side, sigma_lnrho, packets): ragged sides, a box with fewer packets than a
# warp, a box with none, several allocation chunks
SIZES = [(13, 0.3, 50_001), (16, 1.0, 120_000), (8, 1.5, 7), (12, 0.5, 0), (24, 0.8, 200_000)]
SEED = 7


def _batch(precision, mixing="tally", sizes=SIZES):
    from paper_2312_11448_gb300 import rec
    boxes = []
    for i, (n, sig, npk) in enumerate(sizes):
        d, U = make_fields(n, sig, 1.0, seed=20 + i)
        boxes.append((n, d, U, npk))
    return rec.Batch(boxes, precision=precision, mixing=mixing, seed=SEED)


def _fdt(batch):
    return np.float32 if batch.precision == "mixed" else np.float64


def _put(batch, b, name, arr, dtype):
    import torch
    batch.stream.synchronize()
    t = torch.as_tensor(np.ascontiguousarray(arr, dtype=dtype))
    if dtype == np.uint32:
        t = torch.as_tensor(np.ascontiguousarray(arr, dtype=np.uint32).view(np.int32))
    getattr(batch, name)[b].copy_(t)
    torch.cuda.synchronize()


@pytest.mark.parametrize("precision", ["mixed", "fp64"])
def test_batch_transport_bit_exact_per_box(cosmo, precision):
    batch = _batch(precision)
    rng = np.random.default_rng(5)
    fdt = _fdt(batch)
    emis_all, T_all = [], []
    for b, (n, _, _) in enumerate(SIZES):
        emis = rng.lognormal(0.0, 1.2, n ** 3)
        emis[rng.integers(0, n ** 3, 5)] = 0.0
        T = rng.uniform(2500.0, 3500.0, n ** 3)
        _put(batch, b, "emis", emis, fdt)
        _put(batch, b, "T", T, fdt)
        _put(batch, b, "tally", np.zeros(n ** 3), np.uint32)
        emis_all.append(emis)
        T_all.append(T)
    z, step = 1150.0, 4
    batch.transport(step, z)
    stats = batch.stats()
    q = doppler_quantiles().astype(fdt)
    prec = "f32" if precision == "mixed" else "f64"
    for b, (n, _, npk) in enumerate(SIZES):
        gpu = batch.tally_np(b)
        st = stats[b]
        if npk == 0:
            assert gpu.sum() == 0 and st["emitted"] == 0
            continue
        v4 = batch.host("vel4", b)
        tally, cnt, _ = O.transport(cosmo, n, z, SEED, step, npk, batch.host("emis", b), v4, batch.host("T", b), q,
                                    box=b, precision=prec)
        assert np.array_equal(gpu, tally), f"box {b}"
        assert st["emitted"] == cnt["emitted"] == npk
        assert st["absorbed"] == cnt["absorbed"] and st["capped"] == 0
        assert st["crossings"] == cnt["crossings"]
    batch.close()


@pytest.mark.parametrize("precision", ["mixed", "fp64"])
@pytest.mark.parametrize("mixing", ["full", "tally"])
def test_batch_rec_step_per_box(cosmo, precision, mixing):
    batch = _batch(precision, mixing)
    rng = np.random.default_rng(11)
    fdt = _fdt(batch)
    z_from, z_to = 1300.0, 1290.0
    ins = []
    for b, (n, _, _) in enumerate(SIZES):
        d = batch.host("delta", b).astype(np.float64)
        x0 = O.saha_xe(cosmo, z_from, d) * rng.uniform(0.95, 0.99)
        T0 = O.background(cosmo, z_from)["Tg"] * (1.0 + 0.01 * rng.standard_normal(d.size))
        tally = rng.poisson(15 * d ** 1.5).astype(np.uint32)
        _put(batch, b, "x", x0, np.float64)
        _put(batch, b, "T", T0, fdt)
        _put(batch, b, "tally", tally, np.uint32)
        ins.append((d, x0, batch.host("T", b).astype(np.float64), batch.host("vel4", b)[:, :3].astype(np.float64),
                    tally))
    batch.refresh(z_from)
    batch.step(0, z_from, z_to)
    stats = batch.stats()
    tol = TOL[precision]
    for b, (n, _, _) in enumerate(SIZES):
        d, x0, T_in, U, tally = ins[b]
        x1, T1, U1, e1, so = O.rec_step(cosmo, n, z_from, z_to, d, x0, T_in, U=U, tally=tally, mixing=mixing)
        np.testing.assert_allclose(batch.host("x", b), x1, rtol=tol, atol=0, err_msg=f"box {b}")
        np.testing.assert_allclose(batch.host("T", b).astype(np.float64), T1, rtol=tol, atol=0, err_msg=f"box {b}")
        np.testing.assert_allclose(batch.host("vel4", b)[:, :3].astype(np.float64), U1, rtol=tol, atol=1e-12)
        assert stats[b]["X_e"] == pytest.approx(so["Xe"], rel=tol)
        assert stats[b]["flags"] & 1 == 0
        if mixing == "tally":
            assert batch.tally_np(b).sum() == 0
    batch.close()


@pytest.mark.parametrize("precision", ["mixed", "fp64"])
def test_batch_box0_matches_single_box(cosmo, precision):
    """Box 0 uses random-stream box index 0, as a single-box context does: after
    the same state initialisation its first transport is bit-identical."""
    from paper_2312_11448_gb300 import rec
    sizes = [(16, 0.8, 80_000), (20, 0.4, 30_000)]
    batch = _batch(precision, "tally", sizes)
    d, U = make_fields(16, 0.8, 1.0, seed=20)
    single = rec.Box(16, d, U, 80_000, precision=precision, mixing="tally", seed=SEED)
    z0 = 1600.0
    batch.state_init(z0)
    single.state_init(z0)
    assert np.array_equal(batch.host("x", 0), single.host("x"))
    assert np.array_equal(batch.host("emis", 0), single.host("emis"))
    batch.transport(0, 1595.0)
    single.transport(0, 1595.0)
    assert np.array_equal(batch.tally_np(0), single.tally_np())
    sb, ss = batch.stats()[0], single.stats()
    for k in ("emitted", "absorbed", "crossings", "queued"):
        assert sb[k] == ss[k]
    batch.close()
    single.close()


def test_batch_rejects_adjoint_and_bad_boxes():
    from paper_2312_11448_gb300 import rec
    batch = _batch("fp64", "full", SIZES[:2])
    x = batch.x[0]
    with pytest.raises(rec.RecError, match="single-box"):
        batch._check(rec.lib().rec_xe_adjoint(batch.ctx, rec.C.c_void_p(x.data_ptr()), 1.0,
                                              rec.C.c_void_p(x.data_ptr()), rec.C.c_void_p(x.data_ptr())),
                     "rec_xe_adjoint")
    batch.close()
    d, U = make_fields(8, 0.5, 1.0, seed=1)
    with pytest.raises(rec.RecError, match="box 1"):
        rec.Batch([(8, d, U, 10), (8, d, U, 2 ** 32)], precision="fp64")
